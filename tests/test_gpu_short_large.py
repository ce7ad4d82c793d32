"""The short-axis kernel on grids large enough to reach the same kinds of
axis groups as the full-size 8D plans, against stored FP64 oracle results
(tests/golden/make_short_axis_samples.py; one Strang step each, about 15
minutes of oracle time together):
  - 12^7 FP64: a strided group of three 12-point axes with a leading index
    (the 12^8 plan has {5,6,7}, {2,3,4}, {0,1}), compared at 1e-12;
  - 16^6 FP32 (TMA copies): a strided group of two 16-point axes with a
    leading index and a single axis of stride 16^5 (the 16^8 plan has
    {5,6,7}, {3,4}, {1,2}, {0}), compared at the FP32 path's 5e-5.
Compared at the 1024 stored grid points (each within tol of the discrete L2
norm of psi, which relative L2 <= tol implies) and on the grid centres."""
import numpy as np
import pytest

from tests.golden import records

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAM = 0.111803


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1909_06412_gb300 as m

    m.lib()
    return m


@pytest.mark.parametrize("n,D,prec,fname,tol,group", [
    (12, 7, 0, "hh_12p7_strang1.txt", 1e-12, (1, 3)),
    (16, 6, 1, "hh_16p6_strang1.txt", 5e-5, (1, 2)),
])
def test_short_kernel_large_plans_vs_stored_oracle(mg, n, D, prec, fname, tol, group):
    plan = mg.mg_short_axis_plan((n,) * D, prec)
    assert group in plan["groups"], plan
    if prec == 1:
        assert (0, 1) in plan["groups"], plan
    rec = records.read(fname)
    dq = np.sqrt(2 * np.pi / n)
    g = mg.Propagator((n,) * D, (dq,) * D, precision=prec)
    g.set_potential(mg.MG_POT_HENON_HEILES, [LAM])
    g.set_separable([("gauss", 2.0 + 0.1 * l, 0.2 - 0.1 * l, 1.0) for l in range(D)],
                    [2.0 + 0.1 * l for l in range(D)], [0.2 - 0.1 * l for l in range(D)])
    assert g.path == (2 if prec == 1 else 1)
    g.propagate(1, 0.02, "strang")
    _, q, p, _ = g.get_state(want_psi=False)
    ct = max(tol, 1e-12)
    assert np.abs(q - rec["q"]).max() < ct * max(1.0, np.abs(rec["q"]).max()), (q, rec["q"])
    assert np.abs(p - rec["p"]).max() < ct * max(1.0, np.abs(rec["p"]).max()), (p, rec["p"])
    # psi at the stored points, read from the device state (u = psi sqrt(prod dq))
    u = g.psi.view(torch.complex128 if prec == 0 else torch.complex64)
    idx = torch.from_numpy(rec["idx"]).to(u.device)
    vals = u[idx].to(torch.complex128).cpu().numpy() / np.sqrt(dq ** D)
    d = np.abs(vals - rec["psi"]).max()
    assert d < tol * rec["psi_l2"], d / rec["psi_l2"]
    g.close()
    torch.cuda.empty_cache()
