"""GPU parity of the regridding (mg_regrid) and of the naive adaptive grid
(MG_GRID_NAIVE, Sec. II.F) against the FP64 oracle, through the C-ABI.
Tolerance: the FP64 parity bar, relative L2 1e-12 on psi and 1e-12 on the
grid centres."""
import numpy as np
import pytest

import oracle
from tests import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = inputs.ATOM_DIATOM


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1909_06412_gb300 as m

    m.lib()
    return m


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.asarray(b).ravel())


def atom_diatom_pair(mg, N=(48, 36), dq=(0.4, 0.25)):
    minv = (1 / P["mu"][0], 1 / P["mu"][1])
    pot = [P["Dm"], P["a"], P["re"], P["A"], P["beta"]]
    g = mg.Propagator(N, dq, minv=minv)
    g.set_potential(mg.MG_POT_ATOM_DIATOM, pot)
    o = oracle.Grid(N, dq, minv=minv)
    o.set_potential(oracle.POT_ATOM_DIATOM, pot)
    rbar = oracle.morse_mean(P["Dm"], P["a"], P["re"], P["mu"][1])
    fac = [("gauss", 6.0, -10.0, 0.6), ("morse", P["Dm"], P["a"], P["re"], P["mu"][1])]
    g.set_separable(fac, [6.0, rbar], [-10.0, 0.0])
    o.set_separable(fac, [6.0, rbar], [-10.0, 0.0])
    return g, o


@pytest.mark.parametrize("N,prec,tol", [((48, 36), 0, 1e-12), ((12, 18, 16), 0, 1e-12), ((32, 24), 1, 2e-6)])
def test_regrid_matches_oracle(mg, N, prec, tol):
    D = len(N)
    dq = tuple(0.35 + 0.05 * l for l in range(D))
    g = mg.Propagator(N, dq, precision=prec)
    g.set_potential(mg.MG_POT_HARMONIC, list(np.eye(D).ravel()) + [0.0] * D)
    o = oracle.Grid(N, dq)
    u = inputs.random_state(N, 11)
    q0, p0 = inputs.random_centre(D, 12)
    sc = np.sqrt(np.prod(dq))
    g.set_state(u / sc, q0, p0)
    q1 = q0 + np.linspace(0.13, -0.41, D)
    p1 = p0 + np.linspace(-0.7, 0.25, D)
    g.regrid(q1, p1)
    psi, q, p, _ = g.get_state()
    ref = o.apply_f(q1, p1, o.apply_f(q0, p1, u, -1), +1) / sc
    assert rel(psi, ref) < tol
    assert np.allclose(q, q1, rtol=0, atol=1e-15) and np.allclose(p, p1, rtol=0, atol=1e-15)
    g.regrid(q0, p1)  # back to the first positions: the state returns
    psi2, _, _, _ = g.get_state()
    assert rel(psi2 * sc, u * 1.0) < max(tol, 1e-13) * 10


def test_naive_propagation_matches_oracle(mg):
    g, o = atom_diatom_pair(mg)
    g.propagate(6, 5.0, "yoshida4", mg.MG_TVT, mg.MG_GRID_NAIVE)
    o.propagate(6, 5.0, "yoshida4", oracle.SPLIT_TVT, oracle.GRID_NAIVE)
    psi, q, p, _ = g.get_state()
    psi_o, q_o, p_o, _ = o.get_state()
    assert rel(psi, psi_o) < 1e-12
    assert np.abs(q - q_o).max() < 1e-12 * max(1.0, np.abs(q_o).max())
    assert np.abs(p - p_o).max() < 1e-12 * max(1.0, np.abs(p_o).max())


def test_naive_grid_is_not_reversible_on_the_gpu(mg):
    errs = {}
    for motion in (mg.MG_GRID_ADAPTIVE, mg.MG_GRID_NAIVE):
        g, _ = atom_diatom_pair(mg)
        u0 = g.get_state()[0]
        g.propagate(20, 5.0, "yoshida4", mg.MG_TVT, motion)
        g.propagate(20, -5.0, "yoshida4", mg.MG_TVT, motion)
        errs[motion] = rel(g.get_state()[0], u0)
    assert errs[mg.MG_GRID_ADAPTIVE] < 1e-12
    assert errs[mg.MG_GRID_NAIVE] > 1e-6


def e1_pair(mg, q0, prec=0):
    P = inputs.DUSCHINSKY3D
    om = np.array(P["omega"])
    pot = list(np.array(P["K"]).ravel()) + [0.0] * 3
    g = mg.Propagator(P["N"], P["dq"], minv=om, precision=prec)
    g.set_potential(mg.MG_POT_HARMONIC, pot)
    o = oracle.Grid(P["N"], P["dq"], minv=om)
    o.set_potential(oracle.POT_HARMONIC, pot)
    fac = [("gauss", q0[l], 0.0, 1.0) for l in range(3)]
    g.set_separable(fac, q0, [0.0] * 3)
    o.set_separable(fac, q0, [0.0] * 3)
    return g, o


def test_inner_product_matches_oracle_and_leaves_both_states(mg):
    q0 = np.array(inputs.DUSCHINSKY3D["q0"])
    ga, oa = e1_pair(mg, q0)
    gb, ob = e1_pair(mg, q0 + np.array([-1.0, 1.0, 1.0]))
    v = ga.inner_product(gb)
    assert abs(v - np.exp(-0.75)) < 1e-9          # the printed 0.472 of Sec. III.A
    for g, o in ((ga, oa), (gb, ob)):
        g.propagate(7, 0.1, "yoshida4")
        o.propagate(7, 0.1, "yoshida4")
    v = ga.inner_product(gb)
    vo = oracle.inner_product(oa, ob)
    assert abs(v - vo) < 1e-12 * abs(vo)
    # neither context was disturbed: both continue exactly like the oracle
    for g, o in ((ga, oa), (gb, ob)):
        g.propagate(3, 0.1, "yoshida4")
        o.propagate(3, 0.1, "yoshida4")
        psi, q, p, _ = g.get_state()
        psi_o, q_o, p_o, _ = o.get_state()
        assert rel(psi, psi_o) < 1e-12 and np.abs(q - q_o).max() < 1e-12 * max(1.0, np.abs(q_o).max())


def test_inner_product_rejects_mismatched_grids(mg):
    a = mg.Propagator((16, 16), (0.5, 0.5))
    b = mg.Propagator((16, 12), (0.5, 0.5))
    for g in (a, b):
        g.set_potential(mg.MG_POT_HARMONIC, [1.0, 0.0, 0.0, 1.0, 0.0, 0.0])
        g.set_separable([("gauss", 0.0, 0.0, 1.0)] * 2, [0.0, 0.0], [0.0, 0.0])
    with pytest.raises(mg.MgError):
        a.inner_product(b)
