"""GPU parity of the short-axis propagation kernel (grids of D >= 3 axes, all
of one length 8, 12 or 16; several axes transformed per pass) against the
FP64 oracle, through the C-ABI.

Shapes are chosen to exercise every chunking case of the kernel's planner:
one group holding all axes (3D), a contiguous group plus one strided group
of one axis (4D), strided groups of two and three axes (5D, 6D), and chunks
that are only partly filled (3D FP32, where a chunk holds more blocks than the
grid has).  Tolerances: relative L2 1e-12 on psi and 1e-12 on the grid centres
for FP64 (the FP64 parity bar); 5e-5 for FP32 storage, the stated error of
the mixed-precision path on these step counts.
"""
import numpy as np
import pytest

import oracle
from tests import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAM = inputs.HENON_HEILES["lam"]


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1909_06412_gb300 as m

    m.lib()
    return m


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.asarray(b).ravel())


def hh_pair(mg, n, D, prec, q0=2.0, flags=0):
    dq = np.sqrt(2 * np.pi / n)
    N = (n,) * D
    g = mg.Propagator(N, (dq,) * D, precision=prec, flags=flags)
    g.set_potential(mg.MG_POT_HENON_HEILES, [LAM])
    o = oracle.Grid(N, (dq,) * D)
    o.set_potential(oracle.POT_HENON_HEILES, [LAM])
    fac = [("gauss", q0 + 0.1 * l, 0.2 - 0.1 * l, 1.0) for l in range(D)]
    qc = [q0 + 0.1 * l for l in range(D)]
    pc = [0.2 - 0.1 * l for l in range(D)]
    g.set_separable(fac, qc, pc)
    o.set_separable(fac, qc, pc)
    return g, o


def check(g, o, tol):
    psi, q, p, _ = g.get_state()
    psi_o, q_o, p_o, _ = o.get_state()
    err = rel(psi, psi_o)
    assert err < tol, f"psi rel L2 {err:.3e}"
    ct = max(tol, 1e-12)
    assert np.abs(q - q_o).max() < ct * max(1.0, np.abs(q_o).max()), (q, q_o)
    assert np.abs(p - p_o).max() < ct * max(1.0, np.abs(p_o).max()), (p, p_o)
    return err


@pytest.mark.parametrize("n,D,prec,steps", [
    (16, 3, 0, 6), (12, 3, 0, 6), (8, 3, 0, 6),      # one group holds every axis
    (16, 3, 1, 6), (12, 3, 1, 6),                    # FP32: chunks only partly filled
    (16, 5, 1, 1),                                   # TMA copies with a strided group of 2 axes
    (12, 4, 0, 4), (16, 4, 0, 4), (12, 4, 1, 4), (16, 4, 1, 4),
    (12, 5, 0, 1), (8, 5, 1, 4), (8, 6, 0, 2),       # strided groups of 2 and 3 axes
])
def test_short_kernel_henon_heiles_vs_oracle(mg, n, D, prec, steps):
    g, o = hh_pair(mg, n, D, prec)
    # FP32 grids of 16-point axes move their chunks by TMA tensor copies
    assert g.path == (2 if (prec == 1 and n == 16) else 1)
    g.propagate(steps, 0.02, "suzuki4")
    o.propagate(steps, 0.02, "suzuki4")
    check(g, o, 1e-12 if prec == 0 else 5e-5)


@pytest.mark.parametrize("split,motion", [(1, 0), (2, 0), (0, 1), (0, 2)])
def test_short_kernel_splits_and_grid_motion(mg, split, motion):
    g, o = hh_pair(mg, 12, 4, 0)
    g.propagate(3, 0.03, "yoshida4", split, motion)
    o.propagate(3, 0.03, "yoshida4", split, motion)
    check(g, o, 1e-12)


def test_short_kernel_diagonal_harmonic(mg):
    om = np.array([1.0, 1.2, 1.5])
    N, dq = (16, 16, 16), (0.45, 0.45, 0.45)
    pot = list(np.diag(om ** 2).ravel()) + [0.3, -0.2, 0.1]
    g = mg.Propagator(N, dq)
    g.set_potential(mg.MG_POT_HARMONIC, pot)
    o = oracle.Grid(N, dq)
    o.set_potential(oracle.POT_HARMONIC, pot)
    fac = [("gauss", q, p, w ** -0.5) for q, p, w in zip((1.0, -0.5, 0.8), (0.0, 0.5, -0.3), om)]
    g.set_separable(fac, (1.0, -0.5, 0.8), (0.0, 0.5, -0.3))
    o.set_separable(fac, (1.0, -0.5, 0.8), (0.0, 0.5, -0.3))
    assert g.path == 1
    g.propagate(50, 0.01, "strang")
    o.propagate(50, 0.01, "strang")
    check(g, o, 1e-12)


def test_general_harmonic_keeps_the_general_kernel(mg):
    # a coupled force-constant matrix is not of the per-axis + pair form
    K = np.array([[1.0, 0.1, 0.0], [0.1, 1.2, 0.0], [0.0, 0.0, 1.5]])
    g = mg.Propagator((16, 16, 16), (0.45,) * 3)
    g.set_potential(mg.MG_POT_HARMONIC, list(K.ravel()) + [0.0] * 3)
    assert g.path == 0


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 3e-5)])
def test_short_kernel_matches_general_kernel(mg, prec, tol):
    # same grid and state through both kernels (mg_create_ex's
    # MG_CREATE_GENERAL_KERNEL selects the general one)
    gg, _ = hh_pair(mg, 16, 4, prec, flags=mg.MG_CREATE_GENERAL_KERNEL)
    gs, _ = hh_pair(mg, 16, 4, prec)
    assert gg.path == 0 and gs.path == (2 if prec == 1 else 1)
    for g in (gg, gs):
        g.propagate(20, 0.02, "yoshida4")
    a, qa, pa, _ = gs.get_state()
    b, qb, pb, _ = gg.get_state()
    assert rel(a, b) < tol
    assert np.abs(qa - qb).max() < tol and np.abs(pa - pb).max() < tol


def test_short_kernel_norm_energy_and_reversibility(mg):
    g, _ = hh_pair(mg, 12, 5, 0)
    u0 = g.psi.clone()
    _, q0, p0, _ = g.get_state(want_psi=False)
    n0, e0, _, _ = g.observables()
    g.propagate(10, 0.02, "suzuki4")
    n1, e1, _, _ = g.observables()
    assert abs(n1 / n0 - 1) < 1e-13
    assert abs(e1 - e0) < 1e-4 * abs(e0)
    g.propagate(10, -0.02, "suzuki4")
    _, q2, p2, _ = g.get_state(want_psi=False)
    err = float(torch.linalg.vector_norm(g.psi - u0) / torch.linalg.vector_norm(u0))
    assert err < 1e-12
    assert np.abs(q2 - q0).max() < 1e-12 and np.abs(p2 - p0).max() < 1e-11


# --------------------------------------------------------------------------
# The tensor-core variant of the short-axis kernel is refused; the
# tensor-core 16-point DFT runs as its own kernel (test_gpu_probe.py)
# --------------------------------------------------------------------------

def test_tensor_core_flags_are_checked(mg):
    dq = (np.sqrt(2 * np.pi / 16),) * 4
    for flag in (mg.MG_CREATE_TC_TF32X3, mg.MG_CREATE_TC_BF16X3):
        for prec in (mg.MG_FP64, mg.MG_FP32_MIXED):
            with pytest.raises(mg.MgError) as e:
                mg.Propagator((16,) * 4, dq, precision=prec, flags=flag)
            assert e.value.code == mg.MG_ERR_UNSUPPORTED
    with pytest.raises(mg.MgError) as e:  # both splits at once
        mg.Propagator((16,) * 4, dq, precision=mg.MG_FP32_MIXED,
                      flags=mg.MG_CREATE_TC_TF32X3 | mg.MG_CREATE_TC_BF16X3)
    assert e.value.code == mg.MG_ERR_ARG
