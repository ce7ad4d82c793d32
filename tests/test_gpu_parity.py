"""GPU parity: the sm_103a library (through its C-ABI) against the FP64 oracle.

Tolerance: relative L2 distance <= 1e-12 on the wavefunction and on the grid
centres (q_t, p_t), the FP64 parity bar of the hot path.  Inputs are the
seeded synthetic workloads of tests/inputs.py.
"""
import numpy as np
import pytest

import oracle
from tests import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1909_06412_gb300 as m

    m.lib()
    return m


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.asarray(b).ravel())


def pair(mg, N, dq, minv, kind, pot, hbar=1.0):
    g = mg.Propagator(N, dq, minv=minv, hbar=hbar)
    g.set_potential(kind, pot)
    o = oracle.Grid(N, dq, minv=minv, hbar=hbar)
    o.set_potential(kind, pot)
    return g, o


def assert_same(g, o, tol=TOL):
    psi, q, p, t = g.get_state()
    psi_o, q_o, p_o, t_o = o.get_state()
    err = rel(psi, psi_o)
    assert err < tol, f"psi rel L2 {err:.3e}"
    sq = max(1.0, np.abs(q_o).max())
    sp = max(1.0, np.abs(p_o).max())
    assert np.abs(q - q_o).max() < tol * sq, (q, q_o)
    assert np.abs(p - p_o).max() < tol * sp, (p, p_o)
    return err


def atom_diatom(mg, N, dq):
    P = inputs.ATOM_DIATOM
    minv = (1 / P["mu"][0], 1 / P["mu"][1])
    pot = [P["Dm"], P["a"], P["re"], P["A"], P["beta"]]
    g, o = pair(mg, N, dq, minv, oracle.POT_ATOM_DIATOM, pot)
    rbar = oracle.morse_mean(P["Dm"], P["a"], P["re"], P["mu"][1])
    fac = [("gauss", P["R0"], P["P0"], P["sigma"]), ("morse", P["Dm"], P["a"], P["re"], P["mu"][1])]
    g.set_separable(fac, [P["R0"], rbar], [P["P0"], 0.0])
    o.set_separable(fac, [P["R0"], rbar], [P["P0"], 0.0])
    return g, o


def harmonic3d(mg, N=None, dq=None):
    P = inputs.HARMONIC3D
    N = N or P["N"]
    dq = dq or P["dq"]
    om = np.array(P["omega"])
    pot = list(np.diag(om ** 2).ravel()) + [0.0, 0.0, 0.0]
    g, o = pair(mg, N, dq, (1.0, 1.0, 1.0), oracle.POT_HARMONIC, pot)
    fac = [("gauss", P["q0"][l], P["p0"][l], om[l] ** -0.5) for l in range(3)]
    g.set_separable(fac, P["q0"], P["p0"])
    o.set_separable(fac, P["q0"], P["p0"])
    return g, o


# --------------------------------------------------------------------------
# the workloads themselves
# --------------------------------------------------------------------------

def test_initial_state_matches_oracle(mg):
    g, o = atom_diatom(mg, (64, 48), (0.32, 0.2))
    assert_same(g, o, 1e-14)
    assert abs(mg.mg_morse_mean(0.17, 1.0, 1.4, 0.5 * inputs.AMU) -
               oracle.morse_mean(0.17, 1.0, 1.4, 0.5 * inputs.AMU)) < 1e-10


def test_harmonic_3d_strang_1000_steps(mg):
    # 32^3 grid, spacing 0.3, coherent state, Strang dt = 0.01, 1000 steps
    g, o = harmonic3d(mg)
    P = inputs.HARMONIC3D
    g.propagate(P["steps"], P["dt"], "strang")
    o.propagate(P["steps"], P["dt"], "strang")
    assert_same(g, o)


def test_atom_diatom_full_grid_yoshida4(mg):
    # 256 x 256 grid of the benchmark, 20 steps of dt = 1 a.u.
    g, o = atom_diatom(mg, inputs.ATOM_DIATOM["N"], inputs.ATOM_DIATOM["dq"])
    g.propagate(20, 1.0, "yoshida4")
    o.propagate(20, 1.0, "yoshida4")
    assert_same(g, o)


@pytest.mark.parametrize("scheme,steps", [("strang", 12), ("yoshida4", 12), ("suzuki4", 12), ("yoshida6", 12),
                                          ("yoshida8", 12), ("yoshida10", 6), ("suzuki6", 12), ("suzuki8", 4),
                                          ("suzuki10", 2)])
def test_atom_diatom_schemes(mg, scheme, steps):
    # every composition the library offers, up to tenth order (81 and 625
    # stages per step for yoshida10 and suzuki10)
    g, o = atom_diatom(mg, (64, 48), (0.32, 0.2))
    g.propagate(steps, 2.0, scheme)
    o.propagate(steps, 2.0, scheme)
    assert_same(g, o)


@pytest.mark.parametrize("split", [oracle.SPLIT_TVT, oracle.SPLIT_VTV, oracle.SPLIT_TV])
@pytest.mark.parametrize("motion", [oracle.GRID_ADAPTIVE, oracle.GRID_ADAPTIVE_CENTRE_P, oracle.GRID_FIXED])
def test_splits_and_grid_motion(mg, split, motion):
    g, o = atom_diatom(mg, (48, 36), (0.4, 0.25))
    g.propagate(15, 2.0, "yoshida4", split, motion)
    o.propagate(15, 2.0, "yoshida4", split, motion)
    assert_same(g, o)


# --------------------------------------------------------------------------
# other potentials, axis lengths and dimensions (ragged, radix 3, D=1..8)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N", [(2,), (6,), (12,), (64,), (96,), (1024,), (2048,)])
def test_one_dimension(mg, N):
    dq = (8.0 / N[0],) if N[0] > 6 else (0.9,)
    g, o = pair(mg, N, dq, (0.8,), oracle.POT_HARMONIC, [1.7, 0.3])
    fac = [("gauss", 0.6, -0.4, 0.9)]
    g.set_separable(fac, [0.6], [-0.4])
    o.set_separable(fac, [0.6], [-0.4])
    g.propagate(40, 0.05, "yoshida4")
    o.propagate(40, 0.05, "yoshida4")
    assert_same(g, o)


def test_henon_heiles_3d_mixed_radix(mg):
    N, dq = (12, 18, 8), (0.7, 0.55, 0.9)
    g, o = pair(mg, N, dq, (1.0, 1.0, 1.0), oracle.POT_HENON_HEILES, [inputs.HENON_HEILES["lam"]])
    fac = [("gauss", 2.0, 0.0, 1.0)] * 3
    g.set_separable(fac, [2.0] * 3, [0.0] * 3)
    o.set_separable(fac, [2.0] * 3, [0.0] * 3)
    g.propagate(10, 0.05, "suzuki4")
    o.propagate(10, 0.05, "suzuki4")
    assert_same(g, o)


def test_henon_heiles_8d(mg):
    N = (4, 4, 4, 4, 4, 4, 4, 6)
    dq = (1.2,) * 7 + (0.9,)
    g, o = pair(mg, N, dq, (1.0,) * 8, oracle.POT_HENON_HEILES, [inputs.HENON_HEILES["lam"]])
    fac = [("gauss", 2.0, 0.0, 1.0)] * 8
    g.set_separable(fac, [2.0] * 8, [0.0] * 8)
    o.set_separable(fac, [2.0] * 8, [0.0] * 8)
    g.propagate(2, 0.05, "suzuki4")
    o.propagate(2, 0.05, "suzuki4")
    assert_same(g, o)


def test_duschinsky_general_harmonic(mg):
    P = inputs.DUSCHINSKY3D
    N, dq = (16, 16, 16), (0.8, 0.8, 0.8)
    pot = list(np.array(P["K"]).ravel()) + [-1.0, 1.0, 1.0]
    g, o = pair(mg, N, dq, P["omega"], oracle.POT_HARMONIC, pot)
    fac = [("gauss", 0.0, 0.0, 1.0)] * 3
    g.set_separable(fac, [0, 0, 0], [0, 0, 0])
    o.set_separable(fac, [0, 0, 0], [0, 0, 0])
    g.propagate(20, 0.05, "yoshida4")
    o.propagate(20, 0.05, "yoshida4")
    assert_same(g, o)


def test_secrest_johnson_vtv(mg):
    N, rng1, rng2 = (64, 64), 28.0, 48.0
    dq = (rng1 / N[0], rng2 / N[1])
    g, o = pair(mg, N, dq, (1.0, 1.5), oracle.POT_SECREST_JOHNSON, [20.0, 0.158, 0.3])
    fac = [("gauss", 0.0, 0.0, 1.0), ("gauss", 24.0, -3.56, np.sqrt(8.0))]
    g.set_separable(fac, [0.0, 24.0], [0.0, -3.56])
    o.set_separable(fac, [0.0, 24.0], [0.0, -3.56])
    g.propagate(30, 0.1, "yoshida4", oracle.SPLIT_VTV)
    o.propagate(30, 0.1, "yoshida4", oracle.SPLIT_VTV)
    assert_same(g, o)


@pytest.mark.parametrize("N,motion,bits", [
    ((128, 2048), oracle.GRID_FIXED, 3),
    ((128, 2048), oracle.GRID_ADAPTIVE, 3),
    ((64, 1536), oracle.GRID_ADAPTIVE, 1),
])
def test_long_axis_tables_in_workspace(mg, N, motion, bits):
    # Sec. III.B's Secrest-Johnson model on grids whose per-axis tables do not
    # fit shared memory beside the data regions: the general kernel reads them
    # from the workspace (the 128 x 2048 fixed reference grid of the paper)
    rng1, rng2 = 28.0, 96.0
    dq = (rng1 / N[0], rng2 / N[1])
    g, o = pair(mg, N, dq, (1.0, 1.5), oracle.POT_SECREST_JOHNSON, [20.0, 0.158, 0.3])
    assert g.tables_in_workspace == bits
    fac = [("gauss", 0.0, 0.0, 1.0), ("gauss", 24.0, -3.56, np.sqrt(8.0))]
    g.set_separable(fac, [0.0, 24.0], [0.0, -3.56])
    o.set_separable(fac, [0.0, 24.0], [0.0, -3.56])
    g.propagate(6, 0.1, "yoshida4", oracle.SPLIT_VTV, motion)
    o.propagate(6, 0.1, "yoshida4", oracle.SPLIT_VTV, motion)
    assert_same(g, o)
    assert abs(g.observables()[1] - o.observables()[1]) < 1e-11 * abs(o.observables()[1])


def test_random_state_and_centre(mg):
    N, dq = (24, 32), (0.45, 0.35)
    g, o = pair(mg, N, dq, (0.7, 1.3), oracle.POT_HENON_HEILES, [0.2], hbar=0.8)
    u = inputs.random_state(N, seed=42) / np.sqrt(np.prod(dq))
    q, p = inputs.random_centre(2, seed=9, scale=1.0)
    g.set_state(u, q, p, 0.25)
    o.set_state(u, q, p, 0.25)
    g.propagate(8, 0.03, "yoshida6", oracle.SPLIT_VTV)
    o.propagate(8, 0.03, "yoshida6", oracle.SPLIT_VTV)
    assert_same(g, o)
    assert abs(g.get_state()[3] - o.get_state()[3]) < 1e-12


# --------------------------------------------------------------------------
# invariants, observables, determinism, error statuses
# --------------------------------------------------------------------------

def test_observables_match_oracle(mg):
    g, o = atom_diatom(mg, (64, 48), (0.32, 0.2))
    g.propagate(10, 2.0, "yoshida4")
    o.propagate(10, 2.0, "yoshida4")
    n, e, mq, mp = g.observables()
    no, eo, mqo, mpo = o.observables()
    assert abs(n - no) < 1e-13 and abs(e - eo) < 1e-12 * abs(eo)
    assert np.allclose(mq, mqo, rtol=1e-12, atol=1e-12) and np.allclose(mp, mpo, rtol=1e-12, atol=1e-12)


def test_reversibility_and_norm_on_gpu(mg):
    g, _ = atom_diatom(mg, inputs.ATOM_DIATOM["N"], inputs.ATOM_DIATOM["dq"])
    u0, q0, p0, _ = g.get_state()
    n0 = g.observables()[0]
    g.propagate(50, 1.0, "yoshida4")
    assert abs(g.observables()[0] / n0 - 1) < 1e-12
    g.propagate(50, -1.0, "yoshida4")
    u1, q1, p1, _ = g.get_state()
    assert rel(u1, u0) < 1e-11
    assert np.allclose(q1, q0, atol=1e-11, rtol=0) and np.allclose(p1, p0, atol=1e-10, rtol=0)


def test_bitwise_deterministic(mg):
    outs = []
    for _ in range(2):
        g, _ = atom_diatom(mg, (128, 96), (0.16, 0.1))
        g.propagate(10, 1.0, "suzuki4")
        outs.append(g.get_state())
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1]) and np.array_equal(outs[0][2], outs[1][2])


def test_unstable_step_reports_status(mg):
    g, _ = harmonic3d(mg, (16, 16, 16), (0.6, 0.6, 0.6))
    with pytest.raises(mg.MgError) as e:
        g.propagate(50, 40.0, "yoshida4")
        g.get_state()
    assert e.value.code in (mg.MG_ERR_UNSTABLE, mg.MG_ERR_NONFINITE)
    # the context stays usable after the error was reported
    g.set_separable([("gauss", 0.0, 0.0, 1.0)] * 3, [0, 0, 0], [0, 0, 0])
    g.propagate(2, 0.01, "strang")
    g.get_state()


def test_nonfinite_state_reports_status(mg):
    g, _ = harmonic3d(mg, (8, 8, 8), (0.6, 0.6, 0.6))
    u = np.zeros((8, 8, 8), complex)
    u[1, 2, 3] = np.nan
    g.set_state(u, [0, 0, 0], [0, 0, 0])
    g.propagate(1, 0.01, "strang")
    with pytest.raises(mg.MgError) as e:
        g.sync()
    assert e.value.code == mg.MG_ERR_NONFINITE


def test_argument_errors(mg):
    with pytest.raises(mg.MgError) as e:
        mg.Propagator((10, 7), (0.1, 0.1))
    assert e.value.code in (mg.MG_ERR_ARG, mg.MG_ERR_UNSUPPORTED)
    with pytest.raises(mg.MgError) as e:
        mg.Propagator((10, 14), (0.1, 0.1))  # factor 5 and 7
    assert e.value.code == mg.MG_ERR_UNSUPPORTED
    g = mg.Propagator((8, 8), (0.5, 0.5))
    with pytest.raises(mg.MgError) as e:
        g.propagate(1, 0.1)  # no potential, no state
    assert e.value.code == mg.MG_ERR_STATE
    g.set_potential(mg.MG_POT_HENON_HEILES, [0.1])
    g.set_separable([("gauss", 0, 0, 1)] * 2, [0, 0], [0, 0])
    with pytest.raises(mg.MgError):
        g.propagate(1, 0.1, "yoshida5")
    with pytest.raises(mg.MgError):
        g.set_potential(mg.MG_POT_ATOM_DIATOM, [1.0, 2.0])


def test_host_buffer_upload_and_download(mg):
    # mg_upload_u / mg_download_u move the scaled state without conversion;
    # a propagation between them matches the oracle
    g, o = atom_diatom(mg, (64, 48), (0.32, 0.2))
    u = g.psi.view(torch.complex128).cpu().pin_memory()
    _, q0, p0, _ = g.get_state(want_psi=False)
    g.set_separable([("gauss", 0.0, 0.0, 1.0)] * 2, [0.0, 0.0], [0.0, 0.0])  # overwritten below
    g.upload_u(u, q0, p0, 0.0)
    g.propagate(10, 2.0, "yoshida4")
    o.propagate(10, 2.0, "yoshida4")
    out = torch.empty_like(u).pin_memory()
    q, p, t = g.download_u(out)
    psi_o, q_o, p_o, _ = o.get_state()
    cell = np.sqrt(0.32 * 0.2)
    assert rel(out.numpy().reshape(64, 48) / cell, psi_o) < TOL
    assert np.abs(q - q_o).max() < TOL * max(1.0, np.abs(q_o).max())
    assert np.abs(p - p_o).max() < TOL * max(1.0, np.abs(p_o).max())
    assert abs(t - 20.0) < 1e-12


# --------------------------------------------------------------------------
# a full (non-diagonal) inverse mass matrix, eq:KE_operator (general kernel)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["harmonic3d", "henon_heiles3d_fixed", "atom_diatom"])
def test_full_inverse_mass_matrix(mg, case):
    if case == "atom_diatom":
        P = inputs.ATOM_DIATOM
        N, dq = (64, 48), (0.32, 0.2)
        m = np.array([[1 / P["mu"][0], 0.2 / P["mu"][0]], [0.2 / P["mu"][0], 1 / P["mu"][1]]])
        kind, pot = oracle.POT_ATOM_DIATOM, [P["Dm"], P["a"], P["re"], P["A"], P["beta"]]
        rbar = oracle.morse_mean(P["Dm"], P["a"], P["re"], P["mu"][1])
        fac = [("gauss", P["R0"], P["P0"], P["sigma"]), ("morse", P["Dm"], P["a"], P["re"], P["mu"][1])]
        qc, pc, dt, steps, motion = [P["R0"], rbar], [P["P0"], 0.0], 2.0, 12, oracle.GRID_ADAPTIVE
    else:
        N, dq = (16, 18, 12), (0.5, 0.45, 0.6)
        m = np.array([[1.0, 0.25, -0.1], [0.25, 0.8, 0.15], [-0.1, 0.15, 1.2]])
        if case == "harmonic3d":
            kind, pot = oracle.POT_HARMONIC, [1.0, 0, 0, 0, 1.44, 0, 0, 0, 2.25, 0.1, -0.2, 0.0]
            motion = oracle.GRID_ADAPTIVE
        else:
            kind, pot = oracle.POT_HENON_HEILES, [inputs.HENON_HEILES["lam"]]
            motion = oracle.GRID_FIXED
        fac = [("gauss", 1.0, 0.3, 0.9), ("gauss", -0.5, -0.2, 0.8), ("gauss", 0.4, 0.1, 1.0)]
        qc, pc, dt, steps = [1.0, -0.5, 0.4], [0.3, -0.2, 0.1], 0.05, 20
    g, o = pair(mg, N, dq, m, kind, pot)
    assert g.path == 0  # the short-axis kernel takes diagonal matrices only
    g.set_separable(fac, qc, pc)
    o.set_separable(fac, qc, pc)
    g.propagate(steps, dt, "yoshida4", oracle.SPLIT_TVT, motion)
    o.propagate(steps, dt, "yoshida4", oracle.SPLIT_TVT, motion)
    assert_same(g, o)
    n, e, mq, mp = g.observables()
    no, eo, mqo, mpo = o.observables()
    assert abs(n - no) < 1e-13 and abs(e - eo) < 1e-12 * abs(eo)
    assert np.allclose(mp, mpo, rtol=1e-12, atol=1e-12)


def test_full_inverse_mass_matrix_is_refused_where_unsupported(mg):
    m = np.array([[1.0, 0.2, 0.0], [0.2, 1.0, 0.0], [0.0, 0.0, 1.0]])
    g = mg.Propagator((16, 16, 16), (0.5,) * 3, minv=m)
    g.set_potential(mg.MG_POT_HARMONIC, [1.0, 0, 0, 0, 1.0, 0, 0, 0, 1.0, 0, 0, 0])
    g.set_separable([("gauss", 0.0, 0.0, 1.0)] * 3, [0, 0, 0], [0, 0, 0])
    g.propagate(2, 0.05, "strang")
    with pytest.raises(mg.MgError) as e:
        g.adjoint(2, 0.05, "strang", np.zeros((16, 16, 16), complex), np.zeros(3), np.zeros(3))
    assert e.value.code == mg.MG_ERR_UNSUPPORTED
    with pytest.raises(mg.MgError) as e:
        mg.Batch([g])
    assert e.value.code == mg.MG_ERR_UNSUPPORTED
    with pytest.raises(mg.MgError) as e:  # not symmetric
        mg.Propagator((16, 16), (0.5, 0.5), minv=np.array([[1.0, 0.2], [0.1, 1.0]]))
    assert e.value.code == mg.MG_ERR_ARG
