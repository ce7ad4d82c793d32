"""Batched launch (mg_batch_*): every problem of a batch against the oracle
and against the single-grid GPU path, cluster sizes, potentials changed
between launches, failure reporting, and the full 512-grid workload."""
import numpy as np
import pytest

import oracle
from tests import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1909_06412_gb300 as m

    m.lib()
    return m


def pot_params(pr):
    if pr["kind"] == "atom_diatom":
        return list(pr["pot"])
    k, c = pr["pot"]
    D = len(k)
    return list(np.diag(k).ravel()) + list(c)


def factors(pr, morse_mean):
    if pr["kind"] == "atom_diatom":
        Dm, a, re, A, be = pr["pot"]
        mr = pr["mass"][1]
        R0, P0, sg = pr["gauss"][0]
        fac = [("gauss", R0, P0, sg), ("morse", Dm, a, re, mr)]
        return fac, [R0, morse_mean(Dm, a, re, mr)], [P0, 0.0]
    fac = [("gauss", q, p, s) for q, p, s in pr["gauss"]]
    return fac, [f[1] for f in fac], [f[2] for f in fac]


def make_gpu(mg, pr, precision=None):
    precision = mg.MG_FP64 if precision is None else precision
    g = mg.Propagator(pr["N"], pr["dq"], minv=1.0 / np.array(pr["mass"]), precision=precision)
    kind = mg.MG_POT_ATOM_DIATOM if pr["kind"] == "atom_diatom" else mg.MG_POT_HARMONIC
    g.set_potential(kind, pot_params(pr))
    fac, q, p = factors(pr, mg.mg_morse_mean)
    g.set_separable(fac, q, p)
    return g


def make_oracle(pr):
    o = oracle.Grid(pr["N"], pr["dq"], minv=1.0 / np.array(pr["mass"]))
    kind = oracle.POT_ATOM_DIATOM if pr["kind"] == "atom_diatom" else oracle.POT_HARMONIC
    o.set_potential(kind, pot_params(pr))
    fac, q, p = factors(pr, oracle.morse_mean)
    o.set_separable(fac, q, p)
    return o


def small_problems():
    """Six small problems of both kinds and dimensions, with ragged tiles."""
    ad = inputs.ATOM_DIATOM
    return [
        dict(kind="atom_diatom", N=(48, 36), dq=(0.42, 0.28), mass=ad["mu"],
             pot=[0.17, 1.0, 1.4, 5.0, 1.8], gauss=[(8.0, -10.0, 0.5)], dt=2.0),
        dict(kind="atom_diatom", N=(24, 64), dq=(0.8, 0.16), mass=ad["mu"],
             pot=[0.19, 0.9, 1.5, 4.5, 1.7], gauss=[(7.5, -9.0, 0.6)], dt=1.0),
        dict(kind="harmonic", N=(32, 18), dq=(0.45, 0.6), mass=(1.0, 1.0),
             pot=[[1.1, 1.6], [0.0, 0.0]], gauss=[(1.0, 0.3, 0.9), (-0.5, 0.5, 0.8)], dt=0.05),
        dict(kind="harmonic", N=(12, 16, 18), dq=(0.8, 0.6, 0.55), mass=(1.0, 1.0, 1.0),
             pot=[[1.0, 1.44, 2.25], [0.0, 0.0, 0.0]], gauss=[(1.0, 0.0, 1.0), (-0.5, 0.5, 0.9), (0.8, -0.3, 0.8)],
             dt=0.03),
        dict(kind="harmonic", N=(16, 16, 24), dq=(0.6, 0.6, 0.4), mass=(1.0, 1.0, 1.0),
             pot=[[0.8, 1.2, 1.9], [0.1, -0.2, 0.0]], gauss=[(0.5, 0.2, 1.1), (0.0, -0.4, 0.9), (0.3, 0.1, 0.7)],
             dt=0.04),
        dict(kind="harmonic", N=(64, 24), dq=(0.3, 0.5), mass=(1.0, 1.0),
             pot=[[1.3, 0.9], [0.0, 0.0]], gauss=[(0.2, -0.6, 0.88), (1.1, 0.4, 1.05)], dt=0.02),
    ]


def state(g):
    psi, q, p, t = g.get_state()
    return psi, q, p, t


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("cluster", [1, 2, 4])
def test_batch_fp64_matches_oracle(mg, cluster):
    probs = small_problems()
    gs = [make_gpu(mg, pr) for pr in probs]
    b = mg.Batch(gs, cluster=cluster)
    steps = 5
    b.propagate(steps, [pr["dt"] for pr in probs], "yoshida4")
    b.sync()
    for pr, g in zip(probs, gs):
        o = make_oracle(pr)
        o.propagate(steps, pr["dt"], "yoshida4")
        psi, q, p, t = state(g)
        psi_o, q_o, p_o, t_o = o.get_state()
        assert rel(psi, psi_o) < 1e-12, pr["N"]
        assert np.allclose(q, q_o, rtol=1e-12, atol=1e-12) and np.allclose(p, p_o, rtol=1e-12, atol=1e-12)
        assert abs(t - steps * pr["dt"]) < 1e-12


@pytest.mark.parametrize("split,motion", [(1, 0), (2, 0), (0, 1), (0, 2)])
def test_batch_splits_and_grid_motion(mg, split, motion):
    probs = small_problems()[:4]
    gs = [make_gpu(mg, pr) for pr in probs]
    b = mg.Batch(gs, cluster=2)
    b.propagate(3, [pr["dt"] for pr in probs], "suzuki4", split, motion)
    b.sync()
    for pr, g in zip(probs, gs):
        o = make_oracle(pr)
        o.propagate(3, pr["dt"], "suzuki4", split, motion)
        psi, q, p, _ = state(g)
        psi_o, q_o, p_o, _ = o.get_state()
        assert rel(psi, psi_o) < 1e-12
        assert np.allclose(q, q_o, rtol=1e-12, atol=1e-12) and np.allclose(p, p_o, rtol=1e-12, atol=1e-12)


def test_batch_fp32_matches_oracle(mg):
    probs = small_problems()
    gs = [make_gpu(mg, pr, mg.MG_FP32_MIXED) for pr in probs]
    b = mg.Batch(gs, cluster=2)
    b.propagate(20, [pr["dt"] for pr in probs], "yoshida4")
    b.sync()
    for pr, g in zip(probs, gs):
        o = make_oracle(pr)
        o.propagate(20, pr["dt"], "yoshida4")
        psi, q, p, _ = state(g)
        psi_o, q_o, p_o, _ = o.get_state()
        assert rel(psi, psi_o) < 2e-5
        assert np.allclose(q, q_o, atol=2e-5) and np.allclose(p, p_o, atol=2e-4)


def test_batch_matches_single_grid_path_on_the_seeded_workload(mg):
    # 48 problems of the seeded 512-grid workload (every 11th), FP64, 4 steps:
    # the batch and mg_propagate on each context differ only in the order of
    # the reduction sums
    probs = inputs.batch_problems()[::11][:48]
    gb = [make_gpu(mg, pr) for pr in probs]
    b = mg.Batch(gb, cluster=2)
    b.propagate(4, [pr["dt"] for pr in probs], "suzuki4")
    b.sync()
    for pr, g in zip(probs, gb):
        s = make_gpu(mg, pr)
        s.propagate(4, pr["dt"], "suzuki4")
        psi, q, p, _ = state(g)
        psi_s, q_s, p_s, _ = state(s)
        assert rel(psi, psi_s) < 1e-12, pr["N"]
        assert np.allclose(q, q_s, rtol=1e-12, atol=1e-12) and np.allclose(p, p_s, rtol=1e-12, atol=1e-12)
        s.close()


@pytest.mark.parametrize("cluster", [1, 2])
def test_ensemble_of_the_256x256_atom_diatom_run(mg, cluster):
    # copies of the 256 x 256 FP64 atom-diatom run (Sec. III.B model, yoshida4,
    # dt = 1 a.u.) on one or two CTAs each: every member equals the
    # single-grid result up to the order of the reduction sums
    N, dq = (256, 256), (0.08, 0.04)
    amu = 1822.888486
    pot = [0.17, 1.0, 1.4, 5.0, 1.8]

    def member():
        g = mg.Propagator(N, dq, minv=(1 / (2.67 * amu), 1 / (0.5 * amu)))
        g.set_potential(mg.MG_POT_ATOM_DIATOM, pot)
        rbar = mg.mg_morse_mean(pot[0], pot[1], pot[2], 0.5 * amu)
        g.set_separable([("gauss", 8.0, -10.0, 0.5), ("morse", pot[0], pot[1], pot[2], 0.5 * amu)],
                        [8.0, rbar], [-10.0, 0.0])
        return g

    gs = [member() for _ in range(6)]
    b = mg.Batch(gs, cluster=cluster)
    b.propagate(3, 1.0, "yoshida4")
    b.sync()
    s = member()
    s.propagate(3, 1.0, "yoshida4")
    psi_s, q_s, p_s, _ = state(s)
    for g in gs:
        psi, q, p, _ = state(g)
        assert rel(psi, psi_s) < 1e-13
        assert np.allclose(q, q_s, rtol=0, atol=1e-13) and np.allclose(p, p_s, rtol=0, atol=1e-12)
    b.close()
    for g in gs + [s]:
        g.close()


def test_batch_then_single_grid_continues(mg):
    # after a batched launch the contexts carry on with mg_propagate (their
    # demodulation tables are rebuilt for the moved grid centre)
    probs = small_problems()[:3]
    gs = [make_gpu(mg, pr) for pr in probs]
    b = mg.Batch(gs, cluster=1)
    b.propagate(3, [pr["dt"] for pr in probs], "strang")
    b.sync()
    for pr, g in zip(probs, gs):
        g.propagate(2, pr["dt"], "strang")
        o = make_oracle(pr)
        o.propagate(5, pr["dt"], "strang")
        psi, q, p, t = state(g)
        psi_o, q_o, p_o, _ = o.get_state()
        assert rel(psi, psi_o) < 1e-12 and np.allclose(q, q_o, atol=1e-12)
        assert abs(t - 5 * pr["dt"]) < 1e-12


def test_batch_picks_up_potential_changes(mg):
    probs = small_problems()[2:4]
    gs = [make_gpu(mg, pr) for pr in probs]
    b = mg.Batch(gs, cluster=2)
    b.propagate(2, [pr["dt"] for pr in probs], "strang")
    b.sync()
    new = dict(probs[0])
    new["pot"] = [[2.0, 0.7], [0.3, -0.1]]
    gs[0].set_potential(mg.MG_POT_HARMONIC, pot_params(new))
    b.propagate(2, [pr["dt"] for pr in probs], "strang")
    b.sync()
    o = make_oracle(probs[0])
    o.propagate(2, probs[0]["dt"], "strang")
    o.set_potential(oracle.POT_HARMONIC, pot_params(new))
    o.propagate(2, probs[0]["dt"], "strang")
    psi, q, p, _ = state(gs[0])
    psi_o, q_o, p_o, _ = o.get_state()
    assert rel(psi, psi_o) < 1e-12 and np.allclose(p, p_o, rtol=1e-12, atol=1e-12)


def test_batch_reports_the_failed_problem(mg):
    # a harmonic problem with omega dt = 4 (beyond the Verlet stability limit
    # of the grid centre) among stable ones: its centre diverges and the batch
    # names it; the others finish normally
    probs = small_problems()[2:5]
    dts = [pr["dt"] for pr in probs]
    dts[1] = 4.0
    gs = [make_gpu(mg, pr) for pr in probs]
    b = mg.Batch(gs, cluster=2)
    b.propagate(40, dts, "strang")
    with pytest.raises(mg.MgError) as e:
        b.sync()
    assert e.value.code == mg.MG_ERR_UNSTABLE and "problem 1" in str(e.value)
    o = make_oracle(probs[0])
    o.propagate(40, dts[0], "strang")
    psi, _, _, _ = state(gs[0])
    assert rel(psi, o.get_state()[0]) < 1e-12
    with pytest.raises(mg.MgError):
        gs[1].get_state()


def test_full_seeded_workload_fp32(mg):
    # all 512 problems, FP32 storage with FP64 reductions, fourth-order
    # Suzuki: norm kept, and the sampled problems within the FP32 tolerance of
    # the FP64 single-grid path (itself pinned to the oracle at 1e-12)
    probs = inputs.batch_problems()
    gs = [make_gpu(mg, pr, mg.MG_FP32_MIXED) for pr in probs]
    n0 = np.array([g.observables()[0] for g in gs[::16]])
    b = mg.Batch(gs)
    b.propagate(20, [pr["dt"] for pr in probs], "suzuki4")
    b.sync()
    n1 = np.array([g.observables()[0] for g in gs[::16]])
    assert np.abs(n1 / n0 - 1).max() < 1e-5
    for i in range(0, 512, 64):
        s = make_gpu(mg, probs[i])
        s.propagate(20, probs[i]["dt"], "suzuki4")
        psi, q, p, _ = state(gs[i])
        psi_s, q_s, p_s, _ = state(s)
        assert rel(psi, psi_s) < 3e-5, (i, probs[i]["N"])
        assert np.allclose(q, q_s, atol=3e-5)
        s.close()
