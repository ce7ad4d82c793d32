"""Failure detection on the GPU without a GPU fault: a grid-wide barrier that
cannot complete (mg_test_stuck_barrier presets the barrier word so that no
arrival is ever the last one) must end in MG_ERR_TIMEOUT after the short time
limit the hook sets, with every CTA returning, and the context must propagate
normally afterwards (checked against the FP64 oracle)."""
import time

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


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.asarray(b).ravel())


def make(mg, case):
    if case == "general":  # atom-diatom: the general kernel
        P = inputs.ATOM_DIATOM
        N, dq = (64, 48), (0.32, 0.2)
        minv = (1 / P["mu"][0], 1 / P["mu"][1])
        kind, pot = oracle.POT_ATOM_DIATOM, [P["Dm"], P["a"], P["re"], P["A"], P["beta"]]
        rbar = oracle.morse_mean(P["Dm"], P["a"], P["re"], P["mu"][1])
        fac = [("gauss", P["R0"], P["P0"], P["sigma"]), ("morse", P["Dm"], P["a"], P["re"], P["mu"][1])]
        qc, pc, dt, path = [P["R0"], rbar], [P["P0"], 0.0], 2.0, 0
    else:  # Henon-Heiles on 12^3: the short-axis kernel
        n, D = 12, 3
        N, dq, minv = (n,) * D, (np.sqrt(2 * np.pi / n),) * D, (1.0,) * D
        kind, pot = oracle.POT_HENON_HEILES, [inputs.HENON_HEILES["lam"]]
        fac = [("gauss", 2.0, 0.0, 1.0)] * D
        qc, pc, dt, path = [2.0] * D, [0.0] * D, 0.02, 1
    g = mg.Propagator(N, dq, minv=minv)
    g.set_potential(kind, pot)
    g.set_separable(fac, qc, pc)
    o = oracle.Grid(N, dq, minv=minv)
    o.set_potential(kind, pot)
    o.set_separable(fac, qc, pc)
    assert g.path == path
    return g, o, (fac, qc, pc), dt


@pytest.mark.parametrize("case", ["general", "short"])
def test_stuck_barrier_times_out_and_the_context_recovers(mg, case):
    g, o, (fac, qc, pc), dt = make(mg, case)
    g.test_stuck_barrier(2e-3)
    t0 = time.perf_counter()
    g.propagate(3, dt, "yoshida4")
    with pytest.raises(mg.MgError) as e:
        g.sync()
    elapsed = time.perf_counter() - t0
    assert e.value.code == mg.MG_ERR_TIMEOUT
    assert elapsed < 2.0, elapsed  # the 2 ms limit, not the default 5 s
    # the status was reported once; the context works again from a new state
    g.sync()
    g.set_separable(fac, qc, pc)
    g.propagate(3, dt, "yoshida4")
    o.propagate(3, dt, "yoshida4")
    psi, q, p, _ = g.get_state()
    psi_o, q_o, p_o, _ = o.get_state()
    assert rel(psi, psi_o) < 1e-12
    assert np.abs(q - q_o).max() < 1e-12 * max(1.0, np.abs(q_o).max())
    assert np.abs(p - p_o).max() < 1e-12 * max(1.0, np.abs(p_o).max())


def test_stuck_barrier_rejects_bad_limits(mg):
    g, _, _, _ = make(mg, "general")
    for bad in (0.0, -1.0, 6.0, float("nan")):
        with pytest.raises(mg.MgError) as e:
            g.test_stuck_barrier(bad)
        assert e.value.code == mg.MG_ERR_ARG
