"""Pins of the oracle's naive adaptive grid (Sec. II.F) and of the regridding
f~(q', p') f(q, p') it uses: the naive grid keeps the norm but is not time
reversible (eq:naive_t_rev_fail), while the Ehrenfest-driven grid of Sec.
II.G is; the regrid is the exact trigonometric interpolation of a
band-limited state."""
import numpy as np
import pytest

import oracle
from tests import inputs

P = inputs.ATOM_DIATOM


def atom_diatom(N=(48, 36), dq=(0.4, 0.25)):
    o = oracle.Grid(N, dq, minv=(1 / P["mu"][0], 1 / P["mu"][1]))
    o.set_potential(oracle.POT_ATOM_DIATOM, [P["Dm"], P["a"], P["re"], P["A"], P["beta"]])
    rbar = oracle.morse_mean(P["Dm"], P["a"], P["re"], P["mu"][1])
    o.set_separable([("gauss", 6.0, -10.0, 0.6), ("morse", P["Dm"], P["a"], P["re"], P["mu"][1])],
                    [6.0, rbar], [-10.0, 0.0])
    return o


def forward_back(motion, steps=20, dt=5.0):
    o = atom_diatom()
    u0 = o.get_u()
    _, q0, p0, _ = o.get_state()
    o.propagate(steps, dt, "yoshida4", oracle.SPLIT_TVT, motion)
    n1 = np.sum(np.abs(o.get_u()) ** 2)
    o.propagate(steps, -dt, "yoshida4", oracle.SPLIT_TVT, motion)
    _, q2, p2, _ = o.get_state()
    err = np.linalg.norm(o.get_u() - u0) / np.linalg.norm(u0)
    return n1 / np.sum(np.abs(u0) ** 2) - 1, err, np.abs(q2 - q0).max(), np.abs(p2 - p0).max()


def test_naive_grid_keeps_the_norm_but_not_reversibility():
    drift_n, err_n, dq_n, dp_n = forward_back(oracle.GRID_NAIVE)
    drift_e, err_e, dq_e, dp_e = forward_back(oracle.GRID_ADAPTIVE)
    # both norm-preserving (Sec. II.F: U_naive is a product of unitary maps)
    assert abs(drift_n) < 1e-12 and abs(drift_e) < 1e-12
    # the Ehrenfest grid returns to psi0, the naive one does not
    assert err_e < 1e-12 and dq_e < 1e-12 and dp_e < 1e-12
    assert err_n > 1e-6 and max(dq_n, dp_n) > 1e-7
    assert err_n > 1e6 * err_e


def test_naive_step_moves_the_grid_to_the_moments_of_the_propagated_state():
    # Sec. II.F: q1 = <q>, p1 = <p> of U(dt; q0, p0) psi0 on the old grid
    a = atom_diatom()
    a.propagate(1, 5.0, "yoshida4", oracle.SPLIT_TVT, oracle.GRID_FIXED)
    _, _, mq, mp = a.observables()
    b = atom_diatom()
    b.propagate(1, 5.0, "yoshida4", oracle.SPLIT_TVT, oracle.GRID_NAIVE)
    _, q, p, _ = b.get_state()
    assert np.array_equal(q, mq) and np.array_equal(p, mp)
    # the state it carries has those moments up to the grid truncation
    _, _, mq2, mp2 = b.observables()
    assert np.abs(mq2 - q).max() < 1e-5 and np.abs(mp2 - p).max() < 1e-5


def test_regrid_is_exact_for_a_mode_of_the_momentum_grid():
    # u = e^{i P x} sampled on the grid at q is band-limited when P lies on
    # the momentum grid at p; its interpolant on any shifted grid q' is the
    # same plane wave sampled there (up to the common constant).
    N, dq = (16, 12), (0.5, 0.7)
    o = oracle.Grid(N, dq)
    q, p = np.array([0.3, -1.1]), np.array([0.7, 0.2])
    kk = (3, -2)
    P_ = np.array([p[l] + kk[l] * o.dp[l] for l in range(2)])
    def mode(qc):
        X = np.meshgrid(*o.qaxes(qc), indexing="ij")
        return np.exp(1j * (P_[0] * X[0] + P_[1] * X[1]))
    u = mode(q)
    q1 = q + np.array([0.237, -0.61])
    u1 = o.apply_f(q1, p, o.apply_f(q, p, u, -1), +1)
    assert np.abs(u1 - mode(q1)).max() < 1e-12 * np.abs(u).max() * 10


def test_regrid_round_trip_is_identity():
    N, dq = (24, 18), (0.45, 0.6)
    o = oracle.Grid(N, dq)
    u = inputs.random_state(N, 7)
    q, p = np.array([0.2, -0.3]), np.array([1.0, 0.5])
    q1, p1 = q + np.array([0.31, 0.77]), p + np.array([-0.4, 0.9])
    v = o.apply_f(q1, p1, o.apply_f(q, p1, u, -1), +1)
    w = o.apply_f(q, p1, o.apply_f(q1, p1, v, -1), +1)
    assert np.linalg.norm(w - u) < 1e-13
    assert abs(np.linalg.norm(v) - 1) < 1e-14
