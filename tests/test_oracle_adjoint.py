"""Pin of the oracle's taped gradient (oracle/adjoint.py) against central
finite differences of the oracle's own forward propagation."""
import numpy as np
import pytest

import oracle
from oracle.adjoint import Tape
from tests import inputs


def setup_atom_diatom(theta, q0, p0, N=(32, 24), dq=(0.32, 0.2)):
    P = inputs.ATOM_DIATOM
    g = oracle.Grid(N, dq, minv=(1 / P["mu"][0], 1 / P["mu"][1]))
    Dm, a, be, A = theta
    pot = [Dm, a, P["re"], A, be]
    g.set_potential(oracle.POT_ATOM_DIATOM, pot)
    rbar = oracle.morse_mean(P["Dm"], P["a"], P["re"], P["mu"][1])
    g.set_separable([("gauss", P["R0"], P["P0"], P["sigma"]), ("morse", P["Dm"], P["a"], P["re"], P["mu"][1])],
                    [P["R0"], rbar], [P["P0"], 0.0])
    u0 = g.get_u()
    return g, pot, u0


def objective(g, c, alpha, beta):
    psi, q, p, _ = g.get_state()
    u = g.get_u()
    return float(np.real(np.vdot(c, u)) + alpha @ q + beta @ p)


@pytest.mark.parametrize("split,motion", [(oracle.SPLIT_TVT, oracle.GRID_ADAPTIVE),
                                          (oracle.SPLIT_VTV, oracle.GRID_ADAPTIVE),
                                          (oracle.SPLIT_TVT, oracle.GRID_FIXED),
                                          (oracle.SPLIT_TVT, oracle.GRID_ADAPTIVE_CENTRE_P)])
def test_taped_gradient_matches_central_differences(split, motion):
    P = inputs.ATOM_DIATOM
    theta = np.array([P["Dm"], P["a"], P["beta"], P["A"]])
    rng = np.random.default_rng(3)
    g0, pot, u0 = setup_atom_diatom(theta, None, None)
    _, q0, p0, _ = g0.get_state()
    c = inputs.random_state(u0.shape, seed=4) * 0.3
    alpha, beta = rng.normal(size=2), rng.normal(size=2) * 0.1
    steps, dt, scheme = 3, 2.0, "yoshida4"

    def run(u, q, p, th):
        g, pot_, _ = setup_atom_diatom(th, q, p)
        g.set_state(g.get_state()[0], q, p)
        g.set_u(u)
        g.propagate(steps, dt, scheme, split, motion)
        return objective(g, c, alpha, beta)

    g, pot_, _ = setup_atom_diatom(theta, q0, p0)
    tape = Tape(g, oracle.POT_ATOM_DIATOM, pot_)
    tape.run(steps, dt, scheme, split, motion)
    ub, qb, pb, thb_full = tape.backward(c, alpha, beta)
    # the tape differentiates (Dm, a, beta, A) in the potential's own layout
    thb = thb_full

    h = 1e-5
    du = inputs.random_state(u0.shape, seed=9)
    fd_u = (run(u0 + h * du, q0, p0, theta) - run(u0 - h * du, q0, p0, theta)) / (2 * h)
    assert abs(fd_u - np.real(np.vdot(ub, du))) < 1e-6 * max(1.0, abs(fd_u))
    for l in range(2):
        e = np.zeros(2)
        e[l] = 1
        fq = (run(u0, q0 + h * e, p0, theta) - run(u0, q0 - h * e, p0, theta)) / (2 * h)
        fp = (run(u0, q0, p0 + h * e, theta) - run(u0, q0, p0 - h * e, theta)) / (2 * h)
        assert abs(fq - qb[l]) < 1e-6 * max(1.0, abs(fq)), (l, fq, qb[l])
        assert abs(fp - pb[l]) < 1e-6 * max(1.0, abs(fp)), (l, fp, pb[l])
    for k in range(4):
        hk = h * max(1.0, abs(theta[k]))
        e = np.zeros(4)
        e[k] = hk
        ft = (run(u0, q0, p0, theta + e) - run(u0, q0, p0, theta - e)) / (2 * hk)
        assert abs(ft - thb[k]) < 1e-6 * max(1.0, abs(ft)), (k, ft, thb[k])
