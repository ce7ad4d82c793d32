"""Pins of the oracle's inner product of states on different moving grids
(eq:scalar_prod with the trigonometric interpolation of eq:F_defintion)."""
import numpy as np

import oracle
from tests import golden, inputs

P = inputs.DUSCHINSKY3D


def e1_state(q0):
    # Sec. III.A model: masses 1/omega, ground-state width of the first surface
    om = np.array(P["omega"])
    g = oracle.Grid(P["N"], P["dq"], minv=om)
    g.set_potential(oracle.POT_HARMONIC, list(np.array(P["K"]).ravel()) + [0.0] * 3)
    g.set_separable([("gauss", q0[l], 0.0, 1.0) for l in range(3)], q0, [0.0] * 3)
    return g


def test_initial_overlap_of_the_two_states_on_their_own_grids():
    # the paper's printed <psi_0|phi_0> = 0.472 (Sec. III.A): two unit-width
    # Gaussians displaced by (-1, 1, 1), exp(-|d|^2/4) = exp(-0.75); each on
    # a grid centred at its own position
    q0 = np.array(P["q0"])
    a, b = e1_state(q0), e1_state(q0 + np.array([-1.0, 1.0, 1.0]))
    v = oracle.inner_product(a, b)
    assert abs(v - np.exp(-0.75)) < 1e-9
    assert round(abs(v), 3) == golden.PAPER["harmonic_overlap"]
    assert abs(oracle.inner_product(b, a) - np.conj(v)) < 1e-13


def test_inner_product_with_itself_is_the_norm():
    a = e1_state(np.array(P["q0"]))
    assert abs(oracle.inner_product(a, a) - np.sum(np.abs(a.get_u()) ** 2)) < 1e-14


def test_moving_grid_keeps_the_overlap_of_two_gaussians_in_a_harmonic_well():
    # both packets stay Gaussian on grids that follow them: the overlap is
    # conserved to the grid truncation, while a fixed grid of the same size
    # loses the packets
    q0 = np.array(P["q0"])
    res = {}
    for motion in (oracle.GRID_ADAPTIVE, oracle.GRID_FIXED):
        a, b = e1_state(q0), e1_state(q0 + np.array([-1.0, 1.0, 1.0]))
        v0 = oracle.inner_product(a, b)
        for g in (a, b):
            g.propagate(20, 0.1, "yoshida4", oracle.SPLIT_TVT, motion)
        res[motion] = abs(oracle.inner_product(a, b) - v0)
    assert res[oracle.GRID_ADAPTIVE] < 1e-10
    assert res[oracle.GRID_FIXED] > 1e-2
