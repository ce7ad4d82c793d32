"""Convergence order of every composition on the atom-diatom moving grid.

The paper measures the accuracy of a run by its distance to the run with
half the time step (Sec. III); on a moving grid the two runs end on grids
with different centres, so one state is first carried onto the other's grid
by the trigonometric interpolation of eq:F_defintion.  For a composition of
order k the distances of successive halvings fall by 2^k.  This pins the
oracle's compositions (triple jump and Suzuki, Sec. II.A) and its grid
motion together on a non-harmonic two-dimensional problem, where no closed
form exists."""
import numpy as np
import pytest

import oracle
from tests import inputs

P = inputs.ATOM_DIATOM


def run(scheme, dt, t_end=16.0):
    # the 128 x 128 grid of the gradient workload (dR = 0.16, dr = 0.08): the
    # packet is band-limited in both windows, so the interpolation is exact
    g = oracle.Grid((128, 128), dq=(0.16, 0.08), minv=(1 / P["mu"][0], 1 / P["mu"][1]))
    g.set_potential(oracle.POT_ATOM_DIATOM, [P["Dm"], P["a"], P["re"], P["A"], P["beta"]])
    rbar = oracle.morse_mean(P["Dm"], P["a"], P["re"], P["mu"][1])
    g.set_separable([("gauss", P["R0"], P["P0"], P["sigma"]),
                     ("morse", P["Dm"], P["a"], P["re"], P["mu"][1])],
                    [P["R0"], rbar], [P["P0"], 0.0])
    g.propagate(int(round(t_end / dt)), dt, scheme)
    return g


def distance(a, b):
    """||u_a - u_b|| / ||u_b|| with u_a carried onto b's grid."""
    _, qa, _, _ = a.get_state()
    _, qb, pb, _ = b.get_state()
    ua_on_b = a.regrid(a.get_u(), qa, pb, qb)
    ub = b.get_u()
    return np.linalg.norm(ua_on_b - ub) / np.linalg.norm(ub)


@pytest.mark.parametrize("scheme,order,dts", [("strang", 2, [4.0, 2.0, 1.0, 0.5]),
                                              ("yoshida4", 4, [4.0, 2.0, 1.0, 0.5]),
                                              ("suzuki4", 4, [4.0, 2.0, 1.0]),
                                              ("yoshida6", 6, [4.0, 2.0, 1.0])])
def test_self_convergence_order_on_the_atom_diatom_grid(scheme, order, dts):
    runs = [run(scheme, dt) for dt in dts]
    errs = [distance(runs[k], runs[k + 1]) for k in range(len(runs) - 1)]
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - order) < 0.2), (errs, orders)
    # well above the roundoff floor, so the orders measure the compositions
    assert min(errs) > 1e-12, errs
