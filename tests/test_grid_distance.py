"""Pins of the grid-to-grid distance used for the adaptive-vs-fixed comparisons
of Sec. III (tests/grid_distance.py) against closed forms."""
import numpy as np

from tests import grid_distance as gd


def gauss(x, q0, p0, sig):
    # eq:general_GWP, one axis
    return (np.pi * sig ** 2) ** -0.25 * np.exp(-(x - q0) ** 2 / (2 * sig ** 2) + 1j * p0 * (x - q0))


def test_carry_reproduces_a_band_limited_gaussian():
    # a Gaussian sampled on a coarse moving grid, carried onto a finer grid
    # with another centre, equals the Gaussian at the fine points inside the
    # coarse box, and zero outside it
    # (box +-9.6 and momentum window +-10.5 around the centres: the Gaussian
    # and its spectrum are below 1e-19 at their edges)
    src = {"N": [64], "dq": [0.3], "q": [0.3], "p": [0.5]}
    dst = {"N": [128], "dq": [0.21875], "q": [0.1], "p": [0.0]}
    xs = gd.axis_points(64, 0.3, 0.3)
    y = gd.axis_points(128, 0.21875, 0.1)
    out = gd.carry(gauss(xs, 0.4, 0.7, 1.0), src, dst)
    lo, hi = 0.3 - 32 * 0.3, 0.3 + 32 * 0.3
    assert 0 < np.sum(y < lo) and 0 < np.sum(y >= hi)
    inside = (y >= lo) & (y < hi)
    assert np.abs(out[inside] - gauss(y[inside], 0.4, 0.7, 1.0)).max() < 1e-12
    assert np.all(out[~inside] == 0)


def test_distance_of_two_gaussians_matches_the_closed_form():
    # ||a - b||^2 = 2 - 2 Re<a|b>; for unit-width Gaussians at distance d_l
    # with equal momenta p_l, <a|b> = prod_l exp(-d_l^2/4 - i p_l d_l)
    sparse = {"N": [64, 72], "dq": [0.3, 0.29], "q": [0.2, -0.3], "p": [0.0, 0.4]}
    dense = {"N": [120, 160], "dq": [0.25, 0.21], "q": [0.0, 0.0], "p": [0.0, 0.0]}
    x0, x1 = gd.axis_points(64, 0.3, 0.2), gd.axis_points(72, 0.29, -0.3)
    y0, y1 = gd.axis_points(120, 0.25, 0.0), gd.axis_points(160, 0.21, 0.0)
    d, pm = (0.3, -0.2), (0.0, 0.4)
    a = np.outer(gauss(x0, 0.0, pm[0], 1.0), gauss(x1, 0.0, pm[1], 1.0))
    b = np.outer(gauss(y0, d[0], pm[0], 1.0), gauss(y1, d[1], pm[1], 1.0))
    ov = np.prod([np.exp(-d[l] ** 2 / 4 - 1j * pm[l] * d[l]) for l in range(2)])
    exact = np.sqrt(2 - 2 * ov.real)
    assert abs(gd.distance(a, sparse, b, dense) - exact) < 1e-9
    # the same state on both grids: distance at roundoff
    b0 = np.outer(gauss(y0, 0.0, pm[0], 1.0), gauss(y1, 0.0, pm[1], 1.0))
    assert gd.distance(a, sparse, b0, dense) < 1e-12


def test_mean_q_of_a_gaussian():
    g = {"N": [64], "dq": [0.3], "q": [1.0], "p": [0.0]}
    x = gd.axis_points(64, 0.3, 1.0)
    assert abs(gd.mean_q(gauss(x, 1.7, 0.2, 1.0), g)[0] - 1.7) < 1e-12
