"""The composition coefficients the GPU library uses (host code behind
mg_scheme_coefficients, no GPU needed), checked against the conditions that
fix them (Sec. II.A, eq:comp_TVT with the triple-jump and Suzuki-fractal
constructions) and against the oracle's own construction."""
import numpy as np
import pytest

import oracle

# stage counts and largest |gamma| of the two constructions (closed forms of
# the recursive coefficients a = 1/(2 - 2^{1/(2k+1)}), 1/(4 - 4^{1/(2k+1)}))
CASES = [("strang", 2, 1, 1.0),
         ("yoshida4", 4, 3, 1.702), ("yoshida6", 6, 9, 2.297), ("yoshida8", 8, 27, 2.831),
         ("yoshida10", 10, 81, 3.324),
         ("suzuki4", 4, 5, 0.658), ("suzuki6", 6, 25, 0.324), ("suzuki8", 8, 125, 0.142),
         ("suzuki10", 10, 625, 0.0585)]


@pytest.fixture(scope="module")
def capi():
    import os

    from paper_1909_06412_gb300 import _build, capi as c

    if not os.path.exists(c.LIB_PATH):
        _build.build()
    return c


@pytest.mark.parametrize("name,order,stages,gmax", CASES)
def test_composition_conditions(capi, name, order, stages, gmax):
    g = capi.mg_scheme_coefficients(name)
    assert len(g) == stages
    assert abs(g.sum() - 1.0) < 1e-13                  # consistency
    assert np.array_equal(g, g[::-1])                  # symmetric (time-reversible)
    assert abs(np.abs(g).max() - gmax) < 1e-3
    # a symmetric composition of second-order steps has order p only if the
    # odd moments sum_k gamma_k^(2j+1) vanish for 2j+1 < p
    for m in range(3, order, 2):
        scale = np.sum(np.abs(g) ** m)
        assert abs(np.sum(g ** m)) < 1e-12 * scale, (m, np.sum(g ** m))
    if order < 10:  # and the next odd moment does not
        m = order + 1
        assert abs(np.sum(g ** m)) > 1e-6 * np.sum(np.abs(g) ** m)


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_same_coefficients_as_the_oracle(capi, name):
    g = capi.mg_scheme_coefficients(name)
    go = np.asarray(oracle.scheme(name))
    assert g.shape == go.shape and np.allclose(g, go, rtol=0, atol=4e-15)


def test_unknown_schemes(capi):
    for bad in ("yoshida3", "suzuki12", "rk4", ""):
        with pytest.raises(capi.MgError):
            capi.mg_scheme_coefficients(bad)
