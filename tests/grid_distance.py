"""Distance between wavefunctions held on different tensor-product grids.

The comparison of Sec. III (Figs. 3 and 8, Appendix B): a state on a sparser
grid is carried onto the points of a denser grid by trigonometric
interpolation, and the two are compared there with the denser grid's
quadrature.  Used by the GPU accuracy tests and the benchmark to report the
distance between the adaptive-grid result and the fixed-grid reference; it is
analysis of results, not a step of the propagation.

A grid is a dict with "N", "dq", "q" (position centre) and "p" (momentum
centre), per axis; points x_j = q + (j - N/2) dq and momenta
p_k = p + (k - N/2) dp, dp = 2 pi hbar / (N dq).
"""
import numpy as np


def axis_points(N, dq, q):
    return q + (np.arange(N) - N // 2) * dq


def interp_matrix(N, dq, q, p, y, hbar=1.0):
    """Rows: the band-limited interpolant of samples at the N points of one
    source axis (momentum window centred at p), evaluated at the points y.
    psi(y) = sum_k c_k e^{i p_k (y - q)/hbar}, c_k = N^-1 sum_j psi_j
    e^{-i p_k (x_j - q)/hbar}, so row a is N^-1 sum_k e^{i p_k (y_a - x_j)/hbar}.
    Rows of points outside the source box [q - N dq/2, q + N dq/2) are zero:
    the state is zero outside its grid."""
    x = axis_points(N, dq, q)
    dp = 2 * np.pi * hbar / (N * dq)
    pk = p + (np.arange(N) - N // 2) * dp
    y = np.asarray(y, dtype=float)
    M = (np.exp(1j * np.outer(y - q, pk) / hbar) @ np.exp(-1j * np.outer(pk, x - q) / hbar)) / N
    lo, hi = q - (N // 2) * dq, q + (N - N // 2) * dq
    M[(y < lo - 1e-12 * dq) | (y >= hi - 1e-12 * dq)] = 0.0
    return M


def carry(psi_src, src, dst, hbar=1.0):
    """The state psi_src (physical values on grid src) at the points of grid
    dst, by per-axis trigonometric interpolation."""
    out = np.asarray(psi_src, dtype=np.complex128)
    for l in range(out.ndim):
        y = axis_points(dst["N"][l], dst["dq"][l], dst["q"][l])
        M = interp_matrix(src["N"][l], src["dq"][l], src["q"][l], src["p"][l], y, hbar)
        out = np.moveaxis(np.tensordot(M, out, axes=([1], [l])), 0, l)
    return out


def distance(psi_sparse, sparse, psi_dense, dense, hbar=1.0):
    """||psi_sparse - psi_dense|| with psi_sparse carried onto the dense grid
    (zero outside its own box), by the dense grid's quadrature."""
    d = carry(psi_sparse, sparse, dense, hbar) - np.asarray(psi_dense)
    return float(np.sqrt(np.sum(np.abs(d) ** 2) * np.prod(dense["dq"])))


def mean_q(psi, grid):
    """<q_l> of a physical state on its grid (normalised by its norm)."""
    w = np.abs(psi) ** 2
    n = w.sum()
    out = []
    for l in range(psi.ndim):
        x = axis_points(grid["N"][l], grid["dq"][l], grid["q"][l])
        sh = [1] * psi.ndim
        sh[l] = -1
        out.append(float((w * x.reshape(sh)).sum() / n))
    return np.array(out)
