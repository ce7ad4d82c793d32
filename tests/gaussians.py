"""Closed-form Gaussian wavepacket flows used to pin the oracle.

A 1D Gaussian psi(x) = exp{(i/hbar)[A/2 (x-xc)^2 + pi (x-xc) + g]} stays Gaussian
under the exact kinetic flow of T = p^2/2m and under the exact flow of a
quadratic potential V = k/2 (x-c)^2.  Composing these exact flows in the order
of a splitting scheme gives the state the split-operator integrator must
produce on a grid wide enough to hold the packet (Sec. II.A, eq:SO_TVT and
eq:comp_TVT).  The continuum coherent state of the harmonic oscillator gives
the exact, unsplit evolution (for convergence-order checks).

These formulas follow from inserting the Gaussian into the time-dependent
Schroedinger equation (eq:tdse); they share nothing with the oracle code.
"""
import numpy as np


class Gauss1D:
    def __init__(self, q0, p0, sigma, hbar=1.0):
        self.hbar = hbar
        self.A = 1j * hbar / sigma ** 2
        self.xc = float(q0)
        self.pi = float(p0)
        self.g = 0.25j * hbar * np.log(np.pi * sigma ** 2)

    def kinetic(self, tau, m):
        s = 1 + tau * self.A / m
        self.g = self.g + tau * self.pi ** 2 / (2 * m) + 0.5j * self.hbar * np.log(s)
        self.xc = self.xc + tau * self.pi / m
        self.A = self.A / s

    def potential(self, tau, k, c=0.0):
        d = self.xc - c
        self.g = self.g - tau * k * d * d / 2
        self.pi = self.pi - tau * k * d
        self.A = self.A - tau * k

    def __call__(self, x):
        y = x - self.xc
        return np.exp(1j / self.hbar * (0.5 * self.A * y * y + self.pi * y + self.g))


def coherent_state(x, t, omega, x0, p0, hbar=1.0, m=1.0):
    """Exact harmonic-oscillator coherent state (width sigma^2 = hbar/(m omega))."""
    xt = x0 * np.cos(omega * t) + p0 / (m * omega) * np.sin(omega * t)
    pt = p0 * np.cos(omega * t) - m * omega * x0 * np.sin(omega * t)
    y = x - xt
    phase = pt * y / hbar + (pt * xt - p0 * x0) / (2 * hbar) - omega * t / 2
    return (m * omega / (np.pi * hbar)) ** 0.25 * np.exp(-m * omega * y * y / (2 * hbar) + 1j * phase), xt, pt


def product_on_grid(factors, axes):
    """Outer product of per-axis sample vectors."""
    out = np.array(1.0 + 0j)
    for f, x in zip(factors, axes):
        out = np.multiply.outer(out, f(x))
    return out
