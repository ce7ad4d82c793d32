"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

This module holds no arithmetic of the method: only random numbers and the
workload parameters (grids, potentials, initial wavepackets) written down as
data: the physical constants and the grid spacings that the paper leaves open
(1 amu taken as 1822.888486 electron masses).
"""
import numpy as np

AMU = 1822.888486  # electron masses per atomic mass unit


def rng(seed):
    return np.random.default_rng(seed)


def random_state(shape, seed):
    """Random complex array with unit sum of squares (not a physical state)."""
    g = rng(seed)
    u = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    return u / np.sqrt(np.sum(np.abs(u) ** 2))


def random_centre(D, seed, scale=3.0):
    g = rng(seed)
    return scale * g.uniform(-1, 1, D), scale * g.uniform(-1, 1, D)


# 3D anisotropic harmonic oscillator: 32^3 grid, spacing 0.3, coherent state.
HARMONIC3D = dict(
    N=(32, 32, 32), dq=(0.3, 0.3, 0.3), omega=(1.0, 1.2, 1.5), mass=(1.0, 1.0, 1.0),
    q0=(1.0, -0.5, 0.8), p0=(0.0, 0.5, -0.3), dt=0.01, steps=1000, scheme="strang",
)

# Collinear atom-diatom model, axes (R, r), 256 x 256, spacings 0.08 / 0.04.
ATOM_DIATOM = dict(
    N=(256, 256), dq=(0.08, 0.04), Dm=0.17, a=1.0, re=1.4, A=5.0, beta=1.8,
    mu=(2.67 * AMU, 0.5 * AMU), R0=8.0, P0=-10.0, sigma=0.5,
)

# 8D Henon-Heiles: lambda = 0.111803, unit masses, q0 = 2 in every coordinate.
HENON_HEILES = dict(lam=0.111803, q0=2.0)

# Sec. III.A two-surface model (Table I, with the K_13 sign reading).
DUSCHINSKY3D = dict(
    omega=(2.0, 1.0, 2.5),
    K=((1.997, -0.04, 0.017), (-0.04, 1.015, 0.04), (0.017, 0.04, 2.48)),
    q0=(-7.0, 7.0, 7.0), N=(32, 32, 32), dq=(0.4375, 0.4375, 0.4375),
)
