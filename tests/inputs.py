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


# Batched workload: 512 independent grids drawn from one seed (numpy PCG64).
# 256 are 2D with axis lengths drawn per axis from {64, 72, 96, 128, 144, 192,
# 256} over the ranges of the atom-diatom grid (20.48 in R, 10.24 in r); half
# of them carry the atom-diatom potential, half an anisotropic harmonic one.
# 256 are 3D harmonic with lengths from {16, 18, 24, 32, 36, 48} over the 3D
# harmonic range (9.6 per axis).  Every potential parameter is the nominal
# value times U(0.8, 1.2); centres are the nominal ones plus U[-1, 1] per
# coordinate (for the atom-diatom problems on R only: the r factor stays the
# Morse ground state of that problem's potential, centred at its mean).
BATCH_SEED = 20190913
BATCH_2D_LENGTHS = (64, 72, 96, 128, 144, 192, 256)
BATCH_3D_LENGTHS = (16, 18, 24, 32, 36, 48)


def batch_problems(count=512, seed=BATCH_SEED):
    """List of problem dicts: kind ('harmonic' | 'atom_diatom'), N, dq, mass
    (per axis), pot (harmonic: diagonal force constants k_l and centre c_l;
    atom-diatom: Dm, a, re, A, beta), gauss (per Gaussian axis: q0, p0,
    sigma), dt."""
    g = rng(seed)
    out = []
    n2 = count // 2
    ad = ATOM_DIATOM
    for i in range(count):
        if i < n2:
            N = tuple(int(g.choice(BATCH_2D_LENGTHS)) for _ in range(2))
            dq = (20.48 / N[0], 10.24 / N[1])
            if g.uniform() < 0.5:
                f = g.uniform(0.8, 1.2, 5)
                pot = [ad["Dm"] * f[0], ad["a"] * f[1], ad["re"] * f[2], ad["A"] * f[3], ad["beta"] * f[4]]
                u = g.uniform(-1, 1, 2)
                out.append(dict(kind="atom_diatom", N=N, dq=dq, mass=ad["mu"], pot=pot,
                                gauss=[(ad["R0"] + u[0], ad["P0"] + u[1], ad["sigma"])], dt=1.0))
                continue
            om = np.array([1.0, 1.2]) * g.uniform(0.8, 1.2, 2)
            q0 = np.array([1.0, -0.5]) + g.uniform(-1, 1, 2)
            p0 = np.array([0.0, 0.5]) + g.uniform(-1, 1, 2)
            out.append(dict(kind="harmonic", N=N, dq=dq, mass=(1.0, 1.0), pot=[list(om ** 2), [0.0, 0.0]],
                            gauss=[(q0[l], p0[l], om[l] ** -0.5) for l in range(2)], dt=0.01))
        else:
            N = tuple(int(g.choice(BATCH_3D_LENGTHS)) for _ in range(3))
            dq = tuple(9.6 / n for n in N)
            om = np.array([1.0, 1.2, 1.5]) * g.uniform(0.8, 1.2, 3)
            q0 = np.array([1.0, -0.5, 0.8]) + g.uniform(-1, 1, 3)
            p0 = np.array([0.0, 0.5, -0.3]) + g.uniform(-1, 1, 3)
            out.append(dict(kind="harmonic", N=N, dq=dq, mass=(1.0, 1.0, 1.0), pot=[list(om ** 2), [0.0] * 3],
                            gauss=[(q0[l], p0[l], om[l] ** -0.5) for l in range(3)], dt=0.01))
    return out
