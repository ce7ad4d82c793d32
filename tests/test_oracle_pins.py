"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a textbook
or library routine, a closed form, an invariant the paper proves, a number
the paper prints, or brute force on a tiny grid.  No GPU is involved.
"""
import numpy as np
import pytest
from scipy.linalg import expm
from scipy.special import digamma

import oracle
from tests import golden, inputs
from tests.gaussians import Gauss1D, coherent_state, product_on_grid


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.asarray(b).ravel())


# --------------------------------------------------------------------------
# Discrete Fourier transform (Sec. II.B)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 4, 8, 16, 64, 256, 1024, 6, 12, 18, 24, 48, 96])
def test_dft_matches_numpy_and_direct_sum(n):
    x = inputs.random_state(n, seed=n)
    fwd = oracle.dft1d(x, -1)
    assert np.allclose(fwd, np.fft.fft(x) / np.sqrt(n), atol=1e-14, rtol=0)
    assert np.allclose(fwd, oracle.dft1d_direct(x, -1), atol=1e-13, rtol=0)
    inv = oracle.dft1d(fwd, +1)
    assert np.allclose(inv, x, atol=1e-14, rtol=0)
    assert abs(np.sum(abs(fwd) ** 2) - np.sum(abs(x) ** 2)) < 1e-14  # Parseval


# --------------------------------------------------------------------------
# Shifted transform f(q,p) (eq:F_defintion, eq:t_definition)
# --------------------------------------------------------------------------

def kernel_matrix(g, q, p):
    """N^{-1/2} e^{-i p^K . q^J / hbar}: eq:fourier_pos_to_mom with the
    C_q, C_p scalings folded in (C_q C_p = 1/N)."""
    qa = np.meshgrid(*g.qaxes(q), indexing="ij")
    pa = np.meshgrid(*[p[l] + (np.arange(g.N[l]) - g.N[l] / 2) * g.dp[l] for l in range(g.D)],
                     indexing="ij")
    X = np.stack([a.ravel() for a in qa], 1)
    P = np.stack([a.ravel() for a in pa], 1)
    return np.exp(-1j * (P @ X.T) / g.hbar) / np.sqrt(g.npts)


@pytest.mark.parametrize("N,hbar", [((16,), 1.0), ((8, 6), 0.7), ((4, 4, 4), 1.0), ((12,), 2.0)])
def test_shifted_transform_literal_fused_and_kernel(N, hbar):
    D = len(N)
    g = oracle.Grid(N, dq=np.linspace(0.3, 0.5, D), hbar=hbar)
    q, p = inputs.random_centre(D, seed=7)
    x = inputs.random_state(N, seed=3)
    fused = g.apply_f(q, p, x, -1)
    dense = g.apply_f(q, p, x, -1, dense=True)
    assert rel(fused, dense) < 1e-13
    F = kernel_matrix(g, q, p)
    assert rel(dense.ravel(), F @ x.ravel()) < 1e-12
    # f~ = f^dagger = f^{-1} (eq:F_inv_definition)
    back = g.apply_f(q, p, fused, +1)
    assert rel(back, x) < 1e-13
    assert rel(g.apply_f(q, p, x, +1, dense=True).ravel(), F.conj().T @ x.ravel()) < 1e-12


# --------------------------------------------------------------------------
# Substeps on a fixed grid vs brute-force matrix exponentials
# --------------------------------------------------------------------------

def hh_grid_2d():
    g = oracle.Grid((8, 8), dq=(0.8, 0.7), minv=(1.0, 0.8))
    g.set_potential(oracle.POT_HENON_HEILES, [0.2])
    return g


def hamiltonian_matrix(g, q, p):
    F = kernel_matrix(g, q, p)
    pa = np.meshgrid(*[p[l] + (np.arange(g.N[l]) - g.N[l] / 2) * g.dp[l] for l in range(g.D)],
                     indexing="ij")
    P = np.stack([a.ravel() for a in pa], 1)
    T = 0.5 * np.einsum("ka,ab,kb->k", P, g.minv, P)
    X = np.stack([a.ravel() for a in np.meshgrid(*g.qaxes(q), indexing="ij")], 1)
    V, _ = g.potential(X)
    return F.conj().T @ np.diag(T) @ F, np.diag(V)


def test_fixed_grid_kinetic_substep_is_matrix_exponential():
    g = hh_grid_2d()
    q, p = np.array([0.3, -0.2]), np.array([0.5, 0.1])
    u0 = inputs.random_state(g.N, seed=11)
    g.set_u(u0)
    g.set_state(g.get_state()[0], q, p)
    g.set_u(u0)
    Tm, Vm = hamiltonian_matrix(g, q, p)
    g.substep_T(0.37, oracle.GRID_FIXED)
    assert rel(g.get_u().ravel(), expm(-1j * 0.37 * Tm) @ u0.ravel()) < 1e-12
    g.substep_V(0.21, oracle.GRID_FIXED)
    ref = expm(-1j * 0.21 * Vm) @ expm(-1j * 0.37 * Tm) @ u0.ravel()
    assert rel(g.get_u().ravel(), ref) < 1e-12


# Symmetric compositions have even orders, so a wrong coefficient drops the
# measured slope by 2 or more; the step sizes keep every error between the
# asymptotic range and the roundoff floor.
@pytest.mark.parametrize("scheme,order,dts,tol", [
    ("strang", 2, [0.25, 0.125, 0.0625], 0.35), ("yoshida4", 4, [0.25, 0.125, 0.0625], 0.35),
    ("suzuki4", 4, [0.25, 0.125, 0.0625], 0.35), ("yoshida6", 6, [0.125, 0.0625, 0.03125], 0.35),
    ("suzuki6", 6, [0.25, 0.125, 0.0625], 0.5), ("yoshida8", 8, [0.125, 0.0625, 0.03125], 0.5),
    ("yoshida10", 10, [0.125, 0.0625, 0.03125], 0.5)])
def test_fixed_grid_composition_order_vs_expm(scheme, order, dts, tol):
    composition_order_vs_expm(scheme, order, dts, tol, oracle.SPLIT_TVT)


# VTV (T and V exchanged in every stage, eq:SO_TVT) has the same orders; a
# stage in the wrong order (e.g. V(h) T(h/2) ...) is not symmetric and drops
# to first order.  The first-order TV split of eq:SO_TV converges with slope 1.
@pytest.mark.parametrize("scheme,order,dts,tol,split", [
    ("strang", 2, [0.25, 0.125, 0.0625], 0.35, oracle.SPLIT_VTV),
    ("yoshida4", 4, [0.125, 0.0625, 0.03125], 0.35, oracle.SPLIT_VTV),
    ("yoshida6", 6, [0.125, 0.0625, 0.03125], 0.35, oracle.SPLIT_VTV),
    ("suzuki4", 4, [0.125, 0.0625, 0.03125], 0.35, oracle.SPLIT_VTV),
    ("strang", 1, [0.05, 0.025, 0.0125], 0.15, oracle.SPLIT_TV)])
def test_fixed_grid_vtv_and_tv_orders_vs_expm(scheme, order, dts, tol, split):
    composition_order_vs_expm(scheme, order, dts, tol, split)


def composition_order_vs_expm(scheme, order, dts, tol, split):
    g = hh_grid_2d()
    q, p = np.array([0.3, -0.2]), np.array([0.5, 0.1])
    u0 = inputs.random_state(g.N, seed=5)
    Tm, Vm = hamiltonian_matrix(g, q, p)
    t = 1.0
    exact = expm(-1j * t * (Tm + Vm)) @ u0.ravel()
    errs = []
    for dt in dts:
        g.set_u(u0)
        g.set_state(g.get_state()[0], q, p)
        g.set_u(u0)
        g.propagate(round(t / dt), dt, scheme, split, oracle.GRID_FIXED)
        errs.append(rel(g.get_u().ravel(), exact))
    slopes = np.diff(np.log(errs)) / np.diff(np.log(dts))
    assert np.all(np.abs(slopes - order) < tol), (errs, slopes)
    assert min(errs) > 1e-12, errs


def test_fixed_grid_suzuki_8_and_10_vs_expm():
    # Suzuki 8 and 10 reach the roundoff floor before their slopes show; at
    # dt = 0.25 each order gains at least two decades on the one below it
    g = hh_grid_2d()
    q, p = np.array([0.3, -0.2]), np.array([0.5, 0.1])
    u0 = inputs.random_state(g.N, seed=5)
    Tm, Vm = hamiltonian_matrix(g, q, p)
    exact = expm(-1j * (Tm + Vm)) @ u0.ravel()
    errs = {}
    for scheme in ("suzuki6", "suzuki8", "suzuki10"):
        g.set_u(u0)
        g.set_state(g.get_state()[0], q, p)
        g.set_u(u0)
        g.propagate(4, 0.25, scheme, oracle.SPLIT_TVT, oracle.GRID_FIXED)
        errs[scheme] = rel(g.get_u().ravel(), exact)
    assert errs["suzuki8"] < 1e-9 and errs["suzuki10"] < 1e-11, errs
    assert errs["suzuki8"] < 1e-2 * errs["suzuki6"] and errs["suzuki10"] < 1e-2 * errs["suzuki8"], errs


# --------------------------------------------------------------------------
# Moving grid vs closed-form Gaussian flows
# --------------------------------------------------------------------------

def run_split_gaussians(gs, ms, ks, cs, dt, steps, gammas):
    """Compose the exact 1D Gaussian flows in TVT order (eq:comp_TVT)."""
    for _ in range(steps):
        for gm in gammas:
            h = gm * dt
            for G, m in zip(gs, ms):
                G.kinetic(h / 2, m)
            for G, k, c in zip(gs, ks, cs):
                G.potential(h, k, c)
            for G, m in zip(gs, ms):
                G.kinetic(h / 2, m)


# Both readings of the kinetic substep's centre motion: the <p> reduction
# (eq:eom_qt_case_III_T) and the p-centre itself (eq:eom_qt_solution_case_III_T).
# For a Gaussian the two coincide: the p-centre and the packet's momentum
# receive the same kicks -tau k (x_c - c) in every potential substep and start
# equal, so either way the grid centre must follow the packet's centre
# (position Verlet, Sec. II.H).  A wrong branch (other momentum, sign, mass)
# moves the grid away from the packet and fails both checks.
@pytest.mark.parametrize("scheme", ["strang", "yoshida4"])
@pytest.mark.parametrize("motion", [oracle.GRID_ADAPTIVE, oracle.GRID_ADAPTIVE_CENTRE_P])
def test_moving_grid_matches_discrete_gaussian_closed_form(scheme, motion):
    # 1D, omega = 1, spacing 0.3, 64 points: the packet is < 1e-20 at the edges.
    N, dq, dt, steps = (64,), (0.3,), 0.01, 1000 if scheme == "strang" else 300
    q0, p0 = 1.0, 0.5
    g = oracle.Grid(N, dq)
    g.set_potential(oracle.POT_HARMONIC, [1.0, 0.0])
    g.set_separable([("gauss", q0, p0, 1.0)], [q0], [p0])
    g.propagate(steps, dt, scheme, oracle.SPLIT_TVT, motion)
    psi, q, p, t = g.get_state()
    G = Gauss1D(q0, p0, 1.0)
    run_split_gaussians([G], [1.0], [1.0], [0.0], dt, steps, oracle.scheme(scheme))
    exact = G(g.qaxes(q)[0])
    assert rel(psi, exact) < 1e-12
    # the grid centre equals the Gaussian's centre (position Verlet, Sec. II.H)
    assert abs(q[0] - G.xc) < 1e-12 and abs(p[0] - G.pi) < 1e-12
    assert abs(t - steps * dt) < 1e-9


@pytest.mark.parametrize("motion", [oracle.GRID_ADAPTIVE, oracle.GRID_ADAPTIVE_CENTRE_P])
def test_moving_grid_2d_mass_hbar_and_centre_closed_form(motion):
    hbar = 0.7
    minv = np.array([0.5, 2.0])
    k = np.array([1.3, 0.6])
    c = np.array([0.2, -0.1])
    q0, p0 = np.array([1.1, -0.4]), np.array([0.3, 0.6])
    omega = np.sqrt(k * minv)
    sig = np.sqrt(hbar / (omega / minv))  # sigma^2 = hbar/(m omega)
    N, dq = (64, 128), (0.25, 0.22)
    g = oracle.Grid(N, dq, minv=minv, hbar=hbar)
    g.set_potential(oracle.POT_HARMONIC, list(np.diag(k).ravel()) + list(c))
    g.set_separable([("gauss", q0[l], p0[l], sig[l]) for l in range(2)], q0, p0)
    dt, steps = 0.02, 200
    g.propagate(steps, dt, "yoshida4", oracle.SPLIT_TVT, motion)
    psi, q, p, _ = g.get_state()
    gs = [Gauss1D(q0[l], p0[l], sig[l], hbar) for l in range(2)]
    run_split_gaussians(gs, 1 / minv, k, c, dt, steps, oracle.scheme("yoshida4"))
    exact = product_on_grid(gs, g.qaxes(q))
    assert rel(psi, exact) < 1e-11
    assert np.allclose(q, [G.xc for G in gs], atol=1e-11, rtol=0)
    assert np.allclose(p, [G.pi for G in gs], atol=1e-11, rtol=0)


@pytest.mark.parametrize("scheme,order,dts", [("strang", 2, [0.1, 0.05, 0.025]),
                                              ("yoshida4", 4, [0.2, 0.1, 0.05]),
                                              ("suzuki4", 4, [0.4, 0.2, 0.1]),
                                              ("yoshida6", 6, [0.4, 0.2, 0.1])])
def test_moving_grid_convergence_order_vs_coherent_state(scheme, order, dts):
    N, dq, T, x0, p0 = (64,), (0.3,), 2.0, 1.0, 0.5
    errs = []
    for dt in dts:
        g = oracle.Grid(N, dq)
        g.set_potential(oracle.POT_HARMONIC, [1.0, 0.0])
        g.set_separable([("gauss", x0, p0, 1.0)], [x0], [p0])
        g.propagate(round(T / dt), dt, scheme)
        psi, q, _, _ = g.get_state()
        exact, _, _ = coherent_state(g.qaxes(q)[0], T, 1.0, x0, p0)
        errs.append(rel(psi, exact))
    slopes = np.diff(np.log(errs)) / np.diff(np.log(dts))
    assert np.all(np.abs(slopes - order) < 0.3), (errs, slopes)


# --------------------------------------------------------------------------
# Invariants the paper proves (Sec. II.G): norm, reversibility, separability
# --------------------------------------------------------------------------

def atom_diatom_small():
    P = inputs.ATOM_DIATOM
    g = oracle.Grid((64, 48), dq=(0.32, 0.2), minv=(1 / P["mu"][0], 1 / P["mu"][1]))
    g.set_potential(oracle.POT_ATOM_DIATOM, [P["Dm"], P["a"], P["re"], P["A"], P["beta"]])
    rbar = oracle.morse_mean(P["Dm"], P["a"], P["re"], P["mu"][1])
    g.set_separable([("gauss", P["R0"], P["P0"], P["sigma"]),
                     ("morse", P["Dm"], P["a"], P["re"], P["mu"][1])],
                    [P["R0"], rbar], [P["P0"], 0.0])
    return g


@pytest.mark.parametrize("split", [oracle.SPLIT_TVT, oracle.SPLIT_VTV])
def test_norm_and_time_reversibility(split):
    g = atom_diatom_small()
    u0 = g.get_u()
    _, q0, p0, _ = g.get_state()
    n0 = np.sum(abs(u0) ** 2)
    g.propagate(40, 2.0, "yoshida4", split)
    u1 = g.get_u()
    _, q1, p1, _ = g.get_state()
    assert abs(np.sum(abs(u1) ** 2) / n0 - 1) < 1e-12
    assert np.linalg.norm(q1 - q0) > 1e-2  # the grid actually moved
    g.propagate(40, -2.0, "yoshida4", split)
    u2 = g.get_u()
    _, q2, p2, _ = g.get_state()
    assert rel(u2, u0) < 1e-12
    assert np.allclose(q2, q0, atol=1e-12, rtol=0) and np.allclose(p2, p0, atol=1e-11, rtol=0)


def test_first_order_tv_is_not_reversible():
    g = atom_diatom_small()
    u0 = g.get_u()
    g.propagate(40, 2.0, "strang", oracle.SPLIT_TV)
    g.propagate(40, -2.0, "strang", oracle.SPLIT_TV)
    assert rel(g.get_u(), u0) > 1e-6


def test_separable_3d_equals_product_of_1d_runs():
    P = inputs.HARMONIC3D
    N = (16, 12, 20)
    dq = (0.45, 0.5, 0.4)
    om = np.array(P["omega"])
    g3 = oracle.Grid(N, dq)
    g3.set_potential(oracle.POT_HARMONIC, list(np.diag(om ** 2).ravel()) + [0, 0, 0])
    g3.set_separable([("gauss", P["q0"][l], P["p0"][l], om[l] ** -0.5) for l in range(3)],
                     P["q0"], P["p0"])
    g3.propagate(50, 0.05, "suzuki4")
    psi3, q3, p3, _ = g3.get_state()
    facs, qs, ps = [], [], []
    for l in range(3):
        g1 = oracle.Grid((N[l],), (dq[l],))
        g1.set_potential(oracle.POT_HARMONIC, [om[l] ** 2, 0.0])
        g1.set_separable([("gauss", P["q0"][l], P["p0"][l], om[l] ** -0.5)], [P["q0"][l]], [P["p0"][l]])
        g1.propagate(50, 0.05, "suzuki4")
        psi1, q1, p1, _ = g1.get_state()
        facs.append(psi1)
        qs.append(q1[0])
        ps.append(p1[0])
    prod = np.multiply.outer(np.multiply.outer(facs[0], facs[1]), facs[2])
    assert rel(psi3, prod) < 1e-12
    assert np.allclose(q3, qs, atol=1e-13, rtol=0) and np.allclose(p3, ps, atol=1e-13, rtol=0)


# --------------------------------------------------------------------------
# Numbers the paper prints
# --------------------------------------------------------------------------

def duschinsky(K13):
    P = inputs.DUSCHINSKY3D
    g = oracle.Grid(P["N"], P["dq"], minv=P["omega"])
    K = np.array(P["K"])
    K[0, 2] = K[2, 0] = K13
    g.set_potential(oracle.POT_HARMONIC, list(K.ravel()) + list(P["q0"]))
    g.set_separable([("gauss", 0.0, 0.0, 1.0)] * 3, [0, 0, 0], [0, 0, 0])
    return g


def test_initial_energy_of_the_harmonic_model():
    # Sec. III.A, Fig. 4 caption: E0 = 140.389 n.u.; holds with K13 = +0.017.
    E0 = golden.PAPER["harmonic_E0"]
    n, E, mq, mp = duschinsky(+0.017).observables()
    assert abs(n - 1) < 1e-9
    assert abs(E - E0) < 6e-4
    # Table I as printed (K13 = -0.017) misses the printed E0 by more than 1.
    assert abs(duschinsky(-0.017).observables()[1] - E0) > 1.0


def test_initial_energy_of_the_atom_diatom_state():
    # Sec. III.B model on the 256 x 256 grid: a Gaussian in R (eq:general_GWP)
    # times the Morse ground state in r.  Closed forms: <T_R> = (p0^2 +
    # 1/(2 sigma^2)) / (2 mu_R); the Morse ground state's <T_r + V_Morse> =
    # hbar w/2 - (hbar w)^2/(16 D), w = a sqrt(2 D / mu_r); the two exponential
    # terms factor into <e^{-beta R}> = e^{-beta R0 + beta^2 sigma^2/4} times
    # <e^{+-beta r/2}> by quadrature of the Morse density z^(2 lam - 1) e^-z.
    from scipy.integrate import quad

    P = inputs.ATOM_DIATOM
    Dm, a, re, A, be = (P[k] for k in ("Dm", "a", "re", "A", "beta"))
    muR, mur = P["mu"]
    R0, P0, sg = P["R0"], P["P0"], P["sigma"]
    lam = np.sqrt(2 * mur * Dm) / a
    w = a * np.sqrt(2 * Dm / mur)
    morse = w / 2 - w ** 2 / (16 * Dm)
    TR = (P0 ** 2 + 1 / (2 * sg ** 2)) / (2 * muR)

    def dens(r):
        z = 2 * lam * np.exp(-a * (r - re))
        return np.exp((2 * lam - 1) * np.log(z) - z)

    kw = dict(limit=400, epsabs=0, epsrel=1e-13)
    nrm = quad(dens, re - 2.5, re + 6, **kw)[0]
    ex = sum(quad(lambda r, s=s: dens(r) * np.exp(s * be * r / 2), re - 2.5, re + 6, **kw)[0] for s in (1, -1))
    E = TR + morse + A * np.exp(-be * R0 + be ** 2 * sg ** 2 / 4) * ex / nrm

    g = oracle.Grid(P["N"], P["dq"], minv=(1 / muR, 1 / mur))
    g.set_potential(oracle.POT_ATOM_DIATOM, [Dm, a, re, A, be])
    rbar = oracle.morse_mean(Dm, a, re, mur)
    g.set_separable([("gauss", R0, P0, sg), ("morse", Dm, a, re, mur)], [R0, rbar], [P0, 0.0])
    n, Eo, mq, mp = g.observables()
    assert abs(n - 1) < 1e-13
    assert abs(Eo - E) < 1e-12 * E
    assert np.allclose(mq, [R0, rbar], rtol=0, atol=1e-12) and np.allclose(mp, [P0, 0.0], rtol=0, atol=1e-12)


@pytest.mark.parametrize("q0,p0,sig,minv", [
    ((0.0, 24.0), (0.0, -3.56), (1.0, np.sqrt(8.0)), (1.0, 1.5)),
    ((0.4, 21.0), (0.7, -3.0), (0.8, 2.5), (0.7, 1.2))])
def test_initial_energy_of_the_secrest_johnson_state(q0, p0, sig, minv):
    # eq:modified_secrest_johnson, V = D (1 - e^{-beta q1})^2 + e^{-alpha (q2 - q1)},
    # with D = 20, beta = 0.158, alpha = 0.3 (Sec. III.B), under a product of
    # Gaussians of eq:general_GWP.  |psi|^2 is normal with mean q0_l and
    # variance sigma_l^2 / 2 per axis, so <e^{c q_l}> = e^{c q0_l + c^2 sigma_l^2 / 4}
    # and <V> = D (1 - 2 <e^{-beta q1}> + <e^{-2 beta q1}>) + <e^{-alpha q2}> <e^{alpha q1}>;
    # <T> = sum_l minv_l (p0_l^2 + hbar^2 / (2 sigma_l^2)) / 2.  A sign of alpha,
    # an exchange of q1 and q2 or a dropped factor changes E by far more than
    # the tolerance.
    Dm, be, al = 20.0, 0.158, 0.3
    q0, p0, sig, minv = (np.array(v, dtype=float) for v in (q0, p0, sig, minv))

    def mexp(c, l):
        return np.exp(c * q0[l] + c * c * sig[l] ** 2 / 4)

    V = Dm * (1 - 2 * mexp(-be, 0) + mexp(-2 * be, 0)) + mexp(-al, 1) * mexp(al, 0)
    T = np.sum(minv * (p0 ** 2 + 1 / (2 * sig ** 2))) / 2
    N, dq = (64, 64), (28.0 / 64, 48.0 / 64)
    g = oracle.Grid(N, dq, minv=minv)
    g.set_potential(oracle.POT_SECREST_JOHNSON, [Dm, be, al])
    g.set_separable([("gauss", q0[l], p0[l], sig[l]) for l in range(2)], q0, p0)
    n, E, mq, mp = g.observables()
    assert abs(n - 1) < 1e-13
    assert abs(E - (T + V)) < 1e-12 * (T + V), (E, T + V)
    assert np.allclose(mq, q0, rtol=0, atol=1e-12) and np.allclose(mp, p0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("D,N", [(2, 64), (3, 32)])
def test_initial_energy_of_the_henon_heiles_state(D, N):
    # Sec. III.C model: a unit-width Gaussian at q = 2 in every coordinate has
    # <q> = 2, var 1/2, <q^2> = 9/2, <q^3> = 11, <p^2> = 1/2 per coordinate, so
    # E = D/4 + 9D/4 + lambda (D-1) (<q^2><q> - <q^3>/3) = 5D/2 + lambda (D-1) 16/3
    lam = inputs.HENON_HEILES["lam"]
    dq = np.sqrt(2 * np.pi / N)
    g = oracle.Grid((N,) * D, (dq,) * D)
    g.set_potential(oracle.POT_HENON_HEILES, [lam])
    g.set_separable([("gauss", 2.0, 0.0, 1.0)] * D, [2.0] * D, [0.0] * D)
    n, E, mq, mp = g.observables()
    exact = 2.5 * D + lam * (D - 1) * 16.0 / 3.0
    assert abs(n - 1) < 1e-13 and abs(E - exact) < 1e-13 * exact, (E, exact)


def test_overlap_harmonic_displaced_ground_state():
    # Fig. 4 caption: phi0 = psi0 displaced by (-1, 1, 1) has <psi0|phi0> = 0.472.
    P = inputs.DUSCHINSKY3D
    g = oracle.Grid(P["N"], P["dq"])
    g.set_separable([("gauss", 0.0, 0.0, 1.0)] * 3, [0, 0, 0], [0, 0, 0])
    a = g.get_u()
    g.set_separable([("gauss", d, 0.0, 1.0) for d in (-1, 1, 1)], [0, 0, 0], [0, 0, 0])
    b = g.get_u()
    ov = np.vdot(a, b)
    assert abs(ov.real - golden.PAPER["harmonic_overlap"]) < 5e-4 and abs(ov.imag) < 1e-14


def test_overlap_scattering_packets():
    # Fig. 7 caption: p0 = -3.0 instead of -3.56 gives |<psi0|phi0>| = 0.534
    # (eq:general_GWP with sigma0^2 = 8, q0 = 24; grid of Fig. 5 caption).
    N, rng1, rng2 = (128, 128), (-14.0, 14.0), (0.0, 48.0)
    dq = ((rng1[1] - rng1[0]) / N[0], (rng2[1] - rng2[0]) / N[1])
    g = oracle.Grid(N, dq, minv=(1.0, 1.5))
    s0 = np.sqrt(8.0)
    g.set_separable([("gauss", 0.0, 0.0, 1.0), ("gauss", 24.0, -3.56, s0)], [0, 24], [0, -3.56])
    a = g.get_u()
    g.set_separable([("gauss", 0.0, 0.0, 1.0), ("gauss", 24.0, -3.0, s0)], [0, 24], [0, -3.56])
    b = g.get_u()
    assert abs(abs(np.vdot(a, b)) - golden.PAPER["scattering_overlap"]) < 5e-4


# --------------------------------------------------------------------------
# Composition coefficients, Morse ground state, regridding
# --------------------------------------------------------------------------

@pytest.mark.parametrize("name,stages,gmax", [
    ("strang", 1, 1.0), ("yoshida4", 3, 1.7024), ("yoshida6", 9, 2.2971),
    ("yoshida8", 27, 2.8309), ("yoshida10", 81, 3.3237), ("suzuki4", 5, 0.6580),
    ("suzuki6", 25, 0.3239), ("suzuki8", 125, 0.1420), ("suzuki10", 625, 0.05845)])
def test_composition_coefficients(name, stages, gmax):
    g = oracle.scheme(name)
    assert len(g) == stages
    assert abs(g.sum() - 1) < 1e-13
    assert np.array_equal(g, g[::-1])
    assert abs(np.abs(g).max() - gmax) < 1e-4
    order = 2 if name == "strang" else int(name[-2:] if name.endswith("10") else name[-1])
    # order conditions of symmetric compositions of a symmetric 2nd-order method
    for pw in range(3, order, 2):
        assert abs(np.sum(g ** pw)) < 1e-10


@pytest.mark.parametrize("kind,D,params", [
    (oracle.POT_HARMONIC, 3, list(np.array(inputs.DUSCHINSKY3D["K"]).ravel()) + [0.3, -0.2, 0.1]),
    (oracle.POT_ATOM_DIATOM, 2, [inputs.ATOM_DIATOM[k] for k in ("Dm", "a", "re", "A", "beta")]),
    (oracle.POT_HENON_HEILES, 8, [inputs.HENON_HEILES["lam"]]),
    (oracle.POT_SECREST_JOHNSON, 2, [0.17, 1.0, 1.8])])
def test_potential_gradient_matches_finite_differences(kind, D, params):
    # the Ehrenfest force <dV/dq> moves the p-centre (eq:eom_pt_solution_case_III_V);
    # the oracle's analytic gradient against central differences of its V
    g = oracle.Grid((4,) * D, (0.5,) * D)
    g.set_potential(kind, params)
    rng = np.random.default_rng(3)
    x = rng.uniform(-1.5, 1.5, size=(16, D))
    if kind == oracle.POT_ATOM_DIATOM:
        x += np.array([3.0, 1.4])  # R beyond the wall's steepest part, r near re
    V, grad = g.potential(x)
    h = 1e-5
    for a in range(D):
        e = np.zeros(D)
        e[a] = h
        fd = (g.potential(x + e)[0] - g.potential(x - e)[0]) / (2 * h)
        assert np.allclose(grad[:, a], fd, rtol=1e-7, atol=1e-8 * np.abs(V).max()), (a, grad[:, a], fd)


def test_morse_mean_closed_form():
    P = inputs.ATOM_DIATOM
    m = P["mu"][1]
    lam = np.sqrt(2 * m * P["Dm"]) / P["a"]
    # z = 2 lam e^{-a(r-re)} is Gamma(2 lam - 1)-distributed under |phi0|^2
    exact = P["re"] - (digamma(2 * lam - 1) - np.log(2 * lam)) / P["a"]
    assert abs(oracle.morse_mean(P["Dm"], P["a"], P["re"], m) - exact) < 1e-10


def test_regrid_resamples_a_band_limited_packet():
    g = oracle.Grid((64,), (0.3,))
    G = Gauss1D(0.4, 0.7, 1.0)
    qb, qa, p = np.array([0.0]), np.array([0.83]), np.array([0.7])
    ub = G(g.qaxes(qb)[0]) * np.sqrt(0.3)
    ua = G(g.qaxes(qa)[0]) * np.sqrt(0.3)
    assert rel(g.regrid(ub, qb, p, qa), ua) < 1e-12


# --------------------------------------------------------------------------
# A full (non-diagonal) inverse mass matrix (eq:KE_operator)
# --------------------------------------------------------------------------

MINV_FULL = np.array([[1.0, 0.3], [0.3, 0.8]])


def test_fixed_grid_kinetic_substep_with_full_mass_is_matrix_exponential():
    # T(p) = p^T m^-1 p / 2 with off-diagonal m^-1: the cross term makes the
    # kinetic operator non-separable; brute force as in the diagonal case
    g = oracle.Grid((8, 8), dq=(0.8, 0.7), minv=MINV_FULL)
    g.set_potential(oracle.POT_HENON_HEILES, [0.2])
    q, p = np.array([0.3, -0.2]), np.array([0.5, 0.1])
    u0 = inputs.random_state(g.N, seed=13)
    g.set_u(u0)
    g.set_state(g.get_state()[0], q, p)
    g.set_u(u0)
    Tm, Vm = hamiltonian_matrix(g, q, p)
    assert np.abs(Tm - Tm.conj().T).max() < 1e-12
    g.substep_T(0.37, oracle.GRID_FIXED)
    assert rel(g.get_u().ravel(), expm(-1j * 0.37 * Tm) @ u0.ravel()) < 1e-12


@pytest.mark.parametrize("motion", [oracle.GRID_ADAPTIVE, oracle.GRID_ADAPTIVE_CENTRE_P])
def test_moving_grid_centre_with_full_mass_is_position_verlet(motion):
    # H = p^T M p / 2 + (q - c)^T K (q - c) / 2 with M = m^-1 non-diagonal: a
    # Gaussian stays Gaussian and its centre moves exactly as the classical
    # point under the same splitting, i.e. position Verlet for Strang
    # (Sec. II.H): q += tau/2 M p; p -= tau K (q - c); q += tau/2 M p.  The grid
    # centre must follow it; a transposed or diagonal-only M, or a wrong
    # factor, fails at the first step.
    K = np.array([[1.2, 0.0], [0.0, 0.7]])
    c = np.array([0.2, -0.1])
    q0, p0 = np.array([1.0, -0.6]), np.array([0.4, 0.3])
    g = oracle.Grid((64, 64), (0.3, 0.3), minv=MINV_FULL)
    g.set_potential(oracle.POT_HARMONIC, list(K.ravel()) + list(c))
    g.set_separable([("gauss", q0[0], p0[0], 1.0), ("gauss", q0[1], p0[1], 1.0)], q0, p0)
    dt, steps = 0.02, 200
    g.propagate(steps, dt, "strang", oracle.SPLIT_TVT, motion)
    _, q, p, _ = g.get_state()
    qc, pc = q0.copy(), p0.copy()
    for _ in range(steps):
        qc = qc + 0.5 * dt * MINV_FULL @ pc
        pc = pc - dt * K @ (qc - c)
        qc = qc + 0.5 * dt * MINV_FULL @ pc
    assert np.abs(q - qc).max() < 1e-11 and np.abs(p - pc).max() < 1e-11, (q - qc, p - pc)
