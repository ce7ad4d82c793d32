"""The reversible adjoint (mg_adjoint, MovingGridPropagate) against the
oracle's taped FP64 gradient and against central finite differences."""
import numpy as np
import pytest

import oracle
from oracle.adjoint import Tape
from tests import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = inputs.ATOM_DIATOM


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1909_06412_gb300 as m

    m.lib()
    return m


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def atom_diatom_pair(mg, N, dq, R0=None, P0=None, sigma=None, theta=None):
    R0 = P["R0"] if R0 is None else R0
    P0 = P["P0"] if P0 is None else P0
    sigma = P["sigma"] if sigma is None else sigma
    Dm, a, be, A = (P["Dm"], P["a"], P["beta"], P["A"]) if theta is None else theta
    minv = (1 / P["mu"][0], 1 / P["mu"][1])
    pot = [Dm, a, P["re"], A, be]
    rbar = oracle.morse_mean(P["Dm"], P["a"], P["re"], P["mu"][1])
    fac = [("gauss", R0, P0, sigma), ("morse", P["Dm"], P["a"], P["re"], P["mu"][1])]
    g = mg.Propagator(N, dq, minv=minv)
    g.set_potential(mg.MG_POT_ATOM_DIATOM, pot)
    g.set_separable(fac, [R0, rbar], [P0, 0.0])
    o = oracle.Grid(N, dq, minv=minv)
    o.set_potential(oracle.POT_ATOM_DIATOM, pot)
    o.set_separable(fac, [R0, rbar], [P0, 0.0])
    return g, o, pot


@pytest.mark.parametrize("split,motion,R0", [(0, 0, None), (1, 0, None), (0, 2, None), (0, 1, None), (0, 0, 4.0),
                                             (1, 0, 4.0)])
def test_adjoint_matches_oracle_tape(mg, split, motion, R0):
    # R0 = 4: the packet starts inside the atom-diatom coupling region, where
    # the potential's Hessian and parameter derivatives carry the gradient, and
    # runs 50 steps into its deceleration (p from -10 to about -6).  Its grid
    # keeps the R window within R > -1: a window reaching R ~ -6, where V ~
    # 1e6 hartree, leaves the two computations differing by their roundoff in
    # those phases (1e-8 relative on the state cotangent)
    N, dq = ((48, 36), (0.4, 0.25)) if R0 is None else ((64, 24), (0.16, 0.2))
    g, o, pot = atom_diatom_pair(mg, N, dq, R0=R0)
    u0 = g.psi.view(torch.complex128).cpu().numpy().reshape(N).copy()
    _, q0, p0, _ = g.get_state(want_psi=False)
    steps, dt, scheme = (6 if R0 is None else 50), 2.0, "yoshida4"
    rng = np.random.default_rng(1)
    c = inputs.random_state(N, seed=2) * 0.4
    al, be = rng.normal(size=2), rng.normal(size=2) * 0.1
    g.propagate(steps, dt, scheme, split, motion)
    ub, qb, pb, th = g.adjoint(steps, dt, scheme, c, al, be, split, motion)
    tape = Tape(o, oracle.POT_ATOM_DIATOM, pot)
    tape.run(steps, dt, scheme, split, motion)
    ubo, qbo, pbo, tho = tape.backward(c, al, be)
    assert rel(ub, ubo) < 1e-9
    assert np.allclose(qb, qbo, rtol=1e-9, atol=1e-9 * np.abs(qbo).max())
    assert np.allclose(pb, pbo, rtol=1e-9, atol=1e-9 * np.abs(pbo).max())
    assert np.allclose(th, tho, rtol=1e-8, atol=1e-9 * np.abs(tho).max())
    # the context was rewound to the initial state by the reverse sweep
    u1 = g.psi.view(torch.complex128).cpu().numpy().reshape(N)
    _, q1, p1, _ = g.get_state(want_psi=False)
    assert rel(u1, u0) < 1e-12 and np.allclose(q1, q0, atol=1e-12) and np.allclose(p1, p0, atol=1e-11)


def test_adjoint_harmonic_3d_matches_oracle_tape(mg):
    Ph = inputs.HARMONIC3D
    N, dq = (16, 12, 18), (0.6, 0.7, 0.5)
    om = np.array(Ph["omega"])
    pot = list(np.diag(om ** 2).ravel()) + [0.1, -0.2, 0.0]
    fac = [("gauss", Ph["q0"][l], Ph["p0"][l], om[l] ** -0.5) for l in range(3)]
    g = mg.Propagator(N, dq, minv=(1.0, 0.8, 1.3))
    g.set_potential(mg.MG_POT_HARMONIC, pot)
    g.set_separable(fac, Ph["q0"], Ph["p0"])
    o = oracle.Grid(N, dq, minv=(1.0, 0.8, 1.3))
    o.set_potential(oracle.POT_HARMONIC, pot)
    o.set_separable(fac, Ph["q0"], Ph["p0"])
    c = inputs.random_state(N, seed=5) * 0.3
    al, be = np.array([0.3, -0.7, 0.2]), np.array([0.05, 0.1, -0.2])
    g.propagate(8, 0.05, "suzuki4")
    ub, qb, pb, _ = g.adjoint(8, 0.05, "suzuki4", c, al, be)
    tape = Tape(o, oracle.POT_HARMONIC, pot)
    tape.run(8, 0.05, "suzuki4")
    ubo, qbo, pbo, _ = tape.backward(c, al, be)
    assert rel(ub, ubo) < 1e-9
    assert np.allclose(qb, qbo, rtol=1e-9, atol=1e-10) and np.allclose(pb, pbo, rtol=1e-9, atol=1e-10)


def objective_and_cotangents(mg, g, N, dq, hbar=1.0):
    """J = <q_1>(T) + |<phi_target|psi(T)>|^2 with phi_target a Gaussian in R
    (R = 7.6, p = 0, sigma = 0.6) times the Morse ground state in r, evaluated
    on the final grid; returns J and (ubar_T, qbar_T, pbar_T)."""
    u = g.psi.view(torch.complex128).cpu().numpy().reshape(N)
    _, q, p, _ = g.get_state(want_psi=False)
    y = [(np.arange(N[l]) - N[l] / 2) * dq[l] for l in range(2)]
    R, r = np.meshgrid(q[0] + y[0], q[1] + y[1], indexing="ij")
    w = np.abs(u) ** 2
    n = w.sum()
    mq = (R * w).sum() / n
    lam = np.sqrt(2 * P["mu"][1] * P["Dm"]) / P["a"]
    from scipy.special import gammaln
    z = 2 * lam * np.exp(-P["a"] * (r - P["re"]))
    morse = np.exp((lam - 0.5) * np.log(z) - 0.5 * z + 0.5 * (np.log(P["a"]) - gammaln(2 * lam - 1)))
    s2 = 0.6 ** 2
    gR = (np.pi * s2) ** -0.25 * np.exp(-(R - 7.6) ** 2 / (2 * s2))
    f = gR * morse * np.sqrt(dq[0] * dq[1])
    ov = np.vdot(f, u)
    J = mq + abs(ov) ** 2
    ub = 2 * (R - mq) / n * u + 2 * ov * f
    # d/dq of the sampled target and of x^J
    dfR = -(R - 7.6) / s2 * f
    dmorse_dr = ((lam - 0.5) * (-P["a"]) + 0.5 * P["a"] * z) * f
    qb = np.array([1.0 + 2 * np.real(np.conj(ov) * np.vdot(dfR, u)),
                   2 * np.real(np.conj(ov) * np.vdot(dmorse_dr, u))])
    return J, ub, qb, np.zeros(2)


@pytest.mark.parametrize("steps", [200, 2000])
def test_gradient_of_objective_vs_finite_differences(mg, steps):
    # 128 x 128 grid (dR = dr = 0.08), sixth-order triple jump, dt = 1 a.u.;
    # 2000 steps (t = 2000 a.u.) is the full length of the gradient workload,
    # regenerated backwards by the adjoint without a stored trajectory.  With
    # dR = 0.16 the R window (+-10.24 around the centre) reaches R ~ -6 near
    # the turning point, where V ~ 1e6 hartree turns by ~1e5 rad between
    # neighbouring points: there central differences at h = 1e-5 do not
    # converge, while the adjoint and the oracle's taped gradient still agree
    # on the derivative of the discrete map.
    N, dq = (128, 128), (0.08, 0.08)
    dt, scheme = 1.0, "yoshida6"

    def J_of(R0, P0, sigma, theta):
        g, _, _ = atom_diatom_pair(mg, N, dq, R0, P0, sigma, theta)
        g.propagate(steps, dt, scheme)
        return objective_and_cotangents(mg, g, N, dq)[0]

    R0, P0, sigma = P["R0"], P["P0"], P["sigma"]
    theta = np.array([P["Dm"], P["a"], P["beta"], P["A"]])
    g, _, _ = atom_diatom_pair(mg, N, dq, R0, P0, sigma, theta)
    u0 = g.psi.view(torch.complex128).cpu().numpy().reshape(N).copy()
    g.propagate(steps, dt, scheme)
    J, ubT, qbT, pbT = objective_and_cotangents(mg, g, N, dq)
    ub0, qb0, pb0, thb = g.adjoint(steps, dt, scheme, ubT, qbT, pbT)
    # chain to the wavepacket parameters: samples relative to the centre (q0 only
    # moves the grid), p0 in the phase and the grid's p-centre, sigma in the width
    y = ((np.arange(N[0]) - N[0] / 2) * dq[0])[:, None]
    dR0 = qb0[0]
    dP0 = pb0[0] + np.real(np.vdot(ub0, 1j * y * u0))
    dsig = np.real(np.vdot(ub0, (-0.5 / sigma + y * y / sigma ** 3) * u0))
    grads = {"R0": dR0, "P0": dP0, "sigma": dsig}
    for k, name in enumerate(["Dm", "a", "beta", "A"]):
        grads[name] = thb[k]
    h = 1e-5
    fd = {
        "R0": (J_of(R0 + h, P0, sigma, theta) - J_of(R0 - h, P0, sigma, theta)) / (2 * h),
        "P0": (J_of(R0, P0 + h, sigma, theta) - J_of(R0, P0 - h, sigma, theta)) / (2 * h),
        "sigma": (J_of(R0, P0, sigma + h, theta) - J_of(R0, P0, sigma - h, theta)) / (2 * h),
    }
    for k, name in enumerate(["Dm", "a", "beta", "A"]):
        e = np.zeros(4)
        e[k] = h * max(1.0, abs(theta[k]))
        fd[name] = (J_of(R0, P0, sigma, theta + e) - J_of(R0, P0, sigma, theta - e)) / (2 * e[k])
    for name in fd:
        assert abs(grads[name] - fd[name]) < 1e-6 * max(1.0, abs(fd[name])), (name, grads[name], fd[name])


def test_autograd_function(mg):
    from paper_1909_06412_gb300.autograd import MovingGridPropagate

    N, dq = (48, 36), (0.4, 0.25)
    g, o, pot = atom_diatom_pair(mg, N, dq)
    u0 = g.psi.view(torch.complex128).clone().reshape(N).requires_grad_(True)
    _, q0, p0, _ = g.get_state(want_psi=False)
    q0t = torch.tensor(q0, requires_grad=True)
    p0t = torch.tensor(p0, requires_grad=True)
    th = torch.tensor([P["Dm"], P["a"], P["beta"], P["A"]], dtype=torch.float64, requires_grad=True)
    c = torch.from_numpy(inputs.random_state(N, seed=8) * 0.5).to(g.device)
    uT, qT, pT = MovingGridPropagate.apply(u0, q0t, p0t, th, g, 5, 2.0, "yoshida4")
    L = (torch.conj(c) * uT).real.sum() + qT[0] * 0.3 - pT[1] * 0.2
    L.backward()
    tape = Tape(o, oracle.POT_ATOM_DIATOM, pot)
    tape.run(5, 2.0, "yoshida4")
    ubo, qbo, pbo, tho = tape.backward(c.cpu().numpy(), np.array([0.3, 0.0]), np.array([0.0, -0.2]))
    assert rel(u0.grad.cpu().numpy(), ubo) < 1e-9
    assert np.allclose(q0t.grad.numpy(), qbo, rtol=1e-9, atol=1e-10)
    assert np.allclose(p0t.grad.numpy(), pbo, rtol=1e-9, atol=1e-10)
    assert np.allclose(th.grad.numpy(), tho, rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("steps", [100, 2000])
def test_gradient_3d_harmonic_vs_finite_differences(mg, steps):
    # 64^3 grid, dq = 0.3, omega = (1, 1.2, 1.5), unit masses, sixth-order
    # triple jump, dt = 0.01 (2000 steps: the full length of the gradient
    # workload); initial widths sigma_i = s / sqrt(omega_i), s = 1
    N, dq = (64, 64, 64), (0.3, 0.3, 0.3)
    om = np.array([1.0, 1.2, 1.5])
    pot = list(np.diag(om ** 2).ravel()) + [0.0] * 3
    dt, scheme = 0.01, "yoshida6"
    T = steps * dt
    q0n, p0n = np.array([1.0, -0.5, 0.8]), np.array([0.0, 0.5, -0.3])
    # target: coherent state at the classical point at T, shifted by 0.6 in q_1
    # (a shift of 0.3 leaves |overlap|^2 = e^{-0.045}, above 0.9)
    qt = q0n * np.cos(om * T) + p0n / om * np.sin(om * T) + np.array([0.6, 0.0, 0.0])
    pt = p0n * np.cos(om * T) - q0n * om * np.sin(om * T)

    def make(q0, p0, s):
        g = mg.Propagator(N, dq)
        g.set_potential(mg.MG_POT_HARMONIC, pot)
        g.set_separable([("gauss", q0[l], p0[l], s / np.sqrt(om[l])) for l in range(3)], q0, p0)
        return g

    ys = [(np.arange(N[l]) - N[l] / 2) * dq[l] for l in range(3)]

    def objective(g):
        u = g.psi.view(torch.complex128).cpu().numpy().reshape(N)
        _, q, p, _ = g.get_state(want_psi=False)
        X = np.meshgrid(*[q[l] + ys[l] for l in range(3)], indexing="ij")
        w = np.abs(u) ** 2
        n = w.sum()
        mq = (X[0] * w).sum() / n
        logf = sum(0.25 * np.log(om[l] / np.pi) - 0.5 * om[l] * (X[l] - qt[l]) ** 2 + 1j * pt[l] * (X[l] - qt[l])
                   for l in range(3))
        f = np.exp(logf) * np.sqrt(np.prod(dq))
        ov = np.vdot(f, u)
        J = mq + abs(ov) ** 2
        ub = 2 * (X[0] - mq) / n * u + 2 * ov * f
        qb = np.array([float(l == 0) + 2 * np.real(np.conj(ov) * np.vdot((-om[l] * (X[l] - qt[l]) + 1j * pt[l]) * f, u))
                       for l in range(3)])
        return J, ub, qb, 1e-3 < abs(ov) ** 2 < 0.9

    def J_of(q0, p0, s):
        g = make(q0, p0, s)
        g.propagate(steps, dt, scheme)
        return objective(g)[0]

    g = make(q0n, p0n, 1.0)
    u0 = g.psi.view(torch.complex128).cpu().numpy().reshape(N).copy()
    g.propagate(steps, dt, scheme)
    J, ubT, qbT, ok = objective(g)
    assert ok
    ub0, qb0, pb0, _ = g.adjoint(steps, dt, scheme, ubT, qbT, np.zeros(3))
    Y = np.meshgrid(*ys, indexing="ij")
    grads = {}
    for l in range(3):
        grads[f"q0_{l}"] = qb0[l]
        grads[f"p0_{l}"] = pb0[l] + np.real(np.vdot(ub0, 1j * Y[l] * u0))
    dlog_s = sum(-0.5 + om[l] * Y[l] ** 2 for l in range(3))  # at s = 1
    grads["s"] = np.real(np.vdot(ub0, dlog_s * u0))
    h = 1e-5
    fd = {}
    for l in range(3):
        e = np.eye(3)[l] * h
        fd[f"q0_{l}"] = (J_of(q0n + e, p0n, 1.0) - J_of(q0n - e, p0n, 1.0)) / (2 * h)
        fd[f"p0_{l}"] = (J_of(q0n, p0n + e, 1.0) - J_of(q0n, p0n - e, 1.0)) / (2 * h)
    fd["s"] = (J_of(q0n, p0n, 1.0 + h) - J_of(q0n, p0n, 1.0 - h)) / (2 * h)
    for name in fd:
        assert abs(grads[name] - fd[name]) < 1e-6 * max(1.0, abs(fd[name])), (name, grads[name], fd[name])


def test_autograd_two_forwards_before_their_backwards(mg):
    # One context, two forward passes with different potentials and start
    # centres before either backward, then each backward (the second one twice,
    # through a retained graph).  Each gradient must match the oracle's taped
    # gradient of its own forward pass: the backward restores the end state of
    # its forward pass into the context before the reversible adjoint runs.
    from paper_1909_06412_gb300.autograd import MovingGridPropagate

    N, dq = (48, 36), (0.4, 0.25)
    g, _, pot = atom_diatom_pair(mg, N, dq)
    ubase = g.psi.view(torch.complex128).clone().reshape(N)
    _, qbase, pbase, _ = g.get_state(want_psi=False)
    cell = np.sqrt(np.prod(dq))
    c = torch.from_numpy(inputs.random_state(N, seed=8) * 0.5).to(g.device)
    cases = [(np.array([P["Dm"], P["a"], P["beta"], P["A"]]), 0.0),
             (np.array([P["Dm"] * 1.1, P["a"] * 0.95, P["beta"] * 1.05, P["A"] * 0.9]), 0.25)]
    runs = []
    for theta, shift in cases:
        u0 = ubase.clone().requires_grad_(True)
        q0t = torch.tensor(qbase + np.array([shift, 0.0]), requires_grad=True)
        p0t = torch.tensor(pbase, requires_grad=True)
        th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
        uT, qT, pT = MovingGridPropagate.apply(u0, q0t, p0t, th, g, 5, 2.0, "yoshida4")
        L = (torch.conj(c) * uT).real.sum() + qT[0] * 0.3 - pT[1] * 0.2
        runs.append((L, (u0, q0t, p0t, th), theta, shift))
    for k in (1, 0, 1):
        L, leaves, theta, shift = runs[k]
        gu, gq, gp, gth = torch.autograd.grad(L, leaves, retain_graph=True)
        Dm, a, be, A = theta
        o = oracle.Grid(N, dq, minv=(1 / P["mu"][0], 1 / P["mu"][1]))
        pot_k = [Dm, a, P["re"], A, be]
        o.set_potential(oracle.POT_ATOM_DIATOM, pot_k)
        o.set_state(ubase.cpu().numpy() / cell, qbase + np.array([shift, 0.0]), pbase)
        tape = Tape(o, oracle.POT_ATOM_DIATOM, pot_k)
        tape.run(5, 2.0, "yoshida4")
        ubo, qbo, pbo, tho = tape.backward(c.cpu().numpy(), np.array([0.3, 0.0]), np.array([0.0, -0.2]))
        assert rel(gu.cpu().numpy(), ubo) < 1e-9, k
        assert np.allclose(gq.numpy(), qbo, rtol=1e-9, atol=1e-10), k
        assert np.allclose(gp.numpy(), pbo, rtol=1e-9, atol=1e-10), k
        assert np.allclose(gth.numpy(), tho, rtol=1e-8, atol=1e-10), k
