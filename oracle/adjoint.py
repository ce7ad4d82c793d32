"""Taped FP64 gradient of the moving-grid integrator (TEST INFRASTRUCTURE ONLY).

Reverse-mode derivative of the map (u0, q0, p0, theta) -> (uT, qT, pT) that
`oracle.Grid.propagate` computes, obtained by storing every pre-substep state
on a tape and applying, substep by substep in reverse, the vector-Jacobian
product of the two substeps of Sec. II.G:

  potential substep (eq:eom_pt_solution_case_III_V), u' = e^{-i s V(x^J)/hbar} u,
  p' = p - s g, g = sum_J grad V(x^J) |u_J|^2 / sum |u|^2, q' = q;
  kinetic substep (eq:T_split_substep_adaptive), u' = f~(q', p) U_T f(q, p) u,
  q' = q + t m^-1 pi, pi = sum_K p^K |phi_K|^2 / sum |phi|^2, phi = f(q,p) u.

Cotangent convention: for a real objective J, ubar = dJ/dRe u + i dJ/dIm u, so
dJ = Re sum conj(ubar) du + qbar.dq + pbar.dp.  Pinned against central finite
differences of the oracle's forward propagation in tests/test_oracle_adjoint.py.
The only potential parameters differentiated are those of the atom-diatom
model (Dm, a, beta, A).
"""
import numpy as np

import oracle


def _grids(g, q, p):
    ys = [(np.arange(g.N[l]) - g.N[l] / 2) * g.dq[l] for l in range(g.D)]
    cs = [(np.arange(g.N[l]) - g.N[l] / 2) * g.dp[l] for l in range(g.D)]
    X = np.meshgrid(*[q[l] + ys[l] for l in range(g.D)], indexing="ij")
    Y = np.meshgrid(*ys, indexing="ij")
    PK = np.meshgrid(*[p[l] + cs[l] for l in range(g.D)], indexing="ij")
    return X, Y, PK


def potential_derivatives(kind, params, X):
    """V, grad V, Hessian, dV/dtheta, d(grad V)/dtheta at the points X (list
    of D arrays), straight from the formulas of the potential."""
    D = len(X)
    shp = X[0].shape
    if kind == oracle.POT_HARMONIC:
        K = np.asarray(params[: D * D]).reshape(D, D)
        c = np.asarray(params[D * D:])
        d = np.stack([X[a] - c[a] for a in range(D)])
        G = np.einsum("ab,b...->a...", K, d)
        V = 0.5 * np.einsum("a...,a...->...", d, G)
        H = np.broadcast_to(K.reshape(D, D, *([1] * len(shp))), (D, D) + shp)
        return V, G, H, np.zeros((0,) + shp), np.zeros((0, D) + shp)
    if kind == oracle.POT_ATOM_DIATOM:
        Dm, a, re, A, be = params
        R, r = X
        E = np.exp(-a * (r - re))
        ep, en = np.exp(0.5 * be * r), np.exp(-0.5 * be * r)
        h = ep + en                  # e^{b r/2} + e^{-b r/2}
        sh = ep - en
        hp = 0.5 * be * sh           # dh/dr
        gR = A * np.exp(-be * R)     # A e^{-b R}
        f = Dm * (1 - E) ** 2
        fp = 2 * Dm * a * (E - E * E)
        fpp = 2 * Dm * a * a * E * (2 * E - 1)
        V = f + gR * h
        G = np.stack([-be * gR * h, fp + gR * hp])
        H = np.stack([np.stack([be * be * gR * h, -be * gR * hp]),
                      np.stack([-be * gR * hp, fpp + gR * 0.25 * be * be * h])])
        # theta = (Dm, a, beta, A)
        dV = np.stack([(1 - E) ** 2,
                       2 * Dm * (1 - E) * E * (r - re),
                       -R * gR * h + gR * 0.5 * r * sh,
                       gR * h / A])
        dfp_da = 2 * Dm * ((E - E * E) - a * (r - re) * E * (1 - 2 * E))
        dhp_db = 0.5 * sh + 0.25 * be * r * h
        dG = np.stack([
            np.stack([np.zeros(shp), fp / Dm]),
            np.stack([np.zeros(shp), dfp_da]),
            np.stack([-gR * h + be * R * gR * h - be * gR * 0.5 * r * sh, -R * gR * hp + gR * dhp_db]),
            np.stack([-be * gR * h / A, gR * hp / A]),
        ])
        return V, G, H, dV, dG
    raise ValueError("potential kind without derivative formulas")


class Tape:
    """Forward propagation recording every pre-substep state."""

    def __init__(self, g, kind, params):
        self.g, self.kind, self.params = g, kind, np.asarray(params, dtype=float)
        self.ops = []

    def run(self, n_steps, dt, scheme="strang", split=oracle.SPLIT_TVT, motion=oracle.GRID_ADAPTIVE):
        g = self.g
        gam = oracle.scheme(scheme)
        seq = []
        for _ in range(n_steps):
            for gm in gam:
                h = gm * dt
                if split == oracle.SPLIT_TVT:
                    seq += [("T", h / 2), ("V", h), ("T", h / 2)]
                elif split == oracle.SPLIT_VTV:
                    seq += [("V", h / 2), ("T", h), ("V", h / 2)]
                else:
                    seq += [("V", h), ("T", h)]
        for kindop, tau in seq:
            u = g.get_u()
            _, q, p, _ = g.get_state()
            self.ops.append((kindop, tau, u, q.copy(), p.copy()))
            if kindop == "T":
                g.substep_T(tau, motion)
            else:
                g.substep_V(tau, motion)
        self.motion = motion
        _, q, p, t = g.get_state()
        g.set_state(g.get_state()[0], q, p, t + n_steps * dt)

    def vjp_T(self, tau, u, q, p, ub, qb, pb):
        g = self.g
        hb = g.hbar
        minv = g.minv
        _, Y, PK = _grids(g, q, p)
        phi = g.apply_f(q, p, u, -1)
        rho = np.abs(phi) ** 2
        n = rho.sum()
        pi = np.array([(PK[l] * rho).sum() / n for l in range(g.D)])
        if self.motion == oracle.GRID_ADAPTIVE:
            delta = tau * minv @ pi
        elif self.motion == oracle.GRID_ADAPTIVE_CENTRE_P:
            delta = tau * minv @ p
        else:
            delta = np.zeros(g.D)
        T = 0.5 * np.einsum("a...,ab,b...->...", np.stack(PK), minv, np.stack(PK))
        Kf = np.exp(1j * (np.einsum("a,a...->...", delta, np.stack(PK)) - tau * T) / hb)
        phi1 = Kf * phi                      # f(q,p) u' (up to the f~ f identity)
        u1 = g.apply_f(q, p, phi1, +1)       # u' on the moved grid
        phib1 = g.apply_f(q, p, ub, -1)      # f(q,p) ubar'
        im = np.imag(np.conj(phib1) * phi1)
        deltab = qb - np.array([(PK[l] * im).sum() for l in range(g.D)]) / hb
        if self.motion == oracle.GRID_ADAPTIVE:
            pib = tau * minv @ deltab
        else:
            pib = np.zeros(g.D)
        s = sum(pib[l] * (PK[l] - pi[l]) for l in range(g.D)) / n
        phib = np.conj(Kf) * phib1 + 2 * s * phi
        ubar = g.apply_f(q, p, phib, +1)
        qbar = qb.copy()
        pbar = pb + (pib if self.motion == oracle.GRID_ADAPTIVE else 0)
        # dependence of the multiplier on p (p^K = p + c dp) and on delta(p) for centre_p
        mpk = np.stack([sum(minv[a, b] * PK[b] for b in range(g.D)) for a in range(g.D)])
        for l in range(g.D):
            pbar[l] -= ((delta[l] - tau * mpk[l]) * im).sum() / hb
        if self.motion == oracle.GRID_ADAPTIVE_CENTRE_P:
            pbar += tau * minv @ deltab
        # dependence of f(q,p) and f~(q,p) on p (through the sampled kernel)
        for l in range(g.D):
            pbar[l] += (Y[l] * np.imag(np.conj(ubar) * u)).sum() / hb
            pbar[l] -= (Y[l] * np.imag(np.conj(ub) * u1)).sum() / hb
        return ubar, qbar, pbar

    def vjp_V(self, sig, u, q, p, ub, qb, pb, thb):
        g = self.g
        hb = g.hbar
        X, _, _ = _grids(g, q, p)
        V, G, H, dV, dG = potential_derivatives(self.kind, self.params, X)
        w = np.abs(u) ** 2
        n = w.sum()
        gmean = np.array([(G[a] * w).sum() / n for a in range(g.D)])
        u1 = np.exp(-1j * sig * V / hb) * u
        gb = -sig * pb if self.motion != oracle.GRID_FIXED else np.zeros(g.D)
        Vb = sig / hb * np.imag(np.conj(ub) * u1)
        s = sum(gb[a] * (G[a] - gmean[a]) for a in range(g.D)) / n
        ubar = np.exp(1j * sig * V / hb) * ub + 2 * s * u
        qbar = qb + np.array([(Vb * G[a]).sum() for a in range(g.D)]) + \
            np.array([(sum(H[a, b] * gb[b] for b in range(g.D)) * w).sum() / n for a in range(g.D)])
        if len(dV):
            thb = thb + np.array([(Vb * dV[k]).sum() + (sum(dG[k, a] * gb[a] for a in range(g.D)) * w).sum() / n
                                  for k in range(len(dV))])
        return ubar, qbar, pb.copy(), thb

    def backward(self, ub, qb, pb):
        """Cotangents at t = 0 and the potential-parameter gradient."""
        nth = 4 if self.kind == oracle.POT_ATOM_DIATOM else 0
        thb = np.zeros(nth)
        ub, qb, pb = np.asarray(ub, complex), np.asarray(qb, float), np.asarray(pb, float)
        for kindop, tau, u, q, p in reversed(self.ops):
            if kindop == "T":
                ub, qb, pb = self.vjp_T(tau, u, q, p, ub, qb, pb)
            else:
                ub, qb, pb, thb = self.vjp_V(tau, u, q, p, ub, qb, pb, thb)
        return ub, qb, pb, thb
