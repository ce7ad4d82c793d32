"""ctypes wrapper of the plain FP64 CPU oracle (``oracle/mgrid_oracle.c``).

TEST INFRASTRUCTURE ONLY: this is the checker of the GPU library.  Only the
tests, the smoke check and the CPU-baseline leg of the benchmark use it; the
product path never imports it.  It shares no code with the CUDA library.

Parity is pinned by the CPU tests in ``tests/test_oracle_pins.py``; the one
function whose paper-printed accuracy cannot be reproduced (the adaptive vs
fixed-grid errors of Sec. III.A, which need the unprinted optimal
tenth-order coefficients) is not offered here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_DIR = os.path.join(_HERE, "lib")
_LIB_PATH = os.path.join(_LIB_DIR, "libmgrid_oracle.so")
_SRC = os.path.join(_HERE, "mgrid_oracle.c")

POT_HARMONIC, POT_ATOM_DIATOM, POT_HENON_HEILES, POT_SECREST_JOHNSON = 0, 1, 2, 3
SPLIT_TVT, SPLIT_VTV, SPLIT_TV = 0, 1, 2
GRID_ADAPTIVE, GRID_ADAPTIVE_CENTRE_P, GRID_FIXED, GRID_NAIVE = 0, 1, 2, 3


def build_command():
    return ["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", _LIB_PATH, _SRC, "-lm"]


def build(wait=True):
    """Compile the oracle into ``oracle/lib``.  Returns the Popen if not waiting."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    proc = subprocess.Popen(build_command())
    if wait:
        if proc.wait() != 0:
            raise RuntimeError("oracle build failed")
        return None
    return proc


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            build()
        L = ctypes.CDLL(_LIB_PATH)
        d, i64, i32, vp = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        P = ctypes.POINTER
        L.orc_dft1d.argtypes = [i64, vp, i32]
        L.orc_dft1d_direct.argtypes = [i64, vp, vp, i32]
        L.orc_scheme.argtypes = [ctypes.c_char_p, vp, i32]
        L.orc_create.argtypes = [i32, vp, vp, vp, d]
        L.orc_create.restype = vp
        L.orc_destroy.argtypes = [vp]
        L.orc_npoints.argtypes = [vp]
        L.orc_npoints.restype = i64
        L.orc_set_potential.argtypes = [vp, i32, vp, i32]
        L.orc_potential_eval.argtypes = [vp, i64, vp, vp, vp]
        L.orc_set_state.argtypes = [vp, vp, vp, vp, d]
        L.orc_get_state.argtypes = [vp, vp, vp, vp, vp]
        L.orc_set_u.argtypes = [vp, vp]
        L.orc_get_u.argtypes = [vp, vp]
        L.orc_set_separable.argtypes = [vp, vp, vp, vp, vp]
        L.orc_morse_mean.argtypes = [d, d, d, d, d]
        L.orc_morse_mean.restype = d
        L.orc_apply_f.argtypes = [vp, vp, vp, vp, vp, i32]
        L.orc_apply_f_dense.argtypes = [vp, vp, vp, vp, vp, i32]
        L.orc_substep_V.argtypes = [vp, d, i32]
        L.orc_substep_T.argtypes = [vp, d, i32]
        L.orc_propagate.argtypes = [vp, i64, d, ctypes.c_char_p, i32, i32]
        L.orc_observables.argtypes = [vp, vp, vp, vp, vp]
        L.orc_regrid.argtypes = [vp, vp, vp, vp, vp, vp]
        del P
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def dft1d(x, sign=-1):
    """Unitary 1D DFT (radix-2 FFT for powers of two, direct sum otherwise)."""
    y = _c128(x).copy()
    _check(lib().orc_dft1d(len(y), _ptr(y), sign), "dft1d")
    return y


def dft1d_direct(x, sign=-1):
    x = _c128(x)
    y = np.empty_like(x)
    _check(lib().orc_dft1d_direct(len(x), _ptr(x), _ptr(y), sign), "dft1d_direct")
    return y


def scheme(name):
    """Composition coefficients gamma_1..gamma_S of a named symmetric scheme."""
    buf = np.zeros(625)
    s = lib().orc_scheme(name.encode(), _ptr(buf), 625)
    if s <= 0:
        raise ValueError(f"unknown scheme {name!r}")
    return buf[:s].copy()


def inner_product(ga, gb):
    """<psi_a | psi_b> of two oracle states on grids of the same shape and
    spacing but different centres (eq:scalar_prod): b's samples are carried
    onto a's positions with b's momentum window, f~(q_a, p_b) f(q_b, p_b)
    (literal eq:F_defintion), then summed against a's."""
    ua, ub = ga.get_u(), gb.get_u()
    _, qa, _, _ = ga.get_state()
    _, qb, pb, _ = gb.get_state()
    ub_on_a = ga.apply_f(qa, pb, ga.apply_f(qb, pb, ub, -1), +1)
    return complex(np.vdot(ua, ub_on_a))


def morse_mean(Dm, a, re, mass, hbar=1.0):
    return lib().orc_morse_mean(Dm, a, re, mass, hbar)


class Grid:
    """One oracle context: grid, potential and state (q, p, t, u)."""

    def __init__(self, N, dq, minv=None, hbar=1.0):
        self.N = tuple(int(n) for n in N)
        self.D = len(self.N)
        self.dq = _f64(dq).reshape(self.D)
        if minv is None:
            minv = np.eye(self.D)
        minv = np.asarray(minv, dtype=np.float64)
        if minv.ndim == 1:
            minv = np.diag(minv)
        self.minv = _f64(minv).reshape(self.D, self.D)
        self.hbar = float(hbar)
        self.dp = 2 * np.pi * self.hbar / (np.array(self.N) * self.dq)
        n = np.array(self.N, dtype=np.int64)
        self._h = lib().orc_create(self.D, _ptr(n), _ptr(self.dq), _ptr(self.minv), self.hbar)
        if not self._h:
            raise ValueError("oracle grid rejected (N must be even, dq > 0)")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_destroy(h)
            self._h = None

    @property
    def npts(self):
        return int(np.prod(self.N))

    def set_potential(self, kind, params):
        p = _f64(params).ravel()
        _check(lib().orc_set_potential(self._h, kind, _ptr(p), len(p)), "set_potential")

    def potential(self, x):
        x = _f64(x).reshape(-1, self.D)
        V = np.empty(len(x))
        g = np.empty_like(x)
        _check(lib().orc_potential_eval(self._h, len(x), _ptr(x), _ptr(V), _ptr(g)), "potential")
        return V, g

    def set_state(self, psi, q, p, t=0.0):
        psi = _c128(psi).reshape(self.N)
        q, p = _f64(q).reshape(self.D), _f64(p).reshape(self.D)
        _check(lib().orc_set_state(self._h, _ptr(psi), _ptr(q), _ptr(p), float(t)), "set_state")

    def get_state(self):
        psi = np.empty(self.N, dtype=np.complex128)
        q, p, t = np.empty(self.D), np.empty(self.D), np.zeros(1)
        _check(lib().orc_get_state(self._h, _ptr(psi), _ptr(q), _ptr(p), _ptr(t)), "get_state")
        return psi, q, p, float(t[0])

    def set_u(self, u):
        u = _c128(u).reshape(self.N)
        _check(lib().orc_set_u(self._h, _ptr(u)), "set_u")

    def get_u(self):
        u = np.empty(self.N, dtype=np.complex128)
        _check(lib().orc_get_u(self._h, _ptr(u)), "get_u")
        return u

    def set_separable(self, factors, q_ctr, p_ctr):
        """factors: per axis ('gauss', q0, p0, sigma) or ('morse', Dm, a, re, mass)."""
        kinds = np.zeros(self.D, dtype=np.int32)
        params = np.zeros((self.D, 4))
        for l, f in enumerate(factors):
            kinds[l] = {"gauss": 0, "morse": 1}[f[0]]
            params[l, : len(f) - 1] = f[1:]
        q, p = _f64(q_ctr).reshape(self.D), _f64(p_ctr).reshape(self.D)
        _check(lib().orc_set_separable(self._h, _ptr(kinds), _ptr(params), _ptr(q), _ptr(p)),
               "set_separable")

    def apply_f(self, q, p, x, sign=-1, dense=False):
        x = _c128(x).reshape(self.N)
        y = np.empty_like(x)
        q, p = _f64(q).reshape(self.D), _f64(p).reshape(self.D)
        fn = lib().orc_apply_f_dense if dense else lib().orc_apply_f
        _check(fn(self._h, _ptr(q), _ptr(p), _ptr(x), _ptr(y), sign), "apply_f")
        return y

    def substep_V(self, tau, grid_motion=GRID_ADAPTIVE):
        _check(lib().orc_substep_V(self._h, float(tau), grid_motion), "substep_V")

    def substep_T(self, tau, grid_motion=GRID_ADAPTIVE):
        _check(lib().orc_substep_T(self._h, float(tau), grid_motion), "substep_T")

    def propagate(self, n_steps, dt, scheme="strang", split=SPLIT_TVT, grid_motion=GRID_ADAPTIVE):
        if grid_motion == GRID_NAIVE:
            for _ in range(int(n_steps)):
                self.step_naive(dt, scheme, split)
            return
        rc = lib().orc_propagate(self._h, int(n_steps), float(dt), scheme.encode(), split, grid_motion)
        _check(rc, "propagate")

    def step_naive(self, dt, scheme="strang", split=SPLIT_TVT):
        """One step of the naive adaptive grid, Sec. II.F, in the paper's
        order: U(dt; q0, p0) on the fixed grid (eq:naive_wf_solution), then
        q1 = <q>, p1 = <p> of the propagated state, then the state carried to
        the new grid by f~(q1, p1) f(q0, p1) (literal eq:F_defintion)."""
        self.propagate(1, dt, scheme, split, GRID_FIXED)
        _, _, q1, p1 = self.observables()
        _, q0, _, t = self.get_state()
        u1 = self.apply_f(q1, p1, self.apply_f(q0, p1, self.get_u(), -1), +1)
        self.set_u(u1)
        self.set_centre(q1, p1, t)

    def set_centre(self, q, p, t):
        """Move the grid centre without touching the stored samples u."""
        u = self.get_u()
        psi = self.get_state()[0]
        self.set_state(psi, q, p, t)
        self.set_u(u)

    def observables(self):
        n, e = np.zeros(1), np.zeros(1)
        mq, mp = np.empty(self.D), np.empty(self.D)
        _check(lib().orc_observables(self._h, _ptr(n), _ptr(e), _ptr(mq), _ptr(mp)), "observables")
        return float(n[0]), float(e[0]), mq, mp

    def regrid(self, u_b, q_b, p, q_a):
        u_b = _c128(u_b).reshape(self.N)
        out = np.empty_like(u_b)
        q_b, p, q_a = (_f64(v).reshape(self.D) for v in (q_b, p, q_a))
        _check(lib().orc_regrid(self._h, _ptr(u_b), _ptr(q_b), _ptr(p), _ptr(q_a), _ptr(out)), "regrid")
        return out

    def qaxes(self, q):
        """Per-axis coordinates of the q-grid centred at q."""
        return [q[l] + (np.arange(self.N[l]) - self.N[l] / 2) * self.dq[l] for l in range(self.D)]
