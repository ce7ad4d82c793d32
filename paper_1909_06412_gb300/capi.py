"""ctypes binding of the C-ABI in ``include/mgrid.h`` (same names), plus a thin
``Propagator`` that owns torch device buffers and forwards every call.

Only argument marshalling happens here; every step of the propagation runs in
the CUDA kernels of ``lib/libmgrid.so``.  Loading fails with an ImportError if
the library is missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libmgrid.so")

MG_OK, MG_ERR_ARG, MG_ERR_UNSUPPORTED, MG_ERR_CUDA = 0, -1, -2, -3
MG_ERR_TIMEOUT, MG_ERR_NONFINITE, MG_ERR_UNSTABLE, MG_ERR_STATE = -4, -5, -6, -7
MG_FP64, MG_FP32_MIXED = 0, 1
MG_TVT, MG_VTV, MG_TV = 0, 1, 2
MG_GRID_ADAPTIVE, MG_GRID_ADAPTIVE_CENTRE_P, MG_GRID_FIXED, MG_GRID_NAIVE = 0, 1, 2, 3
MG_POT_HARMONIC, MG_POT_ATOM_DIATOM, MG_POT_HENON_HEILES, MG_POT_SECREST_JOHNSON = 0, 1, 2, 3
MG_CREATE_GENERAL_KERNEL, MG_CREATE_NO_TMA, MG_CREATE_TC_TF32X3, MG_CREATE_TC_BF16X3 = 1, 2, 4, 8

__all__ = [n for n in dir() if n.startswith("MG_")] + ["Propagator", "Batch", "MgError", "lib", "mg_workspace_bytes",
                                                        "mg_batch_workspace_bytes", "mg_morse_mean",
                                                        "mg_propagate_noalloc", "mg_short_axis_plan",
                                                        "mg_scheme_coefficients", "mg_probe_fma_rate",
                                                        "mg_probe_expi", "mg_probe_tc_dft16"]


_lib = None


def lib():
    """The loaded CUDA library (raises ImportError if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
        L.mg_workspace_bytes.argtypes = [i32, vp, i32]
        L.mg_workspace_bytes.restype = sz
        L.mg_create.argtypes = [ctypes.POINTER(vp), i32, vp, vp, vp, d, i32, vp, vp, sz, vp]
        L.mg_create_ex.argtypes = [ctypes.POINTER(vp), i32, vp, vp, vp, d, i32, vp, vp, sz, vp, i32]
        L.mg_destroy.argtypes = [vp]
        L.mg_set_potential.argtypes = [vp, i32, vp, i32]
        L.mg_set_state.argtypes = [vp, vp, vp, vp, d]
        L.mg_set_separable.argtypes = [vp, vp, vp, vp, vp]
        L.mg_propagate.argtypes = [vp, i64, d, ctypes.c_char_p, i32, i32]
        L.mg_get_state.argtypes = [vp, vp, vp, vp, vp]
        L.mg_get_observables.argtypes = [vp, vp, vp, vp, vp]
        L.mg_sync.argtypes = [vp]
        L.mg_test_stuck_barrier.argtypes = [vp, d]
        L.mg_upload_u.argtypes = [vp, vp, vp, vp, d]
        L.mg_download_u.argtypes = [vp, vp, vp, vp, vp]
        L.mg_probe_fma_rate.argtypes = [i32, vp, vp]
        L.mg_probe_expi.argtypes = [vp, vp, vp, i64, vp]
        L.mg_probe_tc_dft16.argtypes = [i32, i32, vp, vp, i64, vp, vp, vp]
        L.mg_regrid.argtypes = [vp, vp, vp]
        L.mg_inner_product.argtypes = [vp, vp, vp, vp]
        L.mg_kernel_launches.argtypes = [vp]
        L.mg_kernel_launches.restype = i64
        L.mg_propagate_path.argtypes = [vp]
        L.mg_propagate_path.restype = i32
        L.mg_tables_in_workspace.argtypes = [vp]
        L.mg_tables_in_workspace.restype = i32
        L.mg_short_axis_plan.argtypes = [i32, vp, i32, vp, vp, vp, vp]
        L.mg_short_axis_plan.restype = i32
        L.mg_scheme_coefficients.argtypes = [ctypes.c_char_p, vp, i32]
        L.mg_scheme_coefficients.restype = i32
        L.mg_morse_mean.argtypes = [d, d, d, d, d]
        L.mg_morse_mean.restype = d
        L.mg_status_string.argtypes = [i32]
        L.mg_status_string.restype = ctypes.c_char_p
        L.mg_adjoint.argtypes = [vp, i64, d, ctypes.c_char_p, i32, i32, vp, vp, vp, vp, i32]
        L.mg_batch_workspace_bytes.argtypes = [i32]
        L.mg_batch_workspace_bytes.restype = sz
        L.mg_batch_create.argtypes = [ctypes.POINTER(vp), i32, vp, i32, vp, vp, vp, sz]
        L.mg_batch_propagate.argtypes = [vp, i64, vp, ctypes.c_char_p, i32, i32]
        L.mg_batch_sync.argtypes = [vp, vp]
        L.mg_batch_info.argtypes = [vp, vp, vp, vp, vp]
        L.mg_batch_destroy.argtypes = [vp]
        for name in ("mg_create", "mg_create_ex", "mg_destroy", "mg_set_potential", "mg_set_state", "mg_set_separable",
                     "mg_propagate", "mg_get_state", "mg_get_observables", "mg_sync", "mg_test_stuck_barrier",
                     "mg_adjoint", "mg_regrid", "mg_inner_product",
                     "mg_batch_create", "mg_batch_propagate", "mg_batch_sync", "mg_batch_info",
                     "mg_batch_destroy", "mg_probe_fma_rate", "mg_probe_expi", "mg_upload_u", "mg_download_u",
                     "mg_probe_tc_dft16"):
            getattr(L, name).restype = i32
        _lib = L
    return _lib


class MgError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {lib().mg_status_string(code).decode()} ({code})")


def _check(code, what):
    if code != MG_OK:
        raise MgError(code, what)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(x, n=None):
    a = np.ascontiguousarray(x, dtype=np.float64).ravel()
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def mg_workspace_bytes(N, precision=MG_FP64):
    n = np.ascontiguousarray(N, dtype=np.int64)
    return int(lib().mg_workspace_bytes(len(n), _ptr(n), precision))


def mg_scheme_coefficients(scheme):
    """Host-only: the stage coefficients gamma_k of a named composition."""
    S = lib().mg_scheme_coefficients(scheme.encode(), None, 0)
    if S < 0:
        raise MgError(MG_ERR_ARG, "mg_scheme_coefficients")
    g = np.zeros(S)
    lib().mg_scheme_coefficients(scheme.encode(), _ptr(g), S)
    return g


def mg_short_axis_plan(N, precision=MG_FP64):
    """Host-only: the short-axis kernel's axis groups for a grid of axis
    lengths N, as (first_axis, naxes) pairs, with the CTA size and dynamic
    shared memory; None if the grid does not take that kernel."""
    n = np.ascontiguousarray(N, dtype=np.int64)
    first, nax = np.zeros(8, dtype=np.int32), np.zeros(8, dtype=np.int32)
    thr, smem = np.zeros(1, dtype=np.int32), np.zeros(1, dtype=np.int32)
    ng = lib().mg_short_axis_plan(n.size, _ptr(n), precision, _ptr(first), _ptr(nax), _ptr(thr), _ptr(smem))
    if ng < 0:
        raise MgError(MG_ERR_ARG, "mg_short_axis_plan")
    if ng == 0:
        return None
    return {"groups": [(int(first[g]), int(nax[g])) for g in range(ng)], "threads": int(thr[0]),
            "smem_bytes": int(smem[0])}


def mg_morse_mean(Dm, a, re, mass, hbar=1.0):
    return float(lib().mg_morse_mean(Dm, a, re, mass, hbar))


def mg_probe_fma_rate(precision=MG_FP64, stream=None):
    """Measured FMA rate of the current GPU in TFLOP/s (FP64 or FP32)."""
    out = np.zeros(1)
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(lib().mg_probe_fma_rate(precision, s, _ptr(out)), "mg_probe_fma_rate")
    return float(out[0])


def mg_probe_tc_dft16(x, pre, post=None, split=1, inverse=False, stream=None, out=None):
    """The 16-point DFT with diagonal multipliers on the tensor cores
    (mg_probe_tc_dft16): x a CUDA complex64 tensor of shape (lines, 16);
    pre, post 16 complex values (post None for 1); split 1 = 3xTF32,
    2 = BF16x3, 0 = the FP32 register DFT for comparison.  Returns y like x
    (written to out when given)."""
    import torch

    xx = x.contiguous()
    if xx.dtype != torch.complex64 or not xx.is_cuda or xx.shape[-1] != 16:
        raise ValueError("x must be a CUDA complex64 tensor of lines of 16 values")
    y = torch.empty_like(xx) if out is None else out
    if y.shape != xx.shape or y.dtype != xx.dtype or not y.is_contiguous():
        raise ValueError("out must be a contiguous tensor like x")
    pr = np.ascontiguousarray(np.asarray(pre, dtype=np.complex128).reshape(16))
    po = None if post is None else np.ascontiguousarray(np.asarray(post, dtype=np.complex128).reshape(16))
    st = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(lib().mg_probe_tc_dft16(int(split), int(bool(inverse)), ctypes.c_void_p(xx.data_ptr()),
                                   ctypes.c_void_p(y.data_ptr()), xx.numel() // 16, _ptr(pr),
                                   _ptr(po) if po is not None else None, st), "mg_probe_tc_dft16")
    return y


def mg_probe_expi(theta, stream=None):
    """The kernels' table-driven (sin, cos) at the CUDA float64 tensor theta."""
    import torch

    th = theta.contiguous()
    if th.dtype != torch.float64 or not th.is_cuda:
        raise ValueError("theta must be a CUDA float64 tensor")
    s, c = torch.empty_like(th), torch.empty_like(th)
    st = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(lib().mg_probe_expi(ctypes.c_void_p(th.data_ptr()), ctypes.c_void_p(s.data_ptr()),
                               ctypes.c_void_p(c.data_ptr()), th.numel(), st), "mg_probe_expi")
    return s, c


class Propagator:
    """One grid context whose state and workspace live in torch CUDA tensors."""

    def __init__(self, N, dq, minv=None, hbar=1.0, precision=MG_FP64, device=None, stream=None, flags=0):
        import torch

        self.torch = torch
        self.N = tuple(int(v) for v in N)
        self.D = len(self.N)
        self.npts = int(np.prod(self.N))
        self.dq = _f64(dq, self.D)
        if minv is None:
            minv = np.ones(self.D)
        minv = np.asarray(minv, dtype=np.float64)
        self.minv = _f64(np.diag(minv) if minv.ndim == 1 else minv, self.D * self.D)
        self.hbar = float(hbar)
        self.precision = precision
        self.device = torch.device(device or "cuda")
        ws = mg_workspace_bytes(self.N, precision)
        if ws == 0:
            raise MgError(MG_ERR_UNSUPPORTED, "mg_workspace_bytes")
        fdt = torch.float64 if precision == MG_FP64 else torch.float32
        self.psi = torch.zeros(2 * self.npts, dtype=fdt, device=self.device)
        self.work = torch.zeros(ws, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        n = np.ascontiguousarray(self.N, dtype=np.int64)
        h = ctypes.c_void_p()
        rc = lib().mg_create_ex(ctypes.byref(h), self.D, _ptr(n), _ptr(self.dq), _ptr(self.minv), self.hbar,
                                precision, ctypes.c_void_p(self.psi.data_ptr()),
                                ctypes.c_void_p(self.work.data_ptr()), ws, ctypes.c_void_p(self.stream.cuda_stream),
                                int(flags))
        _check(rc, "mg_create_ex")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().mg_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def set_potential(self, kind, params):
        p = _f64(params)
        _check(lib().mg_set_potential(self._h, kind, _ptr(p), p.size), "mg_set_potential")
        self._pot_kind = kind
        self._pot_params = [float(v) for v in p]

    def set_state(self, psi, q, p, t=0.0):
        q, p = _f64(q, self.D), _f64(p, self.D)
        if psi is None:
            ptr = None
        else:
            arr = np.ascontiguousarray(psi, dtype=np.complex128).reshape(self.N)
            ptr = _ptr(arr)
        _check(lib().mg_set_state(self._h, ptr, _ptr(q), _ptr(p), float(t)), "mg_set_state")

    def upload_u(self, host_u, q, p, t=0.0):
        """mg_upload_u: host_u is a CPU tensor (ideally pinned) of the storage
        dtype (complex128 / complex64) holding the scaled state u."""
        q, p = _f64(q, self.D), _f64(p, self.D)
        self._check_host(host_u)
        _check(lib().mg_upload_u(self._h, ctypes.c_void_p(host_u.data_ptr()), _ptr(q), _ptr(p), float(t)),
               "mg_upload_u")

    def download_u(self, host_u):
        """mg_download_u into a CPU tensor like upload_u's; returns (q, p, t)."""
        self._check_host(host_u)
        q, p, t = np.empty(self.D), np.empty(self.D), np.zeros(1)
        _check(lib().mg_download_u(self._h, ctypes.c_void_p(host_u.data_ptr()), _ptr(q), _ptr(p), _ptr(t)),
               "mg_download_u")
        return q, p, float(t[0])

    def _check_host(self, a):
        torch = self.torch
        want = torch.complex128 if self.precision == MG_FP64 else torch.complex64
        if a.is_cuda or a.dtype != want or a.numel() != self.npts or not a.is_contiguous():
            raise ValueError(f"host buffer must be a contiguous CPU {want} tensor of {self.npts} values")

    def set_separable(self, factors, q_ctr, p_ctr):
        """factors: per axis ('gauss', q0, p0, sigma) or ('morse', Dm, a, re, mass)."""
        kinds = np.zeros(self.D, dtype=np.int32)
        params = np.zeros((self.D, 4))
        for l, f in enumerate(factors):
            kinds[l] = {"gauss": 0, "morse": 1}[f[0]]
            params[l, : len(f) - 1] = f[1:]
        q, p = _f64(q_ctr, self.D), _f64(p_ctr, self.D)
        _check(lib().mg_set_separable(self._h, _ptr(kinds), _ptr(params), _ptr(q), _ptr(p)), "mg_set_separable")

    def propagate(self, n_steps, dt, scheme="strang", split=MG_TVT, grid_motion=MG_GRID_ADAPTIVE):
        rc = lib().mg_propagate(self._h, int(n_steps), float(dt), scheme.encode(), split, grid_motion)
        _check(rc, "mg_propagate")

    def sync(self):
        _check(lib().mg_sync(self._h), "mg_sync")

    def test_stuck_barrier(self, limit_s):
        """Failure-detection test hook (mg_test_stuck_barrier): the next
        propagate() cannot pass its first grid barrier and gives up after
        limit_s seconds with MG_ERR_TIMEOUT."""
        _check(lib().mg_test_stuck_barrier(self._h, float(limit_s)), "mg_test_stuck_barrier")

    def inner_product(self, other):
        """<psi_self | psi_other>, other's state interpolated onto this grid."""
        re, im = np.zeros(1), np.zeros(1)
        _check(lib().mg_inner_product(self._h, other._h, _ptr(re), _ptr(im)), "mg_inner_product")
        return complex(re[0], im[0])

    def regrid(self, q, p):
        """Carry the state onto the grid centred at (q, p) (trigonometric interpolation)."""
        q, p = _f64(q, self.D), _f64(p, self.D)
        _check(lib().mg_regrid(self._h, _ptr(q), _ptr(p)), "mg_regrid")

    def get_state(self, want_psi=True):
        psi = np.empty(self.N, dtype=np.complex128) if want_psi else None
        q, p, t = np.empty(self.D), np.empty(self.D), np.zeros(1)
        rc = lib().mg_get_state(self._h, _ptr(psi) if want_psi else None, _ptr(q), _ptr(p), _ptr(t))
        _check(rc, "mg_get_state")
        return psi, q, p, float(t[0])

    def observables(self):
        n, e = np.zeros(1), np.zeros(1)
        mq, mp = np.empty(self.D), np.empty(self.D)
        _check(lib().mg_get_observables(self._h, _ptr(n), _ptr(e), _ptr(mq), _ptr(mp)), "mg_get_observables")
        return float(n[0]), float(e[0]), mq, mp

    def adjoint(self, n_steps, dt, scheme, ubar, qbar, pbar, split=MG_TVT, grid_motion=MG_GRID_ADAPTIVE):
        """Cotangents at the start of the last propagate(n_steps, dt, scheme, ...)
        call given those at its end (see mg_adjoint).  ubar: complex array of the
        grid's shape (numpy) or a CUDA complex128 tensor; returns
        (ubar0 as numpy complex128, qbar0, pbar0, thetabar); the context's state
        is rewound to the start of that call."""
        torch = self.torch
        if isinstance(ubar, torch.Tensor):
            ub = ubar.detach().to(self.device, torch.complex128).contiguous().clone()
        else:
            ub = torch.from_numpy(np.ascontiguousarray(ubar, dtype=np.complex128)).to(self.device)
        if ub.numel() != int(np.prod(self.N)):
            raise ValueError("ubar must have one complex value per grid point")
        qb, pb = _f64(qbar, self.D).copy(), _f64(pbar, self.D).copy()
        nth = 4 if getattr(self, "_pot_kind", None) == MG_POT_ATOM_DIATOM else 0
        th = np.zeros(max(nth, 1))
        rc = lib().mg_adjoint(self._h, int(n_steps), float(dt), scheme.encode(), split, grid_motion,
                              ctypes.c_void_p(ub.data_ptr()), _ptr(qb), _ptr(pb), _ptr(th), nth)
        _check(rc, "mg_adjoint")
        return ub.cpu().numpy().reshape(self.N), qb, pb, th[:nth]

    @property
    def launches(self):
        return int(lib().mg_kernel_launches(self._h))

    @property
    def path(self):
        """Kernel of mg_propagate: 0 general, 1 short-axis, 2 short-axis with TMA
        copies."""
        return int(lib().mg_propagate_path(self._h))

    @property
    def tables_in_workspace(self):
        """mg_tables_in_workspace: which per-axis tables the general kernel
        reads from the workspace instead of shared memory (bits 1 and 2)."""
        return int(lib().mg_tables_in_workspace(self._h))


def mg_batch_workspace_bytes(nprob):
    return int(lib().mg_batch_workspace_bytes(int(nprob)))


class Batch:
    """Many Propagator contexts advanced together by one batched launch
    (mg_batch_*).  The propagators must share one precision and one stream and
    stay alive with the batch (it keeps references to them)."""

    def __init__(self, props, cluster=0, tile_bytes=None, radix_max=None):
        import torch

        self.props = list(props)
        n = len(self.props)
        if n == 0:
            raise ValueError("empty batch")
        self.n = n
        self.device = self.props[0].device
        self.stream = self.props[0].stream
        ws = mg_batch_workspace_bytes(n)
        self.work = torch.zeros(ws, dtype=torch.uint8, device=self.device)
        handles = (ctypes.c_void_p * n)(*[p.handle.value for p in self.props])
        tb = None if tile_bytes is None else np.ascontiguousarray(tile_bytes, dtype=np.int32)
        rm = None if radix_max is None else np.ascontiguousarray(radix_max, dtype=np.int32)
        for a in (tb, rm):
            if a is not None and a.size != n:
                raise ValueError("tile_bytes and radix_max take one value per problem")
        h = ctypes.c_void_p()
        rc = lib().mg_batch_create(ctypes.byref(h), n, ctypes.cast(handles, ctypes.c_void_p), int(cluster),
                                   _ptr(tb) if tb is not None else None, _ptr(rm) if rm is not None else None,
                                   ctypes.c_void_p(self.work.data_ptr()), ws)
        _check(rc, "mg_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().mg_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def propagate(self, n_steps, dt, scheme="strang", split=MG_TVT, grid_motion=MG_GRID_ADAPTIVE):
        """dt: one time step for all problems, or one per problem."""
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (self.n,)))
        rc = lib().mg_batch_propagate(self._h, int(n_steps), _ptr(d), scheme.encode(), split, grid_motion)
        _check(rc, "mg_batch_propagate")

    def sync(self):
        """Wait for the batch; raises MgError naming the first failed problem."""
        idx = np.full(1, -1, dtype=np.int32)
        rc = lib().mg_batch_sync(self._h, _ptr(idx))
        if rc != MG_OK:
            raise MgError(rc, f"mg_batch_sync (problem {int(idx[0])})")

    def info(self):
        c, t, s = (np.zeros(1, dtype=np.int32) for _ in range(3))
        l = np.zeros(1, dtype=np.int64)
        _check(lib().mg_batch_info(self._h, _ptr(c), _ptr(t), _ptr(s), _ptr(l)), "mg_batch_info")
        return {"cluster": int(c[0]), "teams": int(t[0]), "smem_bytes": int(s[0]), "launches": int(l[0])}


def mg_propagate_noalloc(N, dq, minv, hbar, pot_kind, pot_params, d_psi, q, p, n_steps, dt, scheme="strang",
                         split=MG_TVT, grid_motion=MG_GRID_ADAPTIVE, stream=None):
    """Propagate without any device allocation by the library (for callers that
    cannot allocate device memory).  d_psi: CUDA float64 tensor of 2*prod(N)
    values holding the scaled state, updated in place; q, p: float64 numpy
    arrays of the grid centres, updated in place.  Synchronises the stream."""
    L = lib()
    fn = L.mg_propagate_noalloc
    vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    fn.argtypes = [i32, vp, vp, vp, d, i32, vp, i32, vp, vp, vp, i64, d, ctypes.c_char_p, i32, i32, vp]
    fn.restype = i32
    n = np.ascontiguousarray(N, dtype=np.int64)
    D = n.size
    dqa = _f64(dq, D)
    mi = np.asarray(minv, dtype=np.float64)
    mi = _f64(np.diag(mi) if mi.ndim == 1 else mi, D * D)
    pp = _f64(pot_params)
    for a in (q, p):
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous and a.size == D):
            raise ValueError("q and p must be contiguous float64 arrays of D values (updated in place)")
    if d_psi.dtype != __import__("torch").float64 or d_psi.numel() != 2 * int(np.prod(n)) or not d_psi.is_cuda:
        raise ValueError("d_psi must be a CUDA float64 tensor of 2*prod(N) values")
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    rc = fn(D, _ptr(n), _ptr(dqa), _ptr(mi), float(hbar), pot_kind, _ptr(pp), pp.size,
            ctypes.c_void_p(d_psi.data_ptr()), _ptr(q), _ptr(p), int(n_steps), float(dt), scheme.encode(),
            split, grid_motion, s)
    _check(rc, "mg_propagate_noalloc")
