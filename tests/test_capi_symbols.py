"""The C-ABI library loads on a host without a GPU and exports every entry
point that include/mgrid.h declares; host-only calls behave as documented."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(mg_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1909_06412_gb300 import _build, capi

    if not os.path.exists(capi.LIB_PATH):
        _build.build()
    return capi.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_workspace_size_and_rejections(lib):
    from paper_1909_06412_gb300 import capi

    assert capi.mg_workspace_bytes((256, 256)) >= 256 * 256 * 16
    assert capi.mg_workspace_bytes((10, 7)) == 0      # odd length
    assert capi.mg_workspace_bytes((10, 12)) == 0     # factor 5
    assert capi.mg_workspace_bytes((2048,)) >= 2048 * 16
    assert capi.mg_workspace_bytes((4096,)) == 0      # longer than supported
    assert capi.mg_workspace_bytes((12,) * 8) > 12 ** 8 * 16
    assert capi.mg_workspace_bytes((8, 8), precision=7) == 0


def test_status_strings_and_host_helpers(lib):
    from paper_1909_06412_gb300 import capi

    for code in range(0, -8, -1):
        assert lib.mg_status_string(code)
    # <r> of the Morse ground state (digamma closed form) vs the oracle's quadrature
    import oracle

    m = 0.5 * 1822.888486
    assert abs(capi.mg_morse_mean(0.17, 1.0, 1.4, m) - oracle.morse_mean(0.17, 1.0, 1.4, m)) < 1e-10


def test_create_rejects_bad_arguments_before_touching_the_device(lib):
    import ctypes

    h = ctypes.c_void_p()
    N = np.array([8, 8], dtype=np.int64)
    dq = np.array([0.5, 0.5])
    minv = np.eye(2).ravel()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert lib.mg_create(ctypes.byref(h), 2, p(N), p(dq), p(minv), 1.0, 0, None, None, 0, None) == -1
    fake = ctypes.c_void_p(256)
    # the inverse mass matrix must be symmetric positive definite (eq:KE_operator)
    for bad in ([[1.0, 0.2], [0.3, 1.0]], [[1.0, 2.0], [2.0, 1.0]], [[0.0, 0.0], [0.0, 1.0]]):
        bad = np.array(bad).ravel()
        assert lib.mg_create(ctypes.byref(h), 2, p(N), p(dq), p(bad), 1.0, 0, fake, fake, 1 << 30, None) == -1
    assert lib.mg_create(ctypes.byref(h), 2, p(N), p(dq), p(minv), -1.0, 0, fake, fake, 1 << 30, None) == -1


def test_batch_host_checks(lib):
    import ctypes

    lib.mg_batch_workspace_bytes.argtypes = [ctypes.c_int]
    lib.mg_batch_workspace_bytes.restype = ctypes.c_size_t
    assert lib.mg_batch_workspace_bytes(0) == 0
    assert lib.mg_batch_workspace_bytes(512) > lib.mg_batch_workspace_bytes(1) > 0
    lib.mg_batch_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
    lib.mg_batch_create.restype = ctypes.c_int
    out = ctypes.c_void_p()
    # no contexts / no workspace: rejected before any device call
    assert lib.mg_batch_create(ctypes.byref(out), 1, None, 0, None, None, None, 0) == -1
    assert lib.mg_batch_create(None, 1, None, 0, None, None, None, 0) == -1
    lib.mg_batch_destroy.argtypes = [ctypes.c_void_p]
    lib.mg_batch_destroy.restype = ctypes.c_int
    assert lib.mg_batch_destroy(None) == -1
