"""GB300 (sm_103a) moving-grid split-operator propagator for the
time-dependent Schroedinger equation (Choi & Vanicek, arXiv:1909.06412).

The compute path is the CUDA library ``lib/libmgrid.so`` behind the C-ABI of
``include/mgrid.h``; ``capi`` binds it with ctypes under the same names and
``Propagator`` marshals torch device buffers into it.  There is no CPU
fallback: importing fails loudly if the library has not been built.
"""
from .capi import *  # noqa: F401,F403
from .capi import Propagator, MgError, lib  # noqa: F401
