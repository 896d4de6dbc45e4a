"""ctypes loader of libswiftcl.so: argument types of every exported C symbol.

The library must have been built (``paper_2505_22718_gb300.build.build()``); there is no
fallback implementation, so a missing or unloadable library raises at import time.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libswiftcl.so")

c_int, c_double, c_void_p, c_size_t = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
c_int64 = ctypes.c_int64

# name -> (restype, argtypes); mirrors include/swiftcl.h
SIGNATURES = {
    "swcl_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_size_t, c_void_p]),
    "swcl_destroy": (c_int, [c_void_p]),
    "swcl_set_grids": (c_int, [c_void_p, c_double, c_double, c_int, c_void_p, c_int, c_void_p, c_int,
                               c_void_p, c_int]),
    "swcl_set_tracers": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "swcl_set_windows": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "swcl_set_window_samples": (c_int, [c_void_p, c_int, c_void_p]),
    "swcl_set_power": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "swcl_set_ell_lists": (c_int, [c_void_p, c_void_p, c_void_p]),
    "swcl_compute_cl": (c_int, [c_void_p, c_int, c_void_p]),
    "swcl_vjp": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "swcl_set_limber": (c_int, [c_void_p, c_int]),
    "swcl_jvp": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "swcl_gaussian_fisher": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "swcl_sync": (c_int, [c_void_p]),
    "swcl_selftest_wait_timeout": (c_int, [c_void_p, c_void_p]),
    "swcl_compute_batched": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "swcl_step_host": (c_int, [c_void_p, c_int] + [c_void_p] * 8),
    "swcl_debug_read": (c_int, [c_void_p, c_int, c_void_p, ctypes.POINTER(c_int64)]),
    "swcl_fftlog_noalloc": (c_int, [c_int, c_int, c_int, c_int, c_double, c_double, c_void_p, c_void_p,
                                    c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                    c_void_p]),
    "swcl_profile_enable": (c_int, [c_void_p, c_int]),
    "swcl_profile_read": (c_int, [c_void_p, c_int, c_void_p, ctypes.POINTER(c_int64),
                                  ctypes.POINTER(c_double), ctypes.POINTER(c_int)]),
    "swcl_profile_reset": (c_int, [c_void_p]),
    "swcl_query": (c_int, [c_void_p, c_int, ctypes.POINTER(c_int64)]),
    "swcl_last_error": (ctypes.c_char_p, [c_void_p]),
    "swcl_strerror": (ctypes.c_char_p, [c_int]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library once and attach the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libswiftcl.so is not built (%s); run __graft_entry__.build() or "
                          "python -m paper_2505_22718_gb300.build" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
