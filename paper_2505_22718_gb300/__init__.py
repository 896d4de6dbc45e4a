"""GB300-native (sm_103a) beyond-Limber FFTLog angular power spectra (arXiv:2505.22718).

The compute path is the CUDA library libswiftcl.so (C ABI in include/swiftcl.h).  This package
holds its sources (csrc/), its build script (build.py), the ctypes binding (api.py) and a
torch.autograd.Function wrapper (autograd.py).  There is no fallback implementation: calls fail
with ImportError when the library has not been built.
"""
from .api import (  # noqa: F401
    Context, SwiftClError, PRECISIONS, SWCL_OK, SWCL_ERR_INVALID_ARG, SWCL_ERR_UNSUPPORTED,
    SWCL_ERR_OOM_BUDGET, SWCL_ERR_CUDA, SWCL_ERR_TIMEOUT, SWCL_ERR_NONFINITE, SWCL_ERR_STATE,
    SWCL_FP64, SWCL_3XTF32, SWCL_SPLIT_BF16, SWCL_TF32X6, SWCL_DENSITY, SWCL_LENSING,
    SWCL_MAGNIFICATION, SWCL_RSD,
    SWCL_Q_WORKSPACE_BYTES, SWCL_Q_RECOMPUTE, SWCL_Q_N_HALF, SWCL_Q_KERNEL_LAUNCHES,
    SWCL_Q_PROFILE_RANK, SWCL_Q_TILE_FWD, SWCL_Q_TILE_ADJ,
    swcl_create, swcl_destroy, swcl_set_grids, swcl_set_tracers, swcl_set_windows,
    swcl_set_power, swcl_set_window_samples, swcl_set_ell_lists, swcl_compute_cl, swcl_vjp, swcl_sync, swcl_query,
    swcl_selftest_wait_timeout, swcl_jvp, swcl_gaussian_fisher, swcl_set_limber,
    swcl_profile_enable, swcl_profile_read, swcl_profile_reset, swcl_debug_read,
    SWCL_DBG_COEF, SWCL_DBG_DELTA, SWCL_DBG_GTAB, SWCL_DBG_PHASE, SWCL_DBG_UNIT,
    swcl_last_error, strerror, swcl_fftlog_noalloc, swcl_compute_batched, swcl_step_host, HostStep,
)


def __getattr__(name):
    # the torch wrapper is imported lazily so that the ctypes binding works without torch
    if name == "AngularPowerSpectrum":
        from .autograd import AngularPowerSpectrum
        return AngularPowerSpectrum
    raise AttributeError(name)
