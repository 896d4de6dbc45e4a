"""Thin Python binding of the swiftcl C ABI (include/swiftcl.h).

Argument marshalling only: every function forwards to the C symbol of the same name.  Arrays
may be numpy arrays (host memory) or torch tensors (host or CUDA memory of the context's
device); they must be C-contiguous and of the documented dtype (float64 / int32).  A failing
call raises SwiftClError with the library's message.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib

SWCL_OK = 0
(SWCL_ERR_INVALID_ARG, SWCL_ERR_UNSUPPORTED, SWCL_ERR_OOM_BUDGET, SWCL_ERR_CUDA, SWCL_ERR_TIMEOUT,
 SWCL_ERR_NONFINITE, SWCL_ERR_STATE) = -1, -2, -3, -4, -5, -6, -7
SWCL_DENSITY, SWCL_LENSING, SWCL_MAGNIFICATION, SWCL_RSD = 0, 1, 2, 3
SWCL_FP64, SWCL_3XTF32, SWCL_SPLIT_BF16, SWCL_TF32X6 = 0, 1, 2, 3
SWCL_Q_WORKSPACE_BYTES, SWCL_Q_RECOMPUTE, SWCL_Q_N_HALF, SWCL_Q_KERNEL_LAUNCHES = 1, 2, 3, 4
SWCL_Q_PROFILE_RANK, SWCL_Q_TILE_FWD, SWCL_Q_TILE_ADJ = 5, 6, 7
PRECISIONS = {"fp64": SWCL_FP64, "3xtf32": SWCL_3XTF32, "bf16x9": SWCL_SPLIT_BF16, "tf32x6": SWCL_TF32X6}


class SwiftClError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("swiftcl status %d (%s): %s" % (status, strerror(status), msg))
        self.status = status


def _ptr(a, dtype):
    """(pointer, keepalive) for a numpy array / torch tensor / None."""
    if a is None:
        return None, None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            want = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
            if a.dtype != want or not a.is_contiguous():
                raise TypeError("tensor must be contiguous %s" % want)
            return ctypes.c_void_p(a.data_ptr()), a
    except ImportError:  # pragma: no cover
        pass
    arr = np.ascontiguousarray(a, dtype=dtype)
    return ctypes.c_void_p(arr.ctypes.data), arr


def strerror(status: int) -> str:
    return _lib.load().swcl_strerror(status).decode()


def _check(ctx, status):
    if status != SWCL_OK:
        msg = _lib.load().swcl_last_error(ctx).decode() if ctx else ""
        raise SwiftClError(status, msg)


def swcl_create(device: int = 0, mem_budget_bytes: int = 0, stream=None):
    lib = _lib.load()
    out = ctypes.c_void_p()
    st = lib.swcl_create(ctypes.byref(out), device, mem_budget_bytes,
                         ctypes.c_void_p(stream) if stream else None)
    _check(None, st)
    return out


def swcl_destroy(ctx):
    _check(None, _lib.load().swcl_destroy(ctx))


def swcl_set_grids(ctx, chi_min, chi_max, N, k, ells, knots):
    pk, a = _ptr(k, np.float64)
    pe, b = _ptr(ells, np.int32)
    pn, c = _ptr(knots, np.float64)
    _check(ctx, _lib.load().swcl_set_grids(ctx, chi_min, chi_max, N, pk, len(a), pe, len(b), pn, len(c)))


def swcl_set_tracers(ctx, kind, fft_bias, taper_chi=None, taper_c=None):
    pk, a = _ptr(kind, np.int32)
    pb, _b = _ptr(fft_bias, np.float64)
    pt, _t = _ptr(taper_chi, np.float64)
    pc, _c = _ptr(taper_c, np.float64)
    _check(ctx, _lib.load().swcl_set_tracers(ctx, len(a), pk, pb, pt, pc))


def swcl_set_windows(ctx, n_walk, W, D=None, B=None):
    pw, _w = _ptr(W, np.float64)
    pd, _d = _ptr(D, np.float64)
    pb, _b = _ptr(B, np.float64)
    _check(ctx, _lib.load().swcl_set_windows(ctx, n_walk, pw, pd, pb))


def swcl_set_window_samples(ctx, n_walk, W):
    pw, _w = _ptr(W, np.float64)
    _check(ctx, _lib.load().swcl_set_window_samples(ctx, n_walk, pw))


def swcl_set_power(ctx, n_walk, P, amp):
    pp, _p = _ptr(P, np.float64)
    pa, _a = _ptr(amp, np.float64)
    _check(ctx, _lib.load().swcl_set_power(ctx, n_walk, pp, pa))


def swcl_set_ell_lists(ctx, offsets=None, ell_idx=None):
    po, _o = _ptr(offsets, np.int32)
    pi, _i = _ptr(ell_idx, np.int32)
    _check(ctx, _lib.load().swcl_set_ell_lists(ctx, po, pi))


def swcl_compute_cl(ctx, precision, C_out):
    pc, keep = _ptr(C_out, np.float64)
    if keep is not C_out:
        raise TypeError("C_out must be a contiguous float64 array or tensor (written in place)")
    _check(ctx, _lib.load().swcl_compute_cl(ctx, precision, pc))


def swcl_vjp(ctx, precision, C_bar, P_bar=None, amp_bar=None, W_bar=None):
    outs = []
    for o in (P_bar, amp_bar, W_bar):
        p, keep = _ptr(o, np.float64)
        if o is not None and keep is not o:
            raise TypeError("VJP outputs must be contiguous float64 arrays or tensors")
        outs.append(p)
    pc, _c = _ptr(C_bar, np.float64)
    _check(ctx, _lib.load().swcl_vjp(ctx, precision, pc, *outs))


def swcl_set_limber(ctx, ell_switch):
    """Multipoles >= ell_switch take the Limber branch (Eq. 2.19); 0 turns it off."""
    _check(ctx, _lib.load().swcl_set_limber(ctx, int(ell_switch)))


def swcl_jvp(ctx, precision, n_dir, C_dot, P_dot=None, amp_dot=None, W_dot=None):
    """Forward-mode derivative of C along n_dir tangents (each input may be None = zero)."""
    pc, keep = _ptr(C_dot, np.float64)
    if keep is not C_dot:
        raise TypeError("C_dot must be a contiguous float64 array or tensor (written in place)")
    pp, _p = _ptr(P_dot, np.float64)
    pa, _a = _ptr(amp_dot, np.float64)
    pw, _w = _ptr(W_dot, np.float64)
    _check(ctx, _lib.load().swcl_jvp(ctx, precision, n_dir, pp, pa, pw, pc))


def swcl_gaussian_fisher(ctx, X, modes, F, noise=None):
    """F[a][b] = sum_l (modes_l/2) Tr[Ct^-1 X_a Ct^-1 X_b] with Ct = C + diag(noise)."""
    pf, keep = _ptr(F, np.float64)
    if keep is not F:
        raise TypeError("F must be a contiguous float64 array or tensor (written in place)")
    px, a = _ptr(X, np.float64)
    pm, _m = _ptr(modes, np.float64)
    pn, _n = _ptr(noise, np.float64)
    _check(ctx, _lib.load().swcl_gaussian_fisher(ctx, int(F.shape[0]), px, pn, pm, pf))


def swcl_compute_batched(ctx, precision, C_out, C_bar=None, P_bar=None, amp_bar=None, W_bar=None):
    """Forward (+ VJP when C_bar is given) for all walkers as one CUDA-graph replay; device
    tensors only."""
    ptrs = []
    for a in (C_out, C_bar, P_bar, amp_bar, W_bar):
        p, _k = _ptr(a, np.float64)
        ptrs.append(p)
    _check(ctx, _lib.load().swcl_compute_batched(ctx, precision, *ptrs))


def swcl_step_host(ctx, precision, C_out, W=None, P=None, amp=None, C_bar=None, P_bar=None,
                   amp_bar=None, W_bar=None):
    """One sampler step with page-locked host arrays (pinned torch tensors): inputs in, forward
    (+ VJP when C_bar is given), results out, in one CUDA-graph replay; returns when the host
    outputs are written."""
    ptrs = []
    for a in (W, P, amp, C_bar, C_out, P_bar, amp_bar, W_bar):
        p, _k = _ptr(a, np.float64)
        ptrs.append(p)
    _check(ctx, _lib.load().swcl_step_host(ctx, precision, *ptrs))


class HostStep:
    """swcl_step_host with its arguments prepared once: the page-locked host tensors are checked
    and their addresses taken at construction, and each call of the object runs one step (inputs
    in, forward + VJP, results out) without re-marshalling.  The tensors must stay alive and in
    place; write new parameters into them between steps."""

    def __init__(self, ctx, precision, C_out, W=None, P=None, amp=None, C_bar=None, P_bar=None,
                 amp_bar=None, W_bar=None):
        self._keep = []
        self._args = []
        for a in (W, P, amp, C_bar, C_out, P_bar, amp_bar, W_bar):
            p, k = _ptr(a, np.float64)
            self._keep.append(k)
            self._args.append(p)
        self._ctx = ctx
        self._precision = precision
        self._fn = _lib.load().swcl_step_host

    def __call__(self):
        st = self._fn(self._ctx, self._precision, *self._args)
        if st != SWCL_OK:
            _check(self._ctx, st)


def swcl_profile_enable(ctx, enable=True):
    _check(ctx, _lib.load().swcl_profile_enable(ctx, 1 if enable else 0))


def swcl_profile_reset(ctx):
    _check(ctx, _lib.load().swcl_profile_reset(ctx))


def swcl_profile_read(ctx, max_entries=64):
    """{kernel name: (launches, total device ms)} accumulated since the last reset."""
    names = ctypes.create_string_buffer(32 * max_entries)
    launches = (ctypes.c_int64 * max_entries)()
    ms = (ctypes.c_double * max_entries)()
    n = ctypes.c_int()
    _check(ctx, _lib.load().swcl_profile_read(ctx, max_entries, names, launches, ms, ctypes.byref(n)))
    out = {}
    for i in range(min(n.value, max_entries)):
        nm = names.raw[32 * i:32 * (i + 1)].split(b"\0")[0].decode()
        out[nm] = (int(launches[i]), float(ms[i]))
    return out


SWCL_DBG_COEF, SWCL_DBG_DELTA, SWCL_DBG_GTAB, SWCL_DBG_PHASE, SWCL_DBG_UNIT = 1, 2, 3, 4, 5


def swcl_debug_read(ctx, what):
    """Internal array of the last compute as a flat float64 numpy array (complex interleaved)."""
    lib = _lib.load()
    n = ctypes.c_int64()
    _check(ctx, lib.swcl_debug_read(ctx, what, None, ctypes.byref(n)))
    out = np.empty(n.value, dtype=np.float64)
    _check(ctx, lib.swcl_debug_read(ctx, what, ctypes.c_void_p(out.ctypes.data), ctypes.byref(n)))
    return out


def swcl_fftlog_noalloc(n_walk, N_tr, N_I, N, chi_min, chi_max, kind, fft_bias, taper_chi, taper_c,
                        W, D, B, coef, stream=None):
    """FFTLog coefficients without a context or any device allocation (see include/swiftcl.h).

    kind, fft_bias: host arrays of N_tr entries; taper_chi [N_tr][N], taper_c [N_tr][N/2+1],
    W [n_walk][N_tr][N], D [N_I][N], B [N_tr][N_I][N], coef [n_walk][N_tr][N_I][N/2+1][2]:
    contiguous float64 CUDA tensors of the current device (taper_*, B may be None).  The C call
    takes plain pointers and cannot tell a host array, a tensor of another device or a short
    buffer from a good one, so each of these is checked here and a TypeError or ValueError is
    raised before the library is called.  Returns the status code (0 = ok) instead of raising, so
    a caller can test the size limit."""
    import torch
    n_h = N // 2 + 1
    kind = np.ascontiguousarray(kind, dtype=np.int32)
    fft_bias = np.ascontiguousarray(fft_bias, dtype=np.float64)
    _need(kind, N_tr, "kind [N_tr]")
    _need(fft_bias, N_tr, "fft_bias [N_tr]")
    dev = torch.cuda.current_device()
    sizes = {"taper_chi": (taper_chi, N_tr * N), "taper_c": (taper_c, N_tr * n_h),
             "W": (W, n_walk * N_tr * N), "D": (D, N_I * N), "B": (B, N_tr * N_I * N),
             "coef": (coef, n_walk * N_tr * N_I * n_h * 2)}
    for name, (x, n) in sizes.items():
        if x is None:
            if name in ("W", "D", "coef"):
                raise ValueError("%s is required" % name)
            continue
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.device.index == dev
                and x.dtype == torch.float64 and x.is_contiguous()):
            raise TypeError("%s must be a contiguous float64 CUDA tensor on device %d" % (name, dev))
        _need(x, n, name)
    pk, _k = _ptr(kind, np.int32)
    pb, _b = _ptr(fft_bias, np.float64)
    args = [_ptr(x, np.float64) for x in (taper_chi, taper_c, W, D, B, coef)]
    return _lib.load().swcl_fftlog_noalloc(n_walk, N_tr, N_I, N, chi_min, chi_max, pk, pb,
                                           *[a[0] for a in args],
                                           ctypes.c_void_p(stream) if stream else None)


def swcl_selftest_wait_timeout(ctx):
    """Runs the bounded-wait self-test; returns (status, cycles) without raising."""
    v = ctypes.c_int64()
    st = _lib.load().swcl_selftest_wait_timeout(ctx, ctypes.byref(v))
    return st, v.value


def swcl_sync(ctx):
    _check(ctx, _lib.load().swcl_sync(ctx))


def swcl_query(ctx, key):
    v = ctypes.c_int64()
    _check(ctx, _lib.load().swcl_query(ctx, key, ctypes.byref(v)))
    return v.value


def swcl_last_error(ctx) -> str:
    return _lib.load().swcl_last_error(ctx).decode()


def _need(a, n, what):
    """ValueError unless array or tensor `a` (None allowed) holds exactly n elements: the C ABI
    takes plain pointers, so the sizes are checked here, where the context's shapes are known."""
    if a is None or n is None:
        return
    size = a.numel() if hasattr(a, "numel") else np.asarray(a).size
    if size != n:
        raise ValueError("%s has %d elements, expected %d" % (what, size, n))


class Context:
    """Owning wrapper: one swcl_ctx on one device.  Its methods check every array's element count
    against the shapes set so far before calling the library (the functions above do not)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, stream=None):
        self.ptr = swcl_create(device, mem_budget_bytes, stream)
        self.n_tr = self.n_ell = self.n_k = self.N = self.n_knots = 0
        self.n_walk = 1
        self.n_out = 0

    def _shape(self, *dims):
        """Product of dims, or None (no check) while a dimension is still unset."""
        n = 1
        for d in dims:
            if not d:
                return None
            n *= d
        return n

    def close(self):
        if self.ptr:
            swcl_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_grids(self, chi_min, chi_max, N, k, ells, knots):
        swcl_set_grids(self.ptr, chi_min, chi_max, N, k, ells, knots)
        self.N, self.n_k, self.n_ell, self.n_knots = N, len(k), len(ells), len(knots)
        self.n_out = self.n_walk * self.n_ell

    def set_tracers(self, kind, fft_bias, taper_chi=None, taper_c=None):
        swcl_set_tracers(self.ptr, kind, fft_bias, taper_chi, taper_c)
        self.n_tr = len(kind)

    def set_windows(self, W, D=None, B=None):
        n_walk = 1 if W.ndim == 2 else W.shape[0]
        _need(W, self._shape(n_walk, self.n_tr, self.N), "W [n_walk][N_tr][N]")
        _need(D, self._shape(self.n_knots, self.N), "D [N_knots][N]")
        _need(B, self._shape(self.n_tr, self.n_knots, self.N), "B [N_tr][N_knots][N]")
        swcl_set_windows(self.ptr, n_walk, W, D, B)
        self.n_walk = n_walk
        self.n_out = n_walk * self.n_ell

    def set_window_samples(self, W):
        """New window samples for the same walkers, keeping D and B (no host wait)."""
        _need(W, self._shape(self.n_walk, self.n_tr, self.N), "W [n_walk][N_tr][N]")
        swcl_set_window_samples(self.ptr, self.n_walk, W)

    def set_power(self, P, amp):
        n_walk = 1 if P.ndim == 1 else P.shape[0]
        _need(P, self._shape(n_walk, self.n_k), "P [n_walk][N_k]")
        _need(amp, self._shape(n_walk, self.n_tr), "amp [n_walk][N_tr]")
        swcl_set_power(self.ptr, n_walk, P, amp)
        self.n_walk = n_walk
        self.n_out = n_walk * self.n_ell

    def set_ell_lists(self, lists=None):
        if lists is None:
            swcl_set_ell_lists(self.ptr, None, None)
            self.n_out = self.n_walk * self.n_ell
            return
        off = np.zeros(len(lists) + 1, dtype=np.int32)
        off[1:] = np.cumsum([len(x) for x in lists])
        idx = np.concatenate([np.asarray(x, dtype=np.int32) for x in lists]) if lists else np.zeros(0, np.int32)
        swcl_set_ell_lists(self.ptr, off, idx)
        self.n_out = int(off[-1])

    def compute_cl(self, precision=SWCL_FP64, out=None):
        if out is None:
            out = np.empty((self.n_out, self.n_tr, self.n_tr))
        _need(out, self._shape(self.n_out, self.n_tr, self.n_tr), "C_out [outputs][N_tr][N_tr]")
        swcl_compute_cl(self.ptr, precision, out)
        return out

    def vjp(self, C_bar, precision=SWCL_FP64, want_W=True):
        _need(C_bar, self._shape(self.n_out, self.n_tr, self.n_tr), "C_bar [outputs][N_tr][N_tr]")
        P_bar = np.empty((self.n_walk, self.n_k))
        amp_bar = np.empty((self.n_walk, self.n_tr))
        W_bar = np.empty((self.n_walk, self.n_tr, self.N)) if want_W else None
        swcl_vjp(self.ptr, precision, C_bar, P_bar, amp_bar, W_bar)
        return P_bar, amp_bar, W_bar

    def set_limber(self, ell_switch):
        swcl_set_limber(self.ptr, ell_switch)

    def jvp(self, P_dot=None, amp_dot=None, W_dot=None, precision=SWCL_FP64):
        """dC [n_dir][N_ell][N_tr][N_tr] along tangents P_dot [n_dir][N_k], amp_dot [n_dir][N_tr],
        W_dot [n_dir][N_tr][N] (None = zero) at the context's single parameter point."""
        n_dir = next(len(x) for x in (P_dot, amp_dot, W_dot) if x is not None)
        _need(P_dot, self._shape(n_dir, self.n_k), "P_dot [n_dir][N_k]")
        _need(amp_dot, self._shape(n_dir, self.n_tr), "amp_dot [n_dir][N_tr]")
        _need(W_dot, self._shape(n_dir, self.n_tr, self.N), "W_dot [n_dir][N_tr][N]")
        out = np.empty((n_dir, self.n_ell, self.n_tr, self.n_tr))
        swcl_jvp(self.ptr, precision, n_dir, out, P_dot, amp_dot, W_dot)
        return out

    def gaussian_fisher(self, X, modes, noise=None):
        """Fisher matrix (X = dC/dtheta) or chi^2 (X = C - C_data) with the Gaussian covariance
        of the last forward pass plus diagonal noise; modes[N_ell] = (2l+1) f_sky (bin width)."""
        F = np.empty((len(X), len(X)))
        _need(X, self._shape(len(X), self.n_ell, self.n_tr, self.n_tr), "X [n_x][N_ell][N_tr][N_tr]")
        _need(modes, self._shape(self.n_ell), "modes [N_ell]")
        _need(noise, self._shape(self.n_tr), "noise [N_tr]")
        swcl_gaussian_fisher(self.ptr, X, modes, F, noise)
        return F

    def query(self, key):
        return swcl_query(self.ptr, key)

    def sync(self):
        swcl_sync(self.ptr)
