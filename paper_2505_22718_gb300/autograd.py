"""torch.autograd wrapper of the library: C_ell(W, P, A) with its hand-written VJP.

    spec = AngularPowerSpectrum(chi_min, chi_max, N, k, ells, knots, kind, fft_bias, D, B=None,
                                precision="bf16x9", device=0)
    C = spec(W, P, amp)            # W [n_walk, N_tr, N], P [n_walk, N_k], amp [n_walk, N_tr]
    C.backward(C_bar)              # W.grad, P.grad, amp.grad from swcl_vjp

Tensors are float64 on the context's CUDA device.  The forward pass and the VJP run in the
library's kernels on the module's own stream, ordered after the caller's current stream and
before it again; this module only moves pointers.  The library keeps the intermediate state
of the last forward pass of a context; when another forward pass has run on the same context
before backward, backward first recomputes the forward pass for its own inputs.
"""
from __future__ import annotations

import torch

from . import api


class _OnLibraryStream:
    """Orders the library's stream after the caller's current stream, and the caller's after it."""

    def __init__(self, spec, *tensors):
        self.spec = spec
        self.tensors = [t for t in tensors if t is not None]

    def __enter__(self):
        cur = torch.cuda.current_stream(self.spec.device)
        self.spec.stream.wait_stream(cur)
        for t in self.tensors:
            t.record_stream(self.spec.stream)
        return self

    def __exit__(self, *exc):
        torch.cuda.current_stream(self.spec.device).wait_stream(self.spec.stream)
        return False


class _SwiftCl(torch.autograd.Function):
    @staticmethod
    def forward(fctx, W, P, amp, spec):
        W, P, amp = W.contiguous(), P.contiguous(), amp.contiguous()
        C = torch.empty((spec.n_walk(W) * spec.n_ell, spec.n_tr, spec.n_tr), dtype=torch.float64,
                        device=W.device)
        with _OnLibraryStream(spec, W, P, amp, C):
            spec._load(W, P, amp)
            api.swcl_compute_cl(spec.ctx.ptr, spec.precision, C)
        spec._generation += 1
        fctx.spec = spec
        fctx.generation = spec._generation
        fctx.save_for_backward(W, P, amp)
        return C

    @staticmethod
    def backward(fctx, C_bar):
        spec = fctx.spec
        W, P, amp = fctx.saved_tensors
        C_bar = C_bar.contiguous()
        P_bar = torch.empty_like(P) if fctx.needs_input_grad[1] else None
        A_bar = torch.empty_like(amp) if fctx.needs_input_grad[2] else None
        W_bar = torch.empty_like(W) if fctx.needs_input_grad[0] else None
        with _OnLibraryStream(spec, W, P, amp, C_bar, P_bar, A_bar, W_bar):
            if spec._generation != fctx.generation:
                # another forward pass ran on this context: rebuild this one's state first
                spec._load(W, P, amp)
                scratch = torch.empty_like(C_bar)
                scratch.record_stream(spec.stream)
                api.swcl_compute_cl(spec.ctx.ptr, spec.precision, scratch)
                spec._generation += 1
            api.swcl_vjp(spec.ctx.ptr, spec.precision, C_bar, P_bar, A_bar, W_bar)
        return W_bar, P_bar, A_bar, None


class AngularPowerSpectrum(torch.nn.Module):
    """C_ell^{ij} of Eq. 2.1 by the FFTLog method (Sec. 3.2) for fixed grids and tracers."""

    def __init__(self, chi_min, chi_max, N, k, ells, knots, kind, fft_bias, D=None, B=None,
                 precision="bf16x9", device=0, mem_budget_bytes=0, taper_chi=None, taper_c=None):
        super().__init__()
        self.device = torch.device("cuda", device)
        self.precision = api.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.stream = torch.cuda.Stream(self.device)
        self.ctx = api.Context(device, mem_budget_bytes, self.stream.cuda_stream)
        self.ctx.set_grids(chi_min, chi_max, N, k, ells, knots)
        self.ctx.set_tracers(kind, fft_bias, taper_chi, taper_c)
        as_dev = lambda a: None if a is None else torch.as_tensor(a, dtype=torch.float64, device=self.device).contiguous()  # noqa: E731
        self.D = as_dev(D)
        self.B = as_dev(B)
        self.n_tr = len(kind)
        self.n_ell = len(ells)
        self._generation = 0

    @staticmethod
    def n_walk(W):
        return 1 if W.dim() == 2 else W.shape[0]

    def _load(self, W, P, amp):
        n_walk = self.n_walk(W)
        api.swcl_set_windows(self.ctx.ptr, n_walk, W, self.D, self.B)
        api.swcl_set_power(self.ctx.ptr, n_walk, P, amp)

    def forward(self, W, P, amp):
        return _SwiftCl.apply(W, P, amp, self)
