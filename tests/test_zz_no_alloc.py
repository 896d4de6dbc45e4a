"""swcl_fftlog_noalloc: the FFTLog coefficients for callers that cannot allocate device memory
(for example a JAX process whose memory arena already holds the GPU), against the coefficients the
context path (swcl_compute_cl) computes for the same inputs.

The entry point keeps its tables in a fixed static device array; two calls in a row with
different inputs must each match, so nothing from the first call leaks into the second.
This file is named to be collected last."""
import numpy as np
import pytest

from gpu_helpers import lib_context, make_ragged_case

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the FP64 parity gate of the other tests


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def _context_coefficients(w, tapers):
    import paper_2505_22718_gb300 as S
    ctx = lib_context(w, tapers)
    ctx.set_ell_lists(None)
    ctx.compute_cl(S.SWCL_FP64)
    c = S.swcl_debug_read(ctx.ptr, S.SWCL_DBG_COEF)
    ctx.close()
    return c


def _noalloc(w, tapers):
    import torch
    import paper_2505_22718_gb300 as S
    dev = torch.device("cuda:0")
    t = lambda a: None if a is None else torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)  # noqa: E731
    nw = 1 if w.W.ndim == 2 else w.W.shape[0]
    n_h = w.N // 2 + 1
    coef = torch.full((nw * w.n_tr * len(w.knots) * n_h * 2,), float("nan"), dtype=torch.float64, device=dev)
    tc, tn = (None, None) if tapers is None else tapers
    ins = [t(tc), t(tn), t(w.W), t(w.D), t(w.B)]
    st = S.swcl_fftlog_noalloc(nw, w.n_tr, len(w.knots), w.N, w.chi_min, w.chi_max, w.kind, w.fft_bias,
                               *ins, coef)
    torch.cuda.synchronize()
    assert st == 0, S.strerror(st)
    return coef.cpu().numpy()


def test_noalloc_matches_context_path_on_two_calls_in_a_row(wl):
    w1, tap1 = make_ragged_case()
    w2 = wl("tiny2")
    ref1 = _context_coefficients(w1, tap1)
    ref2 = _context_coefficients(w2, None)
    out1 = _noalloc(w1, tap1)
    out2 = _noalloc(w2, None)
    for out, ref in ((out1, ref1), (out2, ref2)):
        assert out.shape == ref.shape
        assert np.all(np.isfinite(out))
        assert np.max(np.abs(out - ref)) <= TOL * np.abs(ref).max()


def test_noalloc_rejects_tables_beyond_its_static_array(wl):
    import torch
    import paper_2505_22718_gb300 as S
    w = wl("tiny2")
    dev = torch.device("cuda:0")
    big_tr = 64
    N = 8192  # 8 N_tr N + 16 N_tr (N/2+1) bytes > 4 MiB
    W = torch.zeros((big_tr, N), dtype=torch.float64, device=dev)
    D = torch.ones((1, N), dtype=torch.float64, device=dev)
    coef = torch.zeros((big_tr * (N // 2 + 1) * 2,), dtype=torch.float64, device=dev)
    st = S.swcl_fftlog_noalloc(1, big_tr, 1, N, w.chi_min, w.chi_max, np.zeros(big_tr, np.int32),
                               np.full(big_tr, -0.3), None, None, W, D, None, coef)
    assert st == -3  # SWCL_ERR_OOM_BUDGET, reported before any launch
    n = 300   # not a power of two
    W3 = torch.zeros((1, n), dtype=torch.float64, device=dev)
    D3 = torch.ones((1, n), dtype=torch.float64, device=dev)
    c3 = torch.zeros((n // 2 + 1) * 2, dtype=torch.float64, device=dev)
    st = S.swcl_fftlog_noalloc(1, 1, 1, n, w.chi_min, w.chi_max, np.zeros(1, np.int32),
                               np.full(1, -0.3), None, None, W3, D3, None, c3)
    assert st == -1
    # an infinite chi_max is rejected like in swcl_set_grids
    W4 = torch.zeros((1, 256), dtype=torch.float64, device=dev)
    D4 = torch.ones((1, 256), dtype=torch.float64, device=dev)
    c4 = torch.zeros(129 * 2, dtype=torch.float64, device=dev)
    st = S.swcl_fftlog_noalloc(1, 1, 1, 256, w.chi_min, float("inf"), np.zeros(1, np.int32),
                               np.full(1, -0.3), None, None, W4, D4, None, c4)
    assert st == -1


def test_noalloc_binding_rejects_host_and_short_buffers(wl):
    """The entry point takes plain device pointers: the binding refuses a host array and a short
    output buffer before the library sees them."""
    import torch
    import paper_2505_22718_gb300 as S
    w = wl("tiny2")
    dev = torch.device("cuda:0")
    n_h = w.N // 2 + 1
    W = torch.as_tensor(w.W, dtype=torch.float64, device=dev)
    D = torch.as_tensor(w.D, dtype=torch.float64, device=dev)
    coef = torch.zeros(w.n_tr * n_h * 2, dtype=torch.float64, device=dev)
    args = (1, w.n_tr, 1, w.N, w.chi_min, w.chi_max, w.kind, w.fft_bias, None, None)
    with pytest.raises(TypeError):
        S.swcl_fftlog_noalloc(*args, np.ascontiguousarray(w.W), D, None, coef)
    with pytest.raises(ValueError):
        S.swcl_fftlog_noalloc(*args, W, D, None, coef[:-2])
    assert S.swcl_fftlog_noalloc(*args, W, D, None, coef) == 0
