"""Failure detection for non-finite results: a NaN or Inf planted on the host in an input reaches
the outputs, the kernels that write C, P_bar, amp_bar and W_bar raise the context's status word,
and the next synchronising call returns SWCL_ERR_NONFINITE; the status is then cleared and the
context computes correctly again.  Nothing here faults the GPU."""
import numpy as np
import pytest

from gpu_helpers import lib_context, norm_err, oracle_walker

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("prec", ["fp64", "bf16x9"])
def test_nan_window_is_reported_then_cleared(prec, wl):
    import paper_2505_22718_gb300 as S
    w = wl("tiny2")
    p = S.PRECISIONS[prec]
    ctx = lib_context(w)
    bad = w.W.copy()
    bad[1, w.N // 3] = np.nan
    ctx.set_window_samples(bad)
    with pytest.raises(S.SwiftClError) as e:
        ctx.compute_cl(p)
    assert e.value.status == S.SWCL_ERR_NONFINITE
    ctx.set_window_samples(w.W)
    C = ctx.compute_cl(p)
    f, _ = oracle_walker(w)
    assert norm_err(C, f["C"]) < (1e-10 if prec == "fp64" else 1e-4)


def test_nan_cotangent_is_reported_by_the_vjp(wl):
    import paper_2505_22718_gb300 as S
    w = wl("tiny2")
    ctx = lib_context(w)
    C = ctx.compute_cl(S.SWCL_FP64)
    Cb = np.ones_like(C)
    Cb[3, 0, 1] = np.inf
    with pytest.raises(S.SwiftClError) as e:
        ctx.vjp(Cb, S.SWCL_FP64)
    assert e.value.status == S.SWCL_ERR_NONFINITE
    Pb, Ab, Wb = ctx.vjp(np.ones_like(C), S.SWCL_FP64)
    assert np.all(np.isfinite(Pb)) and np.all(np.isfinite(Wb))


def test_batched_graph_reports_through_sync(wl):
    """Device outputs do not synchronise: the CUDA-graph step returns at once and swcl_sync
    reports the status raised inside the replay."""
    import torch
    import paper_2505_22718_gb300 as S
    w = wl("tiny2")
    dev = torch.device("cuda:0")
    ctx = lib_context(w)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)  # noqa: E731
    C = torch.empty((len(w.ells), w.n_tr, w.n_tr), dtype=torch.float64, device=dev)
    Cb = torch.ones_like(C)
    Pb = torch.empty((1, len(w.k)), dtype=torch.float64, device=dev)
    Ab = torch.empty((1, w.n_tr), dtype=torch.float64, device=dev)
    Wb = torch.empty((1, w.n_tr, w.N), dtype=torch.float64, device=dev)
    S.swcl_compute_batched(ctx.ptr, S.SWCL_SPLIT_BF16, C, Cb, Pb, Ab, Wb)
    ctx.sync()
    bad = w.W.copy()
    bad[0, 7] = np.inf
    ctx.set_window_samples(t(bad))
    S.swcl_compute_batched(ctx.ptr, S.SWCL_SPLIT_BF16, C, Cb, Pb, Ab, Wb)
    with pytest.raises(S.SwiftClError) as e:
        ctx.sync()
    assert e.value.status == S.SWCL_ERR_NONFINITE
    ctx.set_window_samples(t(w.W))
    S.swcl_compute_batched(ctx.ptr, S.SWCL_SPLIT_BF16, C, Cb, Pb, Ab, Wb)
    ctx.sync()
    f, _ = oracle_walker(w)
    assert norm_err(C.cpu().numpy(), f["C"]) < 1e-4
