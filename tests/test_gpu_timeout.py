"""Failure detection without a GPU fault: the bounded mbarrier wait shared by the tensor-core
kernels gives up on a phase that nothing completes, the kernel raises the context's status word,
the host reports SWCL_ERR_TIMEOUT, and the context keeps working afterwards."""
import time

import numpy as np
import pytest

from gpu_helpers import lib_context, norm_err, oracle_walker

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def test_bounded_wait_reports_timeout_and_context_recovers(wl):
    import paper_2505_22718_gb300 as S
    w = wl("tiny2")
    ctx = lib_context(w)
    t0 = time.perf_counter()
    st, cycles = S.swcl_selftest_wait_timeout(ctx.ptr)
    dt = time.perf_counter() - t0
    print("bounded wait gave up after %d cycles, %.3f s" % (cycles, dt))
    assert st == S.SWCL_ERR_TIMEOUT
    assert cycles > 0 and dt < 30.0
    assert "gave up" in S.swcl_last_error(ctx.ptr)
    # the status word was cleared: the context computes normally afterwards
    C = ctx.compute_cl(S.SWCL_SPLIT_BF16)
    f, _ = oracle_walker(w)
    assert norm_err(C, f["C"]) < 1e-4
    S.swcl_sync(ctx.ptr)
