"""Parity of the tensor-core (tcgen05) forms with the FP64 oracle.

Gate (reading R9): |C - C_oracle| <= 1e-4 max(|C_ij|, 1e-3 sqrt(C_ii C_jj)) on every entry for
the split-BF16 (bf16x9) and TF32x6 forms.  The classic 3xTF32 form keeps only 22 bits of each
operand and does NOT meet the 1e-4 gate on the N5K-shaped workload (measured about 1.6e-4): its
tests report the error and hold it to a regression bound ten times the gate, which is not a pass
of the gate."""
import numpy as np
import pytest

from gpu_helpers import grad_err, lib_context, make_ragged_case, norm_err, oracle_walker, pbar_err, wbar_err

pytestmark = pytest.mark.gpu

GATE = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


@pytest.fixture(scope="module")
def n5k_ref(wl):
    w = wl("n5k_vjp")
    f, _ = oracle_walker(w)
    return w, f


@pytest.mark.parametrize("prec", ["bf16x9", "tf32x6"])
def test_tiny2(prec, wl):
    import paper_2505_22718_gb300 as S
    w = wl("tiny2")
    ctx = lib_context(w)
    C = ctx.compute_cl(S.PRECISIONS[prec])
    f, _ = oracle_walker(w)
    assert norm_err(C, f["C"]) < GATE
    assert np.array_equal(C, np.transpose(C, (0, 2, 1)))


@pytest.mark.parametrize("prec", ["bf16x9", "tf32x6"])
def test_n5k_forward(prec, n5k_ref):
    import paper_2505_22718_gb300 as S
    w, f = n5k_ref
    ctx = lib_context(w)
    C = ctx.compute_cl(S.PRECISIONS[prec])
    err = norm_err(C, f["C"])
    print("n5k %s normalised C error %.3e" % (prec, err))
    assert err < GATE
    assert np.array_equal(C, np.transpose(C, (0, 2, 1)))
    # the stage itself: Delta against the oracle, relative to each (ell, tracer) row's maximum
    d = S.swcl_debug_read(ctx.ptr, S.SWCL_DBG_DELTA).reshape(f["delta"].shape)
    rel = np.abs(d - f["delta"]) / np.abs(f["delta"]).max(axis=2, keepdims=True)
    assert rel.max() < 1e-4


def test_n5k_3xtf32_misses_gate_and_is_reported(n5k_ref):
    """3xTF32 (2-plane splits, 22 bits per operand) fails the 1e-4 gate on this workload (about
    1.6e-4).  The error is printed and held to a regression bound of 1e-3."""
    import paper_2505_22718_gb300 as S
    w, f = n5k_ref
    ctx = lib_context(w)
    C = ctx.compute_cl(S.SWCL_3XTF32)
    err = norm_err(C, f["C"])
    print("n5k 3xtf32 normalised C error %.3e" % err)
    assert err < 1e-3


@pytest.mark.parametrize("prec", ["bf16x9", "tf32x6"])
def test_ragged_walkers(prec):
    """7 tracers with B(k, z) and tapers, 333 k (ragged tile), 37 ells, 23 knots, 3 walkers with
    ragged ell lists."""
    import paper_2505_22718_gb300 as S
    w, tapers = make_ragged_case()
    ctx = lib_context(w, tapers)
    C = ctx.compute_cl(S.PRECISIONS[prec])
    o = 0
    for wk, lst in enumerate(w.ell_lists):
        n = len(lst)
        f, _ = oracle_walker(w, wk, tapers)
        assert norm_err(C[o:o + n], f["C"][lst]) < GATE, wk
        o += n


def test_mixed_then_fp64_on_one_context(wl):
    """Switching precision on one context rebuilds nothing stale: FP64 after a mixed call is still
    within the FP64 gate."""
    import paper_2505_22718_gb300 as S
    w = wl("tiny2")
    ctx = lib_context(w)
    ctx.compute_cl(S.SWCL_SPLIT_BF16)
    C = ctx.compute_cl(S.SWCL_FP64)
    f, _ = oracle_walker(w)
    assert norm_err(C, f["C"]) < 1e-10


VJP_GATE = 5e-5   # P_bar per entry against the size of its terms, amp_bar per entry, W_bar per row


@pytest.mark.parametrize("prec", ["bf16x9", "tf32x6", "3xtf32"])
def test_n5k_vjp(prec, wl):
    """Gradients of the tensor-core forms; 3xTF32, which misses the forward gate, is held to a
    regression bound of twice the gradient gate instead (reported, not a pass of the gate)."""
    """Reverse mode through the tensor-core transposed contraction against the oracle's gradient."""
    import paper_2505_22718_gb300 as S
    w = wl("n5k_vjp")
    f, (Pbo, Abo, Wbo, ex) = oracle_walker(w, C_bar=w.C_bar)
    ctx = lib_context(w)
    ctx.compute_cl(S.PRECISIONS[prec])
    Pb, Ab, Wb = ctx.vjp(w.C_bar, S.PRECISIONS[prec])
    errs = (pbar_err(Pb[0], Pbo, ex["P_abs"]), grad_err(Ab[0], Abo), wbar_err(Wb[0], Wbo))
    print("n5k %s VJP errors P_bar %.2e amp_bar %.2e W_bar %.2e" % ((prec,) + errs))
    assert max(errs) < (2 * VJP_GATE if prec == "3xtf32" else VJP_GATE)


@pytest.mark.parametrize("prec", ["bf16x9", "tf32x6"])
def test_ragged_vjp(prec):
    import paper_2505_22718_gb300 as S
    w, tapers = make_ragged_case()
    ctx = lib_context(w, tapers)
    C = ctx.compute_cl(S.PRECISIONS[prec])
    rng = np.random.default_rng(9)
    Cb = rng.standard_normal(C.shape)
    Pb, Ab, Wb = ctx.vjp(Cb, S.PRECISIONS[prec])
    o = 0
    for wk, lst in enumerate(w.ell_lists):
        n = len(lst)
        Cbw = np.zeros((len(w.ells), 7, 7))
        Cbw[lst] = Cb[o:o + n]
        f, (Pbo, Abo, Wbo, ex) = oracle_walker(w, wk, tapers, C_bar=Cbw)
        assert pbar_err(Pb[wk], Pbo, ex["P_abs"]) < VJP_GATE
        assert grad_err(Ab[wk], Abo) < VJP_GATE
        assert wbar_err(Wb[wk], Wbo) < VJP_GATE
        o += n
