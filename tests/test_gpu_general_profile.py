"""Parity of the general k-interpolation path (Sec. 3.2: one FFTLog per k-knot, then the 4-point
Lagrange interpolation of the coefficients along k) in the tensor-core forms.

The workload n5k_general has the N5K shape with a growth D(k, z) = D(z) exp(0.02 ln(k/0.1) g(z))
whose knot profiles are of high numerical rank, so the library cannot fold the interpolation into
a few basis profiles: it transforms all 150 knots per tracer and the knot-stencil tcgen05 kernels
form A = sum_a lambda_a c_a e^{-i eta ln k} in their producers.  Every C_ell entry is gated
(reading R9: 1e-4 normalised for the mixed forms) and every gradient entry is gated per element
(grad_err: relative to max(|g|, 1e-3 of its row's largest entry)), forward and VJP, at the full
N5K size.  The ragged edge case (7 tracers, 333 k, 37 ells, 23 knots, tapers, B(k, z), 3 walkers
with ragged ell lists) runs the same kernels with SWCL_PER_KNOT_FFT=1."""
import os

import numpy as np
import pytest

from gpu_helpers import grad_err, lib_context, make_ragged_case, max_rel, norm_err, oracle_walker, pbar_err, wbar_err

pytestmark = pytest.mark.gpu

GATE_C = 1e-4      # normalised C error (R9), mixed forms
GATE_G = 5e-5      # per-element gradient error, mixed forms


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


@pytest.fixture(scope="module")
def general_ref(wl):
    w = wl("n5k_general")
    f, grads = oracle_walker(w, C_bar=w.C_bar)
    return w, f, grads


def _context(w, tapers=None, per_knot=None):
    old = os.environ.get("SWCL_PER_KNOT_FFT")
    if per_knot is not None:
        os.environ["SWCL_PER_KNOT_FFT"] = "1" if per_knot else "0"
    try:
        return lib_context(w, tapers)
    finally:
        if per_knot is not None:
            if old is None:
                del os.environ["SWCL_PER_KNOT_FFT"]
            else:
                os.environ["SWCL_PER_KNOT_FFT"] = old


def test_general_profile_is_not_low_rank(general_ref):
    """The profile factorisation finds no basis of rank <= 4: the per-knot FFT path runs."""
    import paper_2505_22718_gb300 as S
    w, _, _ = general_ref
    ctx = _context(w, per_knot=False)
    ctx.compute_cl(S.SWCL_SPLIT_BF16)
    assert ctx.query(S.SWCL_Q_PROFILE_RANK) == 0


@pytest.mark.parametrize("prec", ["bf16x9", "tf32x6"])
def test_general_forward_and_vjp(prec, general_ref):
    import paper_2505_22718_gb300 as S
    w, f, (Pbo, Abo, Wbo, ex) = general_ref
    ctx = _context(w, per_knot=False)
    C = ctx.compute_cl(S.PRECISIONS[prec])
    assert ctx.query(S.SWCL_Q_PROFILE_RANK) == 0
    err = norm_err(C, f["C"])
    # Delta itself (a3), relative to each (ell, tracer) row's largest entry
    d = S.swcl_debug_read(ctx.ptr, S.SWCL_DBG_DELTA).reshape(f["delta"].shape)
    drel = float((np.abs(d - f["delta"]) / np.abs(f["delta"]).max(axis=2, keepdims=True)).max())
    Pb, Ab, Wb = ctx.vjp(w.C_bar, S.PRECISIONS[prec])
    ge = (pbar_err(Pb[0], Pbo, ex["P_abs"]), grad_err(Ab[0], Abo), wbar_err(Wb[0], Wbo))
    gm = (pbar_err(Pb[0], Pbo, ex["P_abs"]), grad_err(Ab[0], Abo), wbar_err(Wb[0], Wbo))
    print("n5k_general %s: C %.3e, Delta %.3e; per-element P_bar %.2e amp_bar %.2e W_bar %.2e "
          "(max-normalised %.2e %.2e %.2e)" % ((prec, err, drel) + ge + gm))
    assert err < GATE_C
    assert np.array_equal(C, np.transpose(C, (0, 2, 1)))
    assert drel < 1e-4
    assert max(ge) < GATE_G


@pytest.mark.parametrize("prec", ["bf16x9", "tf32x6"])
def test_ragged_per_knot(prec):
    """The per-knot stencil kernels on the ragged edge case: tiles cut at 333 k points and 37
    multipoles, tapers, per-tracer B(k, z), three walkers with ragged multipole lists."""
    import paper_2505_22718_gb300 as S
    w, tapers = make_ragged_case()
    ctx = _context(w, tapers, per_knot=True)
    C = ctx.compute_cl(S.PRECISIONS[prec])
    assert ctx.query(S.SWCL_Q_PROFILE_RANK) == 0
    rng = np.random.default_rng(17)
    Cb = rng.standard_normal(C.shape)
    Pb, Ab, Wb = ctx.vjp(Cb, S.PRECISIONS[prec])
    o = 0
    for wk, lst in enumerate(w.ell_lists):
        n = len(lst)
        Cbw = np.zeros((len(w.ells), w.n_tr, w.n_tr))
        Cbw[lst] = Cb[o:o + n]
        f, (Pbo, Abo, Wbo, ex) = oracle_walker(w, wk, tapers, C_bar=Cbw)
        err = norm_err(C[o:o + n], f["C"][lst])
        ge = (pbar_err(Pb[wk], Pbo, ex["P_abs"]), grad_err(Ab[wk], Abo), wbar_err(Wb[wk], Wbo))
        print("ragged per-knot %s walker %d: C %.3e, P_bar %.2e amp_bar %.2e W_bar %.2e"
              % ((prec, wk, err) + ge))
        assert err < GATE_C, wk
        assert max(ge) < GATE_G, wk
        o += n
