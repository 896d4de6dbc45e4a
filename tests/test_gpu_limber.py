"""The Limber branch (swcl_set_limber, Eq. 2.19, reading R12) on the GPU against the oracle's
hybrid spectrum (oracle/limber.py), through the C ABI: forward, VJP and JVP with several walkers,
ragged multipole lists and the switch inside the list, at the first multipole (everything Limber)
and above the last (nothing Limber); graph replay; the unsupported combinations.

Gates as in reading R9: C 1e-10 (FP64) and 1e-4 (bf16x9) normalised; gradients relative to their
largest entry 1e-10 / 1e-9 (FP64) and 5e-5 (bf16x9).  The Limber rows are FP64 in every form."""
import copy

import numpy as np
import pytest

from gpu_helpers import grad_err, lib_context, make_ragged_case, max_rel, norm_err, wbar_err
from oracle import fftlog as O
from oracle import limber as LB

pytestmark = pytest.mark.gpu

GATES = {"fp64": (1e-10, 1e-10, 1e-9), "bf16x9": (1e-4, 5e-5, 5e-5)}


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


@pytest.fixture(scope="module")
def case():
    w, tapers = make_ragged_case(n_walk=3, seed=41)
    rng = np.random.default_rng(3)
    Cb = [rng.standard_normal((len(x), w.n_tr, w.n_tr)) for x in w.ell_lists]
    return w, tapers, Cb


def _oracle(w, tapers, Cb, sw):
    """Hybrid C (packed by the walkers' lists) and gradients, walker by walker."""
    g = O.Grids(w.N, w.chi_min, w.chi_max, w.k, w.ells, w.knots, w.kind, w.fft_bias)
    Cs, grads = [], []
    for wk, lst in enumerate(w.ell_lists):
        C, f = LB.hybrid_forward(g, w.W[wk], w.D, w.P[wk], w.amp[wk], sw, w.B, *tapers)
        Cs.append(C[lst])
        full = np.zeros_like(C)
        full[lst] = Cb[wk]
        grads.append(LB.hybrid_vjp(g, f, full, w.W[wk], w.D, w.P[wk], w.amp[wk], sw, w.B, *tapers))
    return np.concatenate(Cs), grads


@pytest.mark.parametrize("prec", ["fp64", "bf16x9"])
@pytest.mark.parametrize("sw", [150, 2, 10000])
def test_hybrid_forward_and_vjp(prec, sw, case):
    import paper_2505_22718_gb300 as S
    w, tapers, Cb = case
    tol, gtol, wtol = GATES[prec]
    ptol = 1e-10 if prec == "fp64" else 1e-4
    Co, go = _oracle(w, tapers, Cb, sw)
    ctx = lib_context(w, tapers)
    ctx.set_limber(sw)
    p = S.PRECISIONS[prec]
    C = ctx.compute_cl(p)
    e = norm_err(C, Co)
    Pb, Ab, Wb = ctx.vjp(np.concatenate(Cb), p)
    # P_bar and amp_bar per element (floor 1e-3 of the row), W_bar per row (walker, tracer)
    ge = [max(grad_err(Pb[wk], go[wk][0]) for wk in range(len(go))),
          max(grad_err(Ab[wk], go[wk][1]) for wk in range(len(go))),
          max(wbar_err(Wb[wk], go[wk][2]) for wk in range(len(go)))]
    print("limber %s switch %d: C %.2e  Pbar %.2e  Abar %.2e  Wbar %.2e" % (prec, sw, e, *ge))
    assert e < tol
    assert ge[0] < ptol and ge[1] < gtol and ge[2] < wtol


def test_limber_rows_do_not_depend_on_the_precision_form(case):
    """The Limber rows are FP64 in every form: bf16x9 and FP64 agree on them to rounding."""
    import paper_2505_22718_gb300 as S
    w, tapers, _ = case
    ctx = lib_context(w, tapers)
    ctx.set_ell_lists(None)
    ctx.set_limber(150)
    a = ctx.compute_cl(S.SWCL_FP64).reshape(3, len(w.ells), w.n_tr, w.n_tr)
    b = ctx.compute_cl(S.SWCL_SPLIT_BF16).reshape(3, len(w.ells), w.n_tr, w.n_tr)
    sel = w.ells >= 150
    assert np.max(np.abs(a[:, sel] - b[:, sel])) <= 1e-13 * np.abs(a[:, sel]).max()


@pytest.mark.parametrize("prec", ["fp64", "bf16x9"])
def test_hybrid_jvp(prec, case):
    import paper_2505_22718_gb300 as S
    w0, tapers, _ = case
    w = copy.copy(w0)
    w.W, w.P, w.amp, w.ell_lists = w0.W[0], w0.P[0], w0.amp[0], None
    sw = 150
    g = O.Grids(w.N, w.chi_min, w.chi_max, w.k, w.ells, w.knots, w.kind, w.fft_bias)
    rng = np.random.default_rng(8)
    Pd = rng.standard_normal((2, len(w.k))) * w.P
    Ad = rng.standard_normal((2, w.n_tr))
    if prec == "fp64":
        # broadband window tangents (white noise under each window)
        Wd = rng.standard_normal((2, w.n_tr, w.N)) * w.W
    else:
        # the window tangents a forecast takes: smooth moves of each window (a shift along ln chi
        # and a tilt, with random amplitudes).  White-noise tangents put their FFTLog coefficients
        # at every n, where the contraction cancels most, and are checked in FP64 above.
        dW = np.gradient(w.W, axis=-1)
        tilt = w.W * np.linspace(-1.0, 1.0, w.N)[None, :]
        Wd = np.stack([rng.standard_normal((w.n_tr, 1)) * dW + rng.standard_normal((w.n_tr, 1)) * tilt
                       for _ in range(2)])
    f = O.forward(g, w.W, w.D, w.P, w.amp, w.B, *tapers)
    Jo = np.array([LB.hybrid_jvp(g, f, w.D, w.P, w.amp, sw, w.B, *tapers, P_dot=Pd[t], amp_dot=Ad[t],
                                 W_dot=Wd[t], W=w.W) for t in range(2)])
    ctx = lib_context(w, tapers)
    ctx.set_limber(sw)
    J = ctx.jvp(Pd, Ad, Wd, S.PRECISIONS[prec])
    tol = GATES[prec][0]
    dg = np.abs(np.einsum("lii->li", f["C"]))
    base = np.sqrt(dg[:, :, None] * dg[:, None, :])
    for t in range(2):
        floor = 1e-3 * base * np.abs(Jo[t]).max() / np.abs(f["C"]).max()
        ex = np.max(np.abs(J[t] - Jo[t]) / (tol * np.maximum(np.abs(Jo[t]), floor)))
        print("limber jvp %s tangent %d: error / gate %.3f" % (prec, t, ex))
        assert ex <= 1.0, (t, ex)


def test_graph_replay_with_limber_rows(case):
    torch = pytest.importorskip("torch")
    import paper_2505_22718_gb300 as S
    w, tapers, Cb = case
    ctx = lib_context(w, tapers)
    ctx.set_limber(150)
    C1 = ctx.compute_cl(S.SWCL_SPLIT_BF16)
    Pb1, Ab1, Wb1 = ctx.vjp(np.concatenate(Cb), S.SWCL_SPLIT_BF16)
    dev = "cuda:0"
    C = torch.empty(C1.shape, dtype=torch.float64, device=dev)
    cb = torch.from_numpy(np.concatenate(Cb)).to(dev)
    Pb = torch.empty(Pb1.shape, dtype=torch.float64, device=dev)
    Ab = torch.empty(Ab1.shape, dtype=torch.float64, device=dev)
    Wb = torch.empty(Wb1.shape, dtype=torch.float64, device=dev)
    for _ in range(2):
        S.swcl_compute_batched(ctx.ptr, S.SWCL_SPLIT_BF16, C, cb, Pb, Ab, Wb)
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy(), C1)
    assert np.array_equal(Ab.cpu().numpy(), Ab1)
    assert max_rel(Pb.cpu().numpy(), Pb1) < 1e-14 and max_rel(Wb.cpu().numpy(), Wb1) < 1e-14


def test_unsupported_limber_combinations(case):
    import paper_2505_22718_gb300 as S
    w, tapers, _ = case
    # the knot-stencil tensor-core forms do not take the branch
    ctx = lib_context(w, tapers)
    ctx.set_limber(150)
    with pytest.raises(S.SwiftClError):
        ctx.compute_cl(S.SWCL_TF32X6)
    # RSD has no Limber form
    kind = w.kind.copy()
    kind[0] = O.KIND_RSD
    bias = w.fft_bias.copy()
    bias[0] = 0.4
    w2 = copy.copy(w)
    w2.kind, w2.fft_bias = kind, bias
    ctx2 = lib_context(w2, tapers)
    ctx2.set_limber(150)
    with pytest.raises(S.SwiftClError):
        ctx2.compute_cl(S.SWCL_FP64)
    ctx2.set_limber(0)
    ctx2.compute_cl(S.SWCL_FP64)
