"""Delta recomputed in the backward pass under a memory budget, and the large configuration
(30 tracers, every ell in [2, 3000], N = 4096, 4096 k points, 200 knots, B(k, z)) at full size.

When Delta and Dbar for every multipole do not fit the context's budget, the forward pass
contracts and integrates multipole chunk by chunk and the VJP recomputes each chunk's Delta.
The chunked results must equal the whole-Delta ones (bit for bit where the arithmetic per
element is unchanged, within the reordering of atomic sums otherwise), and the large
configuration must match the FP64 oracle on sampled multipoles and tracers."""
import copy

import numpy as np
import pytest

from gpu_helpers import grad_err, lib_context, max_rel, norm_err, p_abs, pbar_err, wbar_err
from oracle import fftlog as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def _run(w, prec, Cb, budget=0):
    import paper_2505_22718_gb300 as S
    ctx = lib_context(w, budget=budget)
    C = ctx.compute_cl(S.PRECISIONS[prec])
    grads = ctx.vjp(Cb, S.PRECISIONS[prec])
    return ctx, C, grads


@pytest.mark.parametrize("prec", ["fp64", "bf16x9"])
def test_chunked_recompute_matches_whole(prec, wl):
    import paper_2505_22718_gb300 as S
    w = wl("n5k_vjp")
    full, C1, (P1, A1, W1) = _run(w, prec, w.C_bar)
    assert full.query(S.SWCL_Q_RECOMPUTE) == 0
    held = full.query(S.SWCL_Q_WORKSPACE_BYTES)
    es = 8 if prec == "fp64" else 4
    delta_bytes = w.n_tr * len(w.ells) * len(w.k) * es
    ctx, C2, (P2, A2, W2) = _run(w, prec, w.C_bar, budget=held - delta_bytes)
    assert ctx.query(S.SWCL_Q_RECOMPUTE) == 1
    assert ctx.query(S.SWCL_Q_WORKSPACE_BYTES) <= held - delta_bytes
    assert np.array_equal(C1, C2)
    assert np.array_equal(A1, A2)
    assert np.array_equal(P1, P2)
    assert max_rel(W2, W1) < (1e-12 if prec == "fp64" else 1e-5)


def _sub_workload(w, tr, li):
    s = copy.copy(w)
    s.W, s.kind, s.fft_bias, s.amp = w.W[tr], w.kind[tr], w.fft_bias[tr], w.amp[tr]
    s.B = None if w.B is None else w.B[tr]
    s.ells = w.ells[li]
    return s


@pytest.mark.parametrize("prec", ["bf16x9", "fp64"])
def test_large_configuration_sampled_against_oracle(prec):
    """Full-size forward + VJP of the large configuration under the 40 GB budget (and, for the
    mixed form, again under a budget that forces multipole chunks), compared with the FP64 oracle
    on every tracer at 16 multipoles spread logarithmically over [2, 3000]; the cotangent is
    nonzero only there."""
    import paper_2505_22718_gb300 as S
    from workloads import make_workload
    w = make_workload("large")
    tr = np.arange(w.n_tr)
    li = np.unique(np.round(np.geomspace(2, 3000, 16)).astype(int)) - 2   # ell = 2 ... 3000
    rng = np.random.default_rng(31)
    Cb = np.zeros((len(w.ells), w.n_tr, w.n_tr))
    Cb[np.ix_(li, tr, tr)] = rng.standard_normal((len(li), len(tr), len(tr)))
    ctx, C, (Pb, Ab, Wb) = _run(w, prec, Cb, budget=40 << 30)
    assert ctx.query(S.SWCL_Q_PROFILE_RANK) == 1
    s = _sub_workload(w, tr, li)
    g = O.Grids(s.N, s.chi_min, s.chi_max, s.k, s.ells, s.knots, s.kind, s.fft_bias, fft="numpy")
    f = O.forward(g, s.W, s.D, s.P, s.amp, s.B)
    Pbo, Abo, Wbo, _ = O.vjp(g, f, Cb[np.ix_(li, tr, tr)], s.W, s.D, s.P, s.amp, s.B)
    ex = {"P_abs": p_abs(f["delta"], Cb[np.ix_(li, tr, tr)], s.amp, s.k)}
    gate_c, gate_g = (1e-10, 1e-9) if prec == "fp64" else (1e-4, 5e-5)
    e_c = norm_err(C[np.ix_(li, tr, tr)], f["C"])
    print("large %s: C %.2e  Pbar %.2e  Abar %.2e  Wbar %.2e" % (
        prec, e_c, pbar_err(Pb[0], Pbo, ex["P_abs"]), grad_err(Ab[0][tr], Abo), wbar_err(Wb[0][tr], Wbo)))
    assert e_c < gate_c
    assert pbar_err(Pb[0], Pbo, ex["P_abs"]) < gate_g
    assert grad_err(Ab[0][tr], Abo) < gate_g
    assert wbar_err(Wb[0][tr], Wbo) < gate_g
    # symmetry and per-ell PSD of the full output
    assert np.array_equal(C, np.transpose(C, (0, 2, 1)))
    if prec == "bf16x9":
        held = ctx.query(S.SWCL_Q_WORKSPACE_BYTES)
        del ctx
        ctx2, C2, (Pb2, Ab2, Wb2) = _run(w, prec, Cb, budget=held // 3)
        assert ctx2.query(S.SWCL_Q_RECOMPUTE) == 1
        assert np.array_equal(C, C2)
        assert max_rel(Pb2, Pb) < 1e-12
        assert max_rel(Wb2[0][tr], Wb[0][tr]) < 1e-5


@pytest.mark.parametrize("prec", ["fp64", "bf16x9"])
def test_chunked_recompute_with_limber_rows(prec, wl):
    """Limber rows for l >= 500 and a budget that splits the FFTLog multipoles into chunks: the
    results equal the unchunked run's, only the FFTLog multipoles are held as Delta, and Delta is
    then not readable through the debug call."""
    import paper_2505_22718_gb300 as S
    w = wl("n5k_vjp")

    def run(budget):
        ctx = lib_context(w, budget=budget)
        ctx.set_limber(500)
        C = ctx.compute_cl(S.PRECISIONS[prec])
        g = ctx.vjp(w.C_bar, S.PRECISIONS[prec])
        return ctx, C, g

    full, C1, (P1, A1, W1) = run(0)
    assert full.query(S.SWCL_Q_RECOMPUTE) == 0
    with pytest.raises(S.SwiftClError):
        S.swcl_debug_read(full.ptr, S.SWCL_DBG_DELTA)
    n_fft = int(np.sum(w.ells < 500))
    es = 8 if prec == "fp64" else 4
    held = full.query(S.SWCL_Q_WORKSPACE_BYTES)
    ctx, C2, (P2, A2, W2) = run(held - w.n_tr * n_fft * len(w.k) * es // 2)
    assert ctx.query(S.SWCL_Q_RECOMPUTE) == 1
    assert np.array_equal(C1, C2)
    assert np.array_equal(A1, A2)
    assert np.array_equal(P1, P2)
    assert max_rel(W2, W1) < (1e-12 if prec == "fp64" else 1e-5)
