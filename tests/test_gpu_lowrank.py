"""Low-rank knot profiles: the library transforms r basis profiles instead of N_I knots when
D*B is numerically of rank r <= 4.  Results must equal the per-knot FFT (and the oracle) within the
FP64 gate, for rank-1 profiles (the workloads), a rank-2 profile, per-tracer profiles (B) and a
profile of full rank (which keeps the per-knot FFT)."""
import os

import numpy as np
import pytest

from gpu_helpers import lib_context, make_ragged_case, max_rel, norm_err, oracle_walker, pbar_err, wbar_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def _run(w, prec, tapers=None, per_knot=False):
    import paper_2505_22718_gb300 as S
    old = os.environ.get("SWCL_PER_KNOT_FFT")
    os.environ["SWCL_PER_KNOT_FFT"] = "1" if per_knot else "0"
    try:
        ctx = lib_context(w, tapers)
    finally:
        if old is None:
            del os.environ["SWCL_PER_KNOT_FFT"]
        else:
            os.environ["SWCL_PER_KNOT_FFT"] = old
    C = ctx.compute_cl(S.PRECISIONS[prec])
    rank = ctx.query(S.SWCL_Q_PROFILE_RANK)
    rng = np.random.default_rng(12)
    Cb = rng.standard_normal(C.shape)
    grads = ctx.vjp(Cb, S.PRECISIONS[prec])
    coef = S.swcl_debug_read(ctx.ptr, S.SWCL_DBG_COEF)
    return C, grads, rank, coef, Cb


def test_rank_one_profiles_match_per_knot(wl):
    w = wl("n5k_vjp")
    C1, g1, r1, c1, _ = _run(w, "fp64")
    C2, g2, r2, c2, _ = _run(w, "fp64", per_knot=True)
    assert r1 == 1 and r2 == 0
    assert np.max(np.abs(c1 - c2)) <= 1e-13 * np.abs(c2).max()
    assert norm_err(C1, C2) < 1e-11
    for a, b in zip(g1, g2):
        assert max_rel(a, b) < 1e-11


def _with_profile(w, D):
    import copy
    w2 = copy.copy(w)
    w2.D = D
    w2.ell_lists = None
    return w2


@pytest.mark.parametrize("kind", ["rank2", "full"])
def test_other_ranks_against_oracle(kind):
    from workloads import make_workload
    w = make_workload("n5k")
    tr = [0, 4, 10, 14]
    import copy
    w = copy.copy(w)
    w.W, w.kind, w.fft_bias, w.amp = w.W[tr], w.kind[tr], w.fft_bias[tr], w.amp[tr]
    z = 1.0 / w.D[0] * (1.0 + 0.01 * np.log(w.knots[0] / 0.1)) - 1.0
    lk = np.log(w.knots / 0.1)
    if kind == "rank2":
        D = (1.0 / (1.0 + z))[None, :] * (1.0 + 0.01 * lk[:, None] * (1.0 + z[None, :]))
        want = 2
    else:
        rng = np.random.default_rng(0)
        D = (1.0 / (1.0 + z))[None, :] * (1.0 + 0.01 * rng.standard_normal((len(lk), len(z))))
        want = 0
    w = _with_profile(w, D)
    C, (Pb, Ab, Wb), rank, _, Cb = _run(w, "fp64")
    assert rank == want
    f, (Pbo, Abo, Wbo, ex) = oracle_walker(w, C_bar=Cb)
    assert norm_err(C, f["C"]) < 1e-10
    assert pbar_err(Pb[0], Pbo, ex["P_abs"]) < 1e-10
    assert wbar_err(Wb[0], Wbo) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "bf16x9"])
def test_per_tracer_profiles_with_bias(prec):
    """B_i(k, z) present: one profile factorisation per tracer (ragged case, 3 walkers)."""
    w, tapers = make_ragged_case()
    w.ell_lists = None
    C, (Pb, Ab, Wb), rank, _, Cb = _run(w, prec, tapers)
    assert rank == 1
    gate_c, gate_g = (1e-10, 1e-9) if prec == "fp64" else (1e-4, 5e-5)
    nl = len(w.ells)
    for wk in range(w.W.shape[0]):
        f, (Pbo, Abo, Wbo, ex) = oracle_walker(w, wk, tapers, C_bar=Cb[wk * nl:(wk + 1) * nl])
        assert norm_err(C[wk * nl:(wk + 1) * nl], f["C"]) < gate_c
        assert pbar_err(Pb[wk], Pbo, ex["P_abs"]) < gate_g
        assert wbar_err(Wb[wk], Wbo) < gate_g
