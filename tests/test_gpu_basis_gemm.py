"""Basis-mode tensor-core GEMMs (bf16 compensated products against the constant phase operand):
parity with the FP64 oracle at the mixed-precision gate, agreement with the knot-stencil
tensor-core kernels, autotuned tiles, rank > 1 and per-tracer profiles."""
import os

import numpy as np
import pytest

from gpu_helpers import grad_err, lib_context, make_ragged_case, max_rel, norm_err, oracle_walker, pbar_err, wbar_err

pytestmark = pytest.mark.gpu

GATE_C, GATE_G = 1e-4, 5e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def _context(w, tapers=None, basis=True):
    old = os.environ.get("SWCL_BASIS_GEMM")
    os.environ["SWCL_BASIS_GEMM"] = "1" if basis else "0"
    try:
        return lib_context(w, tapers)
    finally:
        if old is None:
            del os.environ["SWCL_BASIS_GEMM"]
        else:
            os.environ["SWCL_BASIS_GEMM"] = old


def _fwd_vjp(ctx, Cb):
    import paper_2505_22718_gb300 as S
    C = ctx.compute_cl(S.SWCL_SPLIT_BF16)
    g = ctx.vjp(Cb, S.SWCL_SPLIT_BF16)
    return C, g


def test_n5k_against_oracle_and_stencil_kernels(wl):
    import paper_2505_22718_gb300 as S
    w = wl("n5k_vjp")
    ctx = _context(w)
    C, (Pb, Ab, Wb) = _fwd_vjp(ctx, w.C_bar)
    assert ctx.query(S.SWCL_Q_PROFILE_RANK) == 1
    code_f, code_a = ctx.query(S.SWCL_Q_TILE_FWD), ctx.query(S.SWCL_Q_TILE_ADJ)
    nt_f, nt_a = code_f & 255, code_a & 255
    assert nt_f in range(32, 241, 16) and nt_a in range(32, 241, 16)
    # plain, two-CTA (bit 8), two-K-block (bit 10), persistent two-K-block (bits 10 and 12),
    # two-SM tile (bits 10 and 13, with bit 11 in the adjoint: table rows staged first), one
    # accumulator slot per buffer (bit 14, with or without bit 10; in the forward also with bit 15,
    # K split over two CTAs) or the persistent form with epilogue warps (bits 10, 12 and 16)
    assert code_f >> 8 in (0, 1, 4, 20, 36, 64, 65, 68, 192, 276)
    assert code_a >> 8 in (0, 1, 4, 20, 36, 44, 64, 65, 68, 276)
    assert (not code_f & 256 or nt_f <= (128 if code_f & 16384 else 64))
    assert (not code_a & 256 or nt_a <= (128 if code_a & 16384 else 64))
    assert (nt_f <= 128 or code_f & 16384) and (nt_a <= 128 or code_a & 16384)
    f, (Pbo, Abo, Wbo, ex) = oracle_walker(w, C_bar=w.C_bar)
    e = (norm_err(C, f["C"]), pbar_err(Pb[0], Pbo, ex["P_abs"]), grad_err(Ab[0], Abo), wbar_err(Wb[0], Wbo))
    print("basis GEMM n5k: C %.2e  Pbar %.2e  Abar %.2e  Wbar %.2e  tile codes %d/%d" % (e + (code_f, code_a)))
    assert e[0] < GATE_C and max(e[1:]) < GATE_G
    assert np.array_equal(C, np.transpose(C, (0, 2, 1)))
    d = S.swcl_debug_read(ctx.ptr, S.SWCL_DBG_DELTA).reshape(f["delta"].shape)
    rel = np.abs(d - f["delta"]) / np.abs(f["delta"]).max(axis=2, keepdims=True)
    assert rel.max() < 1e-4
    # the knot-stencil tensor-core kernels on the same inputs
    ctx2 = _context(w, basis=False)
    C2, (Pb2, Ab2, Wb2) = _fwd_vjp(ctx2, w.C_bar)
    assert ctx2.query(S.SWCL_Q_TILE_FWD) == 0
    assert norm_err(C, C2) < 2 * GATE_C
    assert max_rel(Wb, Wb2) < 2 * GATE_G


def test_repeat_is_stable(wl):
    """A second forward/VJP on the same context (tuned tiles, rebuilt operands) agrees closely;
    the adjoint's atomics may reorder FP64 additions."""
    w = wl("n5k_vjp")
    ctx = _context(w)
    C1, g1 = _fwd_vjp(ctx, w.C_bar)
    C2, g2 = _fwd_vjp(ctx, w.C_bar)
    assert np.array_equal(C1, C2)
    for a, b in zip(g1, g2):
        assert max_rel(a, b) < 1e-12


def test_per_tracer_profiles_walkers_tapers():
    """B_i(k, z) (per-tracer rank-1 profiles), tapers, 333 k, 37 ells, 3 walkers, ragged lists."""
    import paper_2505_22718_gb300 as S
    w, tapers = make_ragged_case()
    ctx = _context(w, tapers)
    C = ctx.compute_cl(S.SWCL_SPLIT_BF16)
    rng = np.random.default_rng(5)
    Cb = rng.standard_normal(C.shape)
    Pb, Ab, Wb = ctx.vjp(Cb, S.SWCL_SPLIT_BF16)
    assert ctx.query(S.SWCL_Q_PROFILE_RANK) == 1 and ctx.query(S.SWCL_Q_TILE_FWD) > 0
    o = 0
    for wk, lst in enumerate(w.ell_lists):
        n = len(lst)
        Cbw = np.zeros((len(w.ells), 7, 7))
        Cbw[lst] = Cb[o:o + n]
        f, (Pbo, Abo, Wbo, ex) = oracle_walker(w, wk, tapers, C_bar=Cbw)
        assert norm_err(C[o:o + n], f["C"][lst]) < GATE_C
        assert pbar_err(Pb[wk], Pbo, ex["P_abs"]) < GATE_G
        assert grad_err(Ab[wk], Abo) < GATE_G
        assert wbar_err(Wb[wk], Wbo) < GATE_G
        o += n


def test_rank_two_profiles():
    """D(k, z) of rank 2: r = 2 basis columns per (tracer, multipole) in the forward tile."""
    import copy

    import paper_2505_22718_gb300 as S
    from workloads import make_workload
    w = copy.copy(make_workload("n5k"))
    tr = [0, 3, 9, 10, 14]
    w.W, w.kind, w.fft_bias, w.amp = w.W[tr], w.kind[tr], w.fft_bias[tr], w.amp[tr]
    z = (1.0 + 0.01 * np.log(w.knots[0] / 0.1)) / w.D[0] - 1.0
    lk = np.log(w.knots / 0.1)
    w.D = (1.0 / (1.0 + z))[None, :] * (1.0 + 0.01 * lk[:, None] * (1.0 + z[None, :]))
    w.ell_lists = None
    ctx = _context(w)
    C = ctx.compute_cl(S.SWCL_SPLIT_BF16)
    Cb = np.random.default_rng(8).standard_normal(C.shape)
    Pb, Ab, Wb = ctx.vjp(Cb, S.SWCL_SPLIT_BF16)
    assert ctx.query(S.SWCL_Q_PROFILE_RANK) == 2
    assert (ctx.query(S.SWCL_Q_TILE_FWD) & 255) % 2 == 0
    f, (Pbo, Abo, Wbo, ex) = oracle_walker(w, C_bar=Cb)
    assert norm_err(C, f["C"]) < GATE_C
    assert pbar_err(Pb[0], Pbo, ex["P_abs"]) < GATE_G
    assert wbar_err(Wb[0], Wbo) < GATE_G


@pytest.mark.parametrize("code", [96, 128, 48, 64 | 256, 32 | 256, 64 | 1024, 96 | 1024, 128 | 1024,
                                  64 | 1024 | 4096, 96 | 1024 | 4096, 64 | 1024 | 8192,
                                  96 | 1024 | 8192, 128 | 1024 | 8192, 96 | 1024 | 8192 | 2048,
                                  96 | 1024 | 16384, 128 | 1024 | 16384, 160 | 1024 | 16384,
                                  192 | 16384, 208 | 16384, 240 | 16384, 160 | 16384 | 32768,
                                  192 | 16384 | 32768, 240 | 16384 | 32768, 64 | 256 | 16384,
                                  96 | 256 | 16384, 128 | 256 | 16384, 64 | 1024 | 4096 | 65536,
                                  96 | 1024 | 4096 | 65536])
def test_every_tile_variant_against_oracle(code):
    """Each GEMM variant, fixed through SWCL_BASIS_TILES: one CTA per SM (48, 96, 128 columns),
    two CTAs per SM (| 256), two K-blocks per pipeline stage (| 1024), the persistent two-K-block
    form (| 1024 | 4096), the two-SM tile (| 1024 | 8192; | 2048: the adjoint's table rows staged
    at two stages), one accumulator slot per buffer (| 16384: up to 240 columns; | 32768: K split
    over a cluster of two CTAs, forward only, with the 208-column one-slot adjoint; | 256: two CTAs
    per SM; | 1024 | 4096 | 65536: persistent with epilogue warps); three walkers,
    a ragged k
    tail (333 points), 17 K-blocks in the forward GEMM (an odd count: the last stage is short),
    against the oracle."""
    import paper_2505_22718_gb300 as S
    w, tapers = make_ragged_case(n_walk=3, seed=51)
    old = os.environ.get("SWCL_BASIS_TILES")
    code_a = 208 | 16384 if code & 32768 else code
    os.environ["SWCL_BASIS_TILES"] = "%d,%d" % (code, code_a)
    try:
        ctx = _context(w, tapers)
    finally:
        if old is None:
            del os.environ["SWCL_BASIS_TILES"]
        else:
            os.environ["SWCL_BASIS_TILES"] = old
    ctx.set_ell_lists(None)
    rng = np.random.default_rng(2)
    Cb = rng.standard_normal((3 * len(w.ells), w.n_tr, w.n_tr))
    try:
        C, (Pb, Ab, Wb) = _fwd_vjp(ctx, Cb)
    except S.SwiftClError as e:
        # a forward tile must hold whole groups of r basis columns
        assert "not a forward tile" in str(e)
        pytest.skip("tile %d does not hold whole basis groups at this rank" % code)
    assert ctx.query(S.SWCL_Q_TILE_FWD) == code and ctx.query(S.SWCL_Q_TILE_ADJ) == code_a
    C = C.reshape(3, len(w.ells), w.n_tr, w.n_tr)
    Cb = Cb.reshape(3, len(w.ells), w.n_tr, w.n_tr)
    for wk in range(3):
        f, (Pbo, Abo, Wbo, ex) = oracle_walker(w, wk, tapers, C_bar=Cb[wk])
        assert norm_err(C[wk], f["C"]) < GATE_C
        assert max(pbar_err(Pb[wk], Pbo, ex["P_abs"]), grad_err(Ab[wk], Abo), wbar_err(Wb[wk], Wbo)) < GATE_G


def test_programmatic_dependent_launch_gives_the_same_results(wl):
    """SWCL_PDL=1: the critical-path kernels start before their predecessors finish and wait with
    griddepcontrol.wait; C must be bit for bit that of the ordinary launches (the same kernels,
    the same sums) and the gradients equal up to the order of the adjoint's FP64 atomics."""
    w = wl("n5k_vjp")
    old_pdl, old_tiles = os.environ.get("SWCL_PDL"), os.environ.get("SWCL_BASIS_TILES")
    os.environ["SWCL_BASIS_TILES"] = "1120,16736"
    try:
        os.environ["SWCL_PDL"] = "1"
        ctx_p = _context(w)
        os.environ["SWCL_PDL"] = "0"
        ctx_0 = _context(w)
    finally:
        for k, v in (("SWCL_PDL", old_pdl), ("SWCL_BASIS_TILES", old_tiles)):
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    Cp, gp = _fwd_vjp(ctx_p, w.C_bar)
    C0, g0 = _fwd_vjp(ctx_0, w.C_bar)
    assert np.array_equal(Cp, C0)
    for a, b in zip(gp, g0):
        assert max_rel(a, b) < 1e-12
