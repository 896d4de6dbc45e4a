"""One evaluation split by multipole (sharding.ell_block) through the C ABI, the ranks run as
independent replicas on one GPU, one after the other: the C_ell blocks put together and the
gradients summed (what reduce_gradients does across ranks) agree with the oracle's full
evaluation.  No replica waits on another."""
import numpy as np
import pytest

from gpu_helpers import grad_err, max_rel, norm_err, oracle_walker, pbar_err, wbar_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("name,prec", [("tiny2", "fp64"), ("n5k_vjp", "bf16x9")])
def test_ell_blocks_on_replicas_match_full_evaluation(name, prec, wl):
    import paper_2505_22718_gb300 as S
    from paper_2505_22718_gb300.sharding import ell_block
    w = wl(name)
    n_ell, world = len(w.ells), 3
    Cb = np.random.default_rng(17).standard_normal((n_ell, w.n_tr, w.n_tr))
    precision = S.PRECISIONS[prec]
    C = np.empty((n_ell, w.n_tr, w.n_tr))
    Pb = np.zeros((1, len(w.k)))
    Ab = np.zeros((1, w.n_tr))
    Wb = np.zeros((1, w.n_tr, w.N))
    for rank in range(world):
        first, count = ell_block(n_ell, world, rank)
        ctx = S.Context(0, 0)
        ctx.set_grids(w.chi_min, w.chi_max, w.N, w.k, w.ells[first:first + count], w.knots)
        ctx.set_tracers(w.kind, w.fft_bias)
        ctx.set_windows(w.W, w.D, w.B)
        ctx.set_power(w.P, w.amp)
        C[first:first + count] = ctx.compute_cl(precision)
        p, a, wb = ctx.vjp(np.ascontiguousarray(Cb[first:first + count]), precision)
        Pb += p
        Ab += a
        Wb += wb
        ctx.close()
    f, (Pbo, Abo, Wbo, ex) = oracle_walker(w, C_bar=Cb)
    gate_c = 1e-10 if prec == "fp64" else 1e-4
    gate_g = 1e-9 if prec == "fp64" else 5e-5
    assert norm_err(C, f["C"]) < gate_c
    assert pbar_err(Pb[0], Pbo, ex["P_abs"]) < gate_g
    assert grad_err(Ab[0], Abo) < gate_g
    assert wbar_err(Wb[0], Wbo) < gate_g


def test_evaluate_ell_split_through_the_library(wl):
    """sharding.evaluate_ell_split without a process group: the whole multipole list is this
    process's block, computed through the C ABI (library_block), equal to the oracle."""
    import paper_2505_22718_gb300 as S
    from paper_2505_22718_gb300.sharding import evaluate_ell_split
    w = wl("tiny2")
    Cb = np.random.default_rng(4).standard_normal((len(w.ells), w.n_tr, w.n_tr))
    setup = dict(chi_min=w.chi_min, chi_max=w.chi_max, N=w.N, k=w.k, ells=w.ells, knots=w.knots,
                 kind=w.kind, fft_bias=w.fft_bias, W=w.W, D=w.D, B=w.B, P=w.P, amp=w.amp)
    C, Pb, Ab, Wb = evaluate_ell_split(setup, Cb, S.SWCL_FP64)
    f, (Pbo, Abo, Wbo, ex) = oracle_walker(w, C_bar=Cb)
    assert norm_err(C.numpy(), f["C"]) < 1e-10
    assert pbar_err(Pb.numpy(), Pbo, ex["P_abs"]) < 1e-10
    assert grad_err(Ab.numpy(), Abo) < 1e-10
    assert wbar_err(Wb.numpy(), Wbo) < 1e-9
