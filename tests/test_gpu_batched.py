"""Batched walkers through swcl_compute_batched (CUDA-graph capture and replay): ragged multipole
lists, per-walker P(k), amplitudes and window shifts; replay after a parameter update."""
import numpy as np
import pytest

from gpu_helpers import grad_err, lib_context, norm_err, oracle_walker, pbar_err, wbar_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


@pytest.fixture(scope="module")
def walkers8():
    from workloads import make_workload
    return make_workload("walkers", seed=123, n_walkers=6)


@pytest.mark.parametrize("prec", ["bf16x9", "fp64"])
def test_batched_graph_against_oracle(prec, walkers8):
    import torch
    import paper_2505_22718_gb300 as S
    w = walkers8
    dev = torch.device("cuda:0")
    ctx = lib_context(w)
    n_out = sum(len(l) for l in w.ell_lists)
    rng = np.random.default_rng(8)
    Cb = rng.standard_normal((n_out, w.n_tr, w.n_tr))
    C = torch.empty((n_out, w.n_tr, w.n_tr), dtype=torch.float64, device=dev)
    Cb_d = torch.tensor(Cb, device=dev)
    Pb = torch.empty(w.P.shape, dtype=torch.float64, device=dev)
    Ab = torch.empty(w.amp.shape, dtype=torch.float64, device=dev)
    Wb = torch.empty(w.W.shape, dtype=torch.float64, device=dev)
    precision = S.PRECISIONS[prec]
    for _ in range(3):  # capture, then two replays
        S.swcl_compute_batched(ctx.ptr, precision, C, Cb_d, Pb, Ab, Wb)
    ctx.sync()
    gate_c = 1e-10 if prec == "fp64" else 1e-4
    gate_g = 1e-9 if prec == "fp64" else 5e-5
    o = 0
    for wk, lst in enumerate(w.ell_lists):
        n = len(lst)
        Cbw = np.zeros((len(w.ells), w.n_tr, w.n_tr))
        Cbw[lst] = Cb[o:o + n]
        f, (Pbo, Abo, Wbo, ex) = oracle_walker(w, wk, C_bar=Cbw)
        assert norm_err(C[o:o + n].cpu().numpy(), f["C"][lst]) < gate_c, wk
        assert pbar_err(Pb[wk].cpu().numpy(), Pbo, ex["P_abs"]) < gate_g
        assert grad_err(Ab[wk].cpu().numpy(), Abo) < gate_g
        assert wbar_err(Wb[wk].cpu().numpy(), Wbo) < gate_g
        o += n


def test_graph_replay_follows_parameter_updates(walkers8):
    """A replay after swcl_set_power reads the new parameters (the graph references the context's
    buffers) and agrees bit for bit with the direct call."""
    import torch
    import paper_2505_22718_gb300 as S
    w = walkers8
    dev = torch.device("cuda:0")
    ctx = lib_context(w)
    n_out = sum(len(l) for l in w.ell_lists)
    C = torch.empty((n_out, w.n_tr, w.n_tr), dtype=torch.float64, device=dev)
    S.swcl_compute_batched(ctx.ptr, S.SWCL_SPLIT_BF16, C)
    S.swcl_compute_batched(ctx.ptr, S.SWCL_SPLIT_BF16, C)
    P2 = torch.tensor(w.P * 1.7, device=dev)
    A2 = torch.tensor(w.amp * 0.9, device=dev)
    S.swcl_set_power(ctx.ptr, w.W.shape[0], P2, A2)
    S.swcl_compute_batched(ctx.ptr, S.SWCL_SPLIT_BF16, C)
    direct = torch.empty_like(C)
    S.swcl_compute_cl(ctx.ptr, S.SWCL_SPLIT_BF16, direct)
    ctx.sync()
    assert torch.equal(C, direct)
    ctx2 = lib_context(w)
    ref = torch.empty_like(C)
    S.swcl_set_power(ctx2.ptr, w.W.shape[0], P2, A2)
    S.swcl_compute_cl(ctx2.ptr, S.SWCL_SPLIT_BF16, ref)
    ctx2.sync()
    assert torch.equal(C, ref)
