"""The batched configuration at its full size: 256 parameter points (seeded P(k) amplitude and
tilt, biases, window shifts) with ragged multipole lists of 50-103 entries, forward + VJP as one
CUDA-graph replay, the launch the bench times with --walkers 256.  Three walkers (first, middle,
last) are compared with the FP64 oracle one by one."""
import numpy as np
import pytest

from gpu_helpers import grad_err, lib_context, norm_err, oracle_walker, pbar_err, wbar_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def test_256_walkers_sampled_against_oracle():
    import torch
    import paper_2505_22718_gb300 as S
    from workloads import make_workload
    w = make_workload("walkers")
    assert w.W.shape[0] == 256
    dev = torch.device("cuda:0")
    ctx = lib_context(w)
    lens = [len(l) for l in w.ell_lists]
    off = np.concatenate([[0], np.cumsum(lens)])
    n_out = int(off[-1])
    Cb = np.random.default_rng(256).standard_normal((n_out, w.n_tr, w.n_tr))
    C = torch.empty((n_out, w.n_tr, w.n_tr), dtype=torch.float64, device=dev)
    Cb_d = torch.tensor(Cb, device=dev)
    Pb = torch.empty(w.P.shape, dtype=torch.float64, device=dev)
    Ab = torch.empty(w.amp.shape, dtype=torch.float64, device=dev)
    Wb = torch.empty(w.W.shape, dtype=torch.float64, device=dev)
    for _ in range(2):  # capture, then a replay
        S.swcl_compute_batched(ctx.ptr, S.SWCL_SPLIT_BF16, C, Cb_d, Pb, Ab, Wb)
    ctx.sync()
    C_h = C.cpu().numpy()
    assert np.all(np.isfinite(C_h))
    assert np.array_equal(C_h, np.transpose(C_h, (0, 2, 1)))
    for wk in (0, 137, 255):
        lst = w.ell_lists[wk]
        o, n = int(off[wk]), lens[wk]
        Cbw = np.zeros((len(w.ells), w.n_tr, w.n_tr))
        Cbw[lst] = Cb[o:o + n]
        f, (Pbo, Abo, Wbo, ex) = oracle_walker(w, wk, C_bar=Cbw)
        assert norm_err(C_h[o:o + n], f["C"][lst]) < 1e-4, wk
        assert pbar_err(Pb[wk].cpu().numpy(), Pbo, ex["P_abs"]) < 1e-4, wk
        assert grad_err(Ab[wk].cpu().numpy(), Abo) < 5e-5, wk
        assert wbar_err(Wb[wk].cpu().numpy(), Wbo) < 5e-5, wk
