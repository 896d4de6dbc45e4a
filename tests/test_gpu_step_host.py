"""swcl_step_host: one sampler step with page-locked host arrays (inputs in, forward + VJP,
results out, in one CUDA-graph replay).  Against the oracle, against swcl_compute_batched on the
same inputs, across steps with new parameters, and its error paths (pageable arrays, a NaN
planted in the inputs on the host)."""
import numpy as np
import pytest

from gpu_helpers import grad_err, lib_context, norm_err, oracle_walker, pbar_err, wbar_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def _pinned(a):
    import torch
    t = torch.empty(np.shape(a), dtype=torch.float64, pin_memory=True)
    t.numpy()[...] = a
    return t


def _outputs(w, n_out):
    import torch
    mk = lambda shape: torch.empty(shape, dtype=torch.float64, pin_memory=True)  # noqa: E731
    return mk((n_out, w.n_tr, w.n_tr)), mk(w.P.shape), mk(w.amp.shape), mk(w.W.shape)


@pytest.fixture(scope="module")
def walkers():
    from workloads import make_workload
    return make_workload("walkers", seed=321, n_walkers=4)


@pytest.mark.parametrize("prec", ["bf16x9", "fp64"])
def test_step_host_against_oracle_and_device_path(prec, walkers):
    import torch
    import paper_2505_22718_gb300 as S
    w = walkers
    ctx = lib_context(w)
    precision = S.PRECISIONS[prec]
    n_out = sum(len(l) for l in w.ell_lists)
    Cb = np.random.default_rng(3).standard_normal((n_out, w.n_tr, w.n_tr))
    W_h, P_h, A_h, Cb_h = _pinned(w.W), _pinned(w.P), _pinned(w.amp), _pinned(Cb)
    C_h, Pb_h, Ab_h, Wb_h = _outputs(w, n_out)
    for _ in range(3):   # capture, then two replays
        S.swcl_step_host(ctx.ptr, precision, C_h, W_h, P_h, A_h, Cb_h, Pb_h, Ab_h, Wb_h)
    gate_c = 1e-10 if prec == "fp64" else 1e-4
    gate_g = 1e-9 if prec == "fp64" else 5e-5
    o = 0
    for wk, lst in enumerate(w.ell_lists):
        n = len(lst)
        Cbw = np.zeros((len(w.ells), w.n_tr, w.n_tr))
        Cbw[lst] = Cb[o:o + n]
        f, (Pbo, Abo, Wbo, ex) = oracle_walker(w, wk, C_bar=Cbw)
        assert norm_err(C_h[o:o + n].numpy(), f["C"][lst]) < gate_c, wk
        assert pbar_err(Pb_h[wk].numpy(), Pbo, ex["P_abs"]) < gate_g
        assert grad_err(Ab_h[wk].numpy(), Abo) < gate_g
        assert wbar_err(Wb_h[wk].numpy(), Wbo) < gate_g
        o += n
    # the device-pointer graph on the same context and inputs: the same kernels
    dev = torch.device("cuda:0")
    C = torch.empty(C_h.shape, dtype=torch.float64, device=dev)
    Pb = torch.empty(Pb_h.shape, dtype=torch.float64, device=dev)
    Ab = torch.empty(Ab_h.shape, dtype=torch.float64, device=dev)
    Wb = torch.empty(Wb_h.shape, dtype=torch.float64, device=dev)
    S.swcl_compute_batched(ctx.ptr, precision, C, Cb_h.to(dev), Pb, Ab, Wb)
    ctx.sync()
    assert np.array_equal(C.cpu().numpy(), C_h.numpy())
    for a, b in ((Pb, Pb_h), (Ab, Ab_h), (Wb, Wb_h)):
        a, b = a.cpu().numpy(), b.numpy()
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))   # FP64 atomics may reorder


def test_step_host_follows_new_inputs(walkers):
    """Each replay reads the host arrays as they are at the call: new window samples, P and
    amplitudes give the results of a context set up with them."""
    import copy

    import paper_2505_22718_gb300 as S
    w = walkers
    ctx = lib_context(w)
    prec = S.SWCL_SPLIT_BF16
    n_out = sum(len(l) for l in w.ell_lists)
    Cb = np.random.default_rng(4).standard_normal((n_out, w.n_tr, w.n_tr))
    W_h, P_h, A_h, Cb_h = _pinned(w.W), _pinned(w.P), _pinned(w.amp), _pinned(Cb)
    C_h, Pb_h, Ab_h, Wb_h = _outputs(w, n_out)
    S.swcl_step_host(ctx.ptr, prec, C_h, W_h, P_h, A_h, Cb_h, Pb_h, Ab_h, Wb_h)
    # new parameters written into the same pinned arrays
    rng = np.random.default_rng(9)
    w2 = copy.copy(w)
    w2.P = w.P * (1.0 + 0.05 * rng.standard_normal(w.P.shape[-1]))
    w2.amp = w.amp * 1.07
    w2.W = np.roll(w.W, 3, axis=-1)
    P_h.numpy()[...] = w2.P
    A_h.numpy()[...] = w2.amp
    W_h.numpy()[...] = w2.W
    S.swcl_step_host(ctx.ptr, prec, C_h, W_h, P_h, A_h, Cb_h, Pb_h, Ab_h, Wb_h)
    # a context set up with the new parameters (its autotuner may choose other GEMM tiles, whose
    # sums round differently: far below the mixed-precision gate, not bit for bit)
    ref = lib_context(w2)
    C2 = ref.compute_cl(prec)
    Pb2, Ab2, Wb2 = ref.vjp(Cb, prec)
    assert norm_err(C_h.numpy(), C2) < 1e-5
    for a, b in ((Pb_h, Pb2), (Ab_h, Ab2), (Wb_h, Wb2)):
        assert np.max(np.abs(a.numpy() - b)) <= 1e-5 * np.max(np.abs(b))
    # forward only, keeping the inputs of the last step
    C_f = _outputs(w, n_out)[0]
    S.swcl_step_host(ctx.ptr, prec, C_f)
    assert np.array_equal(C_f.numpy(), C_h.numpy())


def test_step_host_rejects_pageable_arrays_and_reports_nonfinite(walkers):
    import paper_2505_22718_gb300 as S
    w = walkers
    ctx = lib_context(w)
    prec = S.SWCL_SPLIT_BF16
    n_out = sum(len(l) for l in w.ell_lists)
    C_h = _outputs(w, n_out)[0]
    with pytest.raises(S.SwiftClError) as e:
        S.swcl_step_host(ctx.ptr, prec, np.zeros(C_h.shape), _pinned(w.W))
    assert e.value.status == S.SWCL_ERR_INVALID_ARG and "page-locked" in str(e.value)
    with pytest.raises(S.SwiftClError) as e:
        S.swcl_step_host(ctx.ptr, prec, C_h, None, _pinned(w.P), None)
    assert e.value.status == S.SWCL_ERR_INVALID_ARG
    # a NaN in one window sample, planted on the host
    Wn = w.W.copy()
    Wn[1, 2, 700] = np.nan
    W_h, P_h, A_h = _pinned(Wn), _pinned(w.P), _pinned(w.amp)
    with pytest.raises(S.SwiftClError) as e:
        S.swcl_step_host(ctx.ptr, prec, C_h, W_h, P_h, A_h)
    assert e.value.status == S.SWCL_ERR_NONFINITE
    # the status word is cleared: the next step with finite inputs succeeds
    W_h.numpy()[...] = w.W
    S.swcl_step_host(ctx.ptr, prec, C_h, W_h, P_h, A_h)
    assert np.all(np.isfinite(C_h.numpy()))


def test_host_step_object_matches_the_call(walkers):
    """HostStep (arguments prepared once) runs the same graph as swcl_step_host, and each call
    reads the host arrays as they are then."""
    import paper_2505_22718_gb300 as S
    w = walkers
    ctx = lib_context(w)
    prec = S.SWCL_SPLIT_BF16
    n_out = sum(len(l) for l in w.ell_lists)
    Cb = np.random.default_rng(6).standard_normal((n_out, w.n_tr, w.n_tr))
    W_h, P_h, A_h, Cb_h = _pinned(w.W), _pinned(w.P), _pinned(w.amp), _pinned(Cb)
    C_h, Pb_h, Ab_h, Wb_h = _outputs(w, n_out)
    S.swcl_step_host(ctx.ptr, prec, C_h, W_h, P_h, A_h, Cb_h, Pb_h, Ab_h, Wb_h)
    ref = [t.numpy().copy() for t in (C_h, Pb_h, Ab_h, Wb_h)]
    step = S.HostStep(ctx.ptr, prec, C_h, W_h, P_h, A_h, Cb_h, Pb_h, Ab_h, Wb_h)
    for t in (C_h, Pb_h, Ab_h, Wb_h):
        t.zero_()
    step()
    assert np.array_equal(C_h.numpy(), ref[0])
    for a, b in zip((Pb_h, Ab_h, Wb_h), ref[1:]):
        assert np.max(np.abs(a.numpy() - b)) <= 1e-12 * np.max(np.abs(b))
    A_h.numpy()[...] = w.amp * 2.0       # C is quadratic in the amplitudes
    step()
    assert np.max(np.abs(C_h.numpy() - 4.0 * ref[0])) <= 1e-12 * np.max(np.abs(ref[0]))
