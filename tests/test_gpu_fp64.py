"""Parity of the FP64 CUDA path with the FP64 oracle (gate 1e-10, normalised as
max(|C_ij|, 1e-3 sqrt(C_ii C_jj)) for C; relative to the largest entry for gradients)."""
import numpy as np
import pytest

from gpu_helpers import grad_err, lib_context, make_ragged_case, max_rel, norm_err, oracle_walker, pbar_err, wbar_err

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def test_tiny2_forward(wl):
    from paper_2505_22718_gb300 import SWCL_FP64
    w = wl("tiny2")
    ctx = lib_context(w)
    C = ctx.compute_cl(SWCL_FP64)
    f, _ = oracle_walker(w)
    assert C.shape == f["C"].shape
    assert norm_err(C, f["C"]) < TOL
    assert np.array_equal(C, np.transpose(C, (0, 2, 1)))


def test_n5k_forward_and_vjp(wl):
    from paper_2505_22718_gb300 import SWCL_FP64
    w = wl("n5k_vjp")
    ctx = lib_context(w)
    C = ctx.compute_cl(SWCL_FP64)
    Pb, Ab, Wb = ctx.vjp(w.C_bar, SWCL_FP64)
    f, (Pbo, Abo, Wbo, ex) = oracle_walker(w, C_bar=w.C_bar)
    assert norm_err(C, f["C"]) < TOL
    assert np.array_equal(C, np.transpose(C, (0, 2, 1)))
    for ell in range(C.shape[0]):
        ev = np.linalg.eigvalsh(C[ell])
        assert ev[0] >= -1e-12 * ev[-1]
    assert pbar_err(Pb[0], Pbo, ex["P_abs"]) < TOL
    assert grad_err(Ab[0], Abo) < TOL
    assert wbar_err(Wb[0], Wbo) < 1e-9


def test_ragged_walkers_tapers_bias():
    """7 tracers with B(k, z), tapers, 333 k (ragged k tile), 37 ells, 23 knots, 3 walkers with
    ragged ell lists; forward and VJP per walker against the oracle."""
    from paper_2505_22718_gb300 import SWCL_FP64
    w, tapers = make_ragged_case()
    ctx = lib_context(w, tapers)
    C = ctx.compute_cl(SWCL_FP64)
    rng = np.random.default_rng(2)
    Cb = rng.standard_normal(C.shape)
    Pb, Ab, Wb = ctx.vjp(Cb, SWCL_FP64)
    o = 0
    for wk, lst in enumerate(w.ell_lists):
        n = len(lst)
        Cbw = np.zeros((len(w.ells), 7, 7))
        Cbw[lst] = Cb[o:o + n]
        f, (Pbo, Abo, Wbo, ex) = oracle_walker(w, wk, tapers, C_bar=Cbw)
        assert norm_err(C[o:o + n], f["C"][lst]) < TOL, wk
        assert pbar_err(Pb[wk], Pbo, ex["P_abs"]) < TOL
        assert grad_err(Ab[wk], Abo) < TOL
        assert wbar_err(Wb[wk], Wbo) < 1e-9
        o += n
    assert o == C.shape[0]


def test_device_pointers_and_bitwise_repeat(wl):
    """Inputs and outputs as CUDA tensors (no host copies); two calls agree bit for bit."""
    import torch
    from paper_2505_22718_gb300 import SWCL_FP64, Context
    w = wl("tiny2")
    dev = torch.device("cuda:0")
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    ctx = Context(0)
    ctx.set_grids(w.chi_min, w.chi_max, w.N, t(w.k), t(w.ells, torch.int32), t(w.knots))
    ctx.set_tracers(t(w.kind, torch.int32), t(w.fft_bias))
    ctx.set_windows(t(w.W), t(w.D))
    ctx.set_power(t(w.P), t(w.amp))
    out1 = torch.empty((len(w.ells), 2, 2), dtype=torch.float64, device=dev)
    out2 = torch.empty_like(out1)
    ctx.compute_cl(SWCL_FP64, out1)
    ctx.compute_cl(SWCL_FP64, out2)
    ctx.sync()
    assert torch.equal(out1, out2)
    f, _ = oracle_walker(w)
    assert norm_err(out1.cpu().numpy(), f["C"]) < TOL


def test_errors_are_status_codes(wl):
    from paper_2505_22718_gb300 import SWCL_FP64, Context, SwiftClError
    w = wl("tiny2")
    ctx = Context(0)
    with pytest.raises(SwiftClError) as e:
        ctx.compute_cl(SWCL_FP64, np.empty((20, 2, 2)))
    assert e.value.status == -7
    with pytest.raises(SwiftClError) as e:
        ctx.set_grids(w.chi_min, w.chi_max, 300, w.k, w.ells, w.knots)
    assert e.value.status == -1
    with pytest.raises(SwiftClError) as e:
        ctx.set_grids(w.chi_min, w.chi_max, w.N, w.k[::-1].copy(), w.ells, w.knots)
    assert e.value.status == -1
    ctx.set_grids(w.chi_min, w.chi_max, w.N, w.k, w.ells, w.knots)
    with pytest.raises(SwiftClError) as e:
        ctx.set_tracers(w.kind, np.array([-0.3, 1.2]))
    assert e.value.status == -1
    with pytest.raises(SwiftClError) as e:
        ctx.set_tracers(np.array([0, 7], np.int32), w.fft_bias)
    assert e.value.status == -1
    small = Context(0, mem_budget_bytes=1 << 16)
    with pytest.raises(SwiftClError) as e:
        small.set_grids(w.chi_min, w.chi_max, w.N, w.k, w.ells, w.knots)
    assert e.value.status == -3
