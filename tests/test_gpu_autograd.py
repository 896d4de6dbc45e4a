"""The torch.autograd wrapper: gradients from the hand-written VJP against the oracle's reverse
mode, against central finite differences through the wrapper itself, and the chain rule to the
window mean shifts."""
import numpy as np
import pytest

from gpu_helpers import grad_err, norm_err, oracle_walker, pbar_err, wbar_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def _spec(w, precision):
    from paper_2505_22718_gb300 import AngularPowerSpectrum
    return AngularPowerSpectrum(w.chi_min, w.chi_max, w.N, w.k, w.ells, w.knots, w.kind, w.fft_bias,
                                w.D, w.B, precision=precision)


@pytest.mark.parametrize("precision,gate", [("fp64", 1e-10), ("bf16x9", 5e-5)])
def test_autograd_matches_oracle_gradient(precision, gate, wl):
    import torch
    w = wl("n5k_vjp")
    dev = torch.device("cuda:0")
    W = torch.tensor(w.W, device=dev, requires_grad=True)
    P = torch.tensor(w.P, device=dev, requires_grad=True)
    A = torch.tensor(w.amp, device=dev, requires_grad=True)
    spec = _spec(w, precision)
    C = spec(W, P, A)
    Cb = torch.tensor(w.C_bar, device=dev)
    (C * Cb).sum().backward()
    f, (Pbo, Abo, Wbo, ex) = oracle_walker(w, C_bar=w.C_bar)
    assert norm_err(C.detach().cpu().numpy(), f["C"]) < (1e-10 if precision == "fp64" else 1e-4)
    assert pbar_err(P.grad.cpu().numpy(), Pbo, ex["P_abs"]) < gate
    assert grad_err(A.grad.cpu().numpy(), Abo) < gate
    assert wbar_err(W.grad.cpu().numpy(), Wbo) < gate


def test_autograd_central_differences_fp64(wl):
    """d<C_bar, C>/dP, dA along random directions by central differences (relative step 1e-5)
    through the wrapper in FP64; C is linear in P and quadratic in A, so the differences are exact
    up to rounding."""
    import torch
    w = wl("tiny2")
    dev = torch.device("cuda:0")
    spec = _spec(w, "fp64")
    rng = np.random.default_rng(4)
    Cb = torch.tensor(rng.standard_normal((len(w.ells), 2, 2)), device=dev)
    W = torch.tensor(w.W, device=dev, requires_grad=True)
    P = torch.tensor(w.P, device=dev, requires_grad=True)
    A = torch.tensor(w.amp, device=dev, requires_grad=True)
    (spec(W, P, A) * Cb).sum().backward()
    L = lambda Wx, Px, Ax: float((spec(Wx, Px, Ax) * Cb).sum())  # noqa: E731
    h = 1e-5
    with torch.no_grad():
        dP = torch.tensor(rng.standard_normal(len(w.k)), device=dev) * P
        fd = (L(W, P + h * dP, A) - L(W, P - h * dP, A)) / (2 * h)
        assert abs(fd / float((P.grad * dP).sum()) - 1) < 1e-7
        dA = torch.tensor(rng.standard_normal(2), device=dev) * A
        fd = (L(W, P, A + h * dA) - L(W, P, A - h * dA)) / (2 * h)
        assert abs(fd / float((A.grad * dA).sum()) - 1) < 1e-7
        dW = torch.tensor(rng.standard_normal(W.shape), device=dev) * W
        fd = (L(W + h * dW, P, A) - L(W - h * dW, P, A)) / (2 * h)
        assert abs(fd / float((W.grad * dW).sum()) - 1) < 1e-6


def test_window_shift_gradients_by_chain_rule(wl):
    """d<C_bar, C>/d mu_i (the 15 window mean shifts) = <W_bar, dW/dmu_i>, with dW/dmu_i from the
    input builder, against central differences of the whole pipeline on the GPU (FP64)."""
    import torch
    from workloads.n5k_synth import window_rows
    w = wl("n5k_vjp")
    dev = torch.device("cuda:0")
    spec = _spec(w, "fp64")
    Cb = torch.tensor(w.C_bar, device=dev)
    W = torch.tensor(w.W, device=dev, requires_grad=True)
    P = torch.tensor(w.P, device=dev)
    A = torch.tensor(w.amp, device=dev)
    (spec(W, P, A) * Cb).sum().backward()
    Wb = W.grad.cpu().numpy()
    meta = w.meta
    for t in (0, 9, 10, 14):
        mu = meta["gauss"][t][0] if t < len(meta["gauss"]) else 0.0
        hz = 1e-5 * (1.0 + mu)
        sp = np.zeros(len(w.kind))
        sp[t] = hz
        Wp, Wm = window_rows(meta, sp), window_rows(meta, -sp)
        with torch.no_grad():
            Lp = float((spec(torch.tensor(Wp, device=dev), P, A) * Cb).sum())
            Lm = float((spec(torch.tensor(Wm, device=dev), P, A) * Cb).sum())
        fd = (Lp - Lm) / (2 * hz)
        chain = float(np.sum(Wb * (Wp - Wm)) / (2 * hz))
        assert abs(fd - chain) <= 1e-6 * abs(fd), (t, fd, chain)


def test_backward_after_a_second_forward(wl):
    """Two forward passes on one module, then backward of the first: the state is rebuilt."""
    import torch
    w = wl("tiny2")
    dev = torch.device("cuda:0")
    spec = _spec(w, "fp64")
    W = torch.tensor(w.W, device=dev, requires_grad=True)
    P = torch.tensor(w.P, device=dev, requires_grad=True)
    A = torch.tensor(w.amp, device=dev, requires_grad=True)
    C1 = spec(W, P, A)
    spec(W * 1.3, P * 0.5, A)          # overwrites the context's state
    rng = np.random.default_rng(1)
    Cb = rng.standard_normal(C1.shape)
    C1.backward(torch.tensor(Cb, device=dev))
    f, (Pbo, Abo, Wbo, ex) = oracle_walker(w, C_bar=Cb)
    assert pbar_err(P.grad.cpu().numpy()[0] if P.grad.dim() > 1 else P.grad.cpu().numpy(), Pbo, ex["P_abs"]) < 1e-10
    assert wbar_err(W.grad.cpu().numpy(), Wbo) < 1e-9
