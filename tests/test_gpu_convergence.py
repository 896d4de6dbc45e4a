"""Convergence of the library's C_l in its three numerical parameters (Appendix A: N_FFT, N_interp,
N_k) against the stored truth tests/golden/convergence_truth.txt (the FP64 oracle at converged
settings, spot-checked against brute-force line-of-sight quadrature), on the reduced N5K-shaped
case workloads.n5k_synth.convergence_case (a narrow and a wide clustering bin, one lensing bin,
9 multipoles in [2, 2000], a scale-dependent growth).

For each setting it prints the normalised error of reading R9 against the truth, the Gaussian
chi^2 of the difference (swcl_gaussian_fisher with X = C - C_truth, cosmic variance with
f_sky = 0.4363 and each multipole standing for its N5K log bin) and the forward time.  The
asserts check that each parameter converges: the FP64 error at the largest setting is at least
100x below the error at the smallest, and below 1e-4 (N_FFT, N_interp; the oracle reaches
9e-6 there, the algebraic convergence of the lens efficiency's kinks) or 1e-3 (N_k, whose truth
shares the N_k = 2048 trapezoid rule)."""
import os

import numpy as np
import pytest

from gpu_helpers import lib_context, norm_err

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
F_SKY = 0.4363


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


@pytest.fixture(scope="module")
def truth():
    rows = np.loadtxt(os.path.join(HERE, "golden", "convergence_truth.txt"))
    ells = np.unique(rows[:, 0]).astype(int)
    C = np.zeros((len(ells), 3, 3))
    for ell, i, j, v in rows:
        C[int(np.searchsorted(ells, ell)), int(i), int(j)] = v
    return ells, C


def _modes(ells):
    """(2l+1) f_sky times the width of the 103-bin log grid on [2, 2000] at l (at least 1)."""
    e = np.asarray(ells, dtype=np.float64)
    return (2.0 * e + 1.0) * F_SKY * np.maximum(1.0, e * np.log(1000.0) / 102.0)


def _run(N, n_interp, n_k, truth):
    import torch
    import paper_2505_22718_gb300 as S
    from workloads.n5k_synth import convergence_case
    ells, Ct = truth
    w = convergence_case(N=N, n_interp=n_interp, n_k=n_k)
    assert np.array_equal(w.ells, ells)
    ctx = lib_context(w)
    out = {}
    for name, p in (("bf16x9", S.SWCL_SPLIT_BF16), ("fp64", S.SWCL_FP64)):
        Cd = torch.empty((len(ells), 3, 3), dtype=torch.float64, device="cuda:0")
        for _ in range(2):
            S.swcl_compute_cl(ctx.ptr, p, Cd)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        e0.record(stream)
        reps = 5
        for _ in range(reps):
            S.swcl_compute_cl(ctx.ptr, p, Cd)
        ctx.sync()
        e1.record(stream)
        torch.cuda.synchronize()
        C = Cd.cpu().numpy()
        chi2 = ctx.gaussian_fisher((C - Ct)[None], _modes(ells))[0, 0]
        out[name] = (norm_err(C, Ct), chi2, e0.elapsed_time(e1) / reps)
    ctx.close()
    return out


def _sweep(label, settings, truth):
    res = []
    for N, ni, nk in settings:
        r = _run(N, ni, nk, truth)
        res.append(r)
        print("SWEEP %s N_FFT=%d N_interp=%d N_k=%d | fp64 err %.2e chi2 %.2e %.3f ms | "
              "bf16x9 err %.2e chi2 %.2e %.3f ms" % (label, N, ni, nk, *r["fp64"], *r["bf16x9"]))
    return [r["fp64"][0] for r in res]


def test_n_fft_convergence(truth):
    err = _sweep("N_FFT", [(n, 150, 2048) for n in (256, 512, 1024, 2048, 4096)], truth)
    assert err[-1] < 1e-2 * err[0]
    assert err[-1] < 1e-4


def test_n_interp_convergence(truth):
    err = _sweep("N_interp", [(4096, n, 2048) for n in (10, 20, 50, 100, 200, 400)], truth)
    assert err[-1] < 1e-2 * err[0]
    assert err[-1] < 1e-4


def test_n_k_convergence(truth):
    err = _sweep("N_k", [(4096, 150, n) for n in (128, 256, 512, 1024)], truth)
    assert err[-1] < 1e-2 * err[0]
    assert err[-1] < 1e-3
