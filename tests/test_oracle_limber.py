"""Pins of the oracle's Limber branch (Eq. 2.19, reading R12) and of the hybrid spectrum.

- closed form: Gaussian windows in ln chi, constant P, a growth D(chi) = e^{-gamma ln chi}, for
  density, lensing and magnification kinds (the chi measure, the nu powers and the prefactors);
- an independent Limber integral (oracle.brute.cl_limber: dense trapezoid with P as a function);
- the hand-written reverse mode against central differences and the homogeneity identities;
- the hybrid: FFTLog rows below the switch, Limber rows at and above it, gradients that add;
- the Limber branch approaches the FFTLog C_l at high l (Eq. 2.19 is its large-l limit).
"""
import numpy as np
import pytest

from oracle import fftlog as O
from oracle import limber as LB
from oracle.brute import cl_limber


def _gauss_case(kinds, N=1024, n_k=512):
    k = np.geomspace(1e-5, 1e2, n_k)
    ells = np.array([10, 100, 1000])
    knots = np.geomspace(1e-5, 1e2, 12)
    g = O.Grids(N, 1.0, 1e5, k, ells, knots, kinds, [-0.3] * len(kinds))
    x = np.log(g.chi)
    mus = np.log([900.0, 1100.0, 1300.0])[:len(kinds)]
    sig = np.array([0.15, 0.2, 0.25])[:len(kinds)]
    W = np.exp(-0.5 * ((x[None, :] - mus[:, None]) / sig[:, None]) ** 2)
    return g, x, mus, sig, W


def test_closed_form_gaussian_windows():
    kinds = [O.KIND_DENSITY, O.KIND_LENSING, O.KIND_MAGNIFICATION]
    g, x, mus, sig, W = _gauss_case(kinds)
    gam = 0.3
    D = np.tile(np.exp(-gam * x), (len(g.knots), 1))          # k-independent growth
    P0 = 2.5e4
    amp = np.array([1.3, 1.0, 0.7])
    U, C = LB.limber_cl(g, W, D, np.full(len(g.k), P0), amp)
    for li, ell in enumerate(g.ells):
        nu = ell + 0.5
        for i in range(3):
            for j in range(3):
                # with s = t the integrand of Eq. 2.19 in ln chi is pi_i pi_j nu^{t_i + t_j}
                # chi^-1 W_i W_j D^2 P0:
                # int exp(-(x-mu_i)^2/2s_i^2 - (x-mu_j)^2/2s_j^2 - (2 gam + 1) x) dx
                a = 0.5 / sig[i] ** 2 + 0.5 / sig[j] ** 2
                b = mus[i] / sig[i] ** 2 + mus[j] / sig[j] ** 2 - 2.0 * gam - 1.0
                c = 0.5 * mus[i] ** 2 / sig[i] ** 2 + 0.5 * mus[j] ** 2 / sig[j] ** 2
                integral = np.sqrt(np.pi / a) * np.exp(b * b / (4.0 * a) - c)
                pi_i = O.ell_prefactor([ell], kinds[i])[0]
                pi_j = O.ell_prefactor([ell], kinds[j])[0]
                t = O.k_power(kinds[i]) + O.k_power(kinds[j])
                want = amp[i] * amp[j] * P0 * pi_i * pi_j * nu ** t * integral
                assert abs(C[li, i, j] / want - 1.0) < 1e-12, (ell, i, j)


def test_against_dense_limber_integral(wl):
    """Density windows of the N5K-shaped workload, D = 1, a smooth P(k): the discrete
    form against the trapezoid rule on a 16x denser chi grid, with the windows rebuilt there and
    P evaluated exactly."""
    from workloads.n5k_synth import Cosmology, clustering_window
    w = wl("n5k")
    tr = [0, 4, 9]
    ells = np.array([20, 200, 1500])
    g = O.Grids(w.N, w.chi_min, w.chi_max, w.k, ells, w.knots, w.kind[tr], w.fft_bias[tr])
    # smooth P (no BAO-like wiggle), so the cubic interpolation in ln k of R12 is ~1e-9 of it
    Pf = lambda kk: 3.5e6 * kk ** 0.965 / (1.0 + (kk / 0.02) ** 2) ** 2  # noqa: E731
    D = np.ones((len(w.knots), w.N))
    _, C = LB.limber_cl(g, w.W[tr], D, Pf(w.k), np.ones(3))
    dense = w.chi_min * np.exp(np.arange(16 * w.N) * g.L / (16 * w.N))
    cosmo = Cosmology()
    Wd = np.array([clustering_window(cosmo, dense, *w.meta["gauss"][t]) for t in tr])
    kmax = w.k[-1]
    Pk = lambda kk, chi: np.where(kk <= kmax, Pf(kk), 0.0)          # noqa: E731
    for li, ell in enumerate(ells):
        for i in range(3):
            for j in range(i, 3):
                ref = cl_limber(ell, dense, Wd[i], Wd[j], Pk)
                if abs(ref) < 1e-6 * np.sqrt(abs(C[li, i, i] * C[li, j, j])):
                    continue
                assert abs(C[li, i, j] / ref - 1.0) < 1e-7, (ell, i, j, C[li, i, j], ref)


def _vjp_case(wl):
    w = wl("n5k_vjp")
    tr = np.array([0, 7, 10, 14])
    ells = np.array([150, 400, 1200])
    g = O.Grids(w.N, w.chi_min, w.chi_max, w.k, ells, w.knots, w.kind[tr], w.fft_bias[tr])
    rng = np.random.default_rng(4)
    Cb = rng.standard_normal((len(ells), 4, 4))
    return w, tr, g, Cb


def test_limber_vjp_identities_and_differences(wl):
    w, tr, g, Cb = _vjp_case(wl)
    W, P, amp = w.W[tr], w.P, w.amp[tr]
    _, C = LB.limber_cl(g, W, w.D, P, amp)
    Pb, Ab, Wb = LB.limber_vjp(g, W, w.D, P, amp, Cb)
    ip = np.sum(Cb * C)
    assert abs(np.sum(Pb * P) / ip - 1) < 1e-12
    assert abs(np.sum(Ab * amp) / (2 * ip) - 1) < 1e-12
    assert abs(np.sum(Wb * W) / (2 * ip) - 1) < 1e-12
    L = lambda Wx, Px, Ax: np.sum(Cb * LB.limber_cl(g, Wx, w.D, Px, Ax)[1])  # noqa: E731
    rng = np.random.default_rng(5)
    h = 1e-5
    for v, grad, which in [(rng.standard_normal(len(P)) * P, Pb, 1),
                           (rng.standard_normal(len(amp)), Ab, 2),
                           (rng.standard_normal(W.shape) * W, Wb, 0)]:
        args_p = [W, P, amp]
        args_m = [W, P, amp]
        args_p[which] = args_p[which] + h * v
        args_m[which] = args_m[which] - h * v
        fd = (L(*args_p) - L(*args_m)) / (2 * h)
        assert abs(fd / np.sum(grad * v) - 1) < 1e-6


def test_hybrid_rows_and_gradients(wl):
    w, tr, g, Cb = _vjp_case(wl)
    W, P, amp = w.W[tr], w.P, w.amp[tr]
    sw = 400
    C, f = LB.hybrid_forward(g, W, w.D, P, amp, sw)
    sel = g.ells >= sw
    assert np.array_equal(C[~sel], f["C"][~sel])
    assert np.array_equal(C[sel], LB.limber_cl(g, W, w.D, P, amp, ells=g.ells[sel])[1])
    Pb, Ab, Wb = LB.hybrid_vjp(g, f, Cb, W, w.D, P, amp, sw)
    ip = np.sum(Cb * C)
    assert abs(np.sum(Pb * P) / ip - 1) < 1e-12
    assert abs(np.sum(Wb * W) / (2 * ip) - 1) < 1e-12


def test_limber_approaches_fftlog_at_high_ell(wl):
    """Eq. 2.19 is the large-l limit: for broad clustering windows the relative difference of the
    auto-spectra falls with l and is below 1e-3 at l ~ 1000."""
    w = wl("n5k")
    tr = [2, 6]
    ells = np.array([30, 300, 1000])
    g = O.Grids(w.N, w.chi_min, w.chi_max, w.k, ells, w.knots, w.kind[tr], w.fft_bias[tr])
    f = O.forward(g, w.W[tr], w.D, w.P, w.amp[tr])
    _, CL = LB.limber_cl(g, w.W[tr], w.D, w.P, w.amp[tr])
    rel = np.abs(np.einsum("lii->li", CL) / np.einsum("lii->li", f["C"]) - 1.0)
    assert np.all(np.diff(rel.max(axis=1)) < 0), rel
    assert rel[-1].max() < 1e-3, rel


def test_rsd_has_no_limber_form():
    g = O.Grids(256, 1.0, 1e5, np.geomspace(1e-4, 1, 64), [10], [1e-4, 1.0], [O.KIND_RSD], [0.4])
    with pytest.raises(ValueError):
        LB.limber_cl(g, np.ones((1, 256)), np.ones((2, 256)), np.ones(64), [1.0])


def test_limber_jvp_against_vjp_and_differences(wl):
    """Forward mode of the Limber branch: central differences entry by entry, and
    <C_bar, J v> = <J^T C_bar, v> with the pinned reverse mode."""
    w, tr, g, Cb = _vjp_case(wl)
    W, P, amp = w.W[tr], w.P, w.amp[tr]
    rng = np.random.default_rng(12)
    dP = rng.standard_normal(len(P)) * P
    dA = rng.standard_normal(len(amp))
    dW = rng.standard_normal(W.shape) * W
    J = LB.limber_jvp(g, W, w.D, P, amp, P_dot=dP, amp_dot=dA, W_dot=dW)
    h = 1e-5
    fd = (LB.limber_cl(g, W + h * dW, w.D, P + h * dP, amp + h * dA)[1]
          - LB.limber_cl(g, W - h * dW, w.D, P - h * dP, amp - h * dA)[1]) / (2 * h)
    _, C = LB.limber_cl(g, W, w.D, P, amp)
    dg = np.sqrt(np.abs(np.einsum("lii->li", C)))
    assert np.max(np.abs(J - fd) / (dg[:, :, None] * dg[:, None, :])) < 1e-7
    Pb, Ab, Wb = LB.limber_vjp(g, W, w.D, P, amp, Cb)
    lhs = np.sum(Cb * J)
    rhs = np.sum(Pb * dP) + np.sum(Ab * dA) + np.sum(Wb * dW)
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)
