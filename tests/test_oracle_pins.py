"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test names the passage it pins and the mistake it would catch.  None of
them needs a GPU or the CUDA library.
"""
import os

import numpy as np
import pytest
from scipy.special import spherical_jn

from oracle import fftlog as O
from oracle.brute import cl_limber, delta_brute, spherical_jn_recurrence

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#", ndmin=2)


# ------------------------------------------------------------ tools ----

@pytest.mark.parametrize("ell", [0, 1, 2, 10, 50, 200, 2000])
def test_bessel_recurrence_matches_library(ell):
    """The brute-force checker's j_ell (recurrence) against scipy's spherical_jn."""
    x = np.concatenate([np.geomspace(1e-2, 5 * ell + 10, 300), [np.pi, 2 * np.pi, ell + 1e-9]])
    a, b = spherical_jn_recurrence(ell, x), spherical_jn(ell, x)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.abs(b).max()


# ---------------------------------------------------- Gamma table (a2) ----

def test_gamma_ratio_matches_mellin_integral():
    """Eq. (3.4): the Gamma-ratio equals int x^p j_ell(x) dx computed from the definition
    (stored mpmath quadrature).  This decides reading R1: the printed "+p" in the
    denominator fails by O(1)."""
    tab = _load("mellin_real_p.txt")
    for ell, p, ref in tab:
        ell = int(ell)
        ours = O.bessel_power_integral([ell], [p])[0, 0]
        assert abs(ours.imag) == 0.0
        assert abs(ours.real / ref - 1.0) < 1e-12, (ell, p, ours, ref)
        # printed form, Gamma((2 + ell + p)/2): wrong
        from scipy.special import gamma
        printed = np.sqrt(np.pi) * 2 ** (p - 1) * gamma(0.5 * (1 + ell + p)) / gamma(0.5 * (2 + ell + p))
        assert abs(printed / ref - 1.0) > 1e-2


def test_gamma_ratio_matches_mp50():
    """The table the contraction uses, complex p = b + i eta up to |eta| = 2000 and ell = 3000,
    against 50-digit mpmath.  The oracle starts from log-Gammas at ell = 2, 3 and recurs upward
    (reading R8), so the tolerance is the base error ~eps |lnG(base)| plus ~4 eps per recurrence
    step; at small |eta| this is ~1e-13 even at ell = 3000."""
    from scipy.special import loggamma
    tab = _load("gamma_ratio_mp50.txt")
    eps = np.finfo(float).eps
    for ell, b, eta, re, im in tab:
        ref = complex(re, im)
        ells = [2, 3] + ([int(ell)] if ell > 3 else [])
        ours = O.bessel_power_integral(ells, [complex(b, eta)])[ells.index(int(ell)), 0]
        p = complex(b, eta)
        l0 = 2 if int(ell) % 2 == 0 else 3
        base = abs(loggamma(0.5 * (l0 + 1 + p))) + abs(loggamma(0.5 * (l0 + 2 - p)))
        tol = 8 * eps * base + 4 * eps * (ell - l0) / 2 + 1e-14
        assert abs(ours / ref - 1.0) < tol, (ell, b, eta, ours, ref, tol)
        if abs(eta) < 100:
            assert abs(ours / ref - 1.0) < 2e-13


# --------------------------------------------------------- FFTLog (a1) ----

@pytest.mark.parametrize("b", [-0.3, -1.5])
def test_fftlog_reconstructs_grid_samples(b):
    """Eq. (3.1)-(3.2) with readings R2, R3: sum_n c_n chi_m^{b + i eta_n} = F(chi_m) exactly on the grid.
    Catches a wrong DFT sign, a missing chi_min phase, a wrong eta_n or Nyquist weight."""
    N = 64
    rng = np.random.default_rng(1)
    F = rng.standard_normal(N)
    chi = O.chi_grid(1.0, 1e5, N)
    c = O.fftlog_coefficients(F[None, :], 1.0, 1e5, b)
    # compare in the scale of g = F chi^-b, the sequence that is transformed
    rec = O.fftlog_reconstruct(c, chi, b, 1.0, 1e5)[0] * chi ** (-b)
    gs = F * chi ** (-b)
    assert np.max(np.abs(rec.imag)) < 1e-12 * np.abs(gs).max()
    assert np.max(np.abs(rec.real - gs)) < 1e-12 * np.abs(gs).max()
    # a chi_min other than 1 exercises the chi_min^{-i eta} factor
    chi2 = O.chi_grid(3.7, 2.0e4, N)
    c2 = O.fftlog_coefficients(F[None, :], 3.7, 2.0e4, b)
    rec2 = O.fftlog_reconstruct(c2, chi2, b, 3.7, 2.0e4)[0] * chi2 ** (-b)
    gs2 = F * chi2 ** (-b)
    assert np.max(np.abs(rec2 - gs2)) < 1e-12 * np.abs(gs2).max()


@pytest.mark.parametrize("b", [-0.3, -1.5])
@pytest.mark.parametrize("m", [0, 5, 64])
def test_powerlaw_window_closed_form(b, m):
    """a1 + a3: a window with W chi^-b = cos(eta_m ln(chi/chi_min)) has c_{+-m} = chi_min^{-+i eta_m}/2,
    so Delta(ell, k) = Re[chi_min^{-i eta_m} I_ell(b + i eta_m) k^{-1-b-i eta_m}] in closed form
    (m = N/2 tests the Nyquist weight).  chi_min = 2.5 keeps the chi_min phase non-trivial."""
    N, cmin, cmax = 128, 2.5, 2.5e5
    L = np.log(cmax / cmin)
    k = np.geomspace(1e-3, 1.0, 9)
    ells = [2, 10, 50]
    g = O.Grids(N, cmin, cmax, k, ells, [0.1], [0], [b])
    eta_m = 2 * np.pi * m / L
    W = (np.cos(eta_m * np.log(g.chi / cmin)) * g.chi ** b)[None, :]
    coef = O.window_coefficients(g, W, np.ones((1, N)))
    d, imag = O.delta_from_coefficients(g, coef)
    I = O.bessel_power_integral(ells, [b + 1j * eta_m])[:, 0]
    exact = np.real(cmin ** (-1j * eta_m) * I[:, None] * k[None, :] ** (-1 - b - 1j * eta_m))
    assert imag < 1e-13
    assert np.max(np.abs(d[:, 0, :] - exact)) <= 1e-12 * np.abs(exact).max()


def test_delta_matches_brute_force_quadrature():
    """a1 + a3 truth: Delta_ell(k) = int W j_ell(k chi) dchi (Eq. 2.2) by brute-force quadrature with
    j_ell from the recurrence, for a Gaussian window, ell in {2, 10, 50, 200}, 8 k values."""
    N, cmin, cmax = 2048, 1.0, 1e5
    k = np.geomspace(1e-3, 0.5, 8)
    ells = [2, 10, 50, 200]
    g = O.Grids(N, cmin, cmax, k, ells, [0.1], [0], [-0.3])
    win = lambda x: np.exp(-0.5 * ((x - 1000.0) / 100.0) ** 2)  # noqa: E731
    coef = O.window_coefficients(g, win(g.chi)[None, :], np.ones((1, N)))
    d, _ = O.delta_from_coefficients(g, coef)
    for li, ell in enumerate(ells):
        br = delta_brute(ell, k, win, 1.0, 2500.0)
        sel = np.abs(br) > 1e-3 * np.abs(br).max()
        rel = np.abs(d[li, 0, :] - br)[sel] / np.abs(br[sel])
        assert rel.max() < 1e-8, (ell, rel.max())


def test_lensing_delta_matches_brute_force(wl):
    """Lensing source function (Eq. 2.14): FFTLog of W^kappa chi^-2 with b = -1.5 against brute force
    of sqrt((l+2)!/(l-2)!) k^-2 int W^kappa chi^-2 j_ell(k chi) dchi for one Smail bin."""
    from workloads.n5k_synth import Cosmology, lensing_window, smail_bin_edges
    cosmo = Cosmology()
    edges = smail_bin_edges(5)
    lo, hi = edges[1], edges[2]
    N = 2048
    k = np.geomspace(3e-3, 0.3, 6)
    ells = [2, 20, 100]
    g = O.Grids(N, 1.0, 1e5, k, ells, [0.1], [1], [-1.5])
    W = lensing_window(cosmo, g.chi, lo, hi)[None, :]
    coef = O.window_coefficients(g, W, np.ones((1, N)))
    d, _ = O.delta_from_coefficients(g, coef)
    chi_hi = float(cosmo.chi(hi)) * 1.0000001
    f = lambda x: lensing_window(cosmo, x.ravel(), lo, hi).reshape(x.shape) / x ** 2  # noqa: E731
    for li, ell in enumerate(ells):
        pre = np.sqrt((ell + 2.0) * (ell + 1.0) * ell * (ell - 1.0))
        br = pre * k ** -2 * delta_brute(ell, k, f, 1e-6, chi_hi, tol=1e-10)
        sel = np.abs(br) > 1e-2 * np.abs(br).max()
        rel = np.abs(d[li, 0, :] - br)[sel] / np.abs(br[sel])
        assert rel.max() < 1e-4, (ell, rel.max())


# --------------------------------------------------- interpolation (a3) ----

def test_lagrange_weights_partition_and_cubic_exactness():
    """Reading R5: weights sum to one and reproduce cubics in ln k exactly; one knot is constant."""
    k = np.geomspace(1e-4, 10.0, 301)
    knots = np.geomspace(1e-4, 10.0, 23)
    lam = O.lagrange_matrix(k, knots)
    assert np.allclose(lam.sum(axis=1), 1.0, atol=1e-14)
    assert np.all((lam != 0).sum(axis=1) <= 4)
    x, xk = np.log(k), np.log(knots)
    for poly in ([1.0, -2.0, 0.5, 0.03], [0.0, 0.0, 0.0, 1.0]):
        f = np.polyval(poly, xk)
        assert np.max(np.abs(lam @ f - np.polyval(poly, x))) < 1e-9
    assert np.all(O.lagrange_matrix(k, [0.1]) == 1.0)


def test_interpolation_exact_for_growth_linear_in_lnk(wl):
    """Sec. 3.2: with D(k, z) = D(z)(1 + 0.01 ln(k/0.1)) the coefficients are linear in ln k, so
    Delta from 150 interpolated knots equals Delta with the growth applied at every k."""
    w = wl("n5k")
    tr = [0, 12]
    ells = w.ells[::20]
    q = np.arange(0, len(w.k), 37)
    g1 = O.Grids(w.N, w.chi_min, w.chi_max, w.k, ells, w.knots, w.kind[tr], w.fft_bias[tr])
    c1 = O.window_coefficients(g1, w.W[tr], w.D)
    d1, _ = O.delta_from_coefficients(g1, c1, q_index=q)
    kq = w.k[q]
    Dq = (w.D[0] / (1.0 + 0.01 * np.log(w.knots[0] / 0.1)))[None, :] * (1.0 + 0.01 * np.log(kq / 0.1))[:, None]
    g2 = O.Grids(w.N, w.chi_min, w.chi_max, kq, ells, kq, w.kind[tr], w.fft_bias[tr])
    c2 = O.window_coefficients(g2, w.W[tr], Dq)
    d2, _ = O.delta_from_coefficients(g2, c2)
    assert np.max(np.abs(d1 - d2)) <= 1e-12 * np.abs(d2).max()


# ---------------------------------------------------- k-quadrature (a4) ----

def test_lnk_trapezoid_second_order():
    """Reading R6: the rule integrates int k^2 e^-k dk over [1e-4, 30] with O(h^2) error, and is
    exact for integrands linear in ln k in the measure dln k = dk/k (which fixes the half
    intervals at the two ends), on an uneven grid."""
    k = np.sort(np.random.default_rng(3).uniform(1e-4, 30.0, 57))
    w = O.lnk_trapezoid_weights(k)
    lk = np.log(k)
    for a, b in ((1.0, 0.0), (0.3, -1.7)):
        exact = a * (lk[-1] - lk[0]) + 0.5 * b * (lk[-1] ** 2 - lk[0] ** 2)
        assert abs(np.sum(w * (a + b * lk) / k) - exact) <= 1e-13 * max(abs(exact), 1.0)
    errs = []
    for n in (200, 400, 800):
        k = np.geomspace(1e-4, 30.0, n)
        w = O.lnk_trapezoid_weights(k)
        exact = 2.0 - np.exp(-30.0) * (900 + 60 + 2) - (2.0 - np.exp(-1e-4) * (1e-8 + 2e-4 + 2))
        errs.append(abs(np.sum(w * k ** 2 * np.exp(-k)) - exact))
    assert errs[1] < errs[0] / 3.5 and errs[2] < errs[1] / 3.5


def test_cl_symmetric_psd_and_scaling(wl):
    """C^{ij} = C^{ji}; C_ell is positive semidefinite (a Gram matrix with u_q > 0);
    C scales as A_i A_j and linearly in P."""
    w = wl("tiny2")
    g = O.Grids(w.N, w.chi_min, w.chi_max, w.k, w.ells, w.knots, w.kind, w.fft_bias)
    f = O.forward(g, w.W, w.D, w.P, w.amp)
    C = f["C"]
    assert np.max(np.abs(C - np.transpose(C, (0, 2, 1)))) <= 1e-15 * np.abs(C).max()
    for l in range(C.shape[0]):
        ev = np.linalg.eigvalsh(C[l])
        assert ev[0] >= -1e-12 * ev[-1]
    A2 = w.amp * np.array([3.0, 0.5])
    C2 = O.angular_cl(f["delta"], O.cl_weights(w.k, 2.5 * w.P), A2)
    ratio = np.outer(A2, A2) / np.outer(w.amp, w.amp) * 2.5
    dg = np.abs(np.einsum("lii->li", C2))
    scale = np.sqrt(dg[:, :, None] * dg[:, None, :])
    assert np.max(np.abs(C2 - C * ratio[None]) / scale) < 1e-14


def test_cl_matches_brute_force_double_quadrature():
    """a4 truth, Eq. (2.1) with Eq. (2.2): the oracle's C_ell (FFTLog Delta, ln-k trapezoid of
    reading R6 on a dense k grid) against C_ell with both integrals done by brute force (stored;
    tests/golden/make_golden.py).  Catches a wrong 2/pi or k^2 in the measure, a wrong trapezoid
    end weight, and any Delta error that the per-k pins could miss in the integrated spectrum."""
    tab = _load("cl_brute_gauss.txt")
    ells = sorted({int(r[0]) for r in tab})
    N, cmin, cmax = 4096, 1.0, 1e5
    k = np.geomspace(1e-4, 0.3, 3000)
    wins = [(1000.0, 100.0), (1250.0, 120.0)]
    g = O.Grids(N, cmin, cmax, k, ells, [0.1], [0, 0], [-0.3, -0.3])
    W = np.array([np.exp(-0.5 * ((g.chi - m) / s) ** 2) for m, s in wins])
    f = O.forward(g, W, np.ones((1, N)), k / (1.0 + (k / 0.02) ** 2) ** 2, [1.0, 1.0])
    C = f["C"]
    ref = np.zeros_like(C)
    for ell, i, j, v in tab:
        ref[ells.index(int(ell)), int(i), int(j)] = v
    dg = np.einsum("lii->li", ref)
    scale = np.sqrt(dg[:, :, None] * dg[:, None, :])
    # measured 2e-14: at N = 4096 over [1, 1e5) the FFTLog and the trapezoid are converged here
    assert np.max(np.abs(C - ref) / scale) < 1e-10


def test_limber_limit_at_high_ell():
    """Eq. (2.19): for a broad window the beyond-Limber C_ell approaches the Limber integral as ell grows,
    with an error of order 1/ell (Sec. 2.6)."""
    N, cmin, cmax = 2048, 1.0, 1e5
    k = np.geomspace(1e-4, 10.0, 8192)
    ells = [100, 300, 1000, 3000]
    b = -0.3
    g = O.Grids(N, cmin, cmax, k, ells, [0.1], [0], [b])
    win = lambda x: np.exp(-0.5 * (np.log(x / 2000.0) / 0.35) ** 2) / x  # noqa: E731
    coef = O.window_coefficients(g, win(g.chi)[None, :], np.ones((1, N)))
    d, _ = O.delta_from_coefficients(g, coef)
    Pk = lambda kk: kk / (1.0 + (kk / 0.02) ** 2) ** 2  # noqa: E731
    C = O.angular_cl(d, O.cl_weights(k, Pk(k)), [1.0])[:, 0, 0]
    chi = np.geomspace(20.0, 2e5, 200001)
    CL = np.array([cl_limber(l, chi, win(chi), win(chi), lambda kk, c: Pk(kk)) for l in ells])
    err = np.abs(C / CL - 1.0)
    assert err[0] < 2e-2 and err[1] < 1e-2 and err[-1] < 2e-3
    assert np.all(np.diff(err) < 0)


# ----------------------------------------------------------- reverse (a5) ----

def _small_n5k(wl):
    """The n5k shape reduced to 4 tracers (2 clustering, 2 lensing), 11 ell, 256 k."""
    w = wl("n5k_vjp")
    tr = np.array([0, 7, 10, 14])
    q = np.arange(0, len(w.k), 4)
    ells = w.ells[::10]
    rng = np.random.default_rng(7)
    Cb = rng.standard_normal((len(ells), 4, 4))
    return w, tr, w.k[q], ells, Cb


def test_vjp_homogeneity_identities(wl):
    """C is linear in P and quadratic in both the amplitudes and the windows, so
    sum P_bar P = <C_bar, C>, sum A_bar A = 2 <C_bar, C>, sum W_bar W = 2 <C_bar, C>."""
    w, tr, k, ells, Cb = _small_n5k(wl)
    g = O.Grids(w.N, w.chi_min, w.chi_max, k, ells, w.knots, w.kind[tr], w.fft_bias[tr])
    P = w.P[::4]
    amp = w.amp[tr]
    f = O.forward(g, w.W[tr], w.D, P, amp)
    Pb, Ab, Wb, _ = O.vjp(g, f, Cb, w.W[tr], w.D, P, amp)
    ip = np.sum(Cb * f["C"])
    assert abs(np.sum(Pb * P) / ip - 1) < 1e-12
    assert abs(np.sum(Ab * amp) / (2 * ip) - 1) < 1e-12
    assert abs(np.sum(Wb * w.W[tr]) / (2 * ip) - 1) < 1e-12


def test_vjp_against_central_differences(wl):
    """Hand-written reverse mode against central finite differences (relative step 1e-5) along
    random directions in P, the amplitudes and the window samples, and along each window mean
    shift (windows rebuilt by the input builder)."""
    from workloads.n5k_synth import window_rows
    w, tr, k, ells, Cb = _small_n5k(wl)
    g = O.Grids(w.N, w.chi_min, w.chi_max, k, ells, w.knots, w.kind[tr], w.fft_bias[tr])
    P = w.P[::4]
    amp = w.amp[tr]
    Wt = w.W[tr]
    f = O.forward(g, Wt, w.D, P, amp)
    Pb, Ab, Wb, _ = O.vjp(g, f, Cb, Wt, w.D, P, amp)
    L = lambda Wx, Px, Ax: np.sum(Cb * O.forward(g, Wx, w.D, Px, Ax)["C"])  # noqa: E731
    rng = np.random.default_rng(3)
    h = 1e-5
    dP = rng.standard_normal(len(P)) * P
    fd = (L(Wt, P + h * dP, amp) - L(Wt, P - h * dP, amp)) / (2 * h)
    assert abs(fd / np.sum(Pb * dP) - 1) < 1e-6
    dA = rng.standard_normal(len(amp)) * amp
    fd = (L(Wt, P, amp + h * dA) - L(Wt, P, amp - h * dA)) / (2 * h)
    assert abs(fd / np.sum(Ab * dA) - 1) < 1e-6
    dW = rng.standard_normal(Wt.shape) * Wt
    fd = (L(Wt + h * dW, P, amp) - L(Wt - h * dW, P, amp)) / (2 * h)
    assert abs(fd / np.sum(Wb * dW) - 1) < 1e-6
    # window mean shifts: absolute step 1e-5 (1 + mu) in z
    meta = w.meta
    ntr = len(w.kind)
    for t_local, t in enumerate(tr):
        mu = meta["gauss"][t][0] if t < len(meta["gauss"]) else 0.0
        hz = 1e-5 * (1.0 + mu)
        sp = np.zeros(ntr)
        sp[t] = hz
        Wp = window_rows(meta, sp)[tr]
        Wm = window_rows(meta, -sp)[tr]
        fd = (L(Wp, P, amp) - L(Wm, P, amp)) / (2 * hz)
        chain = np.sum(Wb * (Wp - Wm)) / (2 * hz)
        assert abs(fd - chain) <= 1e-6 * abs(fd), (t, fd, chain)


def test_numpy_fft_matches_direct_sum():
    """Eq. 3.2 evaluated by numpy.fft (the large-workload option) equals the direct DFT sum, for
    the coefficients (both Nyquist bins, tapers, non-unit chi_min) and for the reverse mode."""
    rng = np.random.default_rng(17)
    N, chi_min, chi_max = 64, 3.0, 3.0e4
    F = rng.standard_normal((5, N))
    tchi = rng.uniform(0.5, 1.0, N)
    tc = rng.uniform(0.5, 1.0, N // 2 + 1)
    for b in (-0.3, -1.5):
        c1 = O.fftlog_coefficients(F, chi_min, chi_max, b, tchi, tc, fft="direct")
        c2 = O.fftlog_coefficients(F, chi_min, chi_max, b, tchi, tc, fft="numpy")
        assert np.max(np.abs(c1 - c2)) < 1e-13 * np.max(np.abs(c1))
    # reverse mode through both DFT forms
    k = np.geomspace(1e-3, 1.0, 40)
    ells = np.array([2, 7, 30])
    knots = np.geomspace(1e-3, 1.0, 6)
    kind = np.array([0, 1])
    bias = np.array([-0.3, -1.5])
    chi = O.chi_grid(chi_min, chi_max, N)
    W = np.exp(-0.5 * ((np.log(chi) - rng.uniform(5, 7, 2)[:, None]) / 0.4) ** 2)
    D = 1.0 + 0.01 * rng.standard_normal((len(knots), N))
    P = rng.uniform(1.0, 2.0, len(k))
    amp = np.array([1.3, 1.0])
    Cb = rng.standard_normal((len(ells), 2, 2))
    out = []
    for fft in ("direct", "numpy"):
        g = O.Grids(N, chi_min, chi_max, k, ells, knots, kind, bias, fft=fft)
        f = O.forward(g, W, D, P, amp)
        out.append((f["C"],) + tuple(O.vjp(g, f, Cb, W, D, P, amp)[:3]))
    for a, b in zip(out[0], out[1]):
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


# ------------------------------------------ magnification and RSD kinds ----

def test_rsd_table_equals_three_term_recurrence():
    """The RSD kernel table (Eq. 2.10), formed by integrating by parts twice,
    int x^p j_l''(x) dx = p (p - 1) I_l(p - 2), against an independent route: the recurrences
    j_l' = (l j_{l-1} - (l+1) j_{l+1})/(2l+1) applied twice give j_l'' as a combination of
    j_{l-2}, j_l and j_{l+2}, so the table is the same combination of the l-2, l and l+2 tables.
    The three terms nearly cancel at large l, so the gate is relative to the sum of their
    magnitudes.  Complex p up to |eta| = 300, l = 2..1500."""
    ells = np.array([2, 3, 7, 40, 301, 1500])
    rng = np.random.default_rng(4)
    p = rng.uniform(-0.8, 0.9, 12) + 1j * rng.uniform(-300, 300, 12)
    got = O.bessel2_power_integral(ells, p)
    l = ells.astype(np.float64)[:, None]
    t0 = l * (l - 1.0) / ((2.0 * l - 1.0) * (2.0 * l + 1.0)) * O.bessel_power_integral(ells - 2, p)
    t1 = ((2.0 * l * l + 2.0 * l - 1.0) / ((2.0 * l - 1.0) * (2.0 * l + 3.0))
          * O.bessel_power_integral(ells, p))
    t2 = (l + 1.0) * (l + 2.0) / ((2.0 * l + 1.0) * (2.0 * l + 3.0)) * O.bessel_power_integral(ells + 2, p)
    scale = np.abs(t0) + np.abs(t1) + np.abs(t2)
    assert np.all(np.abs(got - (t0 - t1 + t2)) <= 1e-12 * scale)
    # a dropped p(p-1) factor or a shifted argument is O(1) off
    assert np.max(np.abs(got / (t0 - t1 + t2) - 1.0)[:4]) < 1e-11


def test_rsd_kernel_identity_against_bessel_equation():
    """The recurrence combination for j_l'' equals the second derivative from the Bessel equation
    x^2 j'' + 2 x j' + (x^2 - l(l+1)) j = 0 with scipy's j_l and j_l'."""
    for ell in (2, 5, 30, 200):
        x = np.geomspace(0.05, 4.0 * ell + 20.0, 400)
        l = float(ell)
        comb = (l * (l - 1) / ((2 * l - 1) * (2 * l + 1)) * spherical_jn(ell - 2, x)
                - (2 * l * l + 2 * l - 1) / ((2 * l - 1) * (2 * l + 3)) * spherical_jn(ell, x)
                + (l + 1) * (l + 2) / ((2 * l + 1) * (2 * l + 3)) * spherical_jn(ell + 2, x))
        jd2 = (-2.0 * x * spherical_jn(ell, x, derivative=True)
               - (x * x - l * (l + 1)) * spherical_jn(ell, x)) / (x * x)
        assert np.max(np.abs(comb - jd2)) <= 1e-12 * np.abs(jd2).max(), ell


def test_rsd_delta_matches_brute_force():
    """RSD source function (Eq. 2.10): the FFTLog Delta of a Gaussian window against brute-force
    quadrature of -int W j_l''(k chi) dchi, j_l'' from the Bessel equation (scipy j_l, j_l').
    Reading R10: j_2'' tends to a constant at small argument, so the periodic images of the window
    are damped only through the FFTLog bias; b = 0.4 (inside the strip -l+1 < b < 1) brings l = 2
    to ~6e-7 (b = -0.3 gives 2e-3; l >= 10 agree to ~1e-12 for any of these b)."""
    N = 2048
    k = np.geomspace(1e-3, 0.5, 8)
    ells = [2, 10, 50, 200]
    g = O.Grids(N, 1.0, 1e5, k, ells, [0.1], [O.KIND_RSD], [0.4])
    win = lambda x: np.exp(-0.5 * ((x - 1000.0) / 100.0) ** 2)  # noqa: E731
    coef = O.window_coefficients(g, win(g.chi)[None, :], np.ones((1, N)))
    d, _ = O.delta_from_coefficients(g, coef)
    xg, wg = np.polynomial.legendre.leggauss(24)
    for li, ell in enumerate(ells):
        br = np.empty_like(k)
        for t, kk in enumerate(k):
            e = np.linspace(1.0, 2500.0, int(max(256, 8 * 2500 * kk / (2 * np.pi))) + 1)
            mid, half = 0.5 * (e[1:] + e[:-1]), 0.5 * (e[1:] - e[:-1])
            xs = (mid[:, None] + half[:, None] * xg[None, :]).ravel()
            ws = (half[:, None] * wg[None, :]).ravel()
            x = kk * xs
            jd2 = (-2.0 * x * spherical_jn(ell, x, derivative=True)
                   - (x * x - ell * (ell + 1.0)) * spherical_jn(ell, x)) / (x * x)
            br[t] = -np.sum(ws * win(xs) * jd2)
        sel = np.abs(br) > 1e-3 * np.abs(br).max()
        rel = np.abs(d[li, 0, :] - br)[sel] / np.abs(br[sel])
        assert rel.max() < (2e-6 if ell == 2 else 1e-9), (ell, rel.max())


def test_magnification_delta_matches_brute_force(wl):
    """Magnification bias (Eq. 2.9): l(l+1) k^-2 int W chi^-2 D j_l against brute force, for a lens
    efficiency window; also its ratio to the lensing kind is l(l+1)/sqrt((l+2)!/(l-2)!) exactly."""
    from workloads.n5k_synth import Cosmology, lensing_window, smail_bin_edges
    cosmo = Cosmology()
    edges = smail_bin_edges(5)
    lo, hi = edges[1], edges[2]
    N = 2048
    k = np.geomspace(3e-3, 0.3, 6)
    ells = [2, 20, 100]
    g = O.Grids(N, 1.0, 1e5, k, ells, [0.1], [O.KIND_MAGNIFICATION, O.KIND_LENSING], [-1.5, -1.5])
    W1 = lensing_window(cosmo, g.chi, lo, hi)
    coef = O.window_coefficients(g, np.stack([W1, W1]), np.ones((1, N)))
    d, _ = O.delta_from_coefficients(g, coef)
    chi_hi = float(cosmo.chi(hi)) * 1.0000001
    f = lambda x: lensing_window(cosmo, x.ravel(), lo, hi).reshape(x.shape) / x ** 2  # noqa: E731
    for li, ell in enumerate(ells):
        br = ell * (ell + 1.0) * k ** -2 * delta_brute(ell, k, f, 1e-6, chi_hi, tol=1e-10)
        sel = np.abs(br) > 1e-2 * np.abs(br).max()
        rel = np.abs(d[li, 0, :] - br)[sel] / np.abs(br[sel])
        assert rel.max() < 1e-4, (ell, rel.max())
        ratio = ell * (ell + 1.0) / np.sqrt((ell + 2.0) * (ell + 1.0) * ell * (ell - 1.0))
        assert np.allclose(d[li, 0, :], ratio * d[li, 1, :], rtol=1e-13, atol=0)
