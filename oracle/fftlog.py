"""Plain FP64 reference of the beyond-Limber FFTLog C_ell computation.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every function follows a
passage of arXiv:2505.22718 and is written for a reader who checks it against
the paper, not for speed: direct DFT as a matrix product, the full two-sided
sum over n = -N/2..N/2, complex log-Gamma from scipy, dense interpolation
matrices.

Readings taken where the paper is silent, garbled or inconsistent:

R1  Eq. (3.4) prints Gamma((2 + ell + p)/2) in the denominator; the Mellin
    transform of j_ell gives Gamma((2 + ell - p)/2).  We use "- p" (checked
    against direct numerical integration in the tests).
R2  Eq. (3.2): the sum runs over m = 0..N-1 (printed "N+1") and the exponent
    is e^{-2 pi i n m / N} (the printed exponent lost its pi).  The grid is
    chi_m = chi_min exp(m L / N), L = ln(chi_max/chi_min), chi_max excluded, so
    eta_n = 2 pi n / L (Sec. 3.1) makes the DFT exact on the grid.
R3  Eq. (3.1) sums n = -N/2..N/2 (N+1 terms): the two Nyquist coefficients
    c_{+-N/2} carry half weight (trigonometric interpolation convention).
R4  The "smoothing function at the tails" (Sec. 3.1) is an optional
    caller-supplied taper in chi (applied to the samples) and in n (applied to
    the coefficients); absent means 1.
R5  The k-interpolation of Sec. 3.2 is local 4-point Lagrange in ln k on the
    knots (3- or 2-point when fewer knots exist), stencil clamped at the ends.
R6  The k-integral of Eq. (2.1) "over all N_k points" (Sec. 3.2) is the
    trapezoid rule in ln k: int dk g = int dlnk k g, w_q = k_q h_q with
    h_q = (ln k_{q+1} - ln k_{q-1})/2 and half intervals at the ends.
R8  The Gamma-ratio table is evaluated from log-Gammas at the smallest ell of each parity and
    carried to larger ell by the exact two-step recurrence of Gamma(z+1) = z Gamma(z)
    (see bessel_power_integral).
R10 RSD tracers (kernel j_l'', Eq. 2.10) need a larger FFTLog bias than density ones: j_2''
    tends to a constant at small argument, so the periodic images of the window are damped
    only through b; b = 0.4 (the strip is -l+1 < b < 1) gives l = 2 to ~6e-7 of brute force.
R7  Source functions: density Delta = int W D j_ell (Eq. 2.6, the linear bias
    b_1 is the tracer amplitude); lensing Delta = sqrt((l+2)!/(l-2)!) k^-2
    int W chi^-2 D j_ell (Eq. 2.14; intrinsic alignment, Eq. 2.15, is the same
    kernel with the window n A_IA); magnification Delta = l(l+1) k^-2
    int W chi^-2 D j_ell (Eq. 2.9, C_g in the amplitude; CMB lensing, Eq. 2.16, is
    the same kernel with its own window); RSD Delta = -int W D j_ell'' (Eq. 2.10,
    f(z) in the window).  A per-tracer amplitude A_i multiplies Delta_i; an
    optional k,z-dependent bias B_i(k, chi) multiplies W D (primordial
    non-Gaussianity, Eq. 2.11-2.13, is a density tracer with B = 1/T_alpha).
"""
from __future__ import annotations

import numpy as np
from scipy.special import loggamma

KIND_DENSITY = 0
KIND_LENSING = 1
KIND_MAGNIFICATION = 2    # magnification bias (Eq. 2.9) and CMB lensing (Eq. 2.16): l(l+1) k^-2
KIND_RSD = 3              # redshift-space distortion (Eq. 2.10): -j_l''

_CHI2 = (KIND_LENSING, KIND_MAGNIFICATION)


# ---------------------------------------------------------------- grids ----

def chi_grid(chi_min: float, chi_max: float, N: int) -> np.ndarray:
    """chi_m = chi_min exp(m L/N), m = 0..N-1 (Sec. 3.1, reading R2)."""
    L = np.log(chi_max / chi_min)
    return chi_min * np.exp(np.arange(N) * L / N)


def eta_two_sided(N: int, L: float) -> tuple[np.ndarray, np.ndarray]:
    """n = -N/2..N/2 and eta_n = 2 pi n / L (Sec. 3.1)."""
    n = np.arange(-N // 2, N // 2 + 1)
    return n, 2.0 * np.pi * n / L


def chi_power(kind) -> np.ndarray:
    """Power s of chi multiplying the window: 0 (density Eq. 2.6, RSD Eq. 2.10), -2 (lensing
    Eq. 2.14, magnification Eq. 2.9)."""
    return np.where(np.isin(np.asarray(kind), _CHI2), -2.0, 0.0)


def k_power(kind) -> np.ndarray:
    """Power t of k in front of the chi integral: 0 (density, RSD), -2 (lensing, magnification)."""
    return np.where(np.isin(np.asarray(kind), _CHI2), -2.0, 0.0)


def ell_prefactor(ells, kind: int) -> np.ndarray:
    """c(ell) of Eq. (2.2): 1 for density, sqrt((l+2)!/(l-2)!) for lensing (Eq. 2.14), l(l+1) for
    magnification (Eq. 2.9), -1 for RSD (the sign of Eq. 2.10)."""
    l = np.asarray(ells, dtype=np.float64)
    if kind == KIND_LENSING:
        return np.sqrt((l + 2.0) * (l + 1.0) * l * (l - 1.0))
    if kind == KIND_MAGNIFICATION:
        return l * (l + 1.0)
    if kind == KIND_RSD:
        return -np.ones_like(l)
    return np.ones_like(l)


# ------------------------------------------------------------- FFTLog ------

def fftlog_coefficients(F, chi_min, chi_max, b, taper_chi=None, taper_c=None, fft="direct"):
    """Two-sided FFTLog coefficients c_n, n = -N/2..N/2, of real samples F[..., m].

    Eq. (3.2) with readings R2-R4:
        c_n = T_c(|n|) chi_min^{-i eta_n} (1/N) sum_{m<N} F(chi_m) chi_m^{-b} T_chi(m) e^{-2 pi i n m/N},
    and c_{+-N/2} halved, so that F(chi) = sum_n c_n chi^{b + i eta_n} (Eq. 3.1) on the grid.
    fft="direct": the plain O(N^2) sum, written as a product with the DFT matrix whose phases
    use the exact integer residue (n m mod N).  fft="numpy": the same sum by numpy.fft (a library
    step for large N; the pins check it against the direct sum), with c_{-n} read from bin N - n.
    """
    F = np.asarray(F, dtype=np.float64)
    N = F.shape[-1]
    L = np.log(chi_max / chi_min)
    chi = chi_grid(chi_min, chi_max, N)
    n, eta = eta_two_sided(N, L)
    g = F * chi ** (-b)
    if taper_chi is not None:
        g = g * taper_chi
    if fft == "numpy":
        c = np.fft.fft(g, axis=-1)[..., np.mod(n, N)] / N
    elif fft == "direct":
        m = np.arange(N)
        resid = np.mod(np.outer(m, n), N)             # (n m) mod N, exact
        dft = np.exp(-2j * np.pi * resid / N)         # [N, N+1]
        c = (g @ dft) / N
    else:
        raise ValueError("fft must be 'direct' or 'numpy'")
    c = c * np.exp(-1j * eta * np.log(chi_min))       # chi_min^{-i eta_n}
    if taper_c is not None:
        c = c * taper_c[np.abs(n)]
    c[..., 0] *= 0.5                                  # n = -N/2
    c[..., -1] *= 0.5                                 # n = +N/2
    return c


def fftlog_reconstruct(c, chi, b, chi_min, chi_max):
    """Evaluate sum_n c_n chi^{b + i eta_n} (Eq. 3.1) at arbitrary chi (for tests)."""
    N = c.shape[-1] - 1
    _, eta = eta_two_sided(N, np.log(chi_max / chi_min))
    ph = np.exp(1j * np.outer(np.log(chi), eta))
    return (ph @ c.T).T * chi ** b


# ----------------------------------------------------- Gamma-ratio table ---

def bessel_power_integral(ells, p):
    """I_ell(p) = int_0^inf chi^p j_ell(chi) dchi = sqrt(pi) 2^{p-1} Gamma((l+1+p)/2) / Gamma((l+2-p)/2).

    Eq. (3.4) at k = 1 with reading R1; valid for -ell-1 < Re p < 1.
    Returns the table [len(ells), len(p)].

    Evaluation (reading R8): the Gamma ratio is formed from log-Gammas only at the smallest
    requested ell of each parity; larger ell follow from the exact identity Gamma(z+1) = z Gamma(z),
        I_{ell+2}(p) = I_ell(p) (ell + 1 + p) / (ell + 2 - p),
    applied one step at a time.  A direct difference of log-Gammas of size ~ (ell/2) ln(ell/2)
    would lose ~1e-12 of relative accuracy at ell ~ 2000 to cancellation; the recurrence keeps
    the table within ~1e-14 (checked against 50-digit values in the tests).
    """
    ells = np.asarray(ells, dtype=np.int64)
    p = np.asarray(p, dtype=np.complex128)
    out = np.empty((len(ells), len(p)), dtype=np.complex128)
    for parity in (0, 1):
        sel = np.nonzero(ells % 2 == parity)[0]
        if len(sel) == 0:
            continue
        l0 = int(ells[sel].min())
        cur = np.sqrt(np.pi) * np.exp((p - 1.0) * np.log(2.0)
                                      + loggamma(0.5 * (l0 + 1.0 + p)) - loggamma(0.5 * (l0 + 2.0 - p)))
        want = {int(ells[j]): [] for j in sel}
        for j in sel:
            want[int(ells[j])].append(j)
        l = l0
        lmax = int(ells[sel].max())
        while True:
            for j in want.get(l, ()):
                out[j] = cur
            if l >= lmax:
                break
            cur = cur * (l + 1.0 + p) / (l + 2.0 - p)
            l += 2
    return out


# ------------------------------------------------------ k-interpolation ----

def bessel2_power_integral(ells, p):
    """int_0^inf chi^p j_l''(chi) dchi for the RSD kernel (Eq. 2.10), l >= 2.

    Integrating by parts twice (the boundary terms vanish inside the strip 1 - l < Re p < 1,
    where both integrals converge):
        int chi^p j_l'' dchi = p (p - 1) int chi^{p-2} j_l dchi = p (p - 1) I_l(p - 2).
    This product form is used rather than the three-term Bessel recurrence
    j_l'' = a j_{l-2} - b j_l + c j_{l+2}: at large l and small eta the three terms nearly cancel
    (about seven digits at l ~ 1000) and the result would carry the R8 recurrence error magnified
    by that amount.  The tests check the two forms against each other where the cancellation is
    mild, and the j_l'' combination against the Bessel equation.
    """
    ells = np.asarray(ells, dtype=np.int64)
    if np.any(ells < 2):
        raise ValueError("the RSD kernel needs ell >= 2")
    p = np.asarray(p, dtype=np.complex128)
    return (p * (p - 1.0))[None, :] * bessel_power_integral(ells, p - 2.0)


def lagrange_matrix(k, knots) -> np.ndarray:
    """Dense interpolation matrix Lam[q, a] (reading R5).

    For each k_q: x = ln k_q, interval a with x_a <= x < x_{a+1} (clamped),
    stencil of s = min(4, N_I) consecutive knots starting at clamp(a - 1, 0, N_I - s),
    Lagrange basis polynomials in ln k evaluated at x.
    """
    x = np.log(np.asarray(k, dtype=np.float64))
    xk = np.log(np.asarray(knots, dtype=np.float64))
    NI = len(xk)
    s = min(4, NI)
    lam = np.zeros((len(x), NI))
    for q, xq in enumerate(x):
        a = int(np.searchsorted(xk, xq, side="right")) - 1
        a = min(max(a, 0), NI - 1)
        j0 = min(max(a - 1, 0), NI - s)
        nodes = xk[j0:j0 + s]
        for r in range(s):
            num = 1.0
            for t in range(s):
                if t != r:
                    num *= (xq - nodes[t]) / (nodes[r] - nodes[t])
            lam[q, j0 + r] = num
    return lam


# ---------------------------------------------------------- k-quadrature ---

def lnk_trapezoid_weights(k) -> np.ndarray:
    """w_q with int dk g(k) ~ sum_q w_q g(k_q): trapezoid in ln k (reading R6)."""
    lk = np.log(np.asarray(k, dtype=np.float64))
    h = np.empty_like(lk)
    h[1:-1] = 0.5 * (lk[2:] - lk[:-2])
    h[0] = 0.5 * (lk[1] - lk[0])
    h[-1] = 0.5 * (lk[-1] - lk[-2])
    return np.asarray(k, dtype=np.float64) * h


def cl_weights(k, P) -> np.ndarray:
    """u_q = (2/pi) w_q k_q^2 P(k_q): the measure of Eq. (2.1) on the k grid."""
    k = np.asarray(k, dtype=np.float64)
    return (2.0 / np.pi) * lnk_trapezoid_weights(k) * k * k * np.asarray(P, dtype=np.float64)


# -------------------------------------------------------------- forward ----

def source_samples(W, D, B, chi, kind):
    """F[i, a, m] = W_i(chi_m) chi_m^{s_i} D(kappa_a, chi_m) B_i(kappa_a, chi_m) (Sec. 3.2, R7)."""
    W = np.asarray(W, dtype=np.float64)
    s = chi_power(kind)
    F = (W * chi[None, :] ** s[:, None])[:, None, :] * np.asarray(D)[None, :, :]
    if B is not None:
        F = F * np.asarray(B)
    return F


class Grids:
    """Everything that depends on the grids only (the paper's precomputation, Sec. 3.2)."""

    def __init__(self, N, chi_min, chi_max, k, ells, knots, kind, fft_bias, fft="direct"):
        self.N = int(N)
        self.fft = fft                                            # see fftlog_coefficients
        self.chi_min, self.chi_max = float(chi_min), float(chi_max)
        self.L = np.log(self.chi_max / self.chi_min)
        self.chi = chi_grid(self.chi_min, self.chi_max, self.N)
        self.k = np.asarray(k, dtype=np.float64)
        self.ells = np.asarray(ells)
        self.knots = np.asarray(knots, dtype=np.float64)
        self.kind = np.asarray(kind)
        self.fft_bias = np.asarray(fft_bias, dtype=np.float64)
        self.n, self.eta = eta_two_sided(self.N, self.L)
        self.lam = lagrange_matrix(self.k, self.knots)            # [N_k, N_I]
        self.wq = lnk_trapezoid_weights(self.k)
        # k^{-1-p_n} = k^{-1-b} e^{-i eta_n ln k}: the phase part, [N_k, N+1]
        self.phase = np.exp(-1j * np.outer(np.log(self.k), self.eta))
        self._mtab = {}

    def mtable(self, b: float, ells=None, kind: int = KIND_DENSITY):
        """I_ell(b + i eta_n) of the tracer's kernel (j_l, or j_l'' for RSD) for the requested
        ells (default: all), [N_ell, N+1]."""
        ells = self.ells if ells is None else np.asarray(ells)
        rsd = int(kind) == KIND_RSD
        key = (float(b), rsd, tuple(int(e) for e in ells))
        if key not in self._mtab:
            f = bessel2_power_integral if rsd else bessel_power_integral
            self._mtab[key] = f(ells, b + 1j * self.eta)
        return self._mtab[key]


def window_coefficients(g: Grids, W, D, B=None, taper_chi=None, taper_c=None):
    """c[i][a][n]: FFTLog coefficients of F_i(chi; kappa_a) at every knot (Eq. 3.3)."""
    F = source_samples(W, D, B, g.chi, g.kind)
    out = []
    for i in range(F.shape[0]):
        tc = None if taper_chi is None else taper_chi[i]
        tn = None if taper_c is None else taper_c[i]
        out.append(fftlog_coefficients(F[i], g.chi_min, g.chi_max, g.fft_bias[i], tc, tn, g.fft))
    return np.array(out)                                          # [N_tr, N_I, N+1]


def delta_from_coefficients(g: Grids, coef, ells=None, tracers=None, q_index=None):
    """Delta_i(ell, k_q) (Eq. 2.2 with Eq. 3.3-3.4, readings R5, R7).

    Delta_i(ell, k) = c_i(ell) k^{t_i} sum_n c_{i,n}(k) I_ell(b_i + i eta_n) k^{-1-b_i-i eta_n},
    with c_{i,n}(k) = sum_a Lam(k, a) c_{i,a,n}.  The two-sided sum is real up to
    rounding; its imaginary part is returned as a diagnostic.
    Returns (Delta[N_ell][N_tr][N_q], max |Im| / max |Re|).
    """
    ells = g.ells if ells is None else np.asarray(ells)
    tracers = range(coef.shape[0]) if tracers is None else tracers
    q = np.arange(len(g.k)) if q_index is None else np.asarray(q_index)
    k = g.k[q]
    out = np.zeros((len(ells), len(list(tracers)), len(q)))
    worst = 0.0
    for col, i in enumerate(tracers):
        b = g.fft_bias[i]
        kind = int(g.kind[i])
        ck = g.lam[q] @ coef[i]                                   # [N_q, N+1] c_n(k_q)
        X = ck * g.phase[q]                                       # c_n(k) e^{-i eta_n ln k}
        M = g.mtable(b, ells, kind)                               # [N_ell, N+1]
        S = X @ M.T                                               # [N_q, N_ell]
        worst = max(worst, float(np.abs(S.imag).max() / max(np.abs(S.real).max(), 1e-300)))
        kfac = k ** (k_power(kind) - 1.0 - b)
        d = (S.real * kfac[:, None]) * ell_prefactor(ells, kind)[None, :]
        out[:, col, :] = d.T
    return out, worst


def angular_cl(delta, u, amp):
    """C_ell^{ij} = A_i A_j sum_q u_q Delta_i(ell, k_q) Delta_j(ell, k_q) (Eq. 2.1 discretised, R6)."""
    A = np.asarray(amp, dtype=np.float64)
    U = np.einsum("liq,q,ljq->lij", delta, u, delta)
    return U * A[None, :, None] * A[None, None, :]


def forward(g: Grids, W, D, P, amp, B=None, taper_chi=None, taper_c=None, ells=None):
    """Full forward pass: returns dict with coef, delta, u, C."""
    coef = window_coefficients(g, W, D, B, taper_chi, taper_c)
    delta, imag = delta_from_coefficients(g, coef, ells)
    u = cl_weights(g.k, P)
    C = angular_cl(delta, u, amp)
    return dict(coef=coef, delta=delta, u=u, C=C, imag_ratio=imag)


# -------------------------------------------------------------- reverse ----

def vjp(g: Grids, fwd: dict, C_bar, W, D, P, amp, B=None, taper_chi=None, taper_c=None, ells=None):
    """Reverse mode of `forward`, written by hand step by step.

    Given the cotangent C_bar[ell][i][j] returns (P_bar[N_k], amp_bar[N_tr], W_bar[N_tr][N]).
      S = (C_bar + C_bar^T)/2
      P_bar_q   = (2/pi) w_q k_q^2 sum_ell sum_ij S_ij A_i A_j Delta_i Delta_j
      amp_bar_i = 2 sum_ell sum_j S_ij A_j U_ij,   U = C at unit amplitudes
      Delta_bar_i(ell, q) = 2 A_i u_q sum_j S_ij A_j Delta_j(ell, q)
    then back through the contraction, the k-interpolation, the FFTLog sum and
    the source samples.
    """
    ells = g.ells if ells is None else np.asarray(ells)
    delta, u, coef = fwd["delta"], fwd["u"], fwd["coef"]
    A = np.asarray(amp, dtype=np.float64)
    S = 0.5 * (C_bar + np.transpose(C_bar, (0, 2, 1)))
    SA = S * A[None, :, None] * A[None, None, :]
    # P(k) enters only through u_q
    P_bar = (2.0 / np.pi) * g.wq * g.k ** 2 * np.einsum("lij,liq,ljq->q", SA, delta, delta)
    U = np.einsum("liq,q,ljq->lij", delta, u, delta)
    amp_bar = 2.0 * np.einsum("lij,j,lij->i", S, A, U)
    delta_bar = 2.0 * A[None, :, None] * u[None, None, :] * np.einsum("lij,j,ljq->liq", S, A, delta)

    N = g.N
    n, eta = g.n, g.eta
    if g.fft == "direct":
        m = np.arange(N)
        resid = np.mod(np.outer(m, n), N)
        dft = np.exp(-2j * np.pi * resid / N)                   # [N, N+1]
    chi_phase = np.exp(-1j * eta * np.log(g.chi_min))
    F_bar_all = []
    W_bar = np.zeros((coef.shape[0], N))
    s = chi_power(g.kind)
    for i in range(coef.shape[0]):
        b = g.fft_bias[i]
        kind = int(g.kind[i])
        M = g.mtable(b, ells, kind)                               # [N_ell, N+1]
        kfac = g.k ** (k_power(kind) - 1.0 - b)
        pre = ell_prefactor(ells, kind)
        # Delta = kfac_q pre_l Re(sum_n X_qn M_ln):  X_bar (d/dRe X + i d/dIm X)
        D_bar_ql = delta_bar[:, i, :].T * kfac[:, None] * pre[None, :]   # [N_q, N_ell]
        X_bar = D_bar_ql @ np.conj(M)                             # [N_q, N+1]
        ck_bar = X_bar * np.conj(g.phase)                         # X = c(k) phase
        c_bar = g.lam.T @ ck_bar                                  # [N_I, N+1]
        # undo the Nyquist halving and the tapers/phases of fftlog_coefficients
        c_bar = c_bar.copy()
        c_bar[:, 0] *= 0.5
        c_bar[:, -1] *= 0.5
        if taper_c is not None:
            c_bar = c_bar * taper_c[i][np.abs(n)]
        c_bar = c_bar * np.conj(chi_phase)
        # c = (g @ dft)/N for real g: in the real-pair sense g_bar_m = Re sum_n conj(c_bar_n) dft_mn / N
        if g.fft == "direct":
            g_bar = np.real(np.conj(c_bar) @ dft.T).astype(np.float64) / N  # [N_I, N]
        else:
            # the same sum by numpy.fft: conj(c_bar_n) into bin n mod N (both Nyquist terms in N/2)
            X = np.zeros(c_bar.shape[:-1] + (N,), dtype=np.complex128)
            for col, nn in enumerate(n):
                X[..., nn % N] += np.conj(c_bar[..., col])
            g_bar = np.real(np.fft.fft(X, axis=-1)) / N
        F_bar = g_bar * g.chi ** (-b)
        if taper_chi is not None:
            F_bar = F_bar * taper_chi[i]
        F_bar_all.append(F_bar)
        fac = np.asarray(D) * g.chi[None, :] ** s[i]
        if B is not None:
            fac = fac * np.asarray(B)[i]
        W_bar[i] = np.sum(F_bar * fac, axis=0)
    return P_bar, amp_bar, W_bar, dict(delta_bar=delta_bar, F_bar=np.array(F_bar_all))
