"""Independent checks of the FFTLog oracle: brute-force line-of-sight integrals and Limber.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* spherical_jn_recurrence: j_ell(x) from the three-term recurrence
  j_{n+1} = (2n+1)/x j_n - j_{n-1}, run upward from j_0, j_1 where x > ell
  (stable there) and downward (Miller's algorithm, normalised to j_0) where
  x <= ell.
* delta_brute: Delta_ell(k) = int_0^inf dchi W(chi) j_ell(k chi) (Eq. 2.2 with
  n = 0) by composite Gauss-Legendre quadrature on a window of compact
  numerical support, refined until two resolutions agree.
* cl_limber: Eq. (2.19), C_ell = int dchi/chi^2 W_i W_j P((ell+1/2)/chi).
"""
from __future__ import annotations

import numpy as np

_GLX, _GLW = np.polynomial.legendre.leggauss(24)


def spherical_jn_recurrence(ell: int, x) -> np.ndarray:
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    out = np.empty_like(x)
    up = x > ell
    if np.any(up):
        xu = x[up]
        j0 = np.sin(xu) / xu
        if ell == 0:
            out[up] = j0
        else:
            j1 = np.sin(xu) / xu ** 2 - np.cos(xu) / xu
            jm, jc = j0, j1
            for n in range(1, ell):
                jm, jc = jc, (2 * n + 1) / xu * jc - jm
            out[up] = jc
    dn = ~up
    if np.any(dn):
        xd = x[dn]
        start = ell + 30 + int(np.sqrt(60.0 * (ell + 1)))
        jp = np.zeros_like(xd)              # j_{n+1}
        jc = np.ones_like(xd)               # j_n (arbitrary scale)
        keep = np.zeros_like(xd)
        j1u = np.zeros_like(xd)
        norm = (2 * start + 1) * jc * jc    # sum_n (2n+1) j_n^2 = 1 fixes the scale
        for n in range(start, 0, -1):
            jm = (2 * n + 1) / xd * jc - jp  # j_{n-1}
            jp, jc = jc, jm
            norm = norm + (2 * n - 1) * jc * jc
            if n - 1 == ell:
                keep = jc.copy()
            if n - 1 == 1:
                j1u = jc.copy()
            big = np.abs(jc) > 1e120
            if np.any(big):
                f = np.where(big, 1e-120, 1.0)
                jc, jp, keep, j1u = jc * f, jp * f, keep * f, j1u * f
                norm = norm * f * f
        # jc is the unnormalised j_0; fix the overall sign with the larger of j_0, j_1
        j0t = np.sin(xd) / xd
        j1t = np.sin(xd) / xd ** 2 - np.cos(xd) / xd
        ref_t = np.where(np.abs(j0t) >= np.abs(j1t), j0t, j1t)
        ref_u = np.where(np.abs(j0t) >= np.abs(j1t), jc, j1u)
        sign = np.sign(ref_t) * np.sign(ref_u)
        out[dn] = sign * keep / np.sqrt(norm)
    return out


def delta_brute(ell: int, k, window, chi_lo: float, chi_hi: float, tol: float = 1e-12):
    """int_{chi_lo}^{chi_hi} W(chi) j_ell(k chi) dchi for each k (W negligible outside)."""
    k = np.atleast_1d(np.asarray(k, dtype=np.float64))
    res = np.empty_like(k)
    for t, kk in enumerate(k):
        # pieces resolve both the window and the Bessel oscillation period 2 pi / k
        pieces = int(max(64, 4 * (chi_hi - chi_lo) * kk / (2 * np.pi)))
        prev = None
        for _ in range(6):
            e = np.linspace(chi_lo, chi_hi, pieces + 1)
            a, b = e[:-1], e[1:]
            half = 0.5 * (b - a)
            nodes = (0.5 * (a + b))[:, None] + half[:, None] * _GLX[None, :]
            val = np.sum(half[:, None] * _GLW[None, :] * window(nodes)
                         * spherical_jn_recurrence(ell, kk * nodes.ravel()).reshape(nodes.shape))
            if prev is not None and abs(val - prev) <= tol * max(abs(val), 1e-300):
                break
            prev = val
            pieces *= 2
        res[t] = val
    return res


def cl_limber(ell: float, chi, Wi, Wj, Pk_of_k_chi):
    """Eq. (2.19) by the trapezoid rule in ln chi on the given (dense) chi grid.

    Pk_of_k_chi(k, chi) is the equal-time power spectrum P(k, chi, chi).
    """
    chi = np.asarray(chi, dtype=np.float64)
    integrand = Wi * Wj * Pk_of_k_chi((ell + 0.5) / chi, chi) / chi ** 2
    lc = np.log(chi)
    f = integrand * chi
    return float(np.sum(0.5 * (f[1:] + f[:-1]) * np.diff(lc)))
