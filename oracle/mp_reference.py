"""High-precision (mpmath) values used to pin the FP64 oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* bessel_power_integral_mp: I_ell(p) = sqrt(pi) 2^{p-1} Gamma((l+1+p)/2) / Gamma((l+2-p)/2)
  (Eq. 3.4 with the "- p" reading) in 50-digit arithmetic.
* mellin_quadrature_mp: the same integral int_0^inf x^p j_ell(x) dx computed by
  oscillatory quadrature, i.e. from its definition and not from the Gamma
  formula; it decides between the printed "+ p" and the "- p" reading.
"""
from __future__ import annotations

import mpmath as mp


def bessel_power_integral_mp(ell: int, p: complex, dps: int = 50) -> complex:
    with mp.workdps(dps):
        p = mp.mpc(p)
        l = mp.mpf(ell)
        v = mp.sqrt(mp.pi) * mp.power(2, p - 1) * mp.exp(
            mp.loggamma((l + 1 + p) / 2) - mp.loggamma((l + 2 - p) / 2))
        return complex(v)


def mellin_quadrature_mp(ell: int, p: float, dps: int = 30) -> float:
    """int_0^inf x^p j_ell(x) dx for real -ell-1 < p < 1 by mpmath quadrature.

    The integrand near 0 behaves as x^{p+ell}; [0, x0] is integrated with
    tanh-sinh and [x0, inf) with quadosc (period 2 pi).
    """
    with mp.workdps(dps):
        p = mp.mpf(p)

        def f(x):
            return x ** p * mp.sqrt(mp.pi / (2 * x)) * mp.besselj(ell + mp.mpf(1) / 2, x)
        x0 = mp.mpf(ell + 2)
        head = mp.quad(f, [0, x0 / 4, x0 / 2, x0])
        tail = mp.quadosc(f, [x0, mp.inf], omega=1)
        return float(head + tail)
