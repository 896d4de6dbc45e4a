"""Writes the stored expected values under tests/golden/ (calls only oracle/).

Run from the repository root:  python tests/golden/make_golden.py

* mellin_real_p.txt   int_0^inf x^p j_ell(x) dx by mpmath quadrature of the
                      definition, real p (Eq. 3.4 of arXiv:2505.22718, Sec. 3.2).
* gamma_ratio_mp50.txt  I_ell(b + i eta) = sqrt(pi) 2^{p-1} Gamma((l+1+p)/2)/Gamma((l+2-p)/2)
                      in 50-digit arithmetic at seeded random (ell, b, eta), the
                      table of Eq. (3.4) that the contraction uses.
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle.mp_reference import bessel_power_integral_mp, mellin_quadrature_mp  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    cases = [(2, -1.0), (2, -0.3), (2, -2.2), (3, -2.5), (5, -1.5), (10, 0.5), (20, -1.5), (50, -0.3)]
    with open(os.path.join(HERE, "mellin_real_p.txt"), "w") as f:
        f.write("# int_0^inf x^p j_ell(x) dx by mpmath quadrature (definition, not the Gamma formula)\n")
        f.write("# source: Eq. (3.4), arXiv:2505.22718 Sec. 3.2; written by tests/golden/make_golden.py\n")
        f.write("# ell p value\n")
        for ell, p in cases:
            f.write("%d %.17g %.17g\n" % (ell, p, mellin_quadrature_mp(ell, p)))
    rng = np.random.default_rng(20250528)
    with open(os.path.join(HERE, "gamma_ratio_mp50.txt"), "w") as f:
        f.write("# I_ell(b + i eta) of Eq. (3.4) (denominator Gamma((l+2-p)/2)) in 50-digit mpmath\n")
        f.write("# source: Eq. (3.4), arXiv:2505.22718 Sec. 3.2; written by tests/golden/make_golden.py\n")
        f.write("# ell b eta re im\n")
        pts = []
        for ell in [2, 3, 7, 30, 103, 500, 2000, 3000]:
            for b in [-0.3, -1.5, -2.2, 0.5]:
                for eta in [0.0, 0.37, 5.0, 60.0, 559.0, 1118.0]:
                    pts.append((ell, b, eta))
        for _ in range(40):
            pts.append((int(rng.integers(2, 3001)), float(rng.uniform(-1.9, 0.9)), float(rng.uniform(-2000, 2000))))
        for ell, b, eta in pts:
            v = bessel_power_integral_mp(ell, complex(b, eta))
            f.write("%d %.17g %.17g %.17g %.17g\n" % (ell, b, eta, v.real, v.imag))


if __name__ == "__main__":
    main()
