"""Writes the stored expected values under tests/golden/ (calls only oracle/).

Run from the repository root:  python tests/golden/make_golden.py

* mellin_real_p.txt   int_0^inf x^p j_ell(x) dx by mpmath quadrature of the
                      definition, real p (Eq. 3.4 of arXiv:2505.22718, Sec. 3.2).
* gamma_ratio_mp50.txt  I_ell(b + i eta) = sqrt(pi) 2^{p-1} Gamma((l+1+p)/2)/Gamma((l+2-p)/2)
                      in 50-digit arithmetic at seeded random (ell, b, eta), the
                      table of Eq. (3.4) that the contraction uses.
* convergence_truth.txt  C_ell of the convergence case (workloads.n5k_synth.convergence_case,
                      the numerical-parameter study of Appendix A) from the oracle at converged
                      settings: N_FFT = 16384, the growth given at every one of the 2048 k points
                      (no k-interpolation error), N_k = 2048.  Spot-checked here against
                      brute-force line-of-sight quadrature (oracle.brute.delta_brute) with the
                      windows and the growth evaluated exactly.
* cl_brute_gauss.txt  C_ell^{ij} = (2/pi) int dk k^2 P(k) Delta_i Delta_j (Eq. 2.1) for two
                      Gaussian windows in chi, by brute force on both integrals: Gauss-Legendre
                      in ln k, each Delta_i(ell, k) = int W_i j_ell(k chi) dchi (Eq. 2.2) by
                      oracle.brute.delta_brute; two resolutions in k must agree.

Usage: python tests/golden/make_golden.py [all|convergence|cl]
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle.mp_reference import bessel_power_integral_mp, mellin_quadrature_mp  # noqa: E402
from oracle import fftlog as O  # noqa: E402
from oracle.brute import delta_brute  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def convergence_truth():
    from workloads.n5k_synth import (Cosmology, clustering_window, conv_growth, convergence_case,
                                     lensing_window)
    n_k = 2048
    k = np.geomspace(1e-4, 10.0, n_k)
    w = convergence_case(N=16384, n_k=n_k, knots=k)
    g = O.Grids(w.N, w.chi_min, w.chi_max, w.k, w.ells, w.knots, w.kind, w.fft_bias, fft="numpy")
    f = O.forward(g, w.W, w.D, w.P, w.amp)
    # brute-force spot checks of Delta: adaptive quadrature of the line-of-sight integral with the
    # windows rebuilt at any chi and the growth exact in (k, z)
    cosmo = Cosmology(0.3)
    (mu0, s0), (mu1, s1) = w.meta["gauss"]
    lo, hi = w.meta["lens_edges"]
    wins = [lambda x: clustering_window(cosmo, x.ravel(), mu0, s0).reshape(x.shape),
            lambda x: clustering_window(cosmo, x.ravel(), mu1, s1).reshape(x.shape),
            lambda x: lensing_window(cosmo, x.ravel(), lo, hi).reshape(x.shape) / x ** 2]
    supports = [(cosmo.chi(max(mu0 - 8 * s0, 0.0)), cosmo.chi(mu0 + 8 * s0)),
                (cosmo.chi(max(mu1 - 8 * s1, 0.0)), cosmo.chi(mu1 + 8 * s1)),
                (1e-6, cosmo.chi(hi) * 1.0000001)]
    worst = 0.0
    checks = []
    for i, li, kq in [(0, 2, 0.02), (0, 5, 0.2), (1, 3, 0.01), (1, 6, 0.3), (2, 3, 0.02), (2, 5, 0.1)]:
        q = int(np.argmin(np.abs(np.log(k / kq))))
        kk = k[q]
        ell = int(w.ells[li])
        fn = lambda x, i=i, kk=kk: wins[i](x) * conv_growth(kk, cosmo.z_of_chi(x.ravel())).reshape(x.shape)  # noqa: E731
        br = delta_brute(ell, [kk], fn, float(supports[i][0]), float(supports[i][1]), tol=1e-11)[0]
        if w.kind[i] == O.KIND_LENSING:
            br *= np.sqrt((ell + 2.0) * (ell + 1.0) * ell * (ell - 1.0)) / kk ** 2
        scale = np.abs(f["delta"][li, i, :]).max()
        dev = abs(f["delta"][li, i, q] - br) / scale
        checks.append((i, ell, kk, dev))
        worst = max(worst, dev)
    assert worst < 1e-8, checks
    with open(os.path.join(HERE, "convergence_truth.txt"), "w") as fo:
        fo.write("# C_l^{ij} of workloads.n5k_synth.convergence_case from the FP64 oracle at converged\n")
        fo.write("# settings: N_FFT = 16384, growth at all 2048 k points (no k-interpolation), N_k = 2048\n")
        fo.write("# in [1e-4, 10]; Eq. 2.1 with Eq. 3.1-3.5, arXiv:2505.22718 Sec. 3.2 and Appendix A.\n")
        fo.write("# written by tests/golden/make_golden.py; brute-force spot checks of Delta (tracer, ell,\n")
        fo.write("# k, |diff| / max_k |Delta|): %s\n" % "; ".join(
            "%d %d %.4g %.1e" % c for c in checks))
        fo.write("# ell i j C\n")
        for li, ell in enumerate(w.ells):
            for i in range(3):
                for j in range(3):
                    fo.write("%d %d %d %.17g\n" % (ell, i, j, f["C"][li, i, j]))


# the brute-force C_ell case: two Gaussian windows in chi (Mpc/h), a smooth P(k), three multipoles
CL_BRUTE_WINDOWS = ((1000.0, 100.0), (1250.0, 120.0))
CL_BRUTE_ELLS = (2, 10, 40)
CL_BRUTE_KRANGE = (1e-4, 0.3)


def cl_brute_power(k):
    return k / (1.0 + (k / 0.02) ** 2) ** 2


def cl_brute():
    wins = [lambda x, m=m, s=s: np.exp(-0.5 * ((x - m) / s) ** 2) for m, s in CL_BRUTE_WINDOWS]
    lo, hi = np.log(CL_BRUTE_KRANGE[0]), np.log(CL_BRUTE_KRANGE[1])
    gx, gw = np.polynomial.legendre.leggauss(10)

    def cl(pieces):
        e = np.linspace(lo, hi, pieces + 1)
        half = 0.5 * np.diff(e)
        x = (0.5 * (e[:-1] + e[1:]))[:, None] + half[:, None] * gx[None, :]
        wt = (half[:, None] * gw[None, :]).ravel()
        k = np.exp(x.ravel())
        out = np.empty((len(CL_BRUTE_ELLS), 2, 2))
        for li, ell in enumerate(CL_BRUTE_ELLS):
            d = np.array([delta_brute(ell, k, wf, 200.0, 2300.0, tol=1e-12) for wf in wins])
            meas = (2.0 / np.pi) * wt * k ** 3 * cl_brute_power(k)       # dk = k dln k
            out[li] = np.einsum("q,iq,jq->ij", meas, d, d)
        return out

    c1, c2 = cl(48), cl(96)
    scale = np.sqrt(np.einsum("lii->li", c2)[:, :, None] * np.einsum("lii->li", c2)[:, None, :])
    agree = float(np.max(np.abs(c1 - c2) / scale))
    assert agree < 1e-11, agree
    with open(os.path.join(HERE, "cl_brute_gauss.txt"), "w") as fo:
        fo.write("# C_l^{ij} = (2/pi) int dk k^2 P(k) Delta_i Delta_j (Eq. 2.1, arXiv:2505.22718 Sec. 2),\n")
        fo.write("# Delta_i = int W_i(chi) j_l(k chi) dchi (Eq. 2.2), both integrals by brute force:\n")
        fo.write("# Gauss-Legendre in ln k on [%g, %g] (96 pieces x 10 nodes; 48 pieces agree to %.1e of\n"
                 % (CL_BRUTE_KRANGE + (agree,)))
        fo.write("# sqrt(C_ii C_jj)), Delta by oracle.brute.delta_brute.  W_i = exp(-(chi - mu)^2 / 2 s^2),\n")
        fo.write("# (mu, s) = %s Mpc/h; P(k) = k / (1 + (k/0.02)^2)^2.\n" % (CL_BRUTE_WINDOWS,))
        fo.write("# written by tests/golden/make_golden.py\n")
        fo.write("# ell i j C\n")
        for li, ell in enumerate(CL_BRUTE_ELLS):
            for i in range(2):
                for j in range(2):
                    fo.write("%d %d %d %.17g\n" % (ell, i, j, c2[li, i, j]))


def main():
    what = sys.argv[1] if len(sys.argv) > 1 else "all"
    if what in ("all", "convergence"):
        convergence_truth()
    if what in ("all", "cl"):
        cl_brute()
    if what in ("convergence", "cl"):
        return
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
