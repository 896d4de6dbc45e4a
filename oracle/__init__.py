"""FP64 CPU oracle of the beyond-Limber FFTLog C_ell method (arXiv:2505.22718).

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA library is checked against.  Only the test-suite, the smoke check of the
build entry point and the CPU-baseline leg of the benchmark may import it; the
library itself never does, and this package imports nothing from the library.

Modules:
  fftlog   -- the method step by step (FFTLog coefficients, Gamma-ratio table,
              k-interpolation, contraction, k-quadrature, reverse mode).
  forecast -- forward mode (JVP) and the Gaussian Fisher / chi^2 quadratic form (Sec. 4.3).
  limber   -- the Limber branch (Eq. 2.19) on the same grids, its reverse mode, the hybrid C_ell.
  brute    -- independent checks: spherical Bessel functions by recurrence,
              brute-force line-of-sight integrals, the Limber limit.
"""
