"""Seeded synthetic inputs for the beyond-Limber FFTLog C_ell hot path.

This package builds the *inputs* of the method (window samples on the log-chi
grid, growth and bias at the k-knots, the k grid, P(k), the ell lists, the
tracer amplitudes) for the five workload shapes used by the tests and the
benchmark.  It is shared by the FP64 oracle and by the CUDA path and therefore
holds none of the method's arithmetic: no FFTLog, no Gamma-function table, no
spherical Bessel function, no k-quadrature.  The window builders implement the
probe definitions of Section 2 of the paper (clustering window Sec. 2.2 and the
lens efficiency, Eq. 2.8), which sit upstream of the hot path.
"""
from .n5k_synth import (  # noqa: F401
    Cosmology, Workload, make_workload, ell_list, WORKLOADS,
)
