"""Planted mistakes: each case replaces one function of the oracle, on the CPU, by a plausible
wrong version of it (a dropped term, a wrong sign, index or weight) and checks that one of the
oracle's pins (test_oracle_pins.py, test_oracle_limber.py, test_oracle_forecast.py) then fails.
This is the evidence that the pins constrain the oracle, rather than restate it.  Nothing here
runs on the GPU or touches the CUDA path."""
import numpy as np
import pytest
from scipy.special import loggamma

import test_oracle_forecast as fpins
import test_oracle_limber as lpins
import test_oracle_pins as pins
from conftest import cached_workload
from oracle import fftlog as O
from oracle import forecast as F
from oracle import limber as LB


def _printed_gamma_denominator(orig):
    # Eq. 3.4 as printed: Gamma((2 + l + p)/2) in the denominator
    def f(ells, p):
        l = np.asarray(ells, dtype=np.float64)[:, None]
        p = np.asarray(p, dtype=np.complex128)[None, :]
        return np.sqrt(np.pi) * np.exp((p - 1.0) * np.log(2.0) + loggamma(0.5 * (l + 1.0 + p))
                                       - loggamma(0.5 * (l + 2.0 + p)))
    return f


def _dft_sign_flipped(orig):
    # e^{+2 pi i n m / N}: for real samples, the conjugate of the right sum (the chi_min phase
    # and the Nyquist halving then act on the wrong coefficients)
    def f(samples, chi_min, chi_max, b, *a, **kw):
        c = orig(samples, chi_min, chi_max, b, *a, **kw)
        _, eta = O.eta_two_sided(c.shape[-1] - 1, np.log(chi_max / chi_min))
        ph = np.exp(-1j * eta * np.log(chi_min))
        return np.conj(c / ph) * ph
    return f


def _nyquist_not_halved(orig):
    def f(*a, **kw):
        c = orig(*a, **kw).copy()
        c[..., 0] *= 2.0
        c[..., -1] *= 2.0
        return c
    return f


def _chi_min_phase_dropped(orig):
    def f(samples, chi_min, chi_max, b, *a, **kw):
        c = orig(samples, chi_min, chi_max, b, *a, **kw)
        _, eta = O.eta_two_sided(c.shape[-1] - 1, np.log(chi_max / chi_min))
        return c * np.exp(1j * eta * np.log(chi_min))
    return f


def _full_end_intervals(orig):
    def f(k):
        w = orig(k).copy()
        w[0] *= 2.0
        w[-1] *= 2.0
        return w
    return f


def _k_squared_dropped(orig):
    def f(k, P):
        return orig(k, P) / np.asarray(k, dtype=np.float64) ** 2
    return f


def _stencil_shifted(orig):
    def f(k, knots):
        return np.roll(orig(k, knots), 1, axis=1)
    return f


def _lensing_prefactor_l_l1(orig):
    def f(ells, kind):
        if kind == O.KIND_LENSING:
            l = np.asarray(ells, dtype=np.float64)
            return l * (l + 1.0)
        return orig(ells, kind)
    return f


def _auto_spectra_only(orig):
    # Delta_i Delta_i in place of Delta_i Delta_j: a wrong index in the k-sum
    def f(delta, u, amp):
        C = orig(delta, u, amp)
        d = np.einsum("lii->li", C)
        A = np.asarray(amp, dtype=np.float64)
        return np.sqrt(d[:, :, None] * d[:, None, :]) * np.sign(A[None, :, None] * A[None, None, :])
    return f


def _amp_bar_half(orig):
    def f(*a, **kw):
        Pb, Ab, Wb, rest = orig(*a, **kw)
        return Pb, 0.5 * Ab, Wb, rest
    return f


def _p_bar_without_measure(orig):
    def f(g, *a, **kw):
        Pb, Ab, Wb, rest = orig(g, *a, **kw)
        return Pb / (2.0 / np.pi), Ab, Wb, rest
    return f


def _rsd_moment_sign(orig):
    # p (p + 1) I(p - 2) in place of p (p - 1) I(p - 2)
    def f(ells, p):
        p = np.asarray(p, dtype=np.complex128)
        return orig(ells, p) * ((p + 1.0) / (p - 1.0))[None, :]
    return f


def _magnification_prefactor_sqrt(orig):
    # the lensing prefactor sqrt((l+2)!/(l-2)!) in place of l(l+1)
    def f(ells, kind):
        if kind == O.KIND_MAGNIFICATION:
            return orig(ells, O.KIND_LENSING)
        return orig(ells, kind)
    return f


def _limber_measure_without_inverse_chi(orig):
    def f(g):
        return orig(g) * g.chi
    return f


def _limber_p_bar_half(orig):
    def f(*a, **kw):
        Pb, Ab, Wb = orig(*a, **kw)
        return 0.5 * Pb, Ab, Wb
    return f


def _fisher_full_modes(orig):
    # nu_l in place of nu_l / 2
    def f(C, X, noise, modes):
        return 2.0 * orig(C, X, noise, modes)
    return f


def _jvp_without_amplitude_term(orig):
    def f(*a, **kw):
        kw["amp_dot"] = None
        return orig(*a, **kw)
    return f


CASES = [
    ("printed Gamma denominator", "bessel_power_integral", _printed_gamma_denominator,
     lambda: pins.test_gamma_ratio_matches_mellin_integral()),
    ("DFT sign", "fftlog_coefficients", _dft_sign_flipped,
     lambda: pins.test_fftlog_reconstructs_grid_samples(-0.3)),
    ("Nyquist weight", "fftlog_coefficients", _nyquist_not_halved,
     lambda: pins.test_powerlaw_window_closed_form(-0.3, 64)),
    ("chi_min phase", "fftlog_coefficients", _chi_min_phase_dropped,
     lambda: pins.test_fftlog_reconstructs_grid_samples(-1.5)),
    ("trapezoid end weights", "lnk_trapezoid_weights", _full_end_intervals,
     lambda: pins.test_lnk_trapezoid_second_order()),
    ("k^2 of the measure", "cl_weights", _k_squared_dropped,
     lambda: pins.test_cl_matches_brute_force_double_quadrature()),
    ("Lagrange stencil index", "lagrange_matrix", _stencil_shifted,
     lambda: pins.test_lagrange_weights_partition_and_cubic_exactness()),
    ("lensing prefactor", "ell_prefactor", _lensing_prefactor_l_l1,
     lambda: pins.test_lensing_delta_matches_brute_force(cached_workload)),
    ("pair index of the k-sum", "angular_cl", _auto_spectra_only,
     lambda: pins.test_cl_matches_brute_force_double_quadrature()),
    ("factor 2 of A_bar", "vjp", _amp_bar_half,
     lambda: pins.test_vjp_homogeneity_identities(cached_workload)),
    ("2/pi in P_bar", "vjp", _p_bar_without_measure,
     lambda: pins.test_vjp_homogeneity_identities(cached_workload)),
    ("RSD moment p(p-1)", "bessel2_power_integral", _rsd_moment_sign,
     lambda: pins.test_rsd_delta_matches_brute_force()),
    ("magnification prefactor", "ell_prefactor", _magnification_prefactor_sqrt,
     lambda: pins.test_magnification_delta_matches_brute_force(cached_workload)),
]
CASES = [(name, O, attr, mutate, pin) for name, attr, mutate, pin in CASES] + [
    ("Limber measure dchi/chi^2", LB, "chi_weights", _limber_measure_without_inverse_chi,
     lambda: lpins.test_closed_form_gaussian_windows()),
    ("Limber P_bar", LB, "limber_vjp", _limber_p_bar_half,
     lambda: lpins.test_limber_vjp_identities_and_differences(cached_workload)),
    ("Fisher mode count", F, "gaussian_quad", _fisher_full_modes,
     lambda: fpins.test_single_tracer_closed_form()),
    ("JVP amplitude term", F, "jvp", _jvp_without_amplitude_term,
     lambda: fpins.test_jvp_against_central_differences(cached_workload)),
]


@pytest.mark.parametrize("name,module,attr,mutate,pin", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_a_pin(name, module, attr, mutate, pin, monkeypatch):
    monkeypatch.setattr(module, attr, mutate(getattr(module, attr)))
    with pytest.raises(AssertionError):
        pin()


def test_unmutated_pins_pass():
    """The same pin calls pass against the oracle as it stands."""
    for case in CASES:
        case[-1]()
