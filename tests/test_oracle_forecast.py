"""Pins of the forward mode and of the Gaussian Fisher form of the oracle (Sec. 4.3).

- jvp against central finite differences of forward() along tangents of P, A and W, entry by
  entry, and against the already pinned reverse mode through <C_bar, J v> = <J^T C_bar, v>;
- jvp is exactly linear: the tangent of a sum is the sum of the tangents;
- gaussian_quad (the trace form) against the explicit covariance of the unique pairs solved by
  brute force, for Fisher and chi^2;
- one tracer: the textbook closed form sum_l (nu_l/2) X_a X_b / (C + N)^2.
"""
import numpy as np

from oracle import fftlog as O
from oracle import forecast as F


def _small(wl):
    w = wl("n5k_vjp")
    tr = np.array([0, 7, 10, 14])
    q = np.arange(0, len(w.k), 4)
    ells = w.ells[::10]
    g = O.Grids(w.N, w.chi_min, w.chi_max, w.k[q], ells, w.knots, w.kind[tr], w.fft_bias[tr])
    return w, tr, g, w.P[::4], w.amp[tr], w.W[tr]


def test_jvp_against_central_differences(wl):
    w, tr, g, P, amp, Wt = _small(wl)
    f = O.forward(g, Wt, w.D, P, amp)
    rng = np.random.default_rng(8)
    dP = rng.standard_normal(len(P)) * P
    dA = rng.standard_normal(len(amp)) * amp
    dW = rng.standard_normal(Wt.shape) * Wt
    J = F.jvp(g, f, w.D, P, amp, P_dot=dP, amp_dot=dA, W_dot=dW)
    h = 1e-5
    Cp = O.forward(g, Wt + h * dW, w.D, P + h * dP, amp + h * dA)["C"]
    Cm = O.forward(g, Wt - h * dW, w.D, P - h * dP, amp - h * dA)["C"]
    fd = (Cp - Cm) / (2 * h)
    # entry by entry, relative to the diagonal scale of each spectrum
    dg = np.sqrt(np.abs(np.einsum("lii->li", f["C"])))
    scale = dg[:, :, None] * dg[:, None, :]
    assert np.max(np.abs(J - fd) / scale) < 1e-7


def test_jvp_is_the_transpose_of_the_pinned_vjp(wl):
    w, tr, g, P, amp, Wt = _small(wl)
    f = O.forward(g, Wt, w.D, P, amp)
    rng = np.random.default_rng(9)
    Cb = rng.standard_normal(f["C"].shape)
    Pb, Ab, Wb, _ = O.vjp(g, f, Cb, Wt, w.D, P, amp)
    dP = rng.standard_normal(len(P)) * P
    dA = rng.standard_normal(len(amp))
    dW = rng.standard_normal(Wt.shape) * Wt
    for v in [(dP, None, None), (None, dA, None), (None, None, dW)]:
        J = F.jvp(g, f, w.D, P, amp, P_dot=v[0], amp_dot=v[1], W_dot=v[2])
        lhs = np.sum(Cb * J)
        rhs = sum(np.sum(a * b) for a, b in zip((Pb, Ab, Wb), v) if b is not None)
        assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


def test_jvp_linear_in_the_tangent(wl):
    w, tr, g, P, amp, Wt = _small(wl)
    f = O.forward(g, Wt, w.D, P, amp)
    rng = np.random.default_rng(10)
    a = rng.standard_normal(Wt.shape) * Wt
    b = rng.standard_normal(len(P)) * P
    Ja = F.jvp(g, f, w.D, P, amp, W_dot=a)
    Jb = F.jvp(g, f, w.D, P, amp, P_dot=b)
    Jab = F.jvp(g, f, w.D, P, amp, W_dot=a, P_dot=b)
    assert np.max(np.abs(Jab - Ja - Jb)) <= 1e-13 * np.max(np.abs(Jab))
    # the window tangent W itself: C is quadratic in W, so J(W) = 2 C
    JW = F.jvp(g, f, w.D, P, amp, W_dot=Wt)
    assert np.max(np.abs(JW - 2.0 * f["C"])) <= 1e-12 * np.max(np.abs(f["C"]))


def _random_spd_case(n_l=5, n=4, n_x=3, seed=2):
    rng = np.random.default_rng(seed)
    C = np.empty((n_l, n, n))
    for l in range(n_l):
        a = rng.standard_normal((n, n + 2))
        C[l] = a @ a.T / (n + 2)
    noise = rng.uniform(0.05, 0.2, n)
    X = rng.standard_normal((n_x, n_l, n, n))
    X = 0.5 * (X + np.transpose(X, (0, 1, 3, 2)))
    modes = rng.uniform(5.0, 500.0, n_l)
    return C, X, noise, modes


def test_trace_form_equals_pair_covariance_fisher():
    C, X, noise, modes = _random_spd_case()
    Q = F.gaussian_quad(C, X, noise, modes)
    n = C.shape[1]
    iu = np.triu_indices(n)
    want = np.zeros_like(Q)
    for l in range(C.shape[0]):
        cov, pairs = F.pair_covariance(C[l] + np.diag(noise), modes[l])
        J = np.array([[X[a, l][i, j] for (i, j) in pairs] for a in range(X.shape[0])])
        assert np.array_equal(np.array(pairs).T, np.array(iu))
        want += J @ np.linalg.solve(cov, J.T)
    assert np.max(np.abs(Q - want)) <= 1e-11 * np.max(np.abs(want))
    assert np.allclose(Q, Q.T, rtol=0, atol=1e-13 * np.abs(Q).max())
    # chi^2 of one perturbation is the same form with a = b
    chi2 = F.gaussian_quad(C, X[:1], noise, modes)[0, 0]
    assert abs(chi2 - want[0, 0]) <= 1e-11 * want[0, 0]


def test_single_tracer_closed_form():
    C, X, noise, modes = _random_spd_case(n=1, n_x=2)
    Q = F.gaussian_quad(C, X, noise, modes)
    Ct = C[:, 0, 0] + noise[0]
    want = np.array([[np.sum(0.5 * modes * X[a, :, 0, 0] * X[b, :, 0, 0] / Ct ** 2)
                      for b in range(2)] for a in range(2)])
    assert np.max(np.abs(Q - want)) <= 1e-13 * np.max(np.abs(want))
