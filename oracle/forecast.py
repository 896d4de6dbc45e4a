"""Forward mode and the Gaussian Fisher matrix of the C_ell pipeline (Sec. 4.3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper computes the Fisher information as the Hessian of the Gaussian log-likelihood of the
C_ell data vector, with a Gaussian covariance (cosmic variance plus additive noise) scaled by
1/f_sky (Sec. 4.3), and measures accuracy as a chi^2 against that covariance (Sec. 4.2).  Both are
the same quadratic form of C_ell perturbations.  This module writes out:

  jvp             the forward-mode derivative dC of forward() along tangents of P(k), the
                  amplitudes A_i and the windows W_i (the product rule on Eq. 2.1; Delta is
                  linear in W through Eq. 3.1-3.5);
  gaussian_quad   Q_ab = sum_l (nu_l / 2) Tr[Ct^-1 X_a Ct^-1 X_b],  Ct = C + diag(noise),
                  nu_l = (2l + 1) f_sky (bin width) the number of modes behind C_l: the Fisher
                  matrix when X_a = dC/dtheta_a, and chi^2 when X = C - C_data;
  pair_covariance the explicit Gaussian covariance of the unique pairs (i <= j),
                  Cov[(ij),(mn)] = (Ct_im Ct_jn + Ct_in Ct_jm) / nu_l, for the pins.

Reading R11: the Fisher matrix of the data vector of unique pairs with that covariance equals
the trace form above (the tests check the two against each other by brute force); the trace form
is the one the library evaluates.
"""
from __future__ import annotations

import numpy as np

from . import fftlog as O


def jvp(g: O.Grids, fwd: dict, D, P, amp, B=None, taper_chi=None, taper_c=None,
        P_dot=None, amp_dot=None, W_dot=None):
    """dC[ell][i][j] of forward() along one tangent (P_dot[N_k], amp_dot[N_tr], W_dot[N_tr][N];
    None = zero).  With U = C at unit amplitudes and u = cl_weights(k, P):
        dU_ij = sum_q [u'_q Delta_i Delta_j + u_q (Delta'_i Delta_j + Delta_i Delta'_j)],
        dC_ij = A_i A_j dU_ij + (A'_i A_j + A_i A'_j) U_ij,
    with u' = cl_weights(k, P_dot) and Delta' = the contraction of the FFTLog coefficients of the
    tangent windows (Delta is linear in W)."""
    delta, u = fwd["delta"], fwd["u"]
    A = np.asarray(amp, dtype=np.float64)
    n_tr = delta.shape[1]
    U = np.einsum("liq,q,ljq->lij", delta, u, delta)
    dU = np.zeros_like(U)
    if P_dot is not None:
        du = O.cl_weights(g.k, P_dot)
        dU += np.einsum("liq,q,ljq->lij", delta, du, delta)
    if W_dot is not None:
        coef_dot = O.window_coefficients(g, W_dot, D, B, taper_chi, taper_c)
        ddelta, _ = O.delta_from_coefficients(g, coef_dot)
        t = np.einsum("liq,q,ljq->lij", ddelta, u, delta)
        dU += t + np.transpose(t, (0, 2, 1))
    Ad = np.zeros(n_tr) if amp_dot is None else np.asarray(amp_dot, dtype=np.float64)
    dC = dU * A[None, :, None] * A[None, None, :]
    dC += U * (Ad[None, :, None] * A[None, None, :] + A[None, :, None] * Ad[None, None, :])
    return dC


def gaussian_quad(C, X, noise, modes):
    """Q[a][b] = sum_l (modes_l / 2) Tr[Ct^-1 X_a Ct^-1 X_b], Ct = C + diag(noise).
    C[N_ell][N_tr][N_tr], X[n_x][N_ell][N_tr][N_tr], noise[N_tr], modes[N_ell]."""
    X = np.asarray(X, dtype=np.float64)
    n_x = X.shape[0]
    Q = np.zeros((n_x, n_x))
    for l in range(C.shape[0]):
        Ct = C[l] + np.diag(np.asarray(noise, dtype=np.float64))
        Y = [np.linalg.solve(Ct, X[a, l]) for a in range(n_x)]
        for a in range(n_x):
            for b in range(n_x):
                Q[a, b] += 0.5 * modes[l] * np.trace(Y[a] @ Y[b])
    return Q


def pair_covariance(Ct, nu):
    """Gaussian covariance of the unique pairs (i <= j) of one multipole:
    Cov[(ij),(mn)] = (Ct_im Ct_jn + Ct_in Ct_jm) / nu; returns (Cov, list of pairs)."""
    n = Ct.shape[0]
    pairs = [(i, j) for i in range(n) for j in range(i, n)]
    cov = np.empty((len(pairs), len(pairs)))
    for p, (i, j) in enumerate(pairs):
        for q, (m, r) in enumerate(pairs):
            cov[p, q] = (Ct[i, m] * Ct[j, r] + Ct[i, r] * Ct[j, m]) / nu
    return cov, pairs
