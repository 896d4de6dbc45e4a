"""The Limber branch (Eq. 2.19) on the pipeline's grids, and the hybrid C_ell.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Eq. 2.19 replaces the two line-of-sight integrals of Eq. 2.1-2.2 by one: the closure relation of
the spherical Bessel functions, int dk k^2 j_l(k chi) j_l(k chi') = (pi/2) delta(chi - chi')/chi^2,
taken at chi = nu/k with nu = l + 1/2.  For this pipeline's source functions
f_i(chi, k) = pi_i(l) k^{t_i} chi^{s_i} W_i(chi) D(k, chi) B_i(k, chi) (reading R7) it reads
    C_ij(l) = A_i A_j int dchi / chi^2 f_i(chi, nu/chi) f_j(chi, nu/chi) P(nu/chi),
which is Eq. 2.19 for density tracers (f = W D).

Reading R12 (the discrete form evaluated here and by the library):
  - chi runs over the FFTLog grid chi_m = chi_min e^{m L/N}; dchi = chi dln chi with the
    rectangle rule in ln chi (weight L/N; the grid is periodic, the windows vanish at its ends):
        C_ij(l) = A_i A_j sum_m (L/N) chi_m^{-1} Pt(k_m) G_i(l, m) G_j(l, m),  k_m = nu / chi_m,
        G_i(l, m) = pi_i(l) k_m^{t_i} chi_m^{s_i} W_i(chi_m) sum_a Lam_a(k_m) D_a(chi_m) B_ia(chi_m);
  - Pt is P on the k grid interpolated as the knots are (R5: 4-point Lagrange in ln k, clamped
    stencil) and zero outside [k_0, k_{N_k-1}], the range the FFTLog path integrates over;
  - D B at k_m by the knot interpolation of R5;
  - the windows enter without the tapers of R4 (those belong to the FFTLog sum);
  - RSD tracers (j_l'') have no Limber form here.
The hybrid spectrum takes the FFTLog C_ell below a switch multipole and the Limber C_ell at and
above it.
"""
from __future__ import annotations

import numpy as np

from . import fftlog as O


def chi_weights(g: O.Grids) -> np.ndarray:
    """c_m = (L/N) / chi_m: dchi / chi^2 on the grid."""
    return (g.L / g.N) / g.chi


def interp_rows(x, grid) -> np.ndarray:
    """Lagrange matrix of R5 from `grid` to the points x, rows zeroed outside [grid_0, grid_-1]."""
    x = np.asarray(x, dtype=np.float64)
    lam = O.lagrange_matrix(x, grid)
    out = (x < grid[0]) | (x > grid[-1])
    lam[out] = 0.0
    return lam


def limber_parts(g: O.Grids, ell: int, W, D, B=None):
    """For one multipole: H[i][m] = pi_i k^{t_i} chi^{s_i} sum_a Lam_a(k_m) D_a B_ia (so that
    G_i = W_i H_i) and the matrix Rho[m][q] with Pt(k_m) = sum_q Rho[m][q] P_q."""
    nu = ell + 0.5
    k = nu / g.chi
    Lk = O.lagrange_matrix(k, g.knots)                       # [N, N_I] knot weights
    Rho = interp_rows(k, g.k)                                # [N, N_k]
    n_tr = len(g.kind)
    H = np.empty((n_tr, g.N))
    s = O.chi_power(g.kind)
    t = O.k_power(g.kind)
    D = np.asarray(D, dtype=np.float64)
    for i in range(n_tr):
        if int(g.kind[i]) == O.KIND_RSD:
            raise ValueError("RSD tracers have no Limber form")
        DB = D if B is None else D * np.asarray(B)[i]        # [N_I, N]
        dbk = np.einsum("ma,am->m", Lk, DB)                  # sum_a Lam_a(k_m) DB_a(chi_m)
        pre = O.ell_prefactor([ell], int(g.kind[i]))[0]
        H[i] = pre * k ** t[i] * g.chi ** s[i] * dbk
    return H, Rho


def limber_cl(g: O.Grids, W, D, P, amp, B=None, ells=None):
    """Unit-amplitude U and C of the Limber branch for the given multipoles (R12)."""
    ells = g.ells if ells is None else np.asarray(ells)
    W = np.asarray(W, dtype=np.float64)
    A = np.asarray(amp, dtype=np.float64)
    c = chi_weights(g)
    U = np.empty((len(ells), len(g.kind), len(g.kind)))
    for li, ell in enumerate(ells):
        H, Rho = limber_parts(g, int(ell), W, D, B)
        G = W * H
        pw = c * (Rho @ np.asarray(P, dtype=np.float64))
        U[li] = (G * pw[None, :]) @ G.T
    return U, U * A[None, :, None] * A[None, None, :]


def limber_vjp(g: O.Grids, W, D, P, amp, C_bar, B=None, ells=None):
    """Reverse mode of limber_cl, written by hand: with S = (C_bar + C_bar^T)/2,
    T = S A A^T, R_i = sum_j T_ij G_j,
        W_bar_i(m) = 2 sum_l c_m Pt_lm H_i(l, m) R_i(l, m),
        P_bar_q   = sum_l sum_m Rho_lm,q c_m sum_i G_i R_i,
        A_bar_i   = 2 sum_l sum_j S_ij A_j U_ij."""
    ells = g.ells if ells is None else np.asarray(ells)
    W = np.asarray(W, dtype=np.float64)
    A = np.asarray(amp, dtype=np.float64)
    c = chi_weights(g)
    S = 0.5 * (C_bar + np.transpose(C_bar, (0, 2, 1)))
    W_bar = np.zeros_like(W)
    P_bar = np.zeros(len(g.k))
    A_bar = np.zeros(len(A))
    for li, ell in enumerate(ells):
        H, Rho = limber_parts(g, int(ell), W, D, B)
        G = W * H
        Pt = Rho @ np.asarray(P, dtype=np.float64)
        T = S[li] * A[:, None] * A[None, :]
        R = T @ G                                            # [N_tr, N]
        W_bar += 2.0 * (c * Pt)[None, :] * H * R
        P_bar += Rho.T @ (c * np.sum(G * R, axis=0))
        U = (G * (c * Pt)[None, :]) @ G.T
        A_bar += 2.0 * np.einsum("ij,j,ij->i", S[li], A, U)
    return P_bar, A_bar, W_bar


def limber_jvp(g: O.Grids, W, D, P, amp, B=None, ells=None, P_dot=None, amp_dot=None, W_dot=None):
    """Forward mode of limber_cl along one tangent (None = zero), by the product rule:
    dU = sum_m c_m [Pt' G_i G_j + Pt (G'_i G_j + G_i G'_j)], G' = W' H (G is linear in W),
    dC = A_i A_j dU + (A'_i A_j + A_i A'_j) U."""
    ells = g.ells if ells is None else np.asarray(ells)
    W = np.asarray(W, dtype=np.float64)
    A = np.asarray(amp, dtype=np.float64)
    Ad = np.zeros_like(A) if amp_dot is None else np.asarray(amp_dot, dtype=np.float64)
    c = chi_weights(g)
    out = np.empty((len(ells), len(A), len(A)))
    for li, ell in enumerate(ells):
        H, Rho = limber_parts(g, int(ell), W, D, B)
        G = W * H
        pw = c * (Rho @ np.asarray(P, dtype=np.float64))
        U = (G * pw[None, :]) @ G.T
        dU = np.zeros_like(U)
        if P_dot is not None:
            dU += (G * (c * (Rho @ np.asarray(P_dot, dtype=np.float64)))[None, :]) @ G.T
        if W_dot is not None:
            t = ((np.asarray(W_dot) * H) * pw[None, :]) @ G.T
            dU += t + t.T
        out[li] = dU * A[:, None] * A[None, :] + U * (Ad[:, None] * A[None, :] + A[:, None] * Ad[None, :])
    return out


def hybrid_forward(g: O.Grids, W, D, P, amp, ell_switch, B=None, taper_chi=None, taper_c=None):
    """C of the FFTLog path for l < ell_switch and of the Limber branch for l >= ell_switch."""
    f = O.forward(g, W, D, P, amp, B, taper_chi, taper_c)
    C = f["C"].copy()
    sel = np.asarray(g.ells) >= ell_switch
    if np.any(sel):
        _, CL = limber_cl(g, W, D, P, amp, B, np.asarray(g.ells)[sel])
        C[sel] = CL
    return C, f


def hybrid_vjp(g: O.Grids, fwd: dict, C_bar, W, D, P, amp, ell_switch, B=None, taper_chi=None,
               taper_c=None):
    """Reverse mode of hybrid_forward: the FFTLog rows and the Limber rows add."""
    sel = np.asarray(g.ells) >= ell_switch
    Cb_f = np.where(sel[:, None, None], 0.0, C_bar)
    Pb, Ab, Wb, _ = O.vjp(g, fwd, Cb_f, W, D, P, amp, B, taper_chi, taper_c)
    if np.any(sel):
        Pl, Al, Wl = limber_vjp(g, W, D, P, amp, C_bar[sel], B, np.asarray(g.ells)[sel])
        Pb, Ab, Wb = Pb + Pl, Ab + Al, Wb + Wl
    return Pb, Ab, Wb


def hybrid_jvp(g: O.Grids, fwd: dict, D, P, amp, ell_switch, B=None, taper_chi=None, taper_c=None,
               P_dot=None, amp_dot=None, W_dot=None, W=None):
    """Forward mode of hybrid_forward: oracle.forecast.jvp on the FFTLog rows, limber_jvp on the
    Limber rows (W, the base windows, is needed by the latter)."""
    from . import forecast as F
    J = F.jvp(g, fwd, D, P, amp, B, taper_chi, taper_c, P_dot=P_dot, amp_dot=amp_dot, W_dot=W_dot)
    sel = np.asarray(g.ells) >= ell_switch
    if np.any(sel):
        J[sel] = limber_jvp(g, W, D, P, amp, B, np.asarray(g.ells)[sel], P_dot, amp_dot, W_dot)
    return J
