"""Shared helpers of the GPU parity tests: run a workload through the C ABI and through the
oracle, and the error gates."""
from __future__ import annotations

import numpy as np

from oracle import fftlog as O


def norm_err(C, Co):
    """max |C - Co| / max(|Co_ij|, 1e-3 sqrt(Co_ii Co_jj)) per element (normalised gate)."""
    dg = np.abs(np.einsum("...ii->...i", Co))
    floor = 1e-3 * np.sqrt(dg[..., :, None] * dg[..., None, :])
    return float(np.max(np.abs(C - Co) / np.maximum(np.abs(Co), floor)))


def max_rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.abs(b).max(), 1e-300))


def p_abs(delta, C_bar, amp, k):
    """Size of the terms that form each P_bar_q, from the oracle's Delta [N_ell][N_tr][N_k]:
    (2/pi) w_q k_q^2 sum_l sum_ij |S_ij A_i A_j Delta_i(l, k_q) Delta_j(l, k_q)|, S the
    symmetrised cotangent.  P_bar_q is a sum of terms of both signs (S is a random cotangent), so
    its relative accuracy is that of Delta times the ratio of this sum to |P_bar_q|; gating
    |P_bar - P_bar_oracle| against tol * p_abs is gating every entry at the accuracy the forward
    gate allows for Delta."""
    S = 0.5 * (C_bar + np.transpose(C_bar, (0, 2, 1)))
    A = np.asarray(amp, dtype=np.float64)
    SA = np.abs(S * A[None, :, None] * A[None, None, :])
    d = np.abs(delta)
    return (2.0 / np.pi) * O.lnk_trapezoid_weights(k) * k ** 2 * np.einsum("lij,liq,ljq->q", SA, d, d)


def pbar_err(g, go, pabs):
    """Per-element error of P_bar against the size of the terms that form it (p_abs)."""
    g = np.asarray(g, dtype=np.float64).reshape(-1)
    go = np.asarray(go, dtype=np.float64).reshape(-1)
    return float(np.max(np.abs(g - go) / np.maximum(pabs, 1e-300)))


def wbar_err(g, go):
    """Per-row error of W_bar: max over the rows (walker, tracer) of max_m |g - go| / max_m |go|.
    W_bar_i(chi_m) is an inverse DFT of the coefficient cotangents (the adjoint of Eq. 3.2), so an
    error in any coefficient spreads evenly over the row: the row's largest entry is the scale."""
    g = np.asarray(g, dtype=np.float64)
    go = np.asarray(go, dtype=np.float64).reshape(g.shape)
    rmax = np.abs(go).max(axis=-1)
    return float(np.max(np.abs(g - go).max(axis=-1) / np.maximum(rmax, 1e-300)))


def grad_err(g, go, floor=1e-3):
    """Per-element error of a gradient: max |g - go| / max(|go|, floor * max |go| of its row),
    rows along the last axis (P_bar: one row of N_k per walker; W_bar: one row of N per walker
    and tracer; amp_bar: one row of N_tr).  The floor keeps entries that are zero or
    sign-changing from being gated at an impossible relative tolerance, while every entry of a
    row's upper three decades is gated on its own."""
    g = np.asarray(g, dtype=np.float64)
    go = np.asarray(go, dtype=np.float64).reshape(g.shape)
    rmax = np.abs(go).max(axis=-1, keepdims=True)
    den = np.maximum(np.abs(go), np.maximum(floor * rmax, 1e-300))
    return float(np.max(np.abs(g - go) / den))


def lib_context(w, tapers=None, budget=0):
    from paper_2505_22718_gb300 import Context
    ctx = Context(0, budget)
    ctx.set_grids(w.chi_min, w.chi_max, w.N, w.k, w.ells, w.knots)
    tc, tn = (None, None) if tapers is None else tapers
    ctx.set_tracers(w.kind, w.fft_bias, tc, tn)
    ctx.set_windows(w.W, w.D, w.B)
    ctx.set_power(w.P, w.amp)
    if w.ell_lists is not None:
        ctx.set_ell_lists(w.ell_lists)
    return ctx


def oracle_walker(w, widx=None, tapers=None, C_bar=None, ells_sel=None):
    """Oracle forward (and VJP if C_bar is given) for one walker (widx None = unbatched)."""
    W = w.W if widx is None else w.W[widx]
    P = w.P if widx is None else w.P[widx]
    amp = w.amp if widx is None else w.amp[widx]
    ells = w.ells if ells_sel is None else w.ells[ells_sel]
    g = O.Grids(w.N, w.chi_min, w.chi_max, w.k, ells, w.knots, w.kind, w.fft_bias)
    tc, tn = (None, None) if tapers is None else tapers
    f = O.forward(g, W, w.D, P, amp, w.B, tc, tn)
    if C_bar is None:
        return f, None
    Pb, Ab, Wb, extra = O.vjp(g, f, C_bar, W, w.D, P, amp, w.B, tc, tn)
    extra = dict(extra, P_abs=p_abs(f["delta"], C_bar, amp, w.k))
    return f, (Pb, Ab, Wb, extra)


def make_ragged_case(n_walk=3, seed=11):
    """A small workload that exercises every edge of the kernels: N = 512, 7 tracers (4 density,
    3 lensing), 333 k points (not a tile multiple), 37 multipoles, 23 knots with a growth that is
    not linear in ln k, a k,z-dependent bias, tapers, several walkers and ragged ell lists."""
    from workloads.n5k_synth import (CHI_MAX, CHI_MIN, Cosmology, Workload, clustering_window,
                                     ell_list, lensing_window, power_spectrum, smail_bin_edges)
    rng = np.random.default_rng(seed)
    cosmo = Cosmology()
    N = 512
    L = np.log(CHI_MAX / CHI_MIN)
    chi = CHI_MIN * np.exp(np.arange(N) * L / N)
    z = cosmo.z_of_chi(chi)
    k = np.geomspace(1e-4, 5.0, 333)
    ells = ell_list(2, 700, 37)
    knots = np.geomspace(1e-4, 5.0, 23)
    gauss = [(0.3, 0.1), (0.6, 0.12), (0.9, 0.15), (1.3, 0.2)]
    edges = smail_bin_edges(3)
    kind = np.array([0, 0, 0, 0, 1, 1, 1], dtype=np.int32)
    fft_bias = np.array([-0.3, -0.3, -0.4, -0.3, -1.5, -1.5, -1.2])
    Ws = []
    for wk in range(n_walk):
        sh = rng.uniform(-0.02, 0.02, 7)
        rows = [clustering_window(cosmo, chi, m + sh[t], s, z) for t, (m, s) in enumerate(gauss)]
        rows += [lensing_window(cosmo, chi, edges[t], edges[t + 1], sh[4 + t], z) for t in range(3)]
        Ws.append(np.array(rows))
    W = np.stack(Ws)
    lk = np.log(knots / 0.1)
    D = (1.0 / (1.0 + z))[None, :] * (1.0 + 0.02 * lk + 0.003 * lk ** 2)[:, None]
    B = np.ones((7, len(knots), N))
    B[:4] = (1.0 + 0.5 * z)[None, None, :] * (1.0 + 0.05 * knots)[None, :, None]
    P = np.stack([power_spectrum(k, 3.5e6 * rng.uniform(0.9, 1.1), rng.uniform(0.94, 0.99))
                  for _ in range(n_walk)])
    amp = np.concatenate([rng.uniform(1.0, 2.5, (n_walk, 4)), np.ones((n_walk, 3))], axis=1)
    lists = [np.sort(rng.choice(len(ells), size=int(rng.integers(5, len(ells) + 1)), replace=False))
             .astype(np.int32) for _ in range(n_walk)]
    lists[0] = np.arange(len(ells), dtype=np.int32)
    # tapers: raised cosine on the outer 5 % of the chi range and the top 25 % of n
    x = np.arange(N) / (N - 1)
    tchi = np.ones(N)
    e = 0.05
    tchi[x < e] = 0.5 * (1 - np.cos(np.pi * x[x < e] / e))
    tchi[x > 1 - e] = 0.5 * (1 - np.cos(np.pi * (1 - x[x > 1 - e]) / e))
    nh = N // 2 + 1
    nn = np.arange(nh) / (nh - 1)
    tc = np.ones(nh)
    tc[nn > 0.75] = 0.5 * (1 + np.cos(np.pi * (nn[nn > 0.75] - 0.75) / 0.25))
    taper_chi = np.stack([tchi if t >= 4 else np.ones(N) for t in range(7)])
    taper_c = np.stack([tc if t >= 4 else np.ones(nh) for t in range(7)])
    w = Workload("ragged", N, CHI_MIN, CHI_MAX, k, ells, knots, kind, fft_bias, W, D, B, P, amp,
                 None, lists, None)
    return w, (taper_chi, taper_c)
