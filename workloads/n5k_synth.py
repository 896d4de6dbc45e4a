"""Synthetic N5K-shaped workloads (seeded), inputs only.

Units: chi in Mpc/h, k in h/Mpc, P in (Mpc/h)^3.  c/H0 = 2997.92458 Mpc/h.

Six workload shapes:

* ``tiny2``    2 Gaussian clustering windows (z = 0.5, 1.0, sigma_z = 0.05),
               3 spectra, 20 ell in [2, 200], N = 256, 256 k in [1e-4, 10],
               scale-independent growth D = 1/(1+z) (one k-knot).
* ``n5k``      10 Gaussian clustering windows (means evenly spaced on
               [0.25, 1.25], sigma_z evenly spaced on [0.04, 0.08]) and 5
               lensing windows from a Smail-type source distribution
               n(z) ~ z^2 exp(-(z/0.5)^1.5) on [0, 4] cut into 5 equal-count
               top-hat bins; 120 spectra, 103 ell in [2, 2000], N = 2048,
               1024 k in [1e-4, 10], D(k, z) = (1+z)^-1 (1 + 0.01 ln(k/0.1))
               sampled at 150 log-spaced k-knots.
* ``n5k_vjp``  ``n5k`` plus a seeded N(0, 1) cotangent on every C_ell entry.
* ``n5k_general``  ``n5k`` with a growth that is not of low rank in (k, z):
               D(k, z) = (1+z)^-1 exp(0.02 ln(k/0.1) g(z)) with g a mix of three
               redshift profiles (general_growth_factor), plus the cotangent of
               ``n5k_vjp``.
* ``walkers``  256 parameter points of the ``n5k`` shape, each with its own
               P(k) amplitude (+-10 %), tilt in [0.94, 0.99], clustering
               amplitudes in [1, 2.5], window mean shifts in [-0.02, 0.02]
               and a ragged ell list (50..103 of the 103 ell values).
* ``large``    20 Gaussian windows (sigma_z = 0.03, means on [0.2, 1.8]) and
               10 Smail lensing bins, every ell in [2, 3000], N = 4096, 4096 k
               in [1e-5, 20], N_I = 200, a k- and z-dependent bias
               b(k, z) = b0 (1+z)^0.5 (1 + 0.1 k^2) on the clustering windows.

The window builders follow Sec. 2.2 (clustering window n(z(chi)), with the
Jacobian H(z)/c so that int W dchi = int n dz = 1) and Eq. (2.8) (lens
efficiency of a source distribution).  Nothing here evaluates any part of the
FFTLog method itself.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

C_OVER_H0 = 2997.92458  # Mpc/h

# Fixed log-chi grid of every workload: chi in [1, 1e5) Mpc/h, period end excluded.
CHI_MIN = 1.0
CHI_MAX = 1.0e5
# FFTLog power-law biases per tracer kind (density, lensing).
B_DENSITY = -0.3
B_LENSING = -1.5

KIND_DENSITY = 0
KIND_LENSING = 1

_GL_X, _GL_W = np.polynomial.legendre.leggauss(16)
_GL64_X, _GL64_W = np.polynomial.legendre.leggauss(64)


class Cosmology:
    """Flat LambdaCDM background: E(z), chi(z) and its inverse z(chi)."""

    def __init__(self, omega_m: float = 0.3, z_cap: float = 12.0, nz: int = 24001):
        self.omega_m = float(omega_m)
        self.z_cap = float(z_cap)
        z = np.linspace(0.0, z_cap, nz)
        self._zt = z
        # cumulative chi(z) on the dense table by composite 16-point Gauss-Legendre
        a, b = z[:-1], z[1:]
        half = 0.5 * (b - a)
        mid = 0.5 * (b + a)
        nodes = mid[:, None] + half[:, None] * _GL_X[None, :]
        seg = (half[:, None] * _GL_W[None, :] / self.E(nodes)).sum(axis=1)
        self._chit = C_OVER_H0 * np.concatenate([[0.0], np.cumsum(seg)])

    def E(self, z):
        z = np.asarray(z, dtype=np.float64)
        return np.sqrt(self.omega_m * (1.0 + z) ** 3 + 1.0 - self.omega_m)

    def chi(self, z):
        """Comoving distance (Mpc/h): table value at the node below + 16-point GL remainder."""
        z = np.clip(np.asarray(z, dtype=np.float64), 0.0, self.z_cap)
        h = self._zt[1] - self._zt[0]
        j = np.minimum((z / h).astype(np.int64), len(self._zt) - 2)
        z0 = self._zt[j]
        half = 0.5 * (z - z0)
        mid = 0.5 * (z + z0)
        nodes = mid[..., None] + half[..., None] * _GL_X
        rem = (half[..., None] * _GL_W / self.E(nodes)).sum(axis=-1)
        return self._chit[j] + C_OVER_H0 * rem

    @property
    def chi_cap(self) -> float:
        return float(self._chit[-1])

    def z_of_chi(self, chi):
        """Inverse of chi(z) by Newton iteration; chi beyond chi(z_cap) maps to z_cap."""
        chi = np.asarray(chi, dtype=np.float64)
        inside = chi < self._chit[-1]
        c = np.where(inside, chi, self._chit[-2])
        z = np.interp(c, self._chit, self._zt)
        for _ in range(6):
            f = self.chi(z) - c
            z = z - f * self.E(z) / C_OVER_H0
            z = np.clip(z, 0.0, self.z_cap)
        return np.where(inside, z, self.z_cap)


def _gauss_nz(mu: float, sig: float):
    """Normalised Gaussian n(z) on z >= 0."""
    lo, hi = max(0.0, mu - 12 * sig), mu + 12 * sig
    xs = 0.5 * (hi + lo) + 0.5 * (hi - lo) * _GL64_X
    norm = 0.5 * (hi - lo) * np.sum(_GL64_W * np.exp(-0.5 * ((xs - mu) / sig) ** 2))

    def nz(z):
        z = np.asarray(z, dtype=np.float64)
        return np.where(z >= 0.0, np.exp(-0.5 * ((z - mu) / sig) ** 2) / norm, 0.0)
    return nz


def _smail(z):
    z = np.asarray(z, dtype=np.float64)
    zz = np.maximum(z, 0.0)
    return zz * zz * np.exp(-((zz / 0.5) ** 1.5))


def _gl_integral(f, lo, hi, pieces: int = 64):
    edges = np.linspace(lo, hi, pieces + 1)
    a, b = edges[:-1], edges[1:]
    half = 0.5 * (b - a)
    nodes = 0.5 * (a + b)[:, None] + half[:, None] * _GL_X[None, :]
    return float(np.sum(half[:, None] * _GL_W[None, :] * f(nodes)))


def smail_bin_edges(nbins: int, zmax: float = 4.0):
    """Equal-count bin edges of the Smail-type n(z) on [0, zmax] (CDF quantiles)."""
    zs = np.linspace(0.0, zmax, 40001)
    h = zs[1] - zs[0]
    seg = np.array([0.0] + [0.0] * (len(zs) - 1))
    a, b = zs[:-1], zs[1:]
    nodes = 0.5 * (a + b)[:, None] + 0.5 * h * _GL_X[None, :]
    seg[1:] = 0.5 * h * (_GL_W[None, :] * _smail(nodes)).sum(axis=1)
    cdf = np.cumsum(seg)
    cdf /= cdf[-1]
    edges = [0.0]
    for qv in np.arange(1, nbins) / nbins:
        j = int(np.searchsorted(cdf, qv))
        # refine the quantile by bisection on the exact GL CDF of the last interval
        lo, hi = zs[j - 1], zs[j]
        base = cdf[j - 1]
        total = _gl_integral(_smail, 0.0, zmax, 256)
        for _ in range(60):
            m = 0.5 * (lo + hi)
            val = base + _gl_integral(_smail, zs[j - 1], m, 1) / total
            if val < qv:
                lo = m
            else:
                hi = m
        edges.append(0.5 * (lo + hi))
    edges.append(zmax)
    return np.array(edges)


def clustering_window(cosmo: Cosmology, chi, mu: float, sig: float, z=None):
    """W(chi) = n(z(chi)) H(z)/c for a Gaussian n(z) (Sec. 2.2, with the dz/dchi Jacobian)."""
    z = cosmo.z_of_chi(chi) if z is None else z
    nz = _gauss_nz(mu, sig)
    w = nz(z) * cosmo.E(z) / C_OVER_H0
    return np.where(chi < cosmo.chi_cap * 0.999, w, 0.0)


def lensing_window(cosmo: Cosmology, chi, z_lo: float, z_hi: float, shift: float = 0.0, z=None):
    """Lens efficiency W^kappa(chi) of Eq. (2.8) for a top-hat bin of the Smail n(z).

    The source distribution is n(z) = n_Smail(z - shift) on [z_lo + shift, z_hi + shift]
    (clipped to z >= 0), normalised to unit integral.  In redshift measure
    W(chi) = (3 Om / 2 (c/H0)^2) chi (1 + z(chi)) int_{max(z(chi), lo)}^{hi} dz' n(z') (1 - chi/chi(z')),
    evaluated as chi (1+z) [G0(hi) - G0(a) - chi (G1(hi) - G1(a))] with the running integrals
    G0(x) = int_lo^x n dz', G1(x) = int_lo^x n/chi dz' tabulated by composite Gauss-Legendre.
    """
    lo = max(z_lo + shift, 0.0)
    hi = z_hi + shift
    nz = lambda z: _smail(z - shift)  # noqa: E731
    nt = 512
    zt = np.linspace(lo, hi, nt + 1)
    h = zt[1] - zt[0]
    nodes = 0.5 * (zt[:-1] + zt[1:])[:, None] + 0.5 * h * _GL_X[None, :]
    n_nodes = nz(nodes)
    g0 = np.concatenate([[0.0], np.cumsum(0.5 * h * (_GL_W * n_nodes).sum(axis=1))])
    g1 = np.concatenate([[0.0], np.cumsum(0.5 * h * (_GL_W * n_nodes / cosmo.chi(nodes)).sum(axis=1))])
    norm = g0[-1]
    chi = np.asarray(chi, dtype=np.float64)
    z = cosmo.z_of_chi(chi) if z is None else z
    a = np.clip(z, lo, hi)
    live = z < hi
    j = np.minimum(((a - lo) / h).astype(np.int64), nt - 1)
    za = zt[j]
    half = 0.5 * (a - za)
    rn = 0.5 * (a + za)[:, None] + half[:, None] * _GL_X[None, :]
    nr = nz(rn)
    G0a = g0[j] + half * (_GL_W * nr).sum(axis=1)
    G1a = g1[j] + half * (_GL_W * nr / cosmo.chi(rn)).sum(axis=1)
    inner = (g0[-1] - G0a) - chi * (g1[-1] - G1a)
    pref = 1.5 * cosmo.omega_m / C_OVER_H0 ** 2
    w = pref * chi * (1.0 + z) * inner / norm
    return np.where(live, np.maximum(w, 0.0), 0.0)


def ell_list(lmin: int, lmax: int, n: int):
    """n log-spaced integer multipoles: unique(round(geomspace(lmin, lmax, m))) with the
    smallest m giving exactly n values."""
    if n == lmax - lmin + 1:
        return np.arange(lmin, lmax + 1, dtype=np.int32)
    for m in range(n, 50 * n):
        e = np.unique(np.round(np.geomspace(lmin, lmax, m)).astype(np.int64))
        if len(e) == n:
            return e.astype(np.int32)
        if len(e) > n:
            break
    raise ValueError("no geomspace length gives exactly %d ells" % n)


def power_spectrum(k, amp: float, ns: float = 0.965):
    """Synthetic P(k) = A k^ns / (1 + (k/0.02)^2)^2 (1 + 0.05 sin(105 k))."""
    k = np.asarray(k, dtype=np.float64)
    return amp * k ** ns / (1.0 + (k / 0.02) ** 2) ** 2 * (1.0 + 0.05 * np.sin(105.0 * k))


@dataclasses.dataclass
class Workload:
    """All inputs of one C_ell evaluation (or a batch of walkers)."""
    name: str
    N: int                  # FFTLog points
    chi_min: float
    chi_max: float          # excluded period end
    k: np.ndarray           # [N_k]
    ells: np.ndarray        # [N_ell] int32 (master list)
    knots: np.ndarray       # [N_I]
    kind: np.ndarray        # [N_tr] int32 (0 density, 1 lensing, 2 magnification, 3 RSD)
    fft_bias: np.ndarray    # [N_tr] FFTLog power-law bias b_i
    W: np.ndarray           # [N_tr][N] or [n_walk][N_tr][N]
    D: np.ndarray           # [N_I][N] growth at the knots on the chi grid
    B: Optional[np.ndarray]  # [N_tr][N_I][N] k,z-dependent bias or None
    P: np.ndarray           # [N_k] or [n_walk][N_k]
    amp: np.ndarray         # [N_tr] or [n_walk][N_tr]
    C_bar: Optional[np.ndarray] = None   # cotangent [N_ell][N_tr][N_tr] (or per walker)
    ell_lists: Optional[list] = None     # walkers: list of index arrays into ells
    # window-construction metadata so tests can differentiate through the window builder
    meta: Optional[dict] = None

    @property
    def n_tr(self):
        return len(self.kind)

    @property
    def chi(self):
        return self.chi_min * np.exp(np.arange(self.N) * np.log(self.chi_max / self.chi_min) / self.N)

    @property
    def walkers(self):
        return 0 if self.W.ndim == 2 else self.W.shape[0]


def _windows(cosmo, chi, gauss, lens_edges, shifts=None):
    """Stack clustering (Gaussian) then lensing (Smail-bin) windows on the chi grid."""
    rows = []
    ng = len(gauss)
    z = cosmo.z_of_chi(chi)
    for t, (mu, sig) in enumerate(gauss):
        s = 0.0 if shifts is None else shifts[t]
        rows.append(clustering_window(cosmo, chi, mu + s, sig, z))
    for t in range(len(lens_edges) - 1):
        s = 0.0 if shifts is None else shifts[ng + t]
        rows.append(lensing_window(cosmo, chi, lens_edges[t], lens_edges[t + 1], s, z))
    return np.array(rows)


def window_rows(meta: dict, shifts=None):
    """Rebuild the window samples of a workload for given mean shifts (len N_tr)."""
    cosmo = Cosmology(meta["omega_m"])
    return _windows(cosmo, meta["chi"], meta["gauss"], meta["lens_edges"], shifts)


def make_workload(name: str, seed: int = 20250528, n_walkers: int = 256, first_walker: int = 0) -> Workload:
    rng = np.random.default_rng(seed)
    cosmo = Cosmology(0.3)
    if name == "tiny2":
        N, nk, kmin, kmax = 256, 256, 1e-4, 10.0
        ells = ell_list(2, 200, 20)
        gauss = [(0.5, 0.05), (1.0, 0.05)]
        lens_edges = []
        n_i = 1
    elif name in ("n5k", "n5k_vjp", "walkers", "n5k_general"):
        N, nk, kmin, kmax = 2048, 1024, 1e-4, 10.0
        ells = ell_list(2, 2000, 103)
        gauss = list(zip(np.linspace(0.25, 1.25, 10), np.linspace(0.04, 0.08, 10)))
        lens_edges = smail_bin_edges(5)
        n_i = 150
    elif name == "large":
        N, nk, kmin, kmax = 4096, 4096, 1e-5, 20.0
        ells = np.arange(2, 3001, dtype=np.int32)
        gauss = [(m, 0.03) for m in np.linspace(0.2, 1.8, 20)]
        lens_edges = smail_bin_edges(10)
        n_i = 200
    else:
        raise ValueError(name)
    L = np.log(CHI_MAX / CHI_MIN)
    chi = CHI_MIN * np.exp(np.arange(N) * L / N)
    z = cosmo.z_of_chi(chi)
    k = np.geomspace(kmin, kmax, nk)
    knots = np.geomspace(kmin, kmax, n_i) if n_i > 1 else np.array([0.1])
    ng, nl = len(gauss), max(len(lens_edges) - 1, 0)
    kind = np.array([KIND_DENSITY] * ng + [KIND_LENSING] * nl, dtype=np.int32)
    fft_bias = np.where(kind == KIND_DENSITY, B_DENSITY, B_LENSING).astype(np.float64)
    growth = 1.0 / (1.0 + z)
    if name == "tiny2":
        D = growth[None, :].copy()
    elif name == "n5k_general":
        D = growth[None, :] * general_growth_factor(knots[:, None], z[None, :])
    else:
        D = growth[None, :] * (1.0 + 0.01 * np.log(knots / 0.1))[:, None]
    B = None
    if name == "large":
        b0 = 1.0 + 0.1 * np.arange(ng)
        B = np.ones((ng + nl, n_i, N))
        B[:ng] = (b0[:, None, None] * ((1.0 + z) ** 0.5)[None, None, :]
                  * (1.0 + 0.1 * knots ** 2)[None, :, None])
    meta = dict(omega_m=0.3, chi=chi, gauss=gauss, lens_edges=list(lens_edges))
    A = 3.5e6 * rng.uniform(0.9, 1.1)
    if name == "walkers":
        # each walker draws from its own stream (seed, global index), so any contiguous block of
        # walkers (one rank's shard) can be generated on its own
        nw = n_walkers
        amps, tilts, biases, shifts, lists = [], [], [], [], []
        for wg in range(first_walker, first_walker + nw):
            r = np.random.default_rng([seed, wg])
            amps.append(3.5e6 * r.uniform(0.9, 1.1))
            tilts.append(r.uniform(0.94, 0.99))
            biases.append(r.uniform(1.0, 2.5, ng))
            shifts.append(r.uniform(-0.02, 0.02, ng + nl))
            m = int(r.integers(50, len(ells) + 1))
            lists.append(np.sort(r.choice(len(ells), size=m, replace=False)).astype(np.int32))
        amps, tilts = np.array(amps), np.array(tilts)
        biases, shifts = np.array(biases), np.array(shifts)
        W = np.stack([_windows(cosmo, chi, gauss, lens_edges, shifts[w]) for w in range(nw)])
        P = np.stack([power_spectrum(k, amps[w], tilts[w]) for w in range(nw)])
        amp = np.concatenate([biases, np.ones((nw, nl))], axis=1)
        meta.update(shifts=shifts, amps=amps, tilts=tilts, first_walker=first_walker)
        return Workload(name, N, CHI_MIN, CHI_MAX, k, ells, knots, kind, fft_bias, W, D, B, P, amp,
                        None, lists, meta)
    W = _windows(cosmo, chi, gauss, lens_edges)
    P = power_spectrum(k, A)
    if name == "tiny2":
        amp = np.array([1.5, 2.0])
    elif name == "large":
        amp = np.ones(ng + nl)
    else:
        amp = np.concatenate([1.0 + 0.15 * np.arange(ng), np.ones(nl)])
    C_bar = None
    if name in ("n5k_vjp", "n5k_general"):
        C_bar = rng.standard_normal((len(ells), ng + nl, ng + nl))
    meta.update(A=A)
    return Workload(name, N, CHI_MIN, CHI_MAX, k, ells, knots, kind, fft_bias, W, D, B, P, amp,
                    C_bar, None, meta)


WORKLOADS = ("tiny2", "n5k", "n5k_vjp", "n5k_general", "walkers", "large")


def general_growth_factor(k, z):
    """Scale-dependent growth factor of the n5k_general workload, exp(0.02 ln(k/0.1) g(z)), with
    g(z) a mix of three independent redshift profiles.  Its power series in ln k carries a new
    function of z at every order, so the knot profiles D(k_a, z) are of high numerical rank (about
    ten at a 1e-14 tolerance) and the k-interpolation of Sec. 3.2 cannot be folded into a few basis
    profiles: the library then transforms every knot.  Broadcasts k against z."""
    k = np.asarray(k, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    g = 0.5 + 0.8 * z / (1.0 + z) + 0.3 * np.sin(2.3 * z) * np.exp(-0.5 * z)
    return np.exp(0.02 * np.log(k / 0.1) * g)


# ------------------------------------------------------- convergence study ----

CONV_ELLS = np.array([2, 5, 12, 30, 80, 200, 500, 1200, 2000], dtype=np.int32)


def conv_growth(k, z):
    """Scale-dependent growth of the convergence study: (1+z)^-1 with a smooth 8 % suppression
    above k ~ 0.1 h/Mpc that grows with 1 - a (a massive-neutrino-like step), so the
    k-interpolation of Sec. 3.2 has something to resolve.  Broadcasts k against z."""
    k = np.asarray(k, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    x = (k / 0.1) ** 2
    return (1.0 - 0.08 * (1.0 - 1.0 / (1.0 + z)) * x / (1.0 + x)) / (1.0 + z)


def convergence_case(N: int = 2048, n_interp: int = 150, n_k: int = 2048, knots=None):
    """A reduced N5K-shaped case for the numerical-parameter study of Appendix A: a narrow and a
    wide Gaussian clustering bin and one Smail lensing bin, the multipoles CONV_ELLS, k in
    [1e-4, 10] h/Mpc.  N_FFT = N, N_interp = n_interp log-spaced knots (or the given knots),
    N_k = n_k; D at the knots from conv_growth.  Returns (Workload, meta) where meta holds the
    window parameters so a reference can rebuild the windows at any chi."""
    cosmo = Cosmology(0.3)
    L = np.log(CHI_MAX / CHI_MIN)
    chi = CHI_MIN * np.exp(np.arange(N) * L / N)
    z = cosmo.z_of_chi(chi)
    k = np.geomspace(1e-4, 10.0, n_k)
    knots = np.geomspace(1e-4, 10.0, n_interp) if knots is None else np.asarray(knots, dtype=np.float64)
    gauss = [(0.5, 0.04), (1.0, 0.08)]
    edges = smail_bin_edges(5)
    lens_edges = [edges[2], edges[3]]
    W = _windows(cosmo, chi, gauss, lens_edges)
    kind = np.array([KIND_DENSITY, KIND_DENSITY, KIND_LENSING], dtype=np.int32)
    # lensing bias -2.5: the lens efficiency grows like chi at small chi, so its FFTLog input
    # W chi^{-2-b} is ~ chi^{-1-b}; with b = -1.5 it still holds 2.6 % of its peak at chi_min and
    # jumps there to the (zero) value at chi_max of the periodic extension; b = -2.5 brings the
    # jump to ~2e-5 of the peak
    fft_bias = np.array([B_DENSITY, B_DENSITY, -2.5])
    D = conv_growth(knots[:, None], z[None, :])
    P = power_spectrum(k, 3.5e6)
    amp = np.array([1.3, 1.6, 1.0])
    meta = dict(omega_m=0.3, chi=chi, gauss=gauss, lens_edges=lens_edges)
    return Workload("convergence", N, CHI_MIN, CHI_MAX, k, CONV_ELLS.copy(), knots, kind, fft_bias,
                    W, D, None, P, amp, None, None, meta)
