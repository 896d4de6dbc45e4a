// The Limber branch (Eq. 2.19): multipoles at or above a switch take
//   U_ij(l) = sum_m c_m Pt(k_m) G_i(l, m) G_j(l, m),   k_m = nu / chi_m,  nu = l + 1/2,
//   c_m = (L/N) / chi_m,   G_i = W_i(chi_m) H_i,   H_i = pi_i(l) nu^{t_i} sum_a Lam_a(k_m) D_a(chi_m) B_ia(chi_m)
// on the FFTLog chi grid (rectangle rule in ln chi), with Pt the 4-point Lagrange interpolant in
// ln k of P on the k grid (zero outside it) and Lam the knot weights of the same rule.  Every kind
// that has a Limber form has s = t (density 0, lensing and magnification -2), so
// k^t chi^s = nu^t.  All arithmetic is FP64: the branch costs N_lim N N_tr^2 operations, small
// next to the FFTLog path it replaces.
//
// Kernels: the forward rows (one CTA per Limber multipole and walker, chi in tiles of 32 staged in
// shared memory, one thread per tracer pair); the forward-mode rows (one CTA per multipole and
// tangent); the reverse mode, in two steps: per chi tile and walker, W_bar += 2 c Pt H R summed
// over the multipoles (R_i = sum_j T_ij G_j, T = S A A^T) and the per-(l, chi) weights
// Q = c sum_i G_i R_i; then P_bar_q += sum_{l,m} rho_q(k_lm) Q_lm, gathered per k point in a fixed
// order.
#include <algorithm>

#include "swcl_internal.h"

namespace swcl {
namespace {

constexpr int LT = 256;   // threads
constexpr int MT = 32;    // chi points per tile
constexpr int MAXR = 9;   // tracer pairs per thread (64 tracers)

// Stencil of R5 on a positive, increasing grid at ln-value x: returns the first row and writes the
// s = min(4, n) Lagrange weights in ln(grid) (unused entries 0).
__device__ int stencil_ln(const double* grid, int n, double x, double w[4]) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (log(grid[mid]) <= x) lo = mid + 1; else hi = mid;
  }
  const int s = n < 4 ? n : 4;
  int a = lo - 1;
  a = a < 0 ? 0 : (a > n - 1 ? n - 1 : a);
  int start = a - 1;
  if (start > n - s) start = n - s;
  if (start < 0) start = 0;
  double xs[4];
  for (int r = 0; r < s; ++r) xs[r] = log(grid[start + r]);
  for (int r = 0; r < 4; ++r) {
    double v = 0.0;
    if (r < s) {
      v = 1.0;
      for (int t = 0; t < s; ++t)
        if (t != r) v *= (x - xs[t]) / (xs[r] - xs[t]);
    }
    w[r] = v;
  }
  return start;
}

__device__ __forceinline__ double ell_pre(int kind, double l) {
  if (kind == SWCL_LENSING) return sqrt((l + 2.0) * (l + 1.0) * l * (l - 1.0));
  if (kind == SWCL_MAGNIFICATION) return l * (l + 1.0);
  return 1.0;
}

// Per chi tile: pw[mm] = c_m Pt(k_m) (P of the walker; Pd, if given, the same with the tangent
// in pwd), the knot stencil (st, lam) and cw[mm] = c_m.
struct Tile {
  double pw[MT], pwd[MT], cw[MT], lam[MT][4];
  int st[MT];
};

__device__ void tile_weights(Tile& T, const LimberArgs& a, double lnnu, int m0, const double* P,
                             const double* Pd) {
  for (int mm = threadIdx.x; mm < MT; mm += blockDim.x) {
    const int m = m0 + mm;
    double pw = 0.0, pwd = 0.0, cw = 0.0, lam[4] = {0.0, 0.0, 0.0, 0.0};
    int st = 0;
    if (m < a.N) {
      const double lnchi = a.lnchi_min + (double)m * a.L / (double)a.N;
      const double lnk = lnnu - lnchi;
      cw = (a.L / (double)a.N) * exp(-lnchi);
      if (lnk >= a.lnk_lo && lnk <= a.lnk_hi) {
        double w[4];
        const int s = stencil_ln(a.k, a.N_k, lnk, w);
        double p = 0.0, pd = 0.0;
        for (int r = 0; r < 4; ++r) {
          if (w[r] == 0.0) continue;
          p += w[r] * P[s + r];
          if (Pd) pd += w[r] * Pd[s + r];
        }
        pw = cw * p;
        pwd = cw * pd;
      }
      st = stencil_ln(a.knots, a.N_I, lnk, lam);
    }
    T.pw[mm] = pw;
    T.pwd[mm] = pwd;
    T.cw[mm] = cw;
    T.st[mm] = st;
    for (int r = 0; r < 4; ++r) T.lam[mm][r] = lam[r];
  }
}

// H[i][mm] = pi_i(l) nu^{t_i} sum_r lam_r D_{st+r}(m) B_{i,st+r}(m)
__device__ void tile_h(double* H, const Tile& T, const LimberArgs& a, double l, int m0) {
  const double nu = l + 0.5;
  for (int e = threadIdx.x; e < a.N_tr * MT; e += blockDim.x) {
    const int i = e / MT, mm = e - i * MT, m = m0 + mm;
    double h = 0.0;
    if (m < a.N) {
      const int kind = a.kind[i];
      const bool chi2 = kind == SWCL_LENSING || kind == SWCL_MAGNIFICATION;
      double db = 0.0;
      for (int r = 0; r < 4; ++r) {
        const double lr = T.lam[mm][r];
        if (lr == 0.0) continue;
        const int row = T.st[mm] + r;
        double v = a.D[(size_t)row * a.N + m];
        if (a.B) v *= a.B[((size_t)i * a.N_I + row) * a.N + m];
        db += lr * v;
      }
      h = ell_pre(kind, l) * (chi2 ? 1.0 / (nu * nu) : 1.0) * db;
    }
    H[e] = h;
  }
}

// Forward (and forward-mode) rows.  Grid (n_lim, n_w): walker w of W (and, for the JVP, tangent
// w: windows Wt + w, P' Pd + w N_k against the base walker 0).  Writes U[w][l_first + li].
template <bool JVP>
__global__ void __launch_bounds__(LT)
k_limber_rows(double* __restrict__ U, LimberArgs a, const double* __restrict__ W,
              const double* __restrict__ P, const double* __restrict__ Wt,
              const double* __restrict__ Pd) {
  extern __shared__ double lsm[];
  double* G = lsm;                          // [N_tr][MT]
  double* Gt = lsm + a.N_tr * MT;           // [N_tr][MT] (JVP)
  __shared__ Tile T;
  const int li = blockIdx.x, w = blockIdx.y;
  const double l = (double)a.ells[a.l_first + li];
  const double lnnu = log(l + 0.5);
  const int n = a.N_tr, npair = n * (n + 1) / 2;
  const double* Ww = JVP ? W : W + (size_t)w * n * a.N;
  const double* Pw = JVP ? P : P + (size_t)w * a.N_k;
  const double* Wtw = JVP && Wt ? Wt + (size_t)w * n * a.N : nullptr;
  const double* Pdw = JVP && Pd ? Pd + (size_t)w * a.N_k : nullptr;
  int pi[MAXR], pj[MAXR];
  double acc[MAXR];
#pragma unroll
  for (int r = 0; r < MAXR; ++r) {
    int p = threadIdx.x + r * LT, i = 0;
    acc[r] = 0.0;
    if (p < npair)
      while (p >= n - i) { p -= n - i; ++i; }
    pi[r] = i;
    pj[r] = i + p;
  }
  for (int m0 = 0; m0 < a.N; m0 += MT) {
    tile_weights(T, a, lnnu, m0, Pw, Pdw);
    __syncthreads();
    tile_h(G, T, a, l, m0);
    __syncthreads();
    for (int e = threadIdx.x; e < n * MT; e += blockDim.x) {
      const int i = e / MT, m = m0 + (e - i * MT);
      const double h = G[e];
      G[e] = m < a.N ? h * Ww[(size_t)i * a.N + m] : 0.0;
      if (JVP) Gt[e] = Wtw && m < a.N ? h * Wtw[(size_t)i * a.N + m] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < MAXR; ++r) {
      if (threadIdx.x + r * LT < npair) {
        const double* gi = G + pi[r] * MT;
        const double* gj = G + pj[r] * MT;
        double s = acc[r];
        if (JVP) {
          const double* ti = Gt + pi[r] * MT;
          const double* tj = Gt + pj[r] * MT;
          for (int mm = 0; mm < MT; ++mm)
            s = fma(T.pwd[mm], gi[mm] * gj[mm], fma(T.pw[mm], fma(ti[mm], gj[mm], gi[mm] * tj[mm]), s));
        } else {
          for (int mm = 0; mm < MT; ++mm) s = fma(T.pw[mm], gi[mm] * gj[mm], s);
        }
        acc[r] = s;
      }
    }
    __syncthreads();
  }
  double* out = U + ((size_t)w * a.N_ell + a.l_first + li) * n * n;
#pragma unroll
  for (int r = 0; r < MAXR; ++r) {
    if (threadIdx.x + r * LT < npair) {
      out[pi[r] * n + pj[r]] = acc[r];
      out[pj[r] * n + pi[r]] = acc[r];
    }
  }
}

// Reverse mode, first step.  Grid (chi tiles, n_walk).  For every Limber multipole:
// T = S A A^T (S the symmetrised cotangent), R_i = sum_j T_ij G_j, W_bar_i += 2 c Pt H_i R_i
// (accumulated in registers, added to Wb at the end when Wb is given) and
// Q[w][li][m] = c_m sum_i G_i R_i.
__global__ void __launch_bounds__(LT)
k_limber_vjp(double* __restrict__ Wb, double* __restrict__ Q, LimberArgs a,
             const double* __restrict__ W, const double* __restrict__ P,
             const double* __restrict__ Sfull, const double* __restrict__ amp) {
  extern __shared__ double lsm[];
  const int n = a.N_tr;
  double* H = lsm;                      // [N_tr][MT]
  double* G = H + n * MT;               // [N_tr][MT]
  double* GR = G + n * MT;              // [N_tr][MT]  G_i R_i
  double* Ts = GR + n * MT;             // [N_tr][N_tr]
  __shared__ Tile T;
  const int m0 = blockIdx.x * MT, w = blockIdx.y;
  const double* Ww = W + (size_t)w * n * a.N;
  const double* Aw = amp + (size_t)w * n;
  constexpr int PER = 64 * MT / LT;     // (i, mm) entries per thread
  double wb[PER];
#pragma unroll
  for (int t = 0; t < PER; ++t) wb[t] = 0.0;
  for (int li = 0; li < a.n_lim; ++li) {
    const double l = (double)a.ells[a.l_first + li];
    const double* S = Sfull + ((size_t)w * a.N_ell + a.l_first + li) * n * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e / n, j = e - i * n;
      Ts[e] = S[e] * Aw[i] * Aw[j];
    }
    tile_weights(T, a, log(l + 0.5), m0, P + (size_t)w * a.N_k, nullptr);
    __syncthreads();
    tile_h(H, T, a, l, m0);
    __syncthreads();
    for (int e = threadIdx.x; e < n * MT; e += blockDim.x) {
      const int i = e / MT, m = m0 + (e - i * MT);
      G[e] = m < a.N ? H[e] * Ww[(size_t)i * a.N + m] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      const int e = threadIdx.x + t * LT;
      if (e < n * MT) {
        const int i = e / MT, mm = e - i * MT;
        double r = 0.0;
        for (int j = 0; j < n; ++j) r = fma(Ts[i * n + j], G[j * MT + mm], r);
        wb[t] = fma(2.0 * T.pw[mm] * H[e], r, wb[t]);
        GR[e] = G[e] * r;
      }
    }
    __syncthreads();
    for (int mm = threadIdx.x; mm < MT; mm += blockDim.x) {
      const int m = m0 + mm;
      if (m >= a.N) continue;
      double q = 0.0;
      for (int i = 0; i < n; ++i) q += GR[i * MT + mm];
      Q[((size_t)w * a.n_lim + li) * a.N + m] = T.cw[mm] * q;
    }
    __syncthreads();
  }
  if (!Wb) return;
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int e = threadIdx.x + t * LT;
    if (e < n * MT) {
      const int i = e / MT, m = m0 + (e - i * MT);
      if (m < a.N) Wb[((size_t)w * n + i) * a.N + m] += wb[t];
    }
  }
}

// Reverse mode, second step: P_bar[w][q] += sum_l sum_m rho_q(k_lm) Q[w][l][m], where rho_q is q's
// weight in the stencil of k_lm.  The m whose stencil can hold q have k_lm within
// [k_{q-3}, k_{q+3}]; each is checked against its exact stencil.  One thread per (q, w).
__global__ void k_limber_pbar(double* __restrict__ Pb, const double* __restrict__ Q, LimberArgs a,
                              int n_walk) {
  const long total = (long)n_walk * a.N_k;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int q = (int)(e % a.N_k), w = (int)(e / a.N_k);
    const double klo = log(a.k[q >= 3 ? q - 3 : 0]);
    const double khi = log(a.k[q + 3 < a.N_k ? q + 3 : a.N_k - 1]);
    const double dm = (double)a.N / a.L;
    double s = 0.0;
    for (int li = 0; li < a.n_lim; ++li) {
      const double lnnu = log((double)a.ells[a.l_first + li] + 0.5);
      // ln k_m = lnnu - lnchi_min - m L/N, decreasing in m
      int mlo = (int)floor((lnnu - a.lnchi_min - khi) * dm) - 1;
      int mhi = (int)ceil((lnnu - a.lnchi_min - klo) * dm) + 1;
      mlo = mlo < 0 ? 0 : mlo;
      mhi = mhi > a.N - 1 ? a.N - 1 : mhi;
      const double* Ql = Q + ((size_t)w * a.n_lim + li) * a.N;
      for (int m = mlo; m <= mhi; ++m) {
        const double lnk = lnnu - (a.lnchi_min + (double)m * a.L / (double)a.N);
        if (!(lnk >= a.lnk_lo && lnk <= a.lnk_hi)) continue;
        double wts[4];
        const int st = stencil_ln(a.k, a.N_k, lnk, wts);
        const int r = q - st;
        if (r >= 0 && r < 4) s = fma(wts[r], Ql[m], s);
      }
    }
    Pb[e] += s;
  }
}

}  // namespace

cudaError_t launch_limber_rows(double* U, const LimberArgs& a, const double* W, const double* P,
                               int n_walk, cudaStream_t s) {
  if (a.N_tr > 64 || a.n_lim < 1) return cudaErrorInvalidValue;
  const size_t smem = sizeof(double) * a.N_tr * MT;
  k_limber_rows<false><<<dim3(a.n_lim, n_walk), LT, smem, s>>>(U, a, W, P, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_limber_jvp(double* dU, const LimberArgs& a, const double* W, const double* P,
                              const double* Wt, const double* Pd, int n_dir, cudaStream_t s) {
  if (a.N_tr > 64 || a.n_lim < 1) return cudaErrorInvalidValue;
  const size_t smem = 2 * sizeof(double) * a.N_tr * MT;
  k_limber_rows<true><<<dim3(a.n_lim, n_dir), LT, smem, s>>>(dU, a, W, P, Wt, Pd);
  return cudaGetLastError();
}

cudaError_t launch_limber_vjp(double* Wb, double* Pb, double* Q, const LimberArgs& a,
                              const double* W, const double* P, const double* Sfull,
                              const double* amp, int n_walk, cudaStream_t s_main,
                              cudaStream_t s_pbar, cudaEvent_t q_ready) {
  if (a.N_tr > 64 || a.n_lim < 1) return cudaErrorInvalidValue;
  const size_t smem = sizeof(double) * (3 * a.N_tr * MT + a.N_tr * a.N_tr);
  cudaError_t e = cudaFuncSetAttribute(k_limber_vjp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int tiles = (a.N + MT - 1) / MT;
  k_limber_vjp<<<dim3(tiles, n_walk), LT, smem, s_main>>>(Wb, Q, a, W, P, Sfull, amp);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (s_pbar != s_main) {
    if ((e = cudaEventRecord(q_ready, s_main)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s_pbar, q_ready, 0)) != cudaSuccess) return e;
  }
  const long total = (long)n_walk * a.N_k;
  const int blocks = (int)std::min<long>((total + 127) / 128, 152L * 4);
  k_limber_pbar<<<blocks, 128, 0, s_pbar>>>(Pb, Q, a, n_walk);
  return cudaGetLastError();
}

}  // namespace swcl
