// The Limber branch (Eq. 2.19): multipoles at or above a switch take
//   U_ij(l) = sum_m c_m Pt(k_m) G_i(l, m) G_j(l, m),   k_m = nu / chi_m,  nu = l + 1/2,
//   c_m = (L/N) / chi_m,   G_i = W_i(chi_m) H_i,   H_i = pi_i(l) nu^{t_i} sum_a Lam_a(k_m) D_a(chi_m) B_ia(chi_m)
// on the FFTLog chi grid (rectangle rule in ln chi), with Pt the 4-point Lagrange interpolant in
// ln k of P on the k grid (zero outside it) and Lam the knot weights of the same rule.  Every kind
// that has a Limber form has s = t (density 0, lensing and magnification -2), so
// k^t chi^s = nu^t.  All arithmetic is FP64.
//
// The stencils depend on the grids only: a table built once per grid (k_limber_table) holds, for
// every Limber multipole and chi point, the first k point of the P stencil (-1 outside the k
// range) with its weights times c_m, and the first knot with the knot weights.  Then:
//  - forward rows: one CTA per (multipole, 256-point chi chunk, walker), chi tiles of 32 staged
//    in shared memory, one thread per tracer pair (up to 9 pairs); partial pair sums per chunk are
//    added in a fixed order by the k-quadrature's reduction;
//  - forward-mode rows: the same kernel with the tangent windows and P';
//  - reverse mode: one CTA per (chi tile, 8 multipoles, walker) forms R_i = sum_j T_ij G_j with
//    T = S A A^T, the partial W_bar_i = 2 c Pt H_i R_i of its multipoles and Q = sum_i G_i R_i;
//    the W_bar partials are added in order into W_bar; P_bar_q gathers sum rho_q c Q over the
//    (l, m) whose stencil holds q, 32 multipoles per CTA, partials added in order.
#include <algorithm>

#include "swcl_internal.h"

namespace swcl {
namespace {

constexpr int LT = 256;   // threads
constexpr int MT = 32;    // chi points per staged tile
constexpr int MTS = MT + 1;  // shared row stride of the per-tracer tiles (lanes of different
                             // tracers at one chi point fall in different banks)
constexpr int MC = 256;   // chi points per CTA of the forward rows
constexpr int LCH = 8;    // multipoles per CTA of the reverse mode
constexpr int PCH = 32;   // multipoles per CTA of the P_bar gather
constexpr int MAXR = 9;   // tracer pairs per thread (64 tracers)

// Stencil of R5 at ln-value x on an increasing grid given by its logarithms: returns the first row
// and writes the s = min(4, n) Lagrange weights (unused entries 0).
__device__ int stencil_ln(const double* lng, int n, double x, double w[4]) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (lng[mid] <= x) lo = mid + 1; else hi = mid;
  }
  const int s = n < 4 ? n : 4;
  int a = lo - 1;
  a = a < 0 ? 0 : (a > n - 1 ? n - 1 : a);
  int start = a - 1;
  if (start > n - s) start = n - s;
  if (start < 0) start = 0;
  for (int r = 0; r < 4; ++r) {
    double v = 0.0;
    if (r < s) {
      v = 1.0;
      for (int t = 0; t < s; ++t)
        if (t != r) v *= (x - lng[start + t]) / (lng[start + r] - lng[start + t]);
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

__global__ void k_limber_lngrid(LimberTable t, LimberArgs a) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < a.N_k) t.lnk[e] = log(a.k[e]);
  else if (e < a.N_k + a.N_I) t.lnknots[e - a.N_k] = log(a.knots[e - a.N_k]);
  else if (e < a.N_k + a.N_I + a.n_lim)
    t.lnnu[e - a.N_k - a.N_I] = log((double)a.ells[a.l_first + e - a.N_k - a.N_I] + 0.5);
}

// one thread per (Limber multipole li, chi point m)
__global__ void k_limber_table(LimberTable t, LimberArgs a) {
  const long total = (long)a.n_lim * a.N;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int li = (int)(e / a.N), m = (int)(e - (long)li * a.N);
    const double lnchi = a.lnchi_min + (double)m * a.L / (double)a.N;
    const double lnk = t.lnnu[li] - lnchi;
    const double c = (a.L / (double)a.N) * exp(-lnchi);
    double w[4] = {0.0, 0.0, 0.0, 0.0};
    int pst = -1;
    if (lnk >= a.lnk_lo && lnk <= a.lnk_hi) pst = stencil_ln(t.lnk, a.N_k, lnk, w);
    t.pst[e] = pst;
    for (int r = 0; r < 4; ++r) t.pw[e * 4 + r] = c * w[r];
    double lam[4];
    t.kst[e] = stencil_ln(t.lnknots, a.N_I, lnk, lam);
    for (int r = 0; r < 4; ++r) t.kw[e * 4 + r] = lam[r];
  }
}

// Per chi tile of one multipole: pw[mm] = c_m Pt(k_m) (and pwd with the tangent P'), the knot
// stencil (kst, kw).
struct Tile {
  double pw[MT], pwd[MT], kw[MT][4];
  int kst[MT];
};

__device__ void tile_weights(Tile& T, const LimberArgs& a, const LimberTable& t, int li, int m0,
                             const double* P, const double* Pd) {
  for (int mm = threadIdx.x; mm < MT; mm += blockDim.x) {
    const int m = m0 + mm;
    double p = 0.0, pd = 0.0;
    int kst = 0;
    double kw[4] = {0.0, 0.0, 0.0, 0.0};
    if (m < a.N) {
      const size_t e = (size_t)li * a.N + m;
      const int pst = t.pst[e];
      if (pst >= 0) {
        for (int r = 0; r < 4; ++r) {
          const double wr = t.pw[e * 4 + r];
          p = fma(wr, P[pst + r], p);
          if (Pd) pd = fma(wr, Pd[pst + r], pd);
        }
      }
      kst = t.kst[e];
      for (int r = 0; r < 4; ++r) kw[r] = t.kw[e * 4 + r];
    }
    T.pw[mm] = p;
    T.pwd[mm] = pd;
    T.kst[mm] = kst;
    for (int r = 0; r < 4; ++r) T.kw[mm][r] = kw[r];
  }
}

// H[i][mm] = pi_i(l) nu^{t_i} sum_r kw_r D_{kst+r}(m) B_{i,kst+r}(m)
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
        const double lr = T.kw[mm][r];
        if (lr == 0.0) continue;
        const int row = T.kst[mm] + r;
        double v = a.D[(size_t)row * a.N + m];
        if (a.B) v *= a.B[((size_t)i * a.N_I + row) * a.N + m];
        db = fma(lr, v, db);
      }
      h = ell_pre(kind, l) * (chi2 ? 1.0 / (nu * nu) : 1.0) * db;
    }
    H[i * MTS + mm] = h;
  }
}

// Forward (and forward-mode) partial pair sums over one chi chunk.  Grid (n_lim, n_mc, n_w):
// walker w of W (and, for the JVP, tangent w: windows Wt + w, P' Pd + w N_k against the base
// walker 0).  part[w][li][mc][pair].
template <bool JVP>
__global__ void __launch_bounds__(LT)
k_limber_part(double* __restrict__ part, LimberArgs a, LimberTable t, const double* __restrict__ W,
              const double* __restrict__ P, const double* __restrict__ Wt,
              const double* __restrict__ Pd, int n_mc) {
  extern __shared__ double lsm[];
  double* G = lsm;                          // [N_tr][MTS]
  double* Gt = lsm + a.N_tr * MTS;          // [N_tr][MTS] (JVP)
  __shared__ Tile T;
  const int li = blockIdx.x, mc = blockIdx.y, w = blockIdx.z;
  const double l = (double)a.ells[a.l_first + li];
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
  const int m_end = min((mc + 1) * MC, a.N);
  for (int m0 = mc * MC; m0 < m_end; m0 += MT) {
    tile_weights(T, a, t, li, m0, Pw, Pdw);
    __syncthreads();
    tile_h(G, T, a, l, m0);
    __syncthreads();
    for (int e = threadIdx.x; e < n * MT; e += blockDim.x) {
      const int i = e / MT, mm = e - i * MT, m = m0 + mm, x = i * MTS + mm;
      const double h = G[x];
      G[x] = m < a.N ? h * Ww[(size_t)i * a.N + m] : 0.0;
      if (JVP) Gt[x] = Wtw && m < a.N ? h * Wtw[(size_t)i * a.N + m] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < MAXR; ++r) {
      if (threadIdx.x + r * LT < npair) {
        const double* gi = G + pi[r] * MTS;
        const double* gj = G + pj[r] * MTS;
        double s = acc[r];
        if (JVP) {
          const double* ti = Gt + pi[r] * MTS;
          const double* tj = Gt + pj[r] * MTS;
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
  double* out = part + (((size_t)w * a.n_lim + li) * n_mc + mc) * npair;
#pragma unroll
  for (int r = 0; r < MAXR; ++r)
    if (threadIdx.x + r * LT < npair) out[threadIdx.x + r * LT] = acc[r];
}

// Reverse mode, first step.  Grid (chi tiles, multipole chunks of LCH, n_walk).  For each
// multipole of the chunk: T = S A A^T (S the symmetrised cotangent), R_i = sum_j T_ij G_j; the
// chunk's W_bar partial 2 sum_l c Pt H_i R_i goes to Wpart[w][lc][i][m] (when has_wb) and
// Q[w][li][m] = sum_i G_i R_i.
__global__ void __launch_bounds__(LT)
k_limber_vjp(double* __restrict__ Wpart, double* __restrict__ Q, LimberArgs a, LimberTable t,
             const double* __restrict__ W, const double* __restrict__ P,
             const double* __restrict__ Sfull, const double* __restrict__ amp, int n_lc, int has_wb) {
  extern __shared__ double lsm[];
  const int n = a.N_tr;
  double* H = lsm;                      // [N_tr][MTS]
  double* G = H + n * MTS;              // [N_tr][MTS]
  double* GR = G + n * MTS;             // [N_tr][MTS]  G_i R_i
  double* Ts = GR + n * MTS;            // [N_tr][N_tr]
  __shared__ Tile T;
  const int m0 = blockIdx.x * MT, lc = blockIdx.y, w = blockIdx.z;
  const double* Ww = W + (size_t)w * n * a.N;
  const double* Aw = amp + (size_t)w * n;
  constexpr int PER = 64 * MT / LT;     // (i, mm) entries per thread
  double wb[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) wb[u] = 0.0;
  const int li_end = min((lc + 1) * LCH, a.n_lim);
  for (int li = lc * LCH; li < li_end; ++li) {
    const double l = (double)a.ells[a.l_first + li];
    const double* S = Sfull + ((size_t)w * a.N_ell + a.l_first + li) * n * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e / n, j = e - i * n;
      Ts[e] = S[e] * Aw[i] * Aw[j];
    }
    tile_weights(T, a, t, li, m0, P + (size_t)w * a.N_k, nullptr);
    __syncthreads();
    tile_h(H, T, a, l, m0);
    __syncthreads();
    for (int e = threadIdx.x; e < n * MT; e += blockDim.x) {
      const int i = e / MT, mm = e - i * MT, m = m0 + mm, x = i * MTS + mm;
      G[x] = m < a.N ? H[x] * Ww[(size_t)i * a.N + m] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = threadIdx.x + u * LT;
      if (e < n * MT) {
        const int i = e / MT, mm = e - i * MT, x = i * MTS + mm;
        double r = 0.0;
        for (int j = 0; j < n; ++j) r = fma(Ts[i * n + j], G[j * MTS + mm], r);
        wb[u] = fma(2.0 * T.pw[mm] * H[x], r, wb[u]);
        GR[x] = G[x] * r;
      }
    }
    __syncthreads();
    for (int mm = threadIdx.x; mm < MT; mm += blockDim.x) {
      const int m = m0 + mm;
      if (m >= a.N) continue;
      double q = 0.0;
      for (int i = 0; i < n; ++i) q += GR[i * MTS + mm];
      Q[((size_t)w * a.n_lim + li) * a.N + m] = q;
    }
    __syncthreads();
  }
  if (!has_wb) return;
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int e = threadIdx.x + u * LT;
    if (e < n * MT) {
      const int i = e / MT, m = m0 + (e - i * MT);
      if (m < a.N) Wpart[(((size_t)w * n_lc + lc) * n + i) * a.N + m] = wb[u];
    }
  }
}

// Wb[w][i][m] += sum_lc Wpart[w][lc][i][m] in order
__global__ void k_limber_wreduce(double* __restrict__ Wb, const double* __restrict__ Wpart,
                                 int n_walk, int N_tr, int N, int n_lc, int* __restrict__ status) {
  const long per = (long)N_tr * N, total = (long)n_walk * per;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long w = e / per, r = e - w * per;
    const double* src = Wpart + (size_t)w * n_lc * per + r;
    double s = 0.0;
    for (int c = 0; c < n_lc; ++c) s += src[(size_t)c * per];
    const double v = Wb[e] + s;
    flag_nonfinite(status, v);
    Wb[e] = v;
  }
}

// P_bar gather.  Grid (k blocks, multipole chunks of PCH, n_walk); thread q:
// Ppart[w][pc][q] = sum over the chunk's l and the m whose P stencil holds q of
// (c rho_q)(l, m) Q[w][l][m].  Those m have ln k_lm in [ln k_{q-3}, ln k_{q+3}]; each is checked
// against the table.
__global__ void k_limber_pbar(double* __restrict__ Ppart, const double* __restrict__ Q,
                              LimberArgs a, LimberTable t, int n_pc) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x, pc = blockIdx.y, w = blockIdx.z;
  if (q >= a.N_k) return;
  const double klo = t.lnk[q >= 3 ? q - 3 : 0];
  const double khi = t.lnk[q + 3 < a.N_k ? q + 3 : a.N_k - 1];
  const double dm = (double)a.N / a.L;
  double s = 0.0;
  const int li_end = min((pc + 1) * PCH, a.n_lim);
  for (int li = pc * PCH; li < li_end; ++li) {
    const double x0 = t.lnnu[li] - a.lnchi_min;   // ln k_m = x0 - m L / N
    int mlo = (int)floor((x0 - khi) * dm) - 1;
    int mhi = (int)ceil((x0 - klo) * dm) + 1;
    mlo = mlo < 0 ? 0 : mlo;
    mhi = mhi > a.N - 1 ? a.N - 1 : mhi;
    const double* Ql = Q + ((size_t)w * a.n_lim + li) * a.N;
    for (int m = mlo; m <= mhi; ++m) {
      const size_t e = (size_t)li * a.N + m;
      const int st = t.pst[e];
      const int r = q - st;
      if (st >= 0 && r >= 0 && r < 4) s = fma(t.pw[e * 4 + r], Ql[m], s);
    }
  }
  Ppart[((size_t)w * n_pc + pc) * a.N_k + q] = s;
}

// Pb[w][q] += sum_pc Ppart[w][pc][q] in order
__global__ void k_limber_preduce(double* __restrict__ Pb, const double* __restrict__ Ppart,
                                 int n_walk, int N_k, int n_pc, int* __restrict__ status) {
  const long total = (long)n_walk * N_k;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long w = e / N_k, q = e - w * N_k;
    double s = 0.0;
    for (int c = 0; c < n_pc; ++c) s += Ppart[((size_t)w * n_pc + c) * N_k + q];
    const double v = Pb[e] + s;
    flag_nonfinite(status, v);
    Pb[e] = v;
  }
}

int n_mc(const LimberArgs& a) { return (a.N + MC - 1) / MC; }
int n_lc(const LimberArgs& a) { return (a.n_lim + LCH - 1) / LCH; }
int n_pc(const LimberArgs& a) { return (a.n_lim + PCH - 1) / PCH; }
unsigned grid_of(long total) { return (unsigned)std::min<long>((total + 255) / 256, 152L * 8); }

}  // namespace

size_t limber_table_bytes(const LimberArgs& a) {
  const size_t nm = (size_t)a.n_lim * a.N;
  return nm * (2 * sizeof(int) + 8 * sizeof(double)) + sizeof(double) * (a.N_k + a.N_I + a.n_lim) + 64;
}

LimberTable limber_table_view(void* base, const LimberArgs& a) {
  const size_t nm = (size_t)a.n_lim * a.N;
  LimberTable t;
  double* d = static_cast<double*>(base);
  t.pw = d;
  t.kw = t.pw + nm * 4;
  t.lnk = t.kw + nm * 4;
  t.lnknots = t.lnk + a.N_k;
  t.lnnu = t.lnknots + a.N_I;
  t.pst = reinterpret_cast<int*>(t.lnnu + a.n_lim);
  t.kst = t.pst + nm;
  return t;
}

size_t limber_scratch_bytes(const LimberArgs& a, int n_rows) {
  const size_t npair = (size_t)a.N_tr * (a.N_tr + 1) / 2;
  const size_t part = (size_t)n_rows * a.n_lim * n_mc(a) * npair;
  const size_t q = (size_t)n_rows * a.n_lim * a.N;
  const size_t wp = (size_t)n_rows * n_lc(a) * a.N_tr * a.N;
  const size_t pp = (size_t)n_rows * n_pc(a) * a.N_k;
  return sizeof(double) * (part + q + wp + pp);
}

cudaError_t launch_limber_table(const LimberTable& t, const LimberArgs& a, cudaStream_t s) {
  const int n0 = a.N_k + a.N_I + a.n_lim;
  k_limber_lngrid<<<(n0 + 255) / 256, 256, 0, s>>>(t, a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_limber_table<<<grid_of((long)a.n_lim * a.N), 256, 0, s>>>(t, a);
  return cudaGetLastError();
}

cudaError_t launch_limber_rows(double* U, double* scratch, const LimberArgs& a, const LimberTable& t,
                               const double* W, const double* P, int n_walk, cudaStream_t s) {
  if (a.N_tr > 64 || a.n_lim < 1) return cudaErrorInvalidValue;
  const size_t smem = sizeof(double) * a.N_tr * MTS;
  k_limber_part<false><<<dim3(a.n_lim, n_mc(a), n_walk), LT, smem, s>>>(scratch, a, t, W, P, nullptr,
                                                                         nullptr, n_mc(a));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_pair_reduce(U, scratch, n_walk, a.N_tr, a.N_ell, a.l_first, a.n_lim, n_mc(a), s);
}

cudaError_t launch_limber_jvp(double* dU, double* scratch, const LimberArgs& a, const LimberTable& t,
                              const double* W, const double* P, const double* Wt, const double* Pd,
                              int n_dir, cudaStream_t s) {
  if (a.N_tr > 64 || a.n_lim < 1) return cudaErrorInvalidValue;
  const size_t smem = 2 * sizeof(double) * a.N_tr * MTS;
  k_limber_part<true><<<dim3(a.n_lim, n_mc(a), n_dir), LT, smem, s>>>(scratch, a, t, W, P, Wt, Pd,
                                                                       n_mc(a));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_pair_reduce(dU, scratch, n_dir, a.N_tr, a.N_ell, a.l_first, a.n_lim, n_mc(a), s);
}

cudaError_t launch_limber_vjp(double* Wb, double* Pb, double* scratch, const LimberArgs& a,
                              const LimberTable& t, const double* W, const double* P,
                              const double* Sfull, const double* amp, int n_walk,
                              cudaStream_t s_main, cudaStream_t s_pbar, cudaEvent_t q_ready,
                              int* status) {
  if (a.N_tr > 64 || a.n_lim < 1) return cudaErrorInvalidValue;
  const size_t npair = (size_t)a.N_tr * (a.N_tr + 1) / 2;
  double* Q = scratch + (size_t)n_walk * a.n_lim * n_mc(a) * npair;   // after the forward partials
  double* Wpart = Q + (size_t)n_walk * a.n_lim * a.N;
  double* Ppart = Wpart + (size_t)n_walk * n_lc(a) * a.N_tr * a.N;
  const size_t smem = sizeof(double) * (3 * a.N_tr * MTS + a.N_tr * a.N_tr);
  cudaError_t e = cudaFuncSetAttribute(k_limber_vjp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int tiles = (a.N + MT - 1) / MT;
  k_limber_vjp<<<dim3(tiles, n_lc(a), n_walk), LT, smem, s_main>>>(Wpart, Q, a, t, W, P, Sfull, amp,
                                                                   n_lc(a), Wb ? 1 : 0);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (Wb) {
    k_limber_wreduce<<<grid_of((long)n_walk * a.N_tr * a.N), 256, 0, s_main>>>(Wb, Wpart, n_walk,
                                                                              a.N_tr, a.N, n_lc(a),
                                                                              status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (s_pbar != s_main) {
    if ((e = cudaEventRecord(q_ready, s_main)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s_pbar, q_ready, 0)) != cudaSuccess) return e;
  }
  k_limber_pbar<<<dim3((a.N_k + 127) / 128, n_pc(a), n_walk), 128, 0, s_pbar>>>(Ppart, Q, a, t, n_pc(a));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_limber_preduce<<<grid_of((long)n_walk * a.N_k), 256, 0, s_pbar>>>(Pb, Ppart, n_walk, a.N_k, n_pc(a),
                                                                      status);
  return cudaGetLastError();
}

}  // namespace swcl
