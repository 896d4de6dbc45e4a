// a4: the k-quadrature of Eq. 2.1, C_l^{ij} = A_i A_j sum_q u_q Delta_i(l,q) Delta_j(l,q),
// u_q = wk2[q] P(k_q), and the reductions of its reverse mode (a5):
//   Pbar_q   = wk2[q] sum_l sum_i A_i Delta_i T_i,   T_i = sum_j S_ij A_j Delta_j,
//   Dbar_i   = 2 A_i u_q T_i,
//   Abar_i   = 2 sum_l sum_j S_ij A_j U_ij            (U = C at unit amplitudes),
// with S = (Cbar + Cbar^T)/2 (zero for multipoles outside a walker's list).
//
// The unit-amplitude spectra U of the FP64 form are formed in two passes: partial sums of each
// unordered pair (i <= j) over chunks of 256 k points (one CTA per multipole and chunk), then the
// chunks added in a fixed order and written to both (i,j) and (j,i), so C is symmetric bit for
// bit and the same from run to run.  Delta in FP32 (mixed paths) goes through k_quad_blocks
// below: FP32 products, compensated FP32 sums (TwoSum; the rounding of each addition carried in
// a second float), FP64 above them, in one pass when a multipole's k range fits one CTA.
#include <algorithm>

#include "swcl_internal.h"

namespace swcl {
namespace {

constexpr int QT = 256;    // threads
constexpr int KC = 256;    // k points per CTA (one partial sum per pair and chunk)
constexpr int KS = KC + 1; // shared row stride: lanes reading rows j at the same k point fall in
                           // different banks
static_assert(QT == KC, "k_quad_part stages one k point per thread");

// Partial pair sums over one chunk of KC k points: part[w][l - l_lo][kc][p] for unordered pairs
// p = (i <= j).  Grid (multipole, k chunk, walker).  Thread t handles pair p = t % npair for the
// k points t / npair, t / npair + G, ... of the chunk (G = QT / npair groups); groups are combined
// in shared memory in a fixed order.
template <typename T>
__global__ void __launch_bounds__(QT)
k_quad_part(double* __restrict__ part, const T* __restrict__ delta, const double* __restrict__ P,
            const double* __restrict__ wk2, int N_tr, int N_k, int n_l, int n_kc,
            const int* __restrict__ listed) {
  extern __shared__ double qsm[];
  T* Ds = reinterpret_cast<T*>(qsm);              // [N_tr][KS]
  __shared__ double us[KC];
  __shared__ float usf[KC];
  __shared__ double red[QT];
  const int ll = blockIdx.x, kc = blockIdx.y, w = blockIdx.z;
  const int q0 = kc * KC;
  const int npair = N_tr * (N_tr + 1) / 2;
  if (listed && listed[w * n_l + ll] < 0) {
    // a multipole the walker does not list: zero partials (its Delta rows are not read)
    double* out = part + (((size_t)w * n_l + ll) * n_kc + kc) * npair;
    for (int p = threadIdx.x; p < npair; p += QT) out[p] = 0.0;
    return;
  }
  const T* dl = delta + ((size_t)w * n_l + ll) * N_tr * N_k;
  {
    // one k point per thread (QT == KC); the rows' loads are unrolled so that several are in
    // flight at once
    const int qq = threadIdx.x, q = q0 + qq;
#pragma unroll 8
    for (int t = 0; t < N_tr; ++t) Ds[t * KS + qq] = q < N_k ? dl[(size_t)t * N_k + q] : T(0);
  }
  for (int e = threadIdx.x; e < KC; e += QT) {
    const int q = q0 + e;
    us[e] = q < N_k ? wk2[q] * P[(size_t)w * N_k + q] : 0.0;
    usf[e] = (float)us[e];
  }
  __syncthreads();
  const int ngroups = max(1, QT / npair);
  double* out = part + (((size_t)w * n_l + ll) * n_kc + kc) * npair;
  for (int p0 = 0; p0 < npair; p0 += QT) {
    const int p = p0 + (ngroups > 1 ? threadIdx.x % npair : threadIdx.x);
    const int group = ngroups > 1 ? threadIdx.x / npair : 0;
    const bool active = p < npair && group < ngroups;
    double acc = 0.0;
    if (active) {
      int r = p, i = 0;                           // unordered pair index -> (i <= j)
      while (r >= N_tr - i) { r -= N_tr - i; ++i; }
      const int j = i + r;
      const T* di = Ds + i * KS;
      const T* dj = Ds + j * KS;
      if (sizeof(T) == 4) {
        // FP32 products in one compensated FP32 sum (the rounding error of each addition,
        // from TwoSum, carried in a second float), widened to FP64 once: GB300 runs FP64 at a
        // small fraction of its FP32 rate
        float sum = 0.0f, comp = 0.0f;
        for (int c0 = group * 32; c0 < KC; c0 += ngroups * 32) {
#pragma unroll 8
          for (int qq = c0; qq < c0 + 32; ++qq) {
            const float t = ((float)di[qq] * usf[qq]) * (float)dj[qq];
            const float sn = sum + t;
            const float bp = sn - sum;
            comp += (sum - (sn - bp)) + (t - bp);
            sum = sn;
          }
        }
        acc = (double)sum + (double)comp;
      } else {
        for (int qq = group; qq < KC; qq += ngroups)
          acc = fma((double)di[qq] * us[qq], (double)dj[qq], acc);
      }
    }
    if (ngroups > 1) {
      red[threadIdx.x] = acc;
      __syncthreads();
      if (active && group == 0) {
        double s2 = acc;
        for (int g = 1; g < ngroups; ++g) s2 += red[g * npair + threadIdx.x];
        out[p] = s2;
      }
      __syncthreads();
    } else if (active) {
      out[p] = acc;
    }
  }
}

// U[w][l][i][j] = U[w][l][j][i] = sum over the k chunks of the pair's partial sums (in order)
__global__ void k_quad_reduce(double* __restrict__ U, const double* __restrict__ part, int N_tr,
                              int N_ell, int l_lo, int n_l, int n_kc, int n_walk) {
  const int npair = N_tr * (N_tr + 1) / 2;
  const long total = (long)n_walk * n_l * npair;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int p = (int)(e % npair);
    const long wl = e / npair;                       // w * n_l + ll
    const int ll = (int)(wl % n_l), w = (int)(wl / n_l);
    const double* src = part + (size_t)wl * n_kc * npair + p;
    double s = 0.0;
    for (int kc = 0; kc < n_kc; ++kc) s += src[(size_t)kc * npair];
    int r = p, i = 0;
    while (r >= N_tr - i) { r -= N_tr - i; ++i; }
    const int j = i + r;
    double* u = U + ((size_t)w * N_ell + l_lo + ll) * N_tr * N_tr;
    u[i * N_tr + j] = s;
    u[j * N_tr + i] = s;
  }
}

// ---- FP32 form: register blocks of 4 x 4 tracer pairs ----
//
// One CTA per (multipole, k chunk, walker) copies the chunk's Delta rows into shared memory as
// they lie in global memory ([tracer][k], rows padded to a multiple of four tracers with zeros)
// with asynchronous 16-byte copies, all in flight at once, and u = wk2 P in FP32.  Warp b takes
// the block of pairs (4 ib .. 4 ib + 3) x (4 jb .. 4 jb + 3), ib <= jb; lane l takes the k points
// l, l + 32, ... (consecutive lanes read consecutive words: no bank conflicts).  Per k point a lane
// forms a_i = Delta_i u (four products, rounded as in the two-pass form) and sixteen FMAs a_i
// Delta_j into block sums; every QB_GROUP points the block sums are added into compensated
// (TwoSum) accumulators.  The 32 lanes are then combined by a butterfly that halves the pairs
// each lane holds at every step (each combination a TwoSum), so lane pair (2p, 2p + 1) ends with
// pair p of the block.  The order of every addition is fixed: the result is the same from run to
// run.  With one chunk the sum, widened to FP64, is U itself (both triangles); with several, the
// per-chunk sums go through the chunk reduction of the other form.
constexpr int QB_MAX_WARPS = 20;
constexpr int QB_GROUP = 4;                  // k points per lane between compensated additions
constexpr int QB_SMEM = 100 * 1024;          // staged rows per CTA at most (2 CTAs per SM)

__device__ __forceinline__ void qb_two_sum(float& s, float& c, float b) {
  const float sn = s + b;
  const float bp = sn - s;
  c += (s - (sn - bp)) + (b - bp);
  s = sn;
}

// (s, c) += (rs, rc): the sums' rounding error from TwoSum, the compensations added
__device__ __forceinline__ void qb_combine(float& s, float& c, float rs, float rc) {
  const float sn = s + rs;
  const float bp = sn - s;
  const float e = (s - (sn - bp)) + (rs - bp);
  c = (c + rc) + e;
  s = sn;
}

// one butterfly step: lanes with (lane & OFF) keep the upper half of their H pairs
template <int H, int OFF>
__device__ __forceinline__ void qb_scatter_step(float* s, float* c, int lane) {
  const bool up = lane & OFF;
#pragma unroll
  for (int p = 0; p < H; ++p) {
    const float keep_s = up ? s[p + H] : s[p], keep_c = up ? c[p + H] : c[p];
    const float ss = up ? s[p] : s[p + H], sc = up ? c[p] : c[p + H];
    const float rs = __shfl_xor_sync(0xffffffffu, ss, OFF);
    const float rc = __shfl_xor_sync(0xffffffffu, sc, OFF);
    s[p] = keep_s;
    c[p] = keep_c;
    qb_combine(s[p], c[p], rs, rc);
  }
}

__global__ void __launch_bounds__(QB_MAX_WARPS * 32, 1)
k_quad_blocks(double* __restrict__ U, double* __restrict__ part, const float* __restrict__ delta,
              const double* __restrict__ P, const double* __restrict__ wk2, int N_tr, int N_k,
              int N_ell, int l_lo, int n_l, int kcap, int n_kc, int ks, bool vec4,
              const int* __restrict__ listed) {
  extern __shared__ float4 qb_smv[];
  float* qb_sm = reinterpret_cast<float*>(qb_smv);
  const int ll = blockIdx.x, kc = blockIdx.y, w = blockIdx.z;
  const int n_ib = (N_tr + 3) / 4, nb = n_ib * (n_ib + 1) / 2;
  const int npair = N_tr * (N_tr + 1) / 2;
  const int q0 = kc * kcap;
  const int nk = min(kcap, N_k - q0);
  const int nk32 = (nk + 31) & ~31;
  double* Uw = U + ((size_t)w * N_ell + l_lo + ll) * N_tr * N_tr;
  double* pw = part + (((size_t)w * n_l + ll) * n_kc + kc) * npair;
  if (listed && listed[w * n_l + ll] < 0) {
    // a multipole the walker does not list: zero sums (its Delta rows are not read)
    if (n_kc == 1)
      for (int e = threadIdx.x; e < N_tr * N_tr; e += blockDim.x) Uw[e] = 0.0;
    else
      for (int e = threadIdx.x; e < npair; e += blockDim.x) pw[e] = 0.0;
    return;
  }
  const int rows = 4 * n_ib;
  float* Ds = qb_sm;                                            // [rows][kcap]
  float* us = qb_sm + (size_t)rows * kcap;                      // [kcap]
  const float* dl = delta + ((size_t)w * n_l + ll) * N_tr * N_k + q0;
  if (vec4) {
    // rows start on 16-byte boundaries (N_k and q0 multiples of 4): 16-byte copies, the part of
    // a group past the chunk's end (and every padding row) filled with zeros by the copy itself
    const int ng = nk32 >> 2;
    for (int e = threadIdx.x; e < rows * ng; e += blockDim.x) {
      const int t = e / ng, gq = e - t * ng;
      const int left = nk - 4 * gq;
      const int bytes = t < N_tr ? (left >= 4 ? 16 : left > 0 ? 4 * left : 0) : 0;
      const float* src = bytes ? dl + (size_t)t * N_k + 4 * gq : dl;
      const unsigned dst = (unsigned)__cvta_generic_to_shared(Ds + (size_t)t * kcap + 4 * gq);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
                   "r"(bytes) : "memory");
    }
  } else {
    for (int e = threadIdx.x; e < rows * nk32; e += blockDim.x) {
      const int t = e / nk32, kk = e - t * nk32;
      const int bytes = t < N_tr && kk < nk ? 4 : 0;
      const float* src = bytes ? dl + (size_t)t * N_k + kk : dl;
      const unsigned dst = (unsigned)__cvta_generic_to_shared(Ds + (size_t)t * kcap + kk);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src),
                   "r"(bytes) : "memory");
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (int kk = threadIdx.x; kk < nk32; kk += blockDim.x)
    us[kk] = kk < nk ? (float)(wk2[q0 + kk] * P[(size_t)w * N_k + q0 + kk]) : 0.0f;
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  // warp wi: k part h = wi / wb of ks, blocks bw, bw + wb, ... (bw = wi % wb); part h takes the
  // 32-point groups [h n32 / ks, (h + 1) n32 / ks) of the chunk
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int wb = (blockDim.x >> 5) / ks, h = wi / wb, bw = wi - h * wb;
  const int n32 = nk32 >> 5;
  const int k_lo = 32 * (h * n32 / ks), k_hi = 32 * ((h + 1) * n32 / ks);
  float2* red = reinterpret_cast<float2*>(us + kcap);         // [ks][nb][16] (sum, compensation)
  for (int b = bw; b < nb && h < ks; b += wb) {
    int ib = 0, r = b;                                          // block b -> (ib <= jb)
    while (r >= n_ib - ib) { r -= n_ib - ib; ++ib; }
    const int jb = ib + r;
    const float* ra = Ds + (size_t)(4 * ib) * kcap;
    const float* rb = Ds + (size_t)(4 * jb) * kcap;
    float s[16], c[16];
#pragma unroll
    for (int p = 0; p < 16; ++p) s[p] = c[p] = 0.0f;
    for (int g0 = k_lo; g0 < k_hi; g0 += 32 * QB_GROUP) {
      float bs[16];
#pragma unroll
      for (int p = 0; p < 16; ++p) bs[p] = 0.0f;
      const int g1 = min(k_hi, g0 + 32 * QB_GROUP);
#pragma unroll 2
      for (int kk = g0 + lane; kk < g1; kk += 32) {
        const float u = us[kk];
        float ai[4], dj[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          ai[x] = ra[(size_t)x * kcap + kk] * u;
          dj[x] = rb[(size_t)x * kcap + kk];
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) bs[4 * x + y] = fmaf(ai[x], dj[y], bs[4 * x + y]);
      }
#pragma unroll
      for (int p = 0; p < 16; ++p) qb_two_sum(s[p], c[p], bs[p]);
    }
    qb_scatter_step<8, 16>(s, c, lane);
    qb_scatter_step<4, 8>(s, c, lane);
    qb_scatter_step<2, 4>(s, c, lane);
    qb_scatter_step<1, 2>(s, c, lane);
    qb_combine(s[0], c[0], __shfl_xor_sync(0xffffffffu, s[0], 1),
               __shfl_xor_sync(0xffffffffu, c[0], 1));
    if (!(lane & 1)) red[((size_t)h * nb + b) * 16 + (lane >> 1)] = make_float2(s[0], c[0]);
  }
  __syncthreads();
  // the k parts of each pair, added in order; pair p of block b is (4 ib + p / 4, 4 jb + p % 4)
  for (int e = threadIdx.x; e < nb * 16; e += blockDim.x) {
    const int b = e >> 4, p = e & 15;
    int ib = 0, r = b;
    while (r >= n_ib - ib) { r -= n_ib - ib; ++ib; }
    const int jb = ib + r;
    const int i = 4 * ib + (p >> 2), j = 4 * jb + (p & 3);
    if (i >= N_tr || j >= N_tr || i > j) continue;
    float2 t = red[e];
    for (int hh = 1; hh < ks; ++hh) {
      const float2 o = red[(size_t)hh * nb * 16 + e];
      qb_combine(t.x, t.y, o.x, o.y);
    }
    const double v = (double)t.x + (double)t.y;
    if (n_kc == 1) {
      Uw[i * N_tr + j] = v;
      Uw[j * N_tr + i] = v;
    } else {
      pw[i * N_tr - i * (i - 1) / 2 + (j - i)] = v;
    }
  }
}

// C[o][i][j] = A_i A_j U[w][l][i][j] for the packed (walker, listed multipole) outputs.
__global__ void k_scale_pack(double* __restrict__ C, const double* __restrict__ U,
                             const double* __restrict__ amp, const int* __restrict__ off,
                             const int* __restrict__ idx, int n_walk, int N_tr, int N_ell,
                             long n_out, int* __restrict__ status) {
  long o = blockIdx.x;
  if (o >= n_out) return;
  int w, l;
  if (off) {
    // walker of output o: largest w with off[w] <= o
    int lo = 0, hi = n_walk;
    while (hi - lo > 1) { int mid = (lo + hi) >> 1; if (off[mid] <= o) lo = mid; else hi = mid; }
    w = lo;
    l = idx[o];
  } else {
    w = (int)(o / N_ell);
    l = (int)(o % N_ell);
  }
  const double* u = U + ((size_t)w * N_ell + l) * N_tr * N_tr;
  const double* A = amp + (size_t)w * N_tr;
  for (int e = threadIdx.x; e < N_tr * N_tr; e += blockDim.x) {
    int i = e / N_tr, j = e - i * N_tr;
    double ai = A[i], aj = A[j];
    double s = (i <= j) ? ai * aj : aj * ai;
    const double v = s * u[e];
    flag_nonfinite(status, v);
    C[o * N_tr * N_tr + e] = v;
  }
}

// Cbar_full[w][l] = (Cbar + Cbar^T)/2 on listed multipoles, 0 elsewhere.
__global__ void k_unpack_sym(double* __restrict__ Cf, const double* __restrict__ Cb,
                             const int* __restrict__ off, const int* __restrict__ idx,
                             int n_walk, int N_tr, int N_ell, long n_out) {
  long o = blockIdx.x;
  if (o >= n_out) return;
  int w, l;
  if (off) {
    int lo = 0, hi = n_walk;
    while (hi - lo > 1) { int mid = (lo + hi) >> 1; if (off[mid] <= o) lo = mid; else hi = mid; }
    w = lo;
    l = idx[o];
  } else {
    w = (int)(o / N_ell);
    l = (int)(o % N_ell);
  }
  const double* s = Cb + o * N_tr * N_tr;
  double* d = Cf + ((size_t)w * N_ell + l) * N_tr * N_tr;
  for (int e = threadIdx.x; e < N_tr * N_tr; e += blockDim.x) {
    int i = e / N_tr, j = e - i * N_tr;
    d[e] = 0.5 * (s[i * N_tr + j] + s[j * N_tr + i]);
  }
}

// amp_bar[w][i] = 2 sum_l sum_j S_ij A_j U_ij
__global__ void k_amp_bar(double* __restrict__ abar, const double* __restrict__ Cf,
                          const double* __restrict__ U, const double* __restrict__ amp,
                          int N_tr, int N_ell, int* __restrict__ status) {
  const int w = blockIdx.y;
  const int i = blockIdx.x;
  __shared__ double red[256];
  double s = 0.0;
  const double* A = amp + (size_t)w * N_tr;
  for (int e = threadIdx.x; e < N_ell * N_tr; e += blockDim.x) {
    int l = e / N_tr, j = e - l * N_tr;
    size_t base = (((size_t)w * N_ell + l) * N_tr + i) * N_tr + j;
    s = fma(Cf[base] * A[j], U[base], s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    flag_nonfinite(status, red[0]);
    abar[(size_t)w * N_tr + i] = 2.0 * red[0];
  }
}

// Delta_bar and the P_bar partial sums.  Grid: (k tile of DT QT points, one multipole, walker);
// QT consecutive k points per thread.  S_ij A_j is staged per multipole chunk in shared memory,
// transposed (St[j][i], rows padded to a multiple of DG with zeros) so that DG consecutive rows i
// load as one vector, in the arithmetic type T (FP32 for the mixed paths, FP64 for the FP64 path);
// Delta_j(l, q) sits in a per-thread shared column.  Each thread forms T_i for DG rows i at a time,
// DG independent FMA chains over j in ascending order.  The P_bar partial of each multipole chunk
// is a compensated sum (TwoSum) written as FP64 to pbar_part[chunk][w][q]; k_pbar_reduce adds the
// chunks.  A launch covers the multipoles [l_lo, l_lo + n_l) of the Delta buffer it is given (a
// multipole chunk when Delta is recomputed chunk by chunk); the reduction runs once after the last
// chunk.
constexpr int DT = 256;   // threads per CTA
constexpr int LC = 1;   // multipoles per CTA: one, for enough CTAs to hide the load latency
constexpr int DG = 4;   // rows i per pass

__host__ __device__ inline int delta_bar_pitch(int N_tr) { return (N_tr + DG - 1) / DG * DG; }

__device__ __forceinline__ void lds4(const float* p, float (&v)[4]) {
  const float4 x = *reinterpret_cast<const float4*>(p);
  v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void lds4(const double* p, double (&v)[4]) {
  const double2 x = reinterpret_cast<const double2*>(p)[0];
  const double2 y = reinterpret_cast<const double2*>(p)[1];
  v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
}

template <typename T>
__device__ __forceinline__ void two_sum_acc(T& s, T& c, T x) {
  const T sn = s + x;
  const T bp = sn - s;
  c += (s - (sn - bp)) + (x - bp);
  s = sn;
}

// QT consecutive k points per thread: with QT = 2 every shared load of S feeds 2 DG FMAs and
// Delta and Dbar move as 8-byte pairs, but one point per thread at 256 threads per CTA measured
// faster (more warps to hide the load latency), so both types use QT = 1; the sums of each k
// point are the same in either form.
template <typename T> struct DbarQ { static constexpr int QT = 1; };
template <> struct DbarQ<float> { static constexpr int QT = 1; };

template <typename T>
__global__ void __launch_bounds__(DT)
k_delta_bar(T* __restrict__ dbar, double* __restrict__ pbar_part, const T* __restrict__ delta,
            const double* __restrict__ Cf, const double* __restrict__ amp,
            const double* __restrict__ P, const double* __restrict__ wk2, int N_tr, int N_k,
            int N_ell, int n_walk, int l_lo, int n_l, const int* __restrict__ listed) {
  constexpr int QT = DbarQ<T>::QT, DQ = DT * QT;
  pdl_trigger();   // the next kernel of the step may be scheduled
  pdl_wait();      // Delta and the cotangent come from the kernels before
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  const int NP = delta_bar_pitch(N_tr);
  T* St = reinterpret_cast<T*>(dsm_raw);           // [N_tr][NP]  St[j][i] = S_ij A_j
  T* Dl = St + N_tr * NP;                          // [N_tr][DQ]
  T* As = Dl + N_tr * DQ;                          // [N_tr] A_i
  const int w = blockIdx.z;
  // Delta and Dbar hold multipoles [l_lo, l_lo + n_l); Cf all N_ell (LC = 1 multipole per CTA)
  const int l0 = l_lo + blockIdx.y;
  const int qt = threadIdx.x * QT;                 // this thread's first column of Dl
  const int q0 = blockIdx.x * DQ + qt;
  if (listed && listed[w * n_l + (l0 - l_lo)] < 0) {
    // a multipole the walker does not list: S = 0, so Dbar = 0 and the P_bar partial is 0; its
    // Delta rows are not read and its Dbar rows are not used
#pragma unroll
    for (int u = 0; u < QT; ++u)
      if (q0 + u < N_k) pbar_part[((size_t)l0 * n_walk + w) * N_k + q0 + u] = 0.0;
    return;
  }
  const double* A = amp + (size_t)w * N_tr;
  const double* Cl = Cf + ((size_t)w * N_ell + l0) * N_tr * N_tr;
  for (int e = threadIdx.x; e < N_tr * NP; e += DT) {
    const int j = e / NP, i = e - j * NP;
    St[e] = i < N_tr ? (T)(Cl[i * N_tr + j] * A[j]) : T(0);
  }
  for (int e = threadIdx.x; e < N_tr; e += DT) As[e] = (T)A[e];
  T two_u[QT];
#pragma unroll
  for (int u = 0; u < QT; ++u)
    two_u[u] = (q0 + u < N_k) ? (T)(2.0 * wk2[q0 + u] * P[(size_t)w * N_k + q0 + u]) : T(0);
  const T* dl = delta + ((size_t)w * n_l + l0 - l_lo) * N_tr * N_k;
  const bool pair = QT == 2 && (N_k & 1) == 0 && q0 + 1 < N_k;   // 8-byte aligned pair
#pragma unroll 5
  for (int t = 0; t < N_tr; ++t) {
    if (pair) {
      *reinterpret_cast<float2*>(Dl + t * DQ + qt) = *reinterpret_cast<const float2*>(dl + (size_t)t * N_k + q0);
    } else {
#pragma unroll
      for (int u = 0; u < QT; ++u) Dl[t * DQ + qt + u] = (q0 + u < N_k) ? dl[(size_t)t * N_k + q0 + u] : T(0);
    }
  }
  __syncthreads();
  if (q0 >= N_k) return;
  T ps[QT], pc[QT];
#pragma unroll
  for (int u = 0; u < QT; ++u) ps[u] = pc[u] = T(0);
  const T* dq = Dl + qt;
  T* db = dbar + ((size_t)w * n_l + l0 - l_lo) * N_tr * N_k + q0;
  for (int i0 = 0; i0 < N_tr; i0 += DG) {
    T t[DG][QT];
#pragma unroll
    for (int g = 0; g < DG; ++g)
#pragma unroll
      for (int u = 0; u < QT; ++u) t[g][u] = 0;
#pragma unroll 5
    for (int j = 0; j < N_tr; ++j) {
      T sv[DG];
      lds4(St + j * NP + i0, sv);
      T d[QT];
#pragma unroll
      for (int u = 0; u < QT; ++u) d[u] = dq[j * DQ + u];
#pragma unroll
      for (int g = 0; g < DG; ++g)
#pragma unroll
        for (int u = 0; u < QT; ++u) t[g][u] = fma(sv[g], d[u], t[g][u]);
    }
#pragma unroll
    for (int g = 0; g < DG; ++g) {
      const int ii = i0 + g;
      if (ii < N_tr) {
        const T ai = As[ii];
        T o[QT];
#pragma unroll
        for (int u = 0; u < QT; ++u) {
          two_sum_acc(ps[u], pc[u], ai * dq[ii * DQ + u] * t[g][u]);
          o[u] = two_u[u] * ai * t[g][u];
        }
        if (pair) {
          *reinterpret_cast<float2*>(db + (size_t)ii * N_k) = make_float2((float)o[0], (float)o[QT - 1]);
        } else {
#pragma unroll
          for (int u = 0; u < QT; ++u)
            if (q0 + u < N_k) db[(size_t)ii * N_k + u] = o[u];
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < QT; ++u)
    if (q0 + u < N_k) pbar_part[((size_t)l0 * n_walk + w) * N_k + q0 + u] = (double)ps[u] + (double)pc[u];
}

__global__ void k_pbar_reduce(double* __restrict__ Pbar, const double* __restrict__ part,
                              const double* __restrict__ wk2, int n_chunk, int n_walk, int N_k,
                              int* __restrict__ status) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)n_walk * N_k) return;
  double s = 0.0;
  for (int c = 0; c < n_chunk; ++c) s += part[(size_t)c * n_walk * N_k + t];
  const double v = wk2[t % N_k] * s;
  flag_nonfinite(status, v);
  Pbar[t] = v;
}

}  // namespace

template <typename T>
cudaError_t launch_quad(double* U, const T* delta, const double* P, const double* wk2, int n_walk,
                        int N_tr, int N_k, int N_ell, int l_lo, int n_l, double* scratch,
                        cudaStream_t s, const int* listed = nullptr) {
  size_t smem = (size_t)N_tr * KS * sizeof(T);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_quad_part<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int n_kc = (N_k + KC - 1) / KC;
  dim3 g(n_l, n_kc, n_walk);
  k_quad_part<T><<<g, QT, smem, s>>>(scratch, delta, P, wk2, N_tr, N_k, n_l, n_kc, listed);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long total = (long)n_walk * n_l * N_tr * (N_tr + 1) / 2;
  const unsigned grid = (unsigned)std::min<long>((total + 255) / 256, 152L * 16);
  k_quad_reduce<<<grid, 256, 0, s>>>(U, scratch, N_tr, N_ell, l_lo, n_l, n_kc, n_walk);
  return cudaGetLastError();
}

size_t quad_scratch_bytes(int n_walk, int N_tr, int N_k, int n_l) {
  return sizeof(double) * (size_t)n_walk * n_l * ((N_k + KC - 1) / KC) * (N_tr * (N_tr + 1) / 2);
}

cudaError_t launch_pair_reduce(double* U, const double* part, int n_walk, int N_tr, int N_ell,
                               int l_lo, int n_l, int n_chunk, cudaStream_t s) {
  const long total = (long)n_walk * n_l * (N_tr * (N_tr + 1) / 2);
  const int grid = (int)std::min<long>((total + 255) / 256, 152L * 8);
  k_quad_reduce<<<grid, 256, 0, s>>>(U, part, N_tr, N_ell, l_lo, n_l, n_chunk, n_walk);
  return cudaGetLastError();
}

cudaError_t launch_quad_fp64(double* U, const double* delta, const double* P, const double* wk2,
                             int n_walk, int N_tr, int N_k, int N_ell, int l_lo, int n_l,
                             double* scratch, cudaStream_t s) {
  return launch_quad<double>(U, delta, P, wk2, n_walk, N_tr, N_k, N_ell, l_lo, n_l, scratch, s);
}

cudaError_t launch_quad_f32(double* U, const float* delta, const double* P, const double* wk2,
                            int n_walk, int N_tr, int N_k, int N_ell, int l_lo, int n_l,
                            double* scratch, cudaStream_t s, const int* listed) {
  if (n_walk <= 0 || n_l <= 0) return cudaSuccess;
  const int n_ib = (N_tr + 3) / 4, nb = n_ib * (n_ib + 1) / 2;
  // k parts per block: with few CTAs (one walker), enough warps per CTA to hide the shared-load
  // and FMA latencies; with many, one part (each further part repeats the lane combination)
  const long n_cta0 = (long)n_walk * n_l * ((N_k + 1023) / 1024);
  const int ks = n_cta0 >= 2 * 152 ? 1 : std::max(1, std::min(4, QB_MAX_WARPS / nb));
  const int warps = ks * std::min(nb, QB_MAX_WARPS / ks);
  const size_t red_bytes = sizeof(float2) * (size_t)ks * nb * 16;
  // k points per CTA: the largest power of two up to 1024 whose rows fit QB_SMEM
  int kcap = 1024;
  while (kcap > 32 && (size_t)kcap * (16 * n_ib + 4) + red_bytes > (size_t)QB_SMEM) kcap >>= 1;
  const int n_kc = (N_k + kcap - 1) / kcap;
  const size_t smem = (size_t)kcap * (16 * n_ib + 4) + red_bytes;
  const bool vec4 = N_k % 4 == 0 && ((uintptr_t)delta & 15) == 0;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_quad_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 g(n_l, n_kc, n_walk);
  k_quad_blocks<<<g, warps * 32, smem, s>>>(U, scratch, delta, P, wk2, N_tr, N_k, N_ell, l_lo,
                                            n_l, kcap, n_kc, ks, vec4, listed);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || n_kc == 1) return e;
  const long total = (long)n_walk * n_l * N_tr * (N_tr + 1) / 2;
  const unsigned grid = (unsigned)std::min<long>((total + 255) / 256, 152L * 16);
  k_quad_reduce<<<grid, 256, 0, s>>>(U, scratch, N_tr, N_ell, l_lo, n_l, n_kc, n_walk);
  return cudaGetLastError();
}

cudaError_t launch_scale_pack(double* C, const double* U, const double* amp, const int* off,
                              const int* idx, int n_walk, int N_tr, int N_ell, int64_t n_out,
                              cudaStream_t s, int* status) {
  if (n_out == 0) return cudaSuccess;
  k_scale_pack<<<(unsigned)n_out, 128, 0, s>>>(C, U, amp, off, idx, n_walk, N_tr, N_ell, n_out,
                                               status);
  return cudaGetLastError();
}

cudaError_t launch_unpack_sym(double* Cf, const double* Cb, const int* off, const int* idx,
                              int n_walk, int N_tr, int N_ell, int64_t n_out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(Cf, 0, (size_t)n_walk * N_ell * N_tr * N_tr * sizeof(double), s);
  if (e != cudaSuccess || n_out == 0) return e;
  k_unpack_sym<<<(unsigned)n_out, 128, 0, s>>>(Cf, Cb, off, idx, n_walk, N_tr, N_ell, n_out);
  return cudaGetLastError();
}

cudaError_t launch_amp_bar(double* amp_bar, const double* Cf, const double* U, const double* amp,
                           int n_walk, int N_tr, int N_ell, cudaStream_t s, int* status) {
  dim3 g(N_tr, n_walk);
  k_amp_bar<<<g, 256, 0, s>>>(amp_bar, Cf, U, amp, N_tr, N_ell, status);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_delta_bar(T* dbar, const T* delta, const double* Cf, const double* amp,
                             const double* P, const double* wk2, int n_walk, int N_tr, int N_k,
                             int N_ell, int l_lo, int n_l, double* scratch, cudaStream_t s,
                             const int* listed, bool pdl) {
  constexpr int DQ = DT * DbarQ<T>::QT;
  const size_t smem = (size_t)(N_tr * delta_bar_pitch(N_tr) + N_tr * DQ + N_tr) * sizeof(T);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_delta_bar<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 g((N_k + DQ - 1) / DQ, n_l, n_walk);
  return launch_k(pdl, k_delta_bar<T>, g, dim3(DT), smem, s, dbar, scratch, delta, Cf, amp, P, wk2,
                  N_tr, N_k, N_ell, n_walk, l_lo, n_l, listed);
}

cudaError_t launch_pbar_reduce(double* P_bar, const double* scratch, const double* wk2,
                               int n_walk, int N_k, int N_ell, cudaStream_t s, int* status) {
  const int n_chunk = (N_ell + LC - 1) / LC;
  const long n = (long)n_walk * N_k;
  k_pbar_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P_bar, scratch, wk2, n_chunk, n_walk, N_k,
                                                           status);
  return cudaGetLastError();
}

size_t delta_bar_scratch_bytes(int n_walk, int N_k, int N_ell) {
  return sizeof(double) * (size_t)((N_ell + LC - 1) / LC) * n_walk * N_k;
}

template cudaError_t launch_delta_bar<double>(double*, const double*, const double*,
                                              const double*, const double*, const double*, int,
                                              int, int, int, int, int, double*, cudaStream_t,
                                              const int*, bool);
template cudaError_t launch_delta_bar<float>(float*, const float*, const double*, const double*,
                                             const double*, const double*, int, int, int, int,
                                             int, int, double*, cudaStream_t, const int*, bool);

}  // namespace swcl
