// a4: the k-quadrature of Eq. 2.1, C_l^{ij} = A_i A_j sum_q u_q Delta_i(l,q) Delta_j(l,q),
// u_q = wk2[q] P(k_q), and the reductions of its reverse mode (a5):
//   Pbar_q   = wk2[q] sum_l sum_i A_i Delta_i T_i,   T_i = sum_j S_ij A_j Delta_j,
//   Dbar_i   = 2 A_i u_q T_i,
//   Abar_i   = 2 sum_l sum_j S_ij A_j U_ij            (U = C at unit amplitudes),
// with S = (Cbar + Cbar^T)/2 (zero for multipoles outside a walker's list).
//
// The unit-amplitude spectra U are formed per (walker, multipole) by one CTA; each unordered
// pair (i <= j) is summed once over k and written to both (i,j) and (j,i), so C is symmetric
// bit for bit.  Delta in FP32 (mixed paths): the products are FP32, the partial sums over 32 k
// points are compensated FP32 sums (TwoSum; the rounding of each addition is carried in a second
// float), and the per-pair total over k is FP64.
#include "swcl_internal.h"

namespace swcl {
namespace {

constexpr int QT = 256;    // threads
constexpr int QC = 128;    // k points staged per step

template <typename T>
__global__ void __launch_bounds__(QT)
k_quad(double* __restrict__ U, const T* __restrict__ delta, const double* __restrict__ P,
       const double* __restrict__ wk2, int N_tr, int N_k, int N_ell, int l_lo, int n_l) {
  extern __shared__ double qsm[];
  T* Ds = reinterpret_cast<T*>(qsm);              // [N_tr][QC]
  __shared__ double us[QC];
  __shared__ float usf[QC];
  __shared__ double red[QT];
  // Delta holds multipoles [l_lo, l_lo + n_l) of each walker; U all N_ell
  const int l = l_lo + blockIdx.x;
  const int w = blockIdx.y;
  const int npair = N_tr * (N_tr + 1) / 2;
  const T* dl = delta + ((size_t)w * n_l + blockIdx.x) * N_tr * N_k;
  const double* Pw = P + (size_t)w * N_k;
  // thread -> (pair slot, k-group)
  const int ngroups = max(1, QT / npair);
  const int group = threadIdx.x / npair;
  for (int p0 = 0; p0 < npair; p0 += QT) {
    int p = p0 + (ngroups > 1 ? (threadIdx.x % npair) : threadIdx.x);
    bool active = (ngroups > 1) ? (group < ngroups) : (p < npair);
    int pi = 0, pj = 0;
    if (active && p < npair) {
      // unordered pair index -> (i <= j)
      int r = p, ii = 0;
      while (r >= N_tr - ii) { r -= N_tr - ii; ++ii; }
      pi = ii; pj = ii + r;
    }
    double acc = 0.0;
    for (int qb = 0; qb < N_k; qb += QC) {
      __syncthreads();
      for (int e = threadIdx.x; e < N_tr * QC; e += QT) {
        int t = e / QC, qq = e - t * QC;
        int q = qb + qq;
        Ds[t * QC + qq] = (q < N_k) ? dl[(size_t)t * N_k + q] : T(0);
      }
      for (int e = threadIdx.x; e < QC; e += QT) {
        int q = qb + e;
        us[e] = (q < N_k) ? wk2[q] * Pw[q] : 0.0;
        usf[e] = (float)us[e];
      }
      __syncthreads();
      if (active && p < npair) {
        const T* di = Ds + pi * QC;
        const T* dj = Ds + pj * QC;
        int qs = (ngroups > 1) ? group : 0;
        int qstep = (ngroups > 1) ? ngroups : 1;
        if (sizeof(T) == 4) {
          // FP32 products, compensated FP32 partial sums of 32 points, FP64 total
          for (int c0 = qs * 32; c0 < QC; c0 += qstep * 32) {
            float sum = 0.0f, comp = 0.0f;
#pragma unroll 8
            for (int qq = c0; qq < c0 + 32; ++qq) {
              const float t = ((float)di[qq] * usf[qq]) * (float)dj[qq];
              const float sn = sum + t;
              const float bp = sn - sum;
              comp += (sum - (sn - bp)) + (t - bp);
              sum = sn;
            }
            acc += (double)sum + (double)comp;
          }
        } else {
          for (int qq = qs; qq < QC; qq += qstep)
            acc = fma((double)di[qq] * us[qq], (double)dj[qq], acc);
        }
      }
    }
    // combine k-groups
    __syncthreads();
    red[threadIdx.x] = acc;
    __syncthreads();
    if (active && p < npair && (ngroups == 1 || group == 0)) {
      double s = acc;
      if (ngroups > 1)
        for (int g = 1; g < ngroups; ++g) s += red[g * npair + (threadIdx.x % npair)];
      double* out = U + ((size_t)w * N_ell + l) * N_tr * N_tr;
      out[pi * N_tr + pj] = s;
      out[pj * N_tr + pi] = s;
    }
    if (ngroups > 1) break;
  }
}

// C[o][i][j] = A_i A_j U[w][l][i][j] for the packed (walker, listed multipole) outputs.
__global__ void k_scale_pack(double* __restrict__ C, const double* __restrict__ U,
                             const double* __restrict__ amp, const int* __restrict__ off,
                             const int* __restrict__ idx, int n_walk, int N_tr, int N_ell,
                             long n_out) {
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
    C[o * N_tr * N_tr + e] = s * u[e];
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
                          int N_tr, int N_ell) {
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
  if (threadIdx.x == 0) abar[(size_t)w * N_tr + i] = 2.0 * red[0];
}

// Delta_bar and the P_bar partial sums.  Grid: (k tile of DT points, chunk of LC multipoles,
// walker); one thread per k point.  S_l A_j is staged per multipole chunk in shared memory (in the
// arithmetic type T: FP32 for the mixed paths, FP64 for the FP64 path), Delta_j(l, q) in a
// per-thread shared column.  The P_bar partial of each multipole chunk is a compensated sum
// (TwoSum) written as FP64 to pbar_part[chunk][w][q]; k_pbar_reduce adds the chunks.  A launch
// covers the multipoles [l_lo, l_lo + n_l) of the Delta buffer it is given (a multipole chunk
// when Delta is recomputed chunk by chunk); the reduction runs once after the last chunk.
constexpr int DT = 128;
constexpr int LC = 8;

template <typename T>
__device__ __forceinline__ void two_sum_acc(T& s, T& c, T x) {
  const T sn = s + x;
  const T bp = sn - s;
  c += (s - (sn - bp)) + (x - bp);
  s = sn;
}

template <typename T>
__global__ void __launch_bounds__(DT)
k_delta_bar(T* __restrict__ dbar, double* __restrict__ pbar_part, const T* __restrict__ delta,
            const double* __restrict__ Cf, const double* __restrict__ amp,
            const double* __restrict__ P, const double* __restrict__ wk2, int N_tr, int N_k,
            int N_ell, int n_walk, int l_lo, int n_l) {
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  T* S = reinterpret_cast<T*>(dsm_raw);            // [LC][N_tr][N_tr]  S_ij A_j
  T* Dl = S + LC * N_tr * N_tr;                    // [N_tr][DT]
  const int w = blockIdx.z;
  // Delta and Dbar hold multipoles [l_lo, l_lo + n_l) (l_lo a multiple of LC); Cf all N_ell
  const int lc = l_lo / LC + blockIdx.y;
  const int q = blockIdx.x * DT + threadIdx.x;
  const int l0 = lc * LC;
  const int nl = min(LC, l_lo + n_l - l0);
  const double* A = amp + (size_t)w * N_tr;
  for (int e = threadIdx.x; e < nl * N_tr * N_tr; e += DT) {
    const int ll = e / (N_tr * N_tr), r = e - ll * N_tr * N_tr;
    S[e] = (T)(Cf[((size_t)w * N_ell + l0 + ll) * N_tr * N_tr + r] * A[r % N_tr]);
  }
  const T two_u = (q < N_k) ? (T)(2.0 * wk2[q] * P[(size_t)w * N_k + q]) : T(0);
  T ps = 0, pc = 0;
  for (int ll = 0; ll < nl; ++ll) {
    __syncthreads();
    const T* dl = delta + ((size_t)w * n_l + l0 - l_lo + ll) * N_tr * N_k;
    for (int t = 0; t < N_tr; ++t)
      Dl[t * DT + threadIdx.x] = (q < N_k) ? dl[(size_t)t * N_k + q] : T(0);
    __syncthreads();
    if (q < N_k) {
      const T* Sl = S + ll * N_tr * N_tr;
      T* db = dbar + ((size_t)w * n_l + l0 - l_lo + ll) * N_tr * N_k;
      for (int ii = 0; ii < N_tr; ++ii) {
        T t = 0;
        for (int j = 0; j < N_tr; ++j) t = fma(Sl[ii * N_tr + j], Dl[j * DT + threadIdx.x], t);
        const T ai = (T)A[ii];
        two_sum_acc(ps, pc, ai * Dl[ii * DT + threadIdx.x] * t);
        db[(size_t)ii * N_k + q] = two_u * ai * t;
      }
    }
  }
  if (q < N_k) pbar_part[((size_t)lc * n_walk + w) * N_k + q] = (double)ps + (double)pc;
}

__global__ void k_pbar_reduce(double* __restrict__ Pbar, const double* __restrict__ part,
                              const double* __restrict__ wk2, int n_chunk, int n_walk, int N_k) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)n_walk * N_k) return;
  double s = 0.0;
  for (int c = 0; c < n_chunk; ++c) s += part[(size_t)c * n_walk * N_k + t];
  Pbar[t] = wk2[t % N_k] * s;
}

}  // namespace

template <typename T>
cudaError_t launch_quad(double* U, const T* delta, const double* P, const double* wk2, int n_walk,
                        int N_tr, int N_k, int N_ell, int l_lo, int n_l, cudaStream_t s) {
  size_t smem = (size_t)N_tr * QC * sizeof(T);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_quad<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 g(n_l, n_walk);
  k_quad<T><<<g, QT, smem, s>>>(U, delta, P, wk2, N_tr, N_k, N_ell, l_lo, n_l);
  return cudaGetLastError();
}

cudaError_t launch_quad_fp64(double* U, const double* delta, const double* P, const double* wk2,
                             int n_walk, int N_tr, int N_k, int N_ell, int l_lo, int n_l,
                             cudaStream_t s) {
  return launch_quad<double>(U, delta, P, wk2, n_walk, N_tr, N_k, N_ell, l_lo, n_l, s);
}

cudaError_t launch_quad_f32(double* U, const float* delta, const double* P, const double* wk2,
                            int n_walk, int N_tr, int N_k, int N_ell, int l_lo, int n_l,
                            cudaStream_t s) {
  return launch_quad<float>(U, delta, P, wk2, n_walk, N_tr, N_k, N_ell, l_lo, n_l, s);
}

cudaError_t launch_scale_pack(double* C, const double* U, const double* amp, const int* off,
                              const int* idx, int n_walk, int N_tr, int N_ell, int64_t n_out,
                              cudaStream_t s) {
  if (n_out == 0) return cudaSuccess;
  k_scale_pack<<<(unsigned)n_out, 128, 0, s>>>(C, U, amp, off, idx, n_walk, N_tr, N_ell, n_out);
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
                           int n_walk, int N_tr, int N_ell, cudaStream_t s) {
  dim3 g(N_tr, n_walk);
  k_amp_bar<<<g, 256, 0, s>>>(amp_bar, Cf, U, amp, N_tr, N_ell);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_delta_bar(T* dbar, const T* delta, const double* Cf, const double* amp,
                             const double* P, const double* wk2, int n_walk, int N_tr, int N_k,
                             int N_ell, int l_lo, int n_l, double* scratch, cudaStream_t s) {
  const size_t smem = (size_t)(LC * N_tr * N_tr + N_tr * DT) * sizeof(T);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_delta_bar<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 g((N_k + DT - 1) / DT, (n_l + LC - 1) / LC, n_walk);
  k_delta_bar<T><<<g, DT, smem, s>>>(dbar, scratch, delta, Cf, amp, P, wk2, N_tr, N_k, N_ell,
                                     n_walk, l_lo, n_l);
  return cudaGetLastError();
}

cudaError_t launch_pbar_reduce(double* P_bar, const double* scratch, const double* wk2,
                               int n_walk, int N_k, int N_ell, cudaStream_t s) {
  const int n_chunk = (N_ell + LC - 1) / LC;
  const long n = (long)n_walk * N_k;
  k_pbar_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P_bar, scratch, wk2, n_chunk, n_walk, N_k);
  return cudaGetLastError();
}

size_t delta_bar_scratch_bytes(int n_walk, int N_k, int N_ell) {
  return sizeof(double) * (size_t)((N_ell + LC - 1) / LC) * n_walk * N_k;
}

template cudaError_t launch_delta_bar<double>(double*, const double*, const double*,
                                              const double*, const double*, const double*, int,
                                              int, int, int, int, int, double*, cudaStream_t);
template cudaError_t launch_delta_bar<float>(float*, const float*, const double*, const double*,
                                             const double*, const double*, int, int, int, int,
                                             int, int, double*, cudaStream_t);

}  // namespace swcl
