// Forward mode (JVP) of a4 and the Gaussian Fisher matrix (Sec. 4.3).
//
// JVP.  Delta is linear in the windows (Eq. 3.1-3.5), so the tangent Delta' of a window tangent
// is the ordinary contraction of the tangent windows; the host runs it as extra walkers.  Here:
//   dU_ij(l) = sum_q wk2_q [P'_q Delta_i Delta_j + P_q (Delta'_i Delta_j + Delta_i Delta'_j)],
//   dC_ij    = A_i A_j dU_ij + (A'_i A_j + A_i A'_j) U_ij                 (Eq. 2.1, product rule).
//
// Fisher.  With Ct = C + diag(noise) per multipole and nu_l modes behind C_l,
//   F_ab = sum_l (nu_l / 2) Tr[Ct^-1 X_a Ct^-1 X_b]
// is the Fisher matrix of the Gaussian likelihood of the unique pairs C_l^{ij} (X = dC/dtheta)
// and its chi^2 (X = C - C_data).  With the Cholesky factor Ct = L L^T and Y_a = L^-1 X_a L^-T,
// F_ab = sum_l (nu_l/2) sum_ij Y_a[i][j] Y_b[j][i]: one CTA per multipole factors Ct and whitens
// every X_a (two triangular solves by columns), and one CTA per pair (a <= b) forms the sum in a
// fixed order, so F is symmetric and the same from run to run.
#include <algorithm>

#include "swcl_internal.h"

namespace swcl {
namespace {

constexpr int JT = 256;   // threads of the JVP quadrature
constexpr int KJ = 32;    // k points staged per step
constexpr int KJS = KJ + 1;  // shared row stride (rows of different tracers in different banks)
constexpr int MAXR = 9;   // pairs per thread: ceil(64 * 65 / 2 / 256)

// dU[t][l_lo + ll][i][j] for tangent t; delta [1 + n_w][n_l][N_tr][N_k] holds the base walker
// first, then one walker per tangent when has_w.  Grid (n_l, n_dir).
template <typename T>
__global__ void __launch_bounds__(JT)
k_quad_jvp(double* __restrict__ dU, const T* __restrict__ delta, const double* __restrict__ P,
           const double* __restrict__ Pdot, const double* __restrict__ wk2, int has_w, int N_tr,
           int N_k, int N_ell, int l_lo, int n_l) {
  __shared__ double D0[64 * KJS], Dt[64 * KJS], us[KJ], uds[KJ];
  const int ll = blockIdx.x, t = blockIdx.y;
  const int npair = N_tr * (N_tr + 1) / 2;
  const T* d0 = delta + (size_t)ll * N_tr * N_k;
  const T* dt = delta + ((size_t)(1 + t) * n_l + ll) * N_tr * N_k;
  const double* pd = Pdot + (size_t)t * N_k;
  int pi[MAXR], pj[MAXR];
  double acc[MAXR];
#pragma unroll
  for (int r = 0; r < MAXR; ++r) {
    int p = threadIdx.x + r * JT, i = 0;
    acc[r] = 0.0;
    if (p < npair) {
      while (p >= N_tr - i) { p -= N_tr - i; ++i; }
    }
    pi[r] = i;
    pj[r] = i + p;
  }
  for (int q0 = 0; q0 < N_k; q0 += KJ) {
    for (int e = threadIdx.x; e < N_tr * KJ; e += JT) {
      const int i = e / KJ, qq = e - i * KJ, q = q0 + qq;
      D0[i * KJS + qq] = q < N_k ? (double)d0[(size_t)i * N_k + q] : 0.0;
      Dt[i * KJS + qq] = (has_w && q < N_k) ? (double)dt[(size_t)i * N_k + q] : 0.0;
    }
    for (int e = threadIdx.x; e < KJ; e += JT) {
      const int q = q0 + e;
      us[e] = q < N_k ? wk2[q] * P[q] : 0.0;
      uds[e] = q < N_k ? wk2[q] * pd[q] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < MAXR; ++r) {
      if (threadIdx.x + r * JT < npair) {
        const double* ai = D0 + pi[r] * KJS;
        const double* aj = D0 + pj[r] * KJS;
        const double* bi = Dt + pi[r] * KJS;
        const double* bj = Dt + pj[r] * KJS;
        double s = acc[r];
        for (int qq = 0; qq < KJ; ++qq)
          s = fma(uds[qq], ai[qq] * aj[qq], fma(us[qq], fma(bi[qq], aj[qq], ai[qq] * bj[qq]), s));
        acc[r] = s;
      }
    }
    __syncthreads();
  }
  double* out = dU + ((size_t)t * N_ell + l_lo + ll) * N_tr * N_tr;
#pragma unroll
  for (int r = 0; r < MAXR; ++r) {
    if (threadIdx.x + r * JT < npair) {
      out[pi[r] * N_tr + pj[r]] = acc[r];
      out[pj[r] * N_tr + pi[r]] = acc[r];
    }
  }
}

// Cdot[t][l][i][j] = A_i A_j dU + (A'_i A_j + A_i A'_j) U
__global__ void k_jvp_combine(double* __restrict__ Cdot, const double* __restrict__ dU,
                              const double* __restrict__ U, const double* __restrict__ amp,
                              const double* __restrict__ Adot, int n_dir, int N_tr, int N_ell,
                              int* __restrict__ status) {
  const long n2 = (long)N_tr * N_tr, per = (long)N_ell * n2, total = per * n_dir;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int t = (int)(e / per);
    const long r = e - (long)t * per;
    const int ij = (int)(r % n2);
    const int i = ij / N_tr, j = ij - i * N_tr;
    const double* ad = Adot + (size_t)t * N_tr;
    // every operation symmetric in (i, j), no contraction into FMAs: dC is symmetric bit for bit
    const double aa = __dmul_rn(amp[i], amp[j]);
    const double cross = __dadd_rn(__dmul_rn(ad[i], amp[j]), __dmul_rn(amp[i], ad[j]));
    const double v = __dadd_rn(__dmul_rn(aa, dU[e]), __dmul_rn(cross, U[r]));
    flag_nonfinite(status, v);
    Cdot[e] = v;
  }
}

// One CTA per multipole: Ct = A_i A_j U + diag(noise) in shared memory, its Cholesky factor in
// place (right-looking; a pivot <= 0 marks the multipole in *status and zeroes its output), then
// for every X_a: T = L^-1 X_a (thread j solves column j), Y^T = L^-1 T^T (thread j solves row j
// of T, giving row j of Y), Z_a = sqrt(nu_l / 2) Y.
__global__ void k_fisher_whiten(double* __restrict__ Z, const double* __restrict__ X,
                                const double* __restrict__ U, const double* __restrict__ amp,
                                const double* __restrict__ noise, const double* __restrict__ modes,
                                int* __restrict__ status, int n_x, int N_tr, int N_ell) {
  extern __shared__ double fsm[];
  double* Ls = fsm;                       // [N_tr][N_tr]
  double* Ts = fsm + N_tr * N_tr;         // [N_tr][N_tr]
  double* Ys = fsm + 2 * N_tr * N_tr;     // [N_tr][N_tr]
  __shared__ int bad;
  const int l = blockIdx.x, n = N_tr, n2 = N_tr * N_tr;
  const double* u = U + (size_t)l * n2;
  for (int e = threadIdx.x; e < n2; e += blockDim.x) {
    const int i = e / n, j = e - i * n;
    Ls[e] = amp[i] * amp[j] * u[e] + (i == j && noise ? noise[i] : 0.0);
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      const double d = Ls[k * n + k];
      if (!(d > 0.0)) bad = 1;
      Ls[k * n + k] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double piv = Ls[k * n + k];
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) Ls[i * n + k] /= piv;
    __syncthreads();
    const int m = n - k - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = k + 1 + e / m, j = k + 1 + e % m;
      if (j <= i) Ls[i * n + j] -= Ls[i * n + k] * Ls[j * n + k];
    }
    __syncthreads();
  }
  const double s = sqrt(0.5 * modes[l]);
  for (int a = 0; a < n_x; ++a) {
    const double* x = X + ((size_t)a * N_ell + l) * n2;
    double* z = Z + ((size_t)a * N_ell + l) * n2;
    if (bad) {
      for (int e = threadIdx.x; e < n2; e += blockDim.x) z[e] = 0.0;
      continue;
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      for (int i = 0; i < n; ++i) {
        double v = x[i * n + j];
        for (int m = 0; m < i; ++m) v -= Ls[i * n + m] * Ts[m * n + j];
        Ts[i * n + j] = v / Ls[i * n + i];
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      for (int i = 0; i < n; ++i) {
        double v = Ts[j * n + i];
        for (int m = 0; m < i; ++m) v -= Ls[i * n + m] * Ys[j * n + m];
        Ys[j * n + i] = v / Ls[i * n + i];
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n2; e += blockDim.x) z[e] = s * Ys[e];
    __syncthreads();
  }
  if (threadIdx.x == 0 && bad) atomicOr(status, 1);
}

constexpr int GT = 256;

// F[a][b] = F[b][a] = sum_l sum_ij Z_a[l][i][j] Z_b[l][j][i]; one CTA per pair a <= b
__global__ void __launch_bounds__(GT)
k_fisher_gram(double* __restrict__ F, const double* __restrict__ Z, int n_x, int N_tr, int N_ell) {
  __shared__ double red[GT];
  int p = blockIdx.x, a = 0;
  while (p >= n_x - a) { p -= n_x - a; ++a; }
  const int b = a + p;
  const long n2 = (long)N_tr * N_tr, per = (long)N_ell * n2;
  const double* za = Z + (size_t)a * per;
  const double* zb = Z + (size_t)b * per;
  double s = 0.0;
  for (long e = threadIdx.x; e < per; e += GT) {
    const long l = e / n2;
    const int ij = (int)(e - l * n2);
    const int i = ij / N_tr, j = ij - i * N_tr;
    s = fma(za[e], zb[l * n2 + (long)j * N_tr + i], s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = GT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    F[(size_t)a * n_x + b] = red[0];
    F[(size_t)b * n_x + a] = red[0];
  }
}

}  // namespace

template <typename T>
cudaError_t launch_quad_jvp(double* dU, const T* delta, const double* P, const double* Pdot,
                            const double* wk2, bool has_w, int n_dir, int N_tr, int N_k,
                            int N_ell, int l_lo, int n_l, cudaStream_t s) {
  if (N_tr > 64) return cudaErrorInvalidValue;
  k_quad_jvp<T><<<dim3(n_l, n_dir), JT, 0, s>>>(dU, delta, P, Pdot, wk2, has_w ? 1 : 0, N_tr, N_k,
                                               N_ell, l_lo, n_l);
  return cudaGetLastError();
}
template cudaError_t launch_quad_jvp<double>(double*, const double*, const double*, const double*,
                                             const double*, bool, int, int, int, int, int, int,
                                             cudaStream_t);
template cudaError_t launch_quad_jvp<float>(double*, const float*, const double*, const double*,
                                            const double*, bool, int, int, int, int, int, int,
                                            cudaStream_t);

cudaError_t launch_jvp_combine(double* Cdot, const double* dU, const double* U, const double* amp,
                               const double* Adot, int n_dir, int N_tr, int N_ell, cudaStream_t s,
                               int* status) {
  const long total = (long)n_dir * N_ell * N_tr * N_tr;
  const int blocks = (int)std::min<long>((total + 255) / 256, 152L * 8);
  k_jvp_combine<<<blocks, 256, 0, s>>>(Cdot, dU, U, amp, Adot, n_dir, N_tr, N_ell, status);
  return cudaGetLastError();
}

cudaError_t launch_fisher(double* F, double* Z, const double* X, const double* U,
                          const double* amp, const double* noise, const double* modes,
                          int* status, int n_x, int N_tr, int N_ell, cudaStream_t s) {
  if (N_tr > 64) return cudaErrorInvalidValue;
  const size_t smem = 3 * sizeof(double) * N_tr * N_tr;
  cudaError_t e = cudaFuncSetAttribute(k_fisher_whiten, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_fisher_whiten<<<N_ell, 64, smem, s>>>(Z, X, U, amp, noise, modes, status, n_x, N_tr, N_ell);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_fisher_gram<<<n_x * (n_x + 1) / 2, GT, 0, s>>>(F, Z, n_x, N_tr, N_ell);
  return cudaGetLastError();
}

}  // namespace swcl
