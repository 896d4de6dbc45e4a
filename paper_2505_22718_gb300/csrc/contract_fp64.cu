// a3 in FP64 on CUDA cores: the contraction with k-interpolation (Eq. 3.3-3.5, Sec. 3.2)
//   Delta_i(l, q) = kpow_i[q] Re sum_n X_{i,q,n} G_{cls(i)}[l][n],
//   X_{i,q,n} = (sum_r lw[q][r] c_{i, j0[q]+r, n}) e^{-i eta_n ln k_q},
// and its adjoint for the VJP
//   cbar_{i,a,n} = sum_q lambda_{q,a} conj(E_{q,n}) kpow_i[q] sum_l Dbar_i(l,q) conj(G[l][n]).
// The A operand X is formed in shared memory by the loading threads (interpolation and phase),
// never stored in global memory.
#include "swcl_internal.h"

namespace swcl {
namespace {

constexpr int BQ = 64;    // k points per CTA
constexpr int BL = 128;   // multipoles per CTA
constexpr int BN = 8;     // complex coefficients per K step
constexpr int NT = 256;

__global__ void __launch_bounds__(NT)
k_contract_fp64(double* __restrict__ delta, const cplx* __restrict__ coef,
                const cplx* __restrict__ phase, const cplx* __restrict__ gtab,
                const int* __restrict__ cls_of, const double* __restrict__ kpow,
                const int* __restrict__ j0, const double* __restrict__ lw, long lw_ts, int N_tr,
                int N_I, int n_h, int N_k, int N_ell, int l_lo, int n_l) {
  // multipoles [l_lo, l_lo + n_l) into delta[w][l - l_lo][i][q]
  __shared__ cplx Xs[BN][BQ + 1];
  __shared__ cplx Gs[BN][BL + 1];
  const int q0 = blockIdx.x * BQ;
  const int l0 = blockIdx.y * BL;
  const int wi = blockIdx.z;  // walker * N_tr + tracer
  const int i = wi % N_tr;
  const int w = wi / N_tr;
  const cplx* cf = coef + (size_t)wi * N_I * n_h;
  const cplx* G = gtab + (size_t)cls_of[i] * N_ell * n_h;
  lw += (size_t)i * lw_ts;
  const int tq = threadIdx.x & 15;   // 4 consecutive q
  const int tl = threadIdx.x >> 4;   // 8 multipoles strided by 16
  double acc[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.0;

  for (int n0 = 0; n0 < n_h; n0 += BN) {
    // form X: BQ x BN, n fastest
    for (int e = threadIdx.x; e < BQ * BN; e += NT) {
      int nn = e % BN, ql = e / BN;
      int q = q0 + ql, n = n0 + nn;
      cplx x = {0.0, 0.0};
      if (q < N_k && n < n_h) {
        int s = j0[q];
        const double* wq = lw + (size_t)q * 4;
        double re = 0.0, im = 0.0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          double wr = wq[r];
          if (s + r < N_I && wr != 0.0) {
            cplx c = cf[(size_t)(s + r) * n_h + n];
            re = fma(wr, c.x, re);
            im = fma(wr, c.y, im);
          }
        }
        cplx e2 = phase[(size_t)q * n_h + n];
        x = {fma(re, e2.x, -im * e2.y), fma(re, e2.y, im * e2.x)};
      }
      Xs[nn][ql] = x;
    }
    for (int e = threadIdx.x; e < BL * BN; e += NT) {
      int nn = e % BN, ll = e / BN;
      int l = l0 + ll, n = n0 + nn;
      Gs[nn][ll] = (l < n_l && n < n_h) ? G[(size_t)(l_lo + l) * n_h + n] : cplx{0.0, 0.0};
    }
    __syncthreads();
#pragma unroll
    for (int nn = 0; nn < BN; ++nn) {
      cplx xv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) xv[a] = Xs[nn][tq * 4 + a];
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        cplx g = Gs[nn][tl + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[a][b] = fma(xv[a].x, g.x, fma(-xv[a].y, g.y, acc[a][b]));
      }
    }
    __syncthreads();
  }
  const double* kp = kpow + (size_t)i * N_k;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    int l = l0 + tl + 16 * b;
    if (l >= n_l) continue;
    double* out = delta + (((size_t)w * n_l + l) * N_tr + i) * N_k;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      int q = q0 + tq * 4 + a;
      if (q < N_k) out[q] = kp[q] * acc[a][b];
    }
  }
}

// adjoint tile: 64 k points x 32 complex coefficients, K loop over multipoles
constexpr int AQ = 64;
constexpr int AN = 32;
constexpr int AL = 8;

__global__ void __launch_bounds__(NT)
k_contract_fp64_adj(cplx* __restrict__ cbar, const double* __restrict__ dbar,
                    const cplx* __restrict__ phase, const cplx* __restrict__ gtab,
                    const int* __restrict__ cls_of, const double* __restrict__ kpow,
                    const int* __restrict__ j0, const double* __restrict__ lw, long lw_ts,
                    int N_tr, int N_I, int n_h, int N_k, int N_ell, int l_lo, int n_l) {
  // dbar holds multipoles [l_lo, l_lo + n_l); cbar accumulates (zeroed by the caller)
  __shared__ double Ds[AL][AQ + 1];
  __shared__ cplx Gs[AL][AN + 1];
  __shared__ cplx V[AQ][AN + 1];
  const int q0 = blockIdx.x * AQ;
  const int nb = blockIdx.y * AN;
  const int wi = blockIdx.z;
  const int i = wi % N_tr;
  const int w = wi / N_tr;
  const cplx* G = gtab + (size_t)cls_of[i] * N_ell * n_h;
  lw += (size_t)i * lw_ts;
  // thread micro-tile: 2 q x 4 n
  const int tn = threadIdx.x & 7;    // n = tn + 8 b
  const int tq = threadIdx.x >> 3;   // q = tq + 32 a
  double ar[2][4], ai[2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { ar[a][b] = 0.0; ai[a][b] = 0.0; }
  for (int l0 = 0; l0 < n_l; l0 += AL) {
    for (int e = threadIdx.x; e < AL * AQ; e += NT) {
      int ql = e % AQ, ll = e / AQ;
      int q = q0 + ql, l = l0 + ll;
      Ds[ll][ql] = (q < N_k && l < n_l)
                       ? dbar[(((size_t)w * n_l + l) * N_tr + i) * N_k + q] : 0.0;
    }
    for (int e = threadIdx.x; e < AL * AN; e += NT) {
      int nn = e % AN, ll = e / AN;
      int n = nb + nn, l = l0 + ll;
      Gs[ll][nn] = (n < n_h && l < n_l) ? G[(size_t)(l_lo + l) * n_h + n] : cplx{0.0, 0.0};
    }
    __syncthreads();
#pragma unroll
    for (int ll = 0; ll < AL; ++ll) {
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        double d = Ds[ll][tq + 32 * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          cplx g = Gs[ll][tn + 8 * b];
          ar[a][b] = fma(d, g.x, ar[a][b]);
          ai[a][b] = fma(-d, g.y, ai[a][b]);
        }
      }
    }
    __syncthreads();
  }
  // v = kpow * acc * conj(E)
  const double* kp = kpow + (size_t)i * N_k;
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    int ql = tq + 32 * a;
    int q = q0 + ql;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int nn = tn + 8 * b;
      int n = nb + nn;
      cplx v = {0.0, 0.0};
      if (q < N_k && n < n_h) {
        cplx e2 = phase[(size_t)q * n_h + n];
        double xr = kp[q] * ar[a][b], xi = kp[q] * ai[a][b];
        v = {fma(xr, e2.x, xi * e2.y), fma(xi, e2.x, -xr * e2.y)};
      }
      V[ql][nn] = v;
    }
  }
  __syncthreads();
  // scatter to knots: thread (column nn, segment of 8 q) with a sliding window of 4 knots
  {
    const int nn = threadIdx.x & 31;
    const int seg = threadIdx.x >> 5;  // 8 segments of 8 k points
    const int n = nb + nn;
    if (n < n_h) {
      cplx* out = cbar + (size_t)wi * N_I * n_h + n;
      int base = -1;
      cplx win[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
      for (int t = 0; t < 8; ++t) {
        int ql = seg * 8 + t;
        int q = q0 + ql;
        if (q >= N_k) break;
        int s = j0[q];
        if (base < 0) base = s;
        while (base < s) {  // flush knot `base`
          if (win[0].x != 0.0 || win[0].y != 0.0) {
            atomicAdd(&out[(size_t)base * n_h].x, win[0].x);
            atomicAdd(&out[(size_t)base * n_h].y, win[0].y);
          }
          win[0] = win[1]; win[1] = win[2]; win[2] = win[3]; win[3] = {0.0, 0.0};
          ++base;
        }
        cplx v = V[ql][nn];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          double wr = lw[(size_t)q * 4 + r];
          win[r].x = fma(wr, v.x, win[r].x);
          win[r].y = fma(wr, v.y, win[r].y);
        }
      }
      if (base >= 0) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          if (base + r < N_I && (win[r].x != 0.0 || win[r].y != 0.0)) {
            atomicAdd(&out[(size_t)(base + r) * n_h].x, win[r].x);
            atomicAdd(&out[(size_t)(base + r) * n_h].y, win[r].y);
          }
        }
      }
    }
  }
}

}  // namespace

cudaError_t launch_contract_fp64(double* delta, const cplx* coef, const cplx* phase,
                                 const cplx* gtab, const int* cls_of, const double* kpow,
                                 const int* j0, const double* lw, long lw_ts, int n_walk,
                                 int N_tr, int N_I, int n_h, int N_k, int N_ell, int l_lo,
                                 int n_l, cudaStream_t s) {
  dim3 g((N_k + BQ - 1) / BQ, (n_l + BL - 1) / BL, n_walk * N_tr);
  k_contract_fp64<<<g, NT, 0, s>>>(delta, coef, phase, gtab, cls_of, kpow, j0, lw, lw_ts, N_tr,
                                    N_I, n_h, N_k, N_ell, l_lo, n_l);
  return cudaGetLastError();
}

cudaError_t launch_contract_fp64_adj(cplx* cbar, const double* dbar, const cplx* phase,
                                     const cplx* gtab, const int* cls_of, const double* kpow,
                                     const int* j0, const double* lw, long lw_ts, int n_walk,
                                     int N_tr, int N_I, int n_h, int N_k, int N_ell, int l_lo,
                                     int n_l, bool accumulate, cudaStream_t s) {
  if (!accumulate) {
    cudaError_t e = cudaMemsetAsync(cbar, 0, (size_t)n_walk * N_tr * N_I * n_h * sizeof(cplx), s);
    if (e != cudaSuccess) return e;
  }
  dim3 g((N_k + AQ - 1) / AQ, (n_h + AN - 1) / AN, n_walk * N_tr);
  k_contract_fp64_adj<<<g, NT, 0, s>>>(cbar, dbar, phase, gtab, cls_of, kpow, j0, lw, lw_ts, N_tr,
                                        N_I, n_h, N_k, N_ell, l_lo, n_l);
  return cudaGetLastError();
}

}  // namespace swcl
