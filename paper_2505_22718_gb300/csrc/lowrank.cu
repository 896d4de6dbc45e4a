// Low-rank knot profiles (the GPU path's reorganisation of Sec. 3.2's per-knot FFTLog).
//
// The FFTLog input of tracer i at knot a is g_{i,a}(chi_m) = W'_i(chi_m) G_i[a][m] with the knot
// profile G_i[a][m] = D(kappa_a, chi_m) B_i(kappa_a, chi_m) (B = 1 when absent: one profile for all
// tracers).  When G_i = sum_{s<r} coef_i[a][s] Q_i[s][m] holds to rounding with a small r, the
// FFT is linear, so
//   c_{i,a,n} = sum_s coef_i[a][s] FFT(W'_i Q_i[s])_n,
// and the k-interpolation c_{i,n}(k_q) = sum_a lambda_{q,a} c_{i,a,n} becomes
//   c_{i,n}(k_q) = sum_s mu_i[q][s] F_{i,s,n},   mu_i[q][s] = sum_a lambda_{q,a} coef_i[a][s].
// The contraction kernels read (j0, weights) stencils either way: knots with the 4-point Lagrange
// weights, or the r <= 4 basis profiles with j0 = 0 and the weights mu.  The reverse mode follows
// by the same linearity.
//
// Q and coef come from modified Gram-Schmidt with column pivoting on the rows of G (largest
// residual row first, each new direction orthogonalised twice), all in FP64; the rank is the
// number of directions taken before every residual row norm is below 1e-14 of the largest row
// norm of G (or 4 directions have been taken, in which case the per-knot FFT is used).
#include <algorithm>
#include <cmath>
#include <vector>

#include "swcl_internal.h"

namespace swcl {
namespace {

constexpr int kT = 256;

__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  double r = red[0];
  __syncthreads();
  return r;
}

// res[a] = G[a] (profile rows of tracer-profile p), norms[a] = |res[a]|^2
__global__ void k_lr_init(double* __restrict__ res, double* __restrict__ norms,
                          const double* __restrict__ D, const double* __restrict__ B, int N_I,
                          int N, int p, int per_tracer) {
  __shared__ double red[kT];
  const int a = blockIdx.x;
  double s = 0.0;
  for (int m = threadIdx.x; m < N; m += kT) {
    double v = D[(size_t)a * N + m];
    if (per_tracer) v *= B[((size_t)p * N_I + a) * N + m];
    res[(size_t)a * N + m] = v;
    s = fma(v, v, s);
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) norms[a] = s;
}

// q = res[piv] / |res[piv]|
__global__ void k_lr_pivot(double* __restrict__ q, const double* __restrict__ res,
                           const double* __restrict__ norms, int piv, int N) {
  const double inv = 1.0 / sqrt(norms[piv]);
  for (int m = blockIdx.x * kT + threadIdx.x; m < N; m += gridDim.x * kT)
    q[m] = res[(size_t)piv * N + m] * inv;
}

// coef[a] += <res[a], q>;  res[a] -= <res[a], q> q;  norms[a] = |res[a]|^2
__global__ void k_lr_project(double* __restrict__ res, double* __restrict__ coef,
                             double* __restrict__ norms, const double* __restrict__ q, int N,
                             int r_stride, int s_idx) {
  __shared__ double red[kT];
  const int a = blockIdx.x;
  double* row = res + (size_t)a * N;
  double d = 0.0;
  for (int m = threadIdx.x; m < N; m += kT) d = fma(row[m], q[m], d);
  d = block_sum(d, red);
  double s = 0.0;
  for (int m = threadIdx.x; m < N; m += kT) {
    const double v = fma(-d, q[m], row[m]);
    row[m] = v;
    s = fma(v, v, s);
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    coef[(size_t)a * r_stride + s_idx] += d;
    norms[a] = s;
  }
}

// mu[q][s] = sum_a lambda[q][a] coef[a][s] (lambda as the 4-point stencil j0/lw)
__global__ void k_lr_mu(double* __restrict__ mu, const int* __restrict__ j0,
                        const double* __restrict__ lw, const double* __restrict__ coef, int N_k,
                        int N_I, int r_stride) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N_k) return;
  for (int s = 0; s < 4; ++s) {
    double v = 0.0;
    if (s < r_stride)
      for (int t = 0; t < 4; ++t) {
        const int a = j0[q] + t;
        if (a < N_I) v = fma(lw[(size_t)q * 4 + t], coef[(size_t)a * r_stride + s], v);
      }
    mu[(size_t)q * 4 + s] = v;
  }
}

__global__ void k_zero_int(int* p, int n) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) p[t] = 0;
}

// c[row][a][n] = sum_s coef[a][s] F[row][s][n] (knot coefficients from the basis, for read-back)
__global__ void k_lr_expand(cplx* __restrict__ c, const cplx* __restrict__ F,
                            const double* __restrict__ coef, int n_rows, int N_I, int r, int n_h,
                            long coef_row_stride, int N_tr) {
  // F holds r basis rows per (walker, tracer); coef rows have a stride of 4
  const long total = (long)n_rows * N_I * n_h;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int n = (int)(e % n_h);
    const int a = (int)((e / n_h) % N_I);
    const int row = (int)(e / ((long)n_h * N_I));
    const double* cf = coef + (size_t)(row % N_tr) * coef_row_stride + (size_t)a * 4;
    double xr = 0.0, xi = 0.0;
    for (int s = 0; s < r; ++s) {
      const cplx f = F[((size_t)row * r + s) * n_h + n];
      xr = fma(cf[s], f.x, xr);
      xi = fma(cf[s], f.y, xi);
    }
    c[e] = {xr, xi};
  }
}

__global__ void k_lr_expand_df(cplx* __restrict__ c, const float4* __restrict__ F,
                               const double* __restrict__ coef, int n_rows, int N_I, int r,
                               int n_h, long coef_row_stride, int N_tr) {
  const long total = (long)n_rows * N_I * n_h;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int n = (int)(e % n_h);
    const int a = (int)((e / n_h) % N_I);
    const int row = (int)(e / ((long)n_h * N_I));
    const double* cf = coef + (size_t)(row % N_tr) * coef_row_stride + (size_t)a * 4;
    double xr = 0.0, xi = 0.0;
    for (int s = 0; s < r; ++s) {
      const float4 f = F[((size_t)row * r + s) * n_h + n];
      xr = fma(cf[s], (double)f.x + (double)f.z, xr);
      xi = fma(cf[s], (double)f.y + (double)f.w, xi);
    }
    c[e] = {xr, xi};
  }
}

}  // namespace

// Factorise the knot profiles of the context's D (and B).  On success with rank <= 4 the context
// switches to basis mode: lr_Q [n_prof][4][N] profiles (unused rows zero), lr_coef
// [n_prof][N_I][4], lr_j0 (zeros) and lr_w ([N_tr-shared] mu weights; with per-tracer profiles the
// weights are per tracer: [N_tr][N_k][4]).
int factor_profiles(swcl_ctx* c) {
  c->lr_basis = false;
  c->lr_rank = 0;
  if (c->lr_disabled) return SWCL_OK;
  const int N_I = c->N_I, N = c->N, N_k = c->N_k;
  if (N_I <= 4) return SWCL_OK;               // nothing to gain
  const int n_prof = c->have_B ? c->N_tr : 1;
  constexpr int RMAX = 4;
  int st;
  if ((st = ensure(c, c->lr_res, sizeof(double) * (size_t)N_I * N))) return st;
  if ((st = ensure(c, c->lr_norms, sizeof(double) * N_I))) return st;
  if ((st = ensure(c, c->lr_Q, sizeof(double) * (size_t)n_prof * RMAX * N))) return st;
  if ((st = ensure(c, c->lr_coef, sizeof(double) * (size_t)n_prof * N_I * RMAX))) return st;
  cudaStream_t s = c->stream;
  cudaError_t e = cudaMemsetAsync(c->lr_Q.p, 0, sizeof(double) * (size_t)n_prof * RMAX * N, s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(c->lr_coef.p, 0, sizeof(double) * (size_t)n_prof * N_I * RMAX, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "low-rank init");
  std::vector<double> norms(N_I);
  int rank = 0;
  for (int p = 0; p < n_prof; ++p) {
    double* res = (double*)c->lr_res.p;
    double* nrm = (double*)c->lr_norms.p;
    double* Q = (double*)c->lr_Q.p + (size_t)p * RMAX * N;
    double* coef = (double*)c->lr_coef.p + (size_t)p * N_I * RMAX;
    k_lr_init<<<N_I, kT, 0, s>>>(res, nrm, (const double*)c->d_D.p,
                                 c->have_B ? (const double*)c->d_B.p : nullptr, N_I, N, p,
                                 c->have_B ? 1 : 0);
    e = cudaMemcpyAsync(norms.data(), nrm, sizeof(double) * N_I, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "low-rank norms");
    const double n0 = *std::max_element(norms.begin(), norms.end());
    const double tol2 = 1e-28 * n0;   // (1e-14)^2 of the largest squared row norm
    int r = 0;
    while (true) {
      int piv = (int)(std::max_element(norms.begin(), norms.end()) - norms.begin());
      if (n0 == 0.0 || norms[piv] <= tol2) break;
      if (r == RMAX) { r = RMAX + 1; break; }
      double* q = Q + (size_t)r * N;
      k_lr_pivot<<<(N + kT - 1) / kT, kT, 0, s>>>(q, res, nrm, piv, N);
      // project every row on q twice (the second pass removes what the first left behind)
      k_lr_project<<<N_I, kT, 0, s>>>(res, coef, nrm, q, N, RMAX, r);
      k_lr_project<<<N_I, kT, 0, s>>>(res, coef, nrm, q, N, RMAX, r);
      e = cudaMemcpyAsync(norms.data(), nrm, sizeof(double) * N_I, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(c, e, "low-rank step");
      ++r;
    }
    if (r > RMAX) return SWCL_OK;             // not low rank: keep the per-knot FFT
    rank = std::max(rank, r);
  }
  if (rank == 0) return SWCL_OK;
  // mu weights and zero stencil starts
  const int n_w = n_prof;                     // one weight set per profile
  if ((st = ensure(c, c->lr_w, sizeof(double) * (size_t)n_w * N_k * 4))) return st;
  if ((st = ensure(c, c->lr_j0, sizeof(int) * N_k))) return st;
  for (int p = 0; p < n_w; ++p)
    k_lr_mu<<<(N_k + 127) / 128, 128, 0, s>>>((double*)c->lr_w.p + (size_t)p * N_k * 4,
                                              (const int*)c->d_interp_j0.p,
                                              (const double*)c->d_interp_w.p,
                                              (const double*)c->lr_coef.p + (size_t)p * N_I * RMAX,
                                              N_k, N_I, RMAX);
  k_zero_int<<<(N_k + 255) / 256, 256, 0, s>>>((int*)c->lr_j0.p, N_k);
  // the profile rows the FFT multiplies by: shared Q as "D" (B = null), or per-tracer Q as "B"
  // with an all-ones "D"
  if (c->have_B) {
    if ((st = ensure(c, c->lr_ones, sizeof(double) * (size_t)RMAX * N))) return st;
    std::vector<double> ones((size_t)RMAX * N, 1.0);
    e = cudaMemcpyAsync(c->lr_ones.p, ones.data(), sizeof(double) * ones.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "low-rank ones");
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "low-rank factorisation");
  c->lr_rank = c->have_B ? RMAX : rank;   // per-tracer profiles keep 4 (zero-padded) rows
  c->lr_true_rank = rank;
  c->lr_basis = true;
  for (auto& t : c->tc) t.ready = t.adj_ready = false;   // stencil weights changed
  c->bt_ready = false;
  ++c->alloc_gen;
  return SWCL_OK;
}

// knot coefficients c[w][i][a][n] (FP64) from the basis coefficients in ws_coef, for read-back
int expand_basis_coefficients(swcl_ctx* c, void* out, bool df_input) {
  const int n_rows = c->n_walk * c->N_tr;
  const long total = (long)n_rows * c->N_I * c->n_h;
  const long stride = c->have_B ? (long)c->N_I * 4 : 0;
  const int r = stencil(c).NI;
  const unsigned grid = (unsigned)std::min<long>((total + 255) / 256, 152L * 64);
  if (df_input)
    k_lr_expand_df<<<grid, 256, 0, c->stream>>>((cplx*)out, (const float4*)c->ws_coef.p,
                                                (const double*)c->lr_coef.p, n_rows, c->N_I, r,
                                                c->n_h, stride, c->N_tr);
  else
    k_lr_expand<<<grid, 256, 0, c->stream>>>((cplx*)out, (const cplx*)c->ws_coef.p,
                                             (const double*)c->lr_coef.p, n_rows, c->N_I, r,
                                             c->n_h, stride, c->N_tr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "basis expansion");
  return SWCL_OK;
}

}  // namespace swcl
