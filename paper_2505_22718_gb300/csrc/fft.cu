// a1: FFTLog coefficients of every window at every k-knot (Sec. 3.1-3.2, Eq. 3.2-3.3), FP64,
// and the adjoint used by the VJP.
//
// One CTA transforms one or more rows (walker, tracer, knot).  The real length-N sequence
// g_m = W_i(chi_m) * chipow_i[m] * D_a[m] * B_ia[m] is packed as N/2 complex points
// z_j = g_{2j} + i g_{2j+1}, transformed by a radix-4 (plus one radix-2) Stockham FFT in shared
// memory, and unpacked to X_n = sum_m g_m e^{-2 pi i n m/N}, n = 0..N/2.  The coefficient is
// c_n = psi_i[n] X_n with psi = T_c chi_min^{-i eta_n}/N.  Twiddles come from a table
// e^{-2 pi i t/N}, t < N, so the only FP64 arithmetic is the butterflies themselves.
#include <cooperative_groups.h>

#include "swcl_internal.h"

namespace cg = cooperative_groups;

namespace swcl {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return {fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x)};
}
__device__ __forceinline__ cplx cmulc(cplx a, cplx b) {  // a * conj(b)
  return {fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y)};
}
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cplx cconj(cplx a) { return {a.x, -a.y}; }

// Forward DFT of n2 = N/2 points held in buffers a/b (ping-pong) for `rows` rows laid out
// row-major with stride n2; returns the buffer holding the result.  Stockham autosort:
// pass with radix R and span Ns maps j -> (j/Ns)*Ns*R + j%Ns with twiddle
// e^{-2 pi i (j%Ns) r / (Ns R)} = tw[(j%Ns) r (N/(Ns R))].
__device__ cplx* stockham(cplx* a, cplx* b, int n2, int rows, const cplx* __restrict__ tw,
                          int N) {
  int lg = 31 - __clz(n2);
  int Ns = 1;
  if (lg & 1) {
    // radix-2 pass, trivial twiddles (Ns = 1)
    int nb = n2 / 2;
    for (int g = threadIdx.x; g < rows * nb; g += blockDim.x) {
      int r = g / nb, j = g - r * nb;
      const cplx* x = a + r * n2;
      cplx* y = b + r * n2;
      cplx v0 = x[j], v1 = x[j + nb];
      y[2 * j] = cadd(v0, v1);
      y[2 * j + 1] = csub(v0, v1);
    }
    __syncthreads();
    cplx* t = a; a = b; b = t;
    Ns = 2;
  }
  int nb = n2 / 4;
  for (; Ns < n2; Ns *= 4) {
    int tstep = N / (Ns * 4);
    for (int g = threadIdx.x; g < rows * nb; g += blockDim.x) {
      int r = g / nb, j = g - r * nb;
      const cplx* x = a + r * n2;
      cplx* y = b + r * n2;
      int jm = j & (Ns - 1);
      cplx v0 = x[j], v1 = x[j + nb], v2 = x[j + 2 * nb], v3 = x[j + 3 * nb];
      if (Ns > 1) {
        int t1 = jm * tstep;
        v1 = cmul(v1, tw[t1]);
        v2 = cmul(v2, tw[2 * t1]);
        v3 = cmul(v3, tw[3 * t1]);
      }
      // 4-point DFT (e^{-2 pi i/4} = -i)
      cplx s02 = cadd(v0, v2), d02 = csub(v0, v2);
      cplx s13 = cadd(v1, v3), d13 = csub(v1, v3);
      cplx md13 = {d13.y, -d13.x};  // -i * d13
      int o = (j - jm) * 4 + jm;
      y[o] = cadd(s02, s13);
      y[o + Ns] = cadd(d02, md13);
      y[o + 2 * Ns] = csub(s02, s13);
      y[o + 3 * Ns] = csub(d02, md13);
    }
    __syncthreads();
    cplx* t = a; a = b; b = t;
  }
  return a;
}

// rows per CTA: enough independent transforms to give every thread work
__host__ __device__ inline int rows_per_cta(int N) {
  int n2 = N / 2;
  int r = (4 * kThreads) / n2;
  return r < 1 ? 1 : r;
}

__device__ __forceinline__ void store_coef(cplx* p, cplx v) { *p = v; }
// double-float pair (re_hi, im_hi, re_lo, im_lo): hi = fl32(v), lo = fl32(v - hi)
__device__ __forceinline__ void store_coef(float4* p, cplx v) {
  const float rh = (float)v.x, ih = (float)v.y;
  *p = make_float4(rh, ih, (float)(v.x - (double)rh), (float)(v.y - (double)ih));
}

template <typename CT>
__global__ void __launch_bounds__(kThreads)
k_fftlog_fwd(CT* __restrict__ coef, const double* __restrict__ W,
             const double* __restrict__ chipow, const double* __restrict__ D,
             const double* __restrict__ B, const cplx* __restrict__ psi,
             const cplx* __restrict__ tw, int n_walk, int N_tr, int N_I, int N) {
  pdl_trigger();   // the next kernel of the step may be scheduled
  pdl_wait();      // every earlier kernel of the step has completed
  extern __shared__ cplx smem[];
  const int n2 = N / 2, n_h = N / 2 + 1;
  const int R = rows_per_cta(N);
  const long total_rows = (long)n_walk * N_tr * N_I;
  const long row0 = (long)blockIdx.x * R;
  int rows = (int)min((long)R, total_rows - row0);
  cplx* a = smem;
  cplx* b = smem + R * n2;
  // load and pack
  for (int g = threadIdx.x; g < rows * n2; g += blockDim.x) {
    int r = g / n2, j = g - r * n2;
    long row = row0 + r;
    int ka = (int)(row % N_I);
    long wi = row / N_I;  // walker * N_tr + tracer
    int i = (int)(wi % N_tr);
    const double* w = W + wi * N;
    const double* cp = chipow + (size_t)i * N;
    const double* d = D + (size_t)ka * N;
    int m = 2 * j;
    double g0 = w[m] * cp[m] * d[m];
    double g1 = w[m + 1] * cp[m + 1] * d[m + 1];
    if (B) {
      const double* bb = B + ((size_t)i * N_I + ka) * N;
      g0 *= bb[m];
      g1 *= bb[m + 1];
    }
    a[r * n2 + j] = {g0, g1};
  }
  __syncthreads();
  cplx* Z = stockham(a, b, n2, rows, tw, N);
  // unpack: X_n = E_n + e^{-2 pi i n/N} O_n, E = (Z_n + conj Z_{n2-n})/2, O = (Z_n - conj Z_{n2-n})/(2i)
  for (int g = threadIdx.x; g < rows * n_h; g += blockDim.x) {
    int r = g / n_h, n = g - r * n_h;
    long row = row0 + r;
    int i = (int)((row / N_I) % N_tr);
    const cplx* z = Z + r * n2;
    cplx zn = z[n == n2 ? 0 : n];
    cplx zc = cconj(z[n == 0 ? 0 : n2 - n]);
    cplx e = {0.5 * (zn.x + zc.x), 0.5 * (zn.y + zc.y)};
    cplx dlt = {0.5 * (zn.x - zc.x), 0.5 * (zn.y - zc.y)};
    cplx o = {dlt.y, -dlt.x};  // dlt / i
    cplx x = cadd(e, cmul(tw[n], o));
    store_coef(coef + row * n_h + n, cmul(psi[(size_t)i * n_h + n], x));
  }
}

// Adjoint.  For row (w, i, a): Y_n = conj(psi_n) cbar_n, H_0 = Re Y_0, H_{N/2} = Re Y_{N/2},
// H_n = Y_n / 2 otherwise; gbar_m = sum_{n<N} H_n e^{+2 pi i n m/N} (Hermitian H), computed as
// x_{2j} + i x_{2j+1} = sum_n (E_n + i O_n) e^{+2 pi i n j/(N/2)} with
// E_n = H_n + conj H_{n2-n}, O_n = (H_n - conj H_{n2-n}) e^{+2 pi i n/N}; the inverse transform is
// conj(FFT(conj(.))).  Each CTA sums gbar * chipow * D_a * B_ia over a chunk of knots of one
// (walker, tracer) into scratch[chunk][w*N_tr+i][m].
constexpr int kKnotChunk = 16;

__global__ void __launch_bounds__(kThreads)
k_fftlog_adj(double* __restrict__ scratch, const cplx* __restrict__ cbar,
             const double* __restrict__ chipow, const double* __restrict__ D,
             const double* __restrict__ B, const cplx* __restrict__ psi,
             const cplx* __restrict__ tw, int n_walk, int N_tr, int N_I, int N) {
  pdl_trigger();   // the next kernel of the step may be scheduled
  pdl_wait();      // every earlier kernel of the step has completed
  extern __shared__ cplx smem[];
  const int n2 = N / 2, n_h = N / 2 + 1;
  cplx* a = smem;
  cplx* b = smem + n2;
  double* acc = reinterpret_cast<double*>(smem + 2 * n2);
  const int wi = blockIdx.y;          // walker * N_tr + tracer
  const int i = wi % N_tr;
  const int chunk = blockIdx.x;
  const int a0 = chunk * kKnotChunk;
  const int a1 = min(N_I, a0 + kKnotChunk);
  for (int m = threadIdx.x; m < N; m += blockDim.x) acc[m] = 0.0;
  const cplx* ps = psi + (size_t)i * n_h;
  for (int ka = a0; ka < a1; ++ka) {
    const cplx* cb = cbar + ((size_t)wi * N_I + ka) * n_h;
    for (int n = threadIdx.x; n < n2; n += blockDim.x) {
      // H_n and conj H_{n2-n}
      cplx y = cmulc(cb[n], ps[n]);           // cbar * conj(psi) ... conj(psi) cbar
      cplx h = (n == 0) ? cplx{y.x, 0.0} : cplx{0.5 * y.x, 0.5 * y.y};
      int m = n2 - n;
      cplx ym = cmulc(cb[m], ps[m]);
      cplx hm = (m == n2) ? cplx{ym.x, 0.0} : cplx{0.5 * ym.x, 0.5 * ym.y};
      cplx hmc = cconj(hm);
      cplx e = cadd(h, hmc);
      cplx d = csub(h, hmc);
      cplx o = cmulc(d, tw[n]);                // * e^{+2 pi i n/N}
      // Z = E + i O, store conj(Z) for the forward transform
      cplx z = {e.x - o.y, e.y + o.x};
      a[n] = cconj(z);
    }
    __syncthreads();
    cplx* Z = stockham(a, b, n2, 1, tw, N);
    const double* cp = chipow + (size_t)i * N;
    const double* d = D + (size_t)ka * N;
    const double* bb = B ? B + ((size_t)i * N_I + ka) * N : nullptr;
    for (int j = threadIdx.x; j < n2; j += blockDim.x) {
      cplx v = cconj(Z[j]);
      int m = 2 * j;
      double f0 = cp[m] * d[m], f1 = cp[m + 1] * d[m + 1];
      if (bb) { f0 *= bb[m]; f1 *= bb[m + 1]; }
      acc[m] = fma(v.x, f0, acc[m]);
      acc[m + 1] = fma(v.y, f1, acc[m + 1]);
    }
    __syncthreads();
  }
  double* out = scratch + ((size_t)chunk * n_walk * N_tr + wi) * N;
  for (int m = threadIdx.x; m < N; m += blockDim.x) out[m] = acc[m];
}

__global__ void k_sum_chunks(double* __restrict__ W_bar, const double* __restrict__ scratch,
                             long per_chunk, int nchunk, int* __restrict__ status) {
  pdl_trigger();   // the next kernel of the step may be scheduled
  pdl_wait();      // every earlier kernel of the step has completed
  long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per_chunk) return;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += scratch[(size_t)c * per_chunk + t];
  flag_nonfinite(status, s);
  W_bar[t] = s;
}

// ---------------------------------------------------------------- cluster form ----
// With few rows (one walker in basis mode: one row per tracer) one CTA per row leaves most SMs
// idle, and each row is bound by its SM's FP64 pipe.  A cluster of kCl CTAs then shares a row:
// four-step DFT of the M = N/2 packed points with n = n1 + kCl t (CTA n1 holds t = 0..L-1,
// L = M/kCl) and k = k2 + L k1:
//   X[k2 + L k1] = sum_{n1} w_M^{n1 k2} w_kCl^{n1 k1} Y_{n1}[k2],  Y_{n1} = DFT_L(z[n1 + kCl t]).
// Step 1 runs in each CTA (Stockham in shared memory), step 2 (the kCl-point DFTs, each CTA a
// slice of k2) reads the other CTAs' Y through distributed shared memory.
constexpr int kCl = 8;
constexpr int kClThreads = 256;

__device__ __forceinline__ cplx tw_mod(const cplx* tw, long x, int N) { return tw[x & (N - 1)]; }

// 4-point DFT of (y0, y1, y2, y3) stored at o[off], o[off + 2], o[off + 4], o[off + 6]
__device__ __forceinline__ void dft4_strided(cplx y0, cplx y1, cplx y2, cplx y3, cplx* o, int off) {
  const cplx s02 = cadd(y0, y2), d02 = csub(y0, y2);
  const cplx s13 = cadd(y1, y3), d13 = csub(y1, y3);
  const cplx md13 = {d13.y, -d13.x};  // -i * d13
  o[off] = cadd(s02, s13);
  o[off + 2] = cadd(d02, md13);
  o[off + 4] = csub(s02, s13);
  o[off + 6] = csub(d02, md13);
}

// kCl-point DFTs of step 2 for this CTA's slice of k2: Xo[e kCl + k1] (e = k2 - rank kq),
// X_{k1} = sum_{n1} w_8^{n1 k1} Y_{n1}[k2], as one radix-2 split into two 4-point DFTs (the
// twiddles w_8^j are 1, (1 - i)/sqrt 2, -i, -(1 + i)/sqrt 2)
__device__ __forceinline__ void step2(cg::cluster_group& cl, cplx* Xo, cplx* Y, int L) {
  static_assert(kCl == 8, "step 2 is an 8-point DFT");
  constexpr double h = 0.70710678118654752440;   // 1/sqrt 2
  const int kq = L / kCl;
  const int c = cl.block_rank();
  for (int e = threadIdx.x; e < kq; e += blockDim.x) {
    const int k2 = c * kq + e;
    cplx x[kCl];
#pragma unroll
    for (int n1 = 0; n1 < kCl; ++n1) x[n1] = cl.map_shared_rank(Y, n1)[k2];
    const cplx d1 = csub(x[1], x[5]), d2 = csub(x[2], x[6]), d3 = csub(x[3], x[7]);
    const cplx b1 = {(d1.x + d1.y) * h, (d1.y - d1.x) * h};
    const cplx b2 = {d2.y, -d2.x};
    const cplx b3 = {(d3.y - d3.x) * h, -(d3.x + d3.y) * h};
    cplx* o = Xo + e * kCl;
    dft4_strided(cadd(x[0], x[4]), cadd(x[1], x[5]), cadd(x[2], x[6]), cadd(x[3], x[7]), o, 0);
    dft4_strided(csub(x[0], x[4]), b1, b2, b3, o, 1);
  }
}

// Twiddle tables of one cluster CTA in shared memory, loaded before the first transform:
// tws[m] = tw[m N / L] (the L-point Stockham's own table: the same values it would read from
// tw) and twc[k2] = w_M^{c k2}
__device__ __forceinline__ void load_cluster_twiddles(cplx* tws, cplx* twc, const cplx* tw, int L,
                                                      int N, int c) {
  for (int m = threadIdx.x; m < L; m += blockDim.x) {
    tws[m] = tw[(size_t)m * (N / L)];
    twc[m] = tw_mod(tw, 2L * c * m, N);
  }
}

template <typename CT>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kClThreads)
k_fftlog_fwd_cl(CT* __restrict__ coef, const double* __restrict__ W,
                const double* __restrict__ chipow, const double* __restrict__ D,
                const double* __restrict__ B, const cplx* __restrict__ psi,
                const cplx* __restrict__ tw, int N_tr, int N_I, int N) {
  pdl_trigger();   // the next kernel of the step may be scheduled
  pdl_wait();      // every earlier kernel of the step has completed
  extern __shared__ cplx smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  const int M = N / 2, L = M / kCl, kq = L / kCl, n_h = M + 1;
  cplx* a = smem;
  cplx* b = smem + L;
  cplx* Xo = smem + 2 * L;
  cplx* tws = smem + 3 * L;
  cplx* twc = smem + 4 * L;
  cplx* twn = smem + 5 * L;        // [L + 1]: tw[n] and psi_i[n] of this CTA's unpack outputs
  cplx* psn = smem + 6 * L + 1;    // [L + 1]
  const long row = blockIdx.x / kCl;
  const int ka = (int)(row % N_I);
  const long wi = row / N_I;
  const int i = (int)(wi % N_tr);
  const double* w = W + wi * N;
  const double* cp = chipow + (size_t)i * N;
  const double* d = D + (size_t)ka * N;
  const double* bb = B ? B + ((size_t)i * N_I + ka) * N : nullptr;
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    const int m = 2 * (c + kCl * t);
    double g0 = w[m] * cp[m] * d[m];
    double g1 = w[m + 1] * cp[m + 1] * d[m + 1];
    if (bb) { g0 *= bb[m]; g1 *= bb[m + 1]; }
    a[t] = {g0, g1};
  }
  load_cluster_twiddles(tws, twc, tw, L, N, c);
  for (int o = threadIdx.x; o <= L; o += blockDim.x) {
    int n = M;                                                     // o = L: the Nyquist point
    if (o < L) {
      const int e = o / kCl, k1 = o - e * kCl;
      n = c * kq + e + L * k1;
    }
    twn[o] = tw[n];
    psn[o] = psi[(size_t)i * n_h + n];
  }
  __syncthreads();
  cplx* Y = stockham(a, b, L, 1, tws, L);
  for (int k2 = threadIdx.x; k2 < L; k2 += blockDim.x)
    Y[k2] = cmul(Y[k2], twc[k2]);                                  // w_M^{c k2}
  cl.sync();
  step2(cl, Xo, Y, L);
  cl.sync();
  // unpack X_n = E_n + e^{-2 pi i n/N} O_n with Z_{M-n} from the CTA that holds it
  for (int o = threadIdx.x; o <= L; o += blockDim.x) {
    int n;
    cplx zn, zm;
    if (o < L) {
      const int e = o / kCl, k1 = o - e * kCl;
      const int k2 = c * kq + e;
      n = k2 + L * k1;
      zn = Xo[o];
      const int k2p = k2 == 0 ? 0 : L - k2;
      const int k1p = k2 == 0 ? (kCl - k1) % kCl : kCl - 1 - k1;
      zm = cl.map_shared_rank(Xo, k2p / kq)[(k2p % kq) * kCl + k1p];
    } else {
      if (c != 0) break;
      n = M;                                                       // Nyquist: Z_M = Z_0
      zn = Xo[0];
      zm = Xo[0];
    }
    const cplx zc = cconj(zm);
    const cplx e = {0.5 * (zn.x + zc.x), 0.5 * (zn.y + zc.y)};
    const cplx dl = {0.5 * (zn.x - zc.x), 0.5 * (zn.y - zc.y)};
    const cplx od = {dl.y, -dl.x};
    const cplx x = cadd(e, cmul(twn[o], od));
    store_coef(coef + row * n_h + n, cmul(psn[o], x));
  }
  cl.sync();   // the other CTAs may still read this CTA's shared memory until here
}

// Adjoint in the cluster form for rows (w, i) with all their knots (N_I <= kKnotChunk): the
// inverse transform of each knot's Hermitian-packed input by the same four-step DFT, the
// products with chipow D_a B_ia summed over the knots in registers, one chunk of scratch.
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kClThreads)
k_fftlog_adj_cl(double* __restrict__ scratch, const cplx* __restrict__ cbar,
                const double* __restrict__ chipow, const double* __restrict__ D,
                const double* __restrict__ B, const cplx* __restrict__ psi,
                const cplx* __restrict__ tw, int N_tr, int N_I, int N, int* __restrict__ status) {
  pdl_trigger();   // the next kernel of the step may be scheduled
  extern __shared__ cplx smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  const int M = N / 2, L = M / kCl, kq = L / kCl, n_h = M + 1;
  cplx* a = smem;
  cplx* b = smem + L;
  cplx* Xo = smem + 2 * L;
  cplx* tws = smem + 3 * L;
  cplx* twc = smem + 4 * L;
  cplx* twn = smem + 5 * L;       // [L]: tw[n], psi_i[n] and psi_i[M - n] of n = c + kCl t
  cplx* psn = smem + 6 * L;
  cplx* psm = smem + 7 * L;
  const long wi = blockIdx.x / kCl;
  const int i = (int)(wi % N_tr);
  const cplx* ps = psi + (size_t)i * n_h;
  load_cluster_twiddles(tws, twc, tw, L, N, c);
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    const int n = c + kCl * t;
    twn[t] = tw[n];
    psn[t] = ps[n];
    psm[t] = ps[M - n];
  }
  // the tables above are the grid's; the coefficient cotangents come from the kernels before
  pdl_wait();
  __syncthreads();
  const double* cp = chipow + (size_t)i * N;
  constexpr int kOut = 2;                  // outputs per thread (L <= 2 kClThreads)
  double acc0[kOut], acc1[kOut];
#pragma unroll
  for (int u = 0; u < kOut; ++u) acc0[u] = acc1[u] = 0.0;
  for (int ka = 0; ka < N_I; ++ka) {
    const cplx* cb = cbar + ((size_t)wi * N_I + ka) * n_h;
    for (int t = threadIdx.x; t < L; t += blockDim.x) {
      const int n = c + kCl * t;               // < M
      cplx y = cmulc(cb[n], psn[t]);
      cplx h = (n == 0) ? cplx{y.x, 0.0} : cplx{0.5 * y.x, 0.5 * y.y};
      const int m = M - n;
      cplx ym = cmulc(cb[m], psm[t]);
      cplx hm = (m == M) ? cplx{ym.x, 0.0} : cplx{0.5 * ym.x, 0.5 * ym.y};
      cplx hmc = cconj(hm);
      cplx e = cadd(h, hmc);
      cplx dd = csub(h, hmc);
      cplx od = cmulc(dd, twn[t]);
      cplx z = {e.x - od.y, e.y + od.x};
      a[t] = cconj(z);
    }
    __syncthreads();
    cplx* Y = stockham(a, b, L, 1, tws, L);
    for (int k2 = threadIdx.x; k2 < L; k2 += blockDim.x)
      Y[k2] = cmul(Y[k2], twc[k2]);
    cl.sync();
    step2(cl, Xo, Y, L);
    __syncthreads();   // step 2 writes each k2's eight outputs from one thread
    // x_{2j} + i x_{2j+1} = conj(Z_j), j = k2 + L k1 of this CTA's outputs
    const double* d = D + (size_t)ka * N;
    const double* bb = B ? B + ((size_t)i * N_I + ka) * N : nullptr;
#pragma unroll
    for (int u = 0; u < kOut; ++u) {
      const int o = threadIdx.x + u * kClThreads;
      if (o < L) {
        const int e = o / kCl, k1 = o - e * kCl;
        const int j = c * kq + e + L * k1;
        const cplx v = cconj(Xo[o]);
        const int m = 2 * j;
        double f0 = cp[m] * d[m], f1 = cp[m + 1] * d[m + 1];
        if (bb) { f0 *= bb[m]; f1 *= bb[m + 1]; }
        acc0[u] = fma(v.x, f0, acc0[u]);
        acc1[u] = fma(v.y, f1, acc1[u]);
      }
    }
    cl.sync();   // Y and Xo are reused by the next knot; the other CTAs have finished reading
  }
  double* out = scratch + (size_t)wi * N;
#pragma unroll
  for (int u = 0; u < kOut; ++u) {
    const int o = threadIdx.x + u * kClThreads;
    if (o < L) {
      const int e = o / kCl, k1 = o - e * kCl;
      const int j = c * kq + e + L * k1;
      flag_nonfinite(status, acc0[u] + acc1[u]);
      out[2 * j] = acc0[u];
      out[2 * j + 1] = acc1[u];
    }
  }
}

// The cluster form serves few rows (fewer than a quarter of the SMs' worth) of a length the
// four-step split supports.
bool use_cluster(long rows, int N) {
  return rows * kCl <= 2L * 152 && N >= 256 && N / 2 / kCl <= 2 * kClThreads;
}

}  // namespace

template <typename CT>
static cudaError_t fftlog_fwd(CT* coef, const double* W, const double* chipow, const double* D,
                              const double* B, const cplx* psi, const cplx* twiddle, int n_walk,
                              int N_tr, int N_I, int N, cudaStream_t s) {
  long rows = (long)n_walk * N_tr * N_I;
  if (use_cluster(rows, N)) {
    const size_t smem = ((size_t)7 * (N / 2 / kCl) + 2) * sizeof(cplx);
    k_fftlog_fwd_cl<CT><<<(unsigned)(rows * kCl), kClThreads, smem, s>>>(coef, W, chipow, D, B, psi,
                                                                        twiddle, N_tr, N_I, N);
    return cudaGetLastError();
  }
  int R = rows_per_cta(N);
  long grid = (rows + R - 1) / R;
  size_t smem = (size_t)2 * R * (N / 2) * sizeof(cplx);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_fftlog_fwd<CT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_fftlog_fwd<CT><<<(unsigned)grid, kThreads, smem, s>>>(coef, W, chipow, D, B, psi, twiddle,
                                                           n_walk, N_tr, N_I, N);
  return cudaGetLastError();
}

cudaError_t launch_fftlog_fwd(cplx* coef, const double* W, const double* chipow,
                              const double* D, const double* B, const cplx* psi,
                              const cplx* twiddle, int n_walk, int N_tr, int N_I, int N,
                              cudaStream_t s) {
  return fftlog_fwd(coef, W, chipow, D, B, psi, twiddle, n_walk, N_tr, N_I, N, s);
}

cudaError_t launch_fftlog_fwd_df(float4* coef, const double* W, const double* chipow,
                                  const double* D, const double* B, const cplx* psi,
                                  const cplx* twiddle, int n_walk, int N_tr, int N_I, int N,
                                  cudaStream_t s) {
  return fftlog_fwd(coef, W, chipow, D, B, psi, twiddle, n_walk, N_tr, N_I, N, s);
}

bool fftlog_adj_single_launch(int n_walk, int N_tr, int N_I, int N) {
  return (N_I + kKnotChunk - 1) / kKnotChunk == 1 && use_cluster((long)n_walk * N_tr, N);
}

size_t fftlog_adj_scratch_bytes(int n_walk, int N_tr, int N_I, int N) {
  int nchunk = (N_I + kKnotChunk - 1) / kKnotChunk;
  return (size_t)nchunk * n_walk * N_tr * N * sizeof(double);
}

cudaError_t launch_fftlog_adj(double* W_bar, const cplx* cbar, const double* chipow,
                              const double* D, const double* B, const cplx* psi,
                              const cplx* twiddle, int n_walk, int N_tr, int N_I, int N,
                              double* scratch, cudaStream_t s, int* status, bool pdl) {
  int nchunk = (N_I + kKnotChunk - 1) / kKnotChunk;
  if (nchunk == 1 && use_cluster((long)n_walk * N_tr, N)) {
    // one chunk: the cluster kernel writes W_bar directly
    const size_t csm = (size_t)8 * (N / 2 / kCl) * sizeof(cplx);
    return launch_k(pdl, k_fftlog_adj_cl, dim3((unsigned)((long)n_walk * N_tr * kCl)),
                    dim3(kClThreads), csm, s, W_bar, cbar, chipow, D, B, psi, twiddle, N_tr, N_I,
                    N, status);
  }
  size_t smem = (size_t)(N / 2) * 2 * sizeof(cplx) + (size_t)N * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_fftlog_adj, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 g(nchunk, n_walk * N_tr);
  k_fftlog_adj<<<g, kThreads, smem, s>>>(scratch, cbar, chipow, D, B, psi, twiddle, n_walk, N_tr,
                                          N_I, N);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  long per = (long)n_walk * N_tr * N;
  k_sum_chunks<<<(unsigned)((per + 255) / 256), 256, 0, s>>>(W_bar, scratch, per, nchunk, status);
  return cudaGetLastError();
}

}  // namespace swcl
