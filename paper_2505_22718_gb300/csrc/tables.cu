// Grid- and tracer-dependent tables (the precomputation of Sec. 3.2): FFT twiddles, the
// phase table e^{-i eta_n ln k_q}, Lagrange weights in ln k, ln-k trapezoid weights, the
// Gamma-ratio table of Eq. 3.4 and per-tracer power/phase factors.  All in FP64.
#include "swcl_internal.h"

namespace swcl {
namespace {

__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cplx cscale(cplx a, double s) { return {a.x * s, a.y * s}; }
__device__ __forceinline__ cplx cinv(cplx a) {
  double d = 1.0 / (a.x * a.x + a.y * a.y);
  return {a.x * d, -a.y * d};
}
__device__ __forceinline__ cplx clog(cplx z) { return {log(hypot(z.x, z.y)), atan2(z.y, z.x)}; }
__device__ __forceinline__ cplx cexp(cplx z) {
  double s, c;
  sincos(z.y, &s, &c);
  double e = exp(z.x);
  return {e * c, e * s};
}

// Stirling's remainder S(z) = sum_{k=1}^{9} B_{2k} / (2k (2k-1) z^{2k-1}) of
//   lnG(z) = (z - 1/2) ln z - z + ln(2 pi)/2 + S(z),
// valid for |z| >= 12 (the next term is then below 1e-19 relative).  B_2 .. B_18 are the
// Bernoulli numbers.
__device__ cplx stirling_tail(cplx z) {
  const double c1 = 1.0 / 12.0, c2 = -1.0 / 360.0, c3 = 1.0 / 1260.0, c4 = -1.0 / 1680.0,
               c5 = 1.0 / 1188.0, c6 = -691.0 / 360360.0, c7 = 1.0 / 156.0,
               c8 = -3617.0 / 122400.0, c9 = 43867.0 / 244188.0;
  cplx w = cinv(z);
  cplx w2 = cmul(w, w);
  cplx s = {c9, 0.0};
  s = cadd(cmul(s, w2), {c8, 0.0});
  s = cadd(cmul(s, w2), {c7, 0.0});
  s = cadd(cmul(s, w2), {c6, 0.0});
  s = cadd(cmul(s, w2), {c5, 0.0});
  s = cadd(cmul(s, w2), {c4, 0.0});
  s = cadd(cmul(s, w2), {c3, 0.0});
  s = cadd(cmul(s, w2), {c2, 0.0});
  s = cadd(cmul(s, w2), {c1, 0.0});
  return cmul(s, w);
}

// ln(1 + w) on the principal branch, accurate for small |w|.
__device__ cplx clog1p(cplx w) {
  double re = 0.5 * log1p(w.x * (2.0 + w.x) + w.y * w.y);
  return {re, atan2(w.y, 1.0 + w.x)};
}

// lnG(z1) - lnG(z2) for Re z1, Re z2 > 0, given d = z1 - z2 exactly.
// Both arguments are first raised by the same integer m (G(z) = G(z+m) / prod_{j<m} (z+j))
// until both moduli reach 12.  Then, with Stirling's formula for each and
// ln z2 = ln z1 + ln(1 + (z2 - z1)/z1) (no branch jump: both arguments lie in the right half
// plane),
//   lnG(z1) - lnG(z2) = d ln z1 - (z2 - 1/2) ln(1 - d/z1) - d + S(z1) - S(z2),
// which never forms the two large log-Gammas (|lnG| ~ |z| ln|z|) whose difference would lose
// ~eps |z| ln|z| to cancellation.  The result is exact only modulo 2 pi i, which cancels in
// the exponential.
__device__ cplx lgamma_diff(cplx z1, cplx z2, cplx d) {
  cplx num = {1.0, 0.0}, den = {1.0, 0.0};
  bool shifted = false;
  while (fmin(z1.x * z1.x + z1.y * z1.y, z2.x * z2.x + z2.y * z2.y) < 144.0) {
    num = cmul(num, z1);
    den = cmul(den, z2);
    z1.x += 1.0;
    z2.x += 1.0;
    shifted = true;
  }
  cplx lz1 = clog(z1);
  cplx iz1 = cinv(z1);
  cplx l12 = clog1p(cmul({-d.x, -d.y}, iz1));  // ln(z2/z1)
  cplx r = csub(cmul(d, lz1), cmul({z2.x - 0.5, z2.y}, l12));
  r = csub(r, d);
  r = cadd(r, csub(stirling_tail(z1), stirling_tail(z2)));
  if (shifted) r = csub(r, clog(cmul(num, cinv(den))));
  return r;
}

// e^{-2 pi i x} for x = n * r reduced exactly: f = n r - rint(n r) computed with one rounding.
__device__ __forceinline__ cplx phase_of(double n, double r) {
  double p = n * r;
  double f = fma(n, r, -rint(p));
  double s, c;
  sincospi(2.0 * f, &s, &c);
  return {c, -s};
}

__global__ void k_twiddles(cplx* tw, int N) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  double s, c;
  sincospi(-2.0 * (double)t / (double)N, &s, &c);
  tw[t] = {c, s};
}

// phase[q][n] = e^{-i eta_n ln k_q} = e^{-2 pi i n ln(k_q)/L}
__global__ void k_phase(cplx* phase, const double* k, int N_k, int n_h, double L) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  int q = blockIdx.y;
  if (n >= n_h || q >= N_k) return;
  double r = log(k[q]) / L;
  phase[(size_t)q * n_h + n] = phase_of((double)n, r);
}

// 4-point (or fewer) Lagrange weights in ln k on the knots; stencil start clamp(a-1, 0, N_I-s)
// where a is the knot interval holding ln k_q (clamped to [0, N_I-1]).
__global__ void k_interp(int* j0, double* w, const double* k, int N_k, const double* knots,
                         int N_I) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N_k) return;
  double x = log(k[q]);
  int s = N_I < 4 ? N_I : 4;
  // largest a with ln knot_a <= x  (searchsorted right - 1)
  int lo = 0, hi = N_I;  // invariant: answer in [lo-1, hi-1]
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (log(knots[mid]) <= x) lo = mid + 1; else hi = mid;
  }
  int a = lo - 1;
  if (a < 0) a = 0;
  if (a > N_I - 1) a = N_I - 1;
  int start = a - 1;
  if (start > N_I - s) start = N_I - s;
  if (start < 0) start = 0;
  j0[q] = start;
  double xs[4];
  for (int r = 0; r < s; ++r) xs[r] = log(knots[start + r]);
  for (int r = 0; r < 4; ++r) {
    double v = 0.0;
    if (r < s) {
      v = 1.0;
      for (int t = 0; t < s; ++t)
        if (t != r) v *= (x - xs[t]) / (xs[r] - xs[t]);
    }
    w[(size_t)q * 4 + r] = v;
  }
}

// wk2[q] = (2/pi) w_q k_q^2 with w_q = k_q h_q, h_q the ln-k trapezoid half-spacing.
__global__ void k_quadw(double* wk2, const double* k, int N_k) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N_k) return;
  double h;
  if (q == 0) h = 0.5 * (log(k[1]) - log(k[0]));
  else if (q == N_k - 1) h = 0.5 * (log(k[N_k - 1]) - log(k[N_k - 2]));
  else h = 0.5 * (log(k[q + 1]) - log(k[q - 1]));
  double kk = k[q];
  wk2[q] = (2.0 / 3.14159265358979323846) * h * kk * kk * kk;
}

// gtab[l][n] = w_n pi_kind(l) M(l, p), p = b + i eta_n, with the Bessel moment of Eq. 3.4
//   M(l, p) = sqrt(pi) 2^{p-1} G((l+1+p)/2) / G((l+2-p)/2)            (j_l kernels),
//   M''(l, p) = p (p-1) M(l, p-2) = M(l, p) p (p-1) / ((l-1+p)(l+2-p))  (RSD, j_l'' of Eq. 2.10),
// the second form by integrating by parts twice and G(z+1) = z G(z) on both Gammas.
// pi_kind(l): 1 (density), sqrt((l+2)!/(l-2)!) (lensing, Eq. 2.14), l(l+1) (magnification,
// Eq. 2.9), -1 (RSD, the sign of Eq. 2.10).
__global__ void k_gamma(cplx* gtab, const int* ells, int N_ell, int n_h, double L, double b,
                        int kind) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  int li = blockIdx.y;
  if (n >= n_h || li >= N_ell) return;
  double l = (double)ells[li];
  double eta = 2.0 * 3.14159265358979323846 * (double)n / L;
  cplx z1 = {0.5 * (l + 1.0 + b), 0.5 * eta};
  cplx z2 = {0.5 * (l + 2.0 - b), -0.5 * eta};
  cplx lg = lgamma_diff(z1, z2, {b - 0.5, eta});
  const double ln2 = 0.69314718055994530942;
  lg.x += (b - 1.0) * ln2;
  lg.y += eta * ln2;
  cplx m = cexp(lg);
  double pre = 1.7724538509055160273;  // sqrt(pi)
  if (kind == SWCL_LENSING) pre *= sqrt((l + 2.0) * (l + 1.0) * l * (l - 1.0));
  if (kind == SWCL_MAGNIFICATION) pre *= l * (l + 1.0);
  if (kind == SWCL_RSD) {
    const cplx num = cmul({b, eta}, {b - 1.0, eta});
    const cplx den = cmul({l - 1.0 + b, eta}, {l + 2.0 - b, -eta});
    m = cmul(m, cmul(num, cinv(den)));
    pre = -pre;
  }
  double wn = (n == 0 || n == n_h - 1) ? 1.0 : 2.0;
  gtab[(size_t)li * n_h + n] = cscale(m, pre * wn);
}

__global__ void k_tracer(double* chipow, cplx* psi, double* kpow, const double* k, int N_k,
                         int N, double chi_min, double L, double b, int kind,
                         const double* taper_chi, const double* taper_c) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int n_h = N / 2 + 1;
  // chi^s in the FFTLog input and k^t in front of it: s = t = -2 for the kinds with the lensing
  // chi^-2 (lensing, magnification), 0 otherwise
  const bool chi2 = kind == SWCL_LENSING || kind == SWCL_MAGNIFICATION;
  double s = chi2 ? -2.0 : 0.0;
  if (t < N) {
    double lnchi = log(chi_min) + (double)t * L / (double)N;
    double v = exp((s - b) * lnchi);
    if (taper_chi) v *= taper_chi[t];
    chipow[t] = v;
  }
  if (t < n_h) {
    // chi_min^{-i eta_n} / N
    cplx ph = phase_of((double)t, log(chi_min) / L);
    double sc = 1.0 / (double)N;
    if (taper_c) sc *= taper_c[t];
    psi[t] = cscale(ph, sc);
  }
  if (t < N_k) {
    double tk = chi2 ? -2.0 : 0.0;
    kpow[t] = exp((tk - 1.0 - b) * log(k[t]));
  }
}

}  // namespace

cudaError_t launch_fft_twiddles(cplx* tw, int N, cudaStream_t s) {
  k_twiddles<<<(N + 255) / 256, 256, 0, s>>>(tw, N);
  return cudaGetLastError();
}

cudaError_t launch_phase_table(cplx* phase, const double* k, int N_k, int n_h, double L,
                               cudaStream_t s) {
  dim3 g((n_h + 255) / 256, N_k);
  k_phase<<<g, 256, 0, s>>>(phase, k, N_k, n_h, L);
  return cudaGetLastError();
}

cudaError_t launch_interp_weights(int* j0, double* w, const double* k, int N_k,
                                  const double* knots, int N_I, cudaStream_t s) {
  k_interp<<<(N_k + 127) / 128, 128, 0, s>>>(j0, w, k, N_k, knots, N_I);
  return cudaGetLastError();
}

cudaError_t launch_quad_weights(double* wk2, const double* k, int N_k, cudaStream_t s) {
  k_quadw<<<(N_k + 255) / 256, 256, 0, s>>>(wk2, k, N_k);
  return cudaGetLastError();
}

cudaError_t launch_gamma_table(cplx* gtab, const int* ells, int N_ell, int n_h, double L,
                               double b, int kind, cudaStream_t s) {
  dim3 g((n_h + 127) / 128, N_ell);
  k_gamma<<<g, 128, 0, s>>>(gtab, ells, N_ell, n_h, L, b, kind);
  return cudaGetLastError();
}

cudaError_t launch_tracer_tables(double* chipow, cplx* psi, double* kpow, const double* k,
                                 int N_k, int N, double chi_min, double L, double b, int kind,
                                 const double* taper_chi, const double* taper_c,
                                 cudaStream_t s) {
  int n = N > N_k ? N : N_k;
  k_tracer<<<(n + 255) / 256, 256, 0, s>>>(chipow, psi, kpow, k, N_k, N, chi_min, L, b, kind,
                                           taper_chi, taper_c);
  return cudaGetLastError();
}

}  // namespace swcl
