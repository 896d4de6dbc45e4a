/*
 * swiftcl.h -- C ABI of the GB300 (sm_103a) beyond-Limber FFTLog C_ell library.
 *
 * The library computes the angular power spectra of arXiv:2505.22718 (SwiftCl):
 *
 *   a1  FFTLog of every window at every k-knot (Sec. 3.1-3.2, Eq. 3.2-3.3):
 *         c_{i,a,n} = T_c(n) chi_min^{-i eta_n} (1/N) sum_{m<N} g_m e^{-2 pi i n m/N},
 *         g_m = W_i(chi_m) chi_m^{s_i - b_i} T_chi(m) D(kappa_a, chi_m) B_i(kappa_a, chi_m),
 *         n = 0..N/2, chi_m = chi_min exp(m L/N), L = ln(chi_max/chi_min), eta_n = 2 pi n/L.
 *   a2  the Gamma-ratio table of Eq. 3.4 (denominator Gamma((l+2-p)/2)):
 *         M_{l,n} = sqrt(pi) 2^{p-1} Gamma((l+1+p)/2) / Gamma((l+2-p)/2),  p = b_i + i eta_n.
 *   a3  the contraction with k-interpolation (Eq. 3.3-3.5, Sec. 3.2):
 *         Delta_i(l, k_q) = pi_i(l) k_q^{t_i-1-b_i} Re sum_{n=0}^{N/2} w_n c_{i,n}(k_q) M_{l,n} e^{-i eta_n ln k_q},
 *         c_{i,n}(k_q) = sum_a lambda_a(k_q) c_{i,a,n} (4-point Lagrange in ln k), w_0 = w_{N/2} = 1, else 2.
 *   a4  the k-quadrature of Eq. 2.1:
 *         C_l^{ij} = A_i A_j sum_q u_q Delta_i(l,k_q) Delta_j(l,k_q),  u_q = (2/pi) w_q k_q^2 P(k_q),
 *         w_q = k_q (ln k_{q+1} - ln k_{q-1})/2 (trapezoid in ln k, half intervals at the ends).
 *   a5  the vector-Jacobian product of a1-a4 with respect to P(k), the amplitudes A_i and the
 *       window samples W_i(chi_m).
 *
 * Tracer kinds (chi power s in the FFTLog input, k power t in front of the chi integral,
 * multipole prefactor pi, spherical-Bessel kernel):
 *   SWCL_DENSITY       s = 0,  t = 0,  pi = 1,                 j_l    (galaxy clustering, Eq. 2.6;
 *                      primordial non-Gaussianity, Eq. 2.11-2.13, is this kind with its B(k,z));
 *   SWCL_LENSING       s = -2, t = -2, pi = sqrt((l+2)!/(l-2)!), j_l  (cosmic shear, Eq. 2.14;
 *                      intrinsic alignments, Eq. 2.15, are this kind with their own window);
 *   SWCL_MAGNIFICATION s = -2, t = -2, pi = l(l+1),            j_l    (magnification bias,
 *                      Eq. 2.9; CMB lensing, Eq. 2.16, is this kind with its own window);
 *   SWCL_RSD           s = 0,  t = 0,  pi = -1,                j_l''  (redshift-space
 *                      distortions, Eq. 2.10).
 * A tracer that sums several of these (clustering + RSD + magnification of one bin) is the sum
 * of its parts: its C_l are block sums of the C_l of the component tracers.
 *
 * Conventions
 *  - Every call returns an int status: SWCL_OK (0) or a negative SWCL_ERR_* code.  No call
 *    aborts, exits or throws across the ABI.  swcl_last_error() returns a message for the
 *    last failing call on a context.
 *  - Pointers are caller-owned.  Input arrays may live in host memory or in device memory
 *    of the context's GPU (unified addressing decides which); set_* calls copy them into
 *    library-owned device buffers, so the caller may free or reuse its arrays once the call
 *    returns.  Outputs are written into caller buffers (host or device).
 *  - All arrays are dense, row-major, FP64 (double) unless stated.
 *  - Work is queued on the context's stream.  Calls that take host output pointers
 *    synchronise that stream before returning; calls with device outputs do not
 *    (swcl_sync waits and reports deferred device errors).
 *  - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef SWIFTCL_H
#define SWIFTCL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct swcl_ctx swcl_ctx;

/* status codes */
#define SWCL_OK               0
#define SWCL_ERR_INVALID_ARG (-1)  /* a size, pointer or value outside its documented range */
#define SWCL_ERR_UNSUPPORTED (-2)  /* valid request this build does not implement */
#define SWCL_ERR_OOM_BUDGET  (-3)  /* the request does not fit the context's memory budget */
#define SWCL_ERR_CUDA        (-4)  /* a CUDA runtime call failed (message has the CUDA error) */
#define SWCL_ERR_TIMEOUT     (-5)  /* a bounded device wait gave up */
#define SWCL_ERR_NONFINITE   (-6)  /* an output holds a NaN or Inf: the kernels that write C,
                                      P_bar, amp_bar, W_bar and dC test every value they store
                                      and raise the context's status word, which the next
                                      synchronising call (swcl_sync, or a call with host outputs)
                                      reports and clears.  Inputs are not scanned: a NaN or Inf
                                      input shows up in the outputs it reaches */
#define SWCL_ERR_STATE       (-7)  /* call out of order (e.g. compute before set_grids) */

/* tracer kinds */
#define SWCL_DENSITY       0
#define SWCL_LENSING       1
#define SWCL_MAGNIFICATION 2
#define SWCL_RSD           3

/* arithmetic of the contraction (a3) and of the k-quadrature (a4) */
#define SWCL_FP64        0  /* FP64 CUDA cores throughout */
#define SWCL_3XTF32      1  /* tcgen05 kind::tf32, 2-plane splits of both operands, 3 products */
#define SWCL_SPLIT_BF16  2  /* tcgen05 kind::f16 (bf16) compensated products, FP32 accumulation:
                               basis mode (low-rank profiles) 3 + 3 planes, 6 products; knot
                               stencil A in 3 planes, B in 4, 9 products ("bf16x9") */
#define SWCL_TF32X6      3  /* tcgen05 kind::tf32, 3-plane splits of both operands, 6 products */
/* All tensor-core forms accumulate in FP32 (TMEM); the FFTLog (a1), the Gamma table (a2) and the
 * per-pair k-sums of a4 stay FP64, the a4 products are FP32 with compensated partial sums. */

/* swcl_query keys */
#define SWCL_Q_WORKSPACE_BYTES 1  /* device bytes the context holds now */
#define SWCL_Q_RECOMPUTE       2  /* 1 if the VJP recomputes Delta instead of storing it */
#define SWCL_Q_N_HALF          3  /* N/2 + 1 */
#define SWCL_Q_KERNEL_LAUNCHES 4  /* kernels launched by the last compute/vjp call */
#define SWCL_Q_PROFILE_RANK    5  /* rank r of the knot profiles D*B used (0 = one FFT per knot) */
#define SWCL_Q_TILE_FWD        6  /* autotuned tile of the basis-mode forward GEMM (0 = none yet):
                                     column tile in bits 0-7, bit 8 set for the variant that runs
                                     two CTAs per SM, bit 10 for two K-blocks per stage */
#define SWCL_Q_TILE_ADJ        7  /* the same for the basis-mode adjoint GEMM */

/* Create a context on CUDA device `device`.  mem_budget_bytes bounds the device memory the
 * context may hold (0 = no bound).  `stream` is a cudaStream_t (NULL = the context creates
 * its own non-blocking stream).  On success *out receives the context. */
int swcl_create(swcl_ctx** out, int device, size_t mem_budget_bytes, void* stream);

/* Release every device buffer of the context and the context itself (NULL is accepted). */
int swcl_destroy(swcl_ctx* ctx);

/* Grids (Sec. 3.1-3.2, Appendix A).  chi grid: N points chi_min exp(m L/N), chi_max excluded;
 * N a power of two, 16 <= N <= 8192.  k[N_k]: strictly increasing, > 0, N_k >= 2.
 * ells[N_ell]: integers >= 0 (>= 2 for lensing tracers).  knots[N_I]: strictly increasing, > 0,
 * N_I >= 1 (one knot = scale-independent growth).  Drops tracers and windows set before. */
int swcl_set_grids(swcl_ctx* ctx, double chi_min, double chi_max, int N,
                   const double* k, int N_k, const int* ells, int N_ell,
                   const double* knots, int N_I);

/* Tracers.  kind[N_tr] (SWCL_DENSITY, SWCL_LENSING, SWCL_MAGNIFICATION, SWCL_RSD), fft_bias[N_tr]
 * = b_i with -ell_min - 1 < b_i < 1 (Eq. 3.4 range; 1 - ell_min < b_i < 1 for SWCL_RSD, whose
 * j_l'' moment is taken at b_i - 2; lensing and RSD need every ell >= 2), taper_chi[N_tr][N] and taper_c[N_tr][N/2+1] optional
 * smoothing of the tails (Sec. 3.1; NULL = none).  Builds the Gamma-ratio (a2) and phase tables. */
int swcl_set_tracers(swcl_ctx* ctx, int N_tr, const int* kind, const double* fft_bias,
                     const double* taper_chi, const double* taper_c);

/* Windows for n_walk parameter points (n_walk >= 1).  The FFTLog input of tracer i at knot a is
 * W_i chi^{s_i - b_i} D_a B_ia; when the knot profiles D_a B_ia are numerically of rank r <= 4
 * (row residuals below 1e-14 of the largest row after r steps of pivoted Gram-Schmidt), the
 * library transforms r basis profiles per tracer instead of N_I knots and carries the
 * interpolation weights through the basis (exact by linearity, up to rounding; set the environment
 * variable SWCL_PER_KNOT_FFT=1 before creating a context to always transform every knot).  W[n_walk][N_tr][N] window samples on the
 * chi grid; D[N_I][N] growth at the knots (NULL = 1); B[N_tr][N_I][N] k,z-dependent bias at the
 * knots (NULL = 1).  Window samples may differ per walker; D and B are shared. */
int swcl_set_windows(swcl_ctx* ctx, int n_walk, const double* W, const double* D, const double* B);

/* New window samples W[n_walk][N_tr][N] for the same parameter points, keeping D, B and the
 * profile factorisation of the last swcl_set_windows (no comparison of D and B, hence no host
 * wait: a host W up to 1 MiB goes through the context's pinned staging ring and the call returns
 * at once; a larger host W is waited for).  n_walk must equal that of the last swcl_set_windows.
 * This is the per-step input of a sampler whose windows move (mean shifts, Sec. 4.3) while the
 * growth and bias tables stay fixed.  Errors: SWCL_ERR_STATE before swcl_set_windows,
 * SWCL_ERR_INVALID_ARG. */
int swcl_set_window_samples(swcl_ctx* ctx, int n_walk, const double* W);

/* Power spectrum and amplitudes: P[n_walk][N_k] = P(k_q, z_fid) (Eq. 2.3), amp[n_walk][N_tr] = A_i
 * (linear bias for density, amplitude for lensing). */
int swcl_set_power(swcl_ctx* ctx, int n_walk, const double* P, const double* amp);

/* Optional ragged multipole lists: walker w uses master-list entries
 * ell_idx[offsets[w] .. offsets[w+1]), strictly increasing.  offsets == NULL restores "all ells for
 * every walker".  Outputs of compute/vjp are then packed walker after walker. */
int swcl_set_ell_lists(swcl_ctx* ctx, const int* offsets, const int* ell_idx);

/* Limber branch (Eq. 2.19).  Multipoles l >= ell_switch of the master list (which must then be
 * ascending) take the Limber form instead of the FFTLog path, in swcl_compute_cl, swcl_vjp and
 * swcl_jvp (0 = off, the default):
 *   C_ij(l) = A_i A_j sum_m (L/N) chi_m^-1 Pt(k_m) G_i G_j,   k_m = (l + 1/2)/chi_m,
 *   G_i = pi_i(l) k_m^{t_i} chi_m^{s_i} W_i(chi_m) sum_a Lam_a(k_m) D_a(chi_m) B_ia(chi_m),
 * on the FFTLog chi grid (rectangle rule in ln chi), Pt the 4-point Lagrange interpolant in ln k
 * of P on the k grid (zero outside it), Lam the knot interpolation; tapers do not apply.  FP64
 * arithmetic in every precision form.  Needs SWCL_FP64 or the basis-mode SWCL_SPLIT_BF16 form
 * and no SWCL_RSD tracer (else the compute call returns SWCL_ERR_UNSUPPORTED).  The Limber error
 * is O(1/l) (Eq. 2.19); the switch trades it for the FFTLog work of those multipoles. */
int swcl_set_limber(swcl_ctx* ctx, int ell_switch);

/* Forward pass a1-a4 for every walker.  C_out[sum_w n_ell(w)][N_tr][N_tr] (full symmetric
 * matrices, C^{ij} = C^{ji} bit for bit).  A host C_out makes the call synchronous and reports
 * SWCL_ERR_NONFINITE or SWCL_ERR_TIMEOUT from the device status word. */
int swcl_compute_cl(swcl_ctx* ctx, int precision, double* C_out);

/* Vector-Jacobian product (a5) of the last swcl_compute_cl for the same precision.
 * C_bar has the layout of C_out.  Outputs (each may be NULL to skip):
 * P_bar[n_walk][N_k], amp_bar[n_walk][N_tr], W_bar[n_walk][N_tr][N]. */
int swcl_vjp(swcl_ctx* ctx, int precision, const double* C_bar,
             double* P_bar, double* amp_bar, double* W_bar);

/* Batched evaluation as one CUDA-graph replay.  Runs swcl_compute_cl for every walker and, when
 * C_bar is not NULL, swcl_vjp with the given outputs (P_bar, amp_bar, W_bar may be NULL), with all
 * of their kernels captured once into a CUDA graph on the context's stream and replayed on later
 * calls with the same arguments, precision and sizes.  Walkers, their parameter arrays and
 * ragged multipole lists are those of the last swcl_set_* calls (Sec. 4.3 runs many parameter
 * points of one survey setup; SwiftCl batches them with vmap).  All pointers must be device
 * pointers of the context's GPU.  The first call of a configuration also runs it once outside
 * the graph (building tables and buffers) and captures; a change of any set_* size, of the
 * precision or of a pointer re-captures.  Calls are asynchronous on the context stream. */
int swcl_compute_batched(swcl_ctx* ctx, int precision, double* C_out, const double* C_bar,
                         double* P_bar, double* amp_bar, double* W_bar);

/* One step of a sampler that keeps its parameter points in host memory (Sec. 4.3: every step
 * evaluates C_l and its gradient at new parameters).  The step's inputs go host -> device, the
 * kernels of swcl_compute_batched run, and the results come back device -> host, all inside one
 * CUDA-graph replay on the context stream; the call returns when the host outputs are written.
 * Inputs (NULL keeps the values of the last set call or step):
 *   W[n_walk][N_tr][N] window samples (as swcl_set_window_samples: D, B and the profile
 *   factorisation stay), P[n_walk][N_k] and amp[n_walk][N_tr] (as swcl_set_power; both or
 *   neither), C_bar (layout of C_out; NULL = forward only).
 * Outputs: C_out (required), P_bar, amp_bar, W_bar (NULL to skip; they need C_bar), laid out as
 * in swcl_compute_cl / swcl_vjp.
 * Every non-NULL pointer must be page-locked host memory (cudaHostAlloc, cudaHostRegister, a
 * pinned torch tensor): two kernels of the graph read and write it directly (copy nodes where
 * the device cannot address it).  Pointers equal to those of the captured graph are not checked
 * again.  The library-owned device side of the outputs and cotangent is sized at the first call.
 * The first call of a configuration (pointers, precision, sizes) runs the step once outside the
 * graph and captures it; later calls replay it.  The call waits for the replay by polling (it
 * keeps one host thread busy for the step's duration).  Needs set_grids, set_tracers, set_windows and set_power
 * first.  Errors: SWCL_ERR_INVALID_ARG (a pointer that is not page-locked host memory, P without
 * amp, gradients without C_bar), SWCL_ERR_STATE, and SWCL_ERR_NONFINITE / SWCL_ERR_TIMEOUT from
 * the device status word of this step (then cleared). */
int swcl_step_host(swcl_ctx* ctx, int precision, const double* W, const double* P,
                   const double* amp, const double* C_bar, double* C_out, double* P_bar,
                   double* amp_bar, double* W_bar);

/* Forward-mode derivative (JVP) of a1-a4 at one parameter point (Sec. 4.3: the Fisher forecasts
 * differentiate C_l along the parameters).  The context must hold one walker (n_walk = 1).  For
 * n_dir tangents (1..256) of the inputs
 *   P_dot[n_dir][N_k], amp_dot[n_dir][N_tr], W_dot[n_dir][N_tr][N]   (each may be NULL = zero),
 * writes C_dot[n_dir][N_ell][N_tr][N_tr] (every multipole of the master list, full symmetric
 * matrices): dC_ij = A_i A_j dU_ij + (A'_i A_j + A_i A'_j) U_ij with
 * dU_ij = sum_q wk2_q [P'_q Delta_i Delta_j + P_q (Delta'_i Delta_j + Delta_i Delta'_j)] (Eq. 2.1
 * by the product rule); Delta' is the contraction of the tangent windows, since Delta is linear
 * in W (Eq. 3.1-3.5).  D and B are held fixed.  Host or device arrays; a host C_dot makes the call
 * synchronous.  Runs the forward kernels over 1 + n_dir walkers, so it replaces the state of the
 * last swcl_compute_cl: a following swcl_vjp needs a new swcl_compute_cl.  Errors:
 * SWCL_ERR_UNSUPPORTED (n_walk != 1), SWCL_ERR_INVALID_ARG, SWCL_ERR_OOM_BUDGET. */
int swcl_jvp(swcl_ctx* ctx, int precision, int n_dir, const double* P_dot, const double* amp_dot,
             const double* W_dot, double* C_dot);

/* Gaussian Fisher matrix / chi^2 of C_l perturbations (Sec. 4.2-4.3: Gaussian covariance with
 * cosmic variance and additive noise, scaled by 1/f_sky).  With Ct_l = C_l + diag(noise) from the
 * last swcl_compute_cl or swcl_jvp (one walker) and nu_l = modes[l] the number of modes behind
 * C_l (e.g. (2l+1) f_sky times the bin width):
 *   F[a][b] = sum_l (nu_l / 2) Tr[Ct_l^-1 X_a,l Ct_l^-1 X_b,l],   X[n_x][N_ell][N_tr][N_tr],
 * which is the Fisher matrix of the Gaussian likelihood of the unique pairs C_l^{ij} when
 * X_a = dC/dtheta_a (swcl_jvp output) and chi^2 when X = C - C_data.  noise[N_tr] (NULL = 0) and
 * modes[N_ell] finite and >= 0; n_x in 1..1024; F[n_x][n_x] host or device.  Every Ct_l must be
 * positive definite, else SWCL_ERR_INVALID_ARG.  Synchronous.  SWCL_ERR_STATE without a forward. */
int swcl_gaussian_fisher(swcl_ctx* ctx, int n_x, const double* X, const double* noise,
                         const double* modes, double* F);

/* Per-kernel device timing.  While enabled, every kernel the context launches is bracketed by
 * CUDA events on the context stream (a few microseconds of overhead per launch).
 * swcl_profile_read synchronises the stream and returns, for up to max_entries kernels,
 * a NUL-terminated name (32 bytes per entry in names[max_entries][32]), the launch count and the
 * total device milliseconds accumulated since the last reset; *n_entries receives the count.
 * swcl_profile_reset clears the accumulators. */
int swcl_profile_enable(swcl_ctx* ctx, int enable);
int swcl_profile_read(swcl_ctx* ctx, int max_entries, char* names, int64_t* launches, double* ms,
                      int* n_entries);
int swcl_profile_reset(swcl_ctx* ctx);

/* Stage read-back for element-wise testing of each step.  Copies an internal array of the last
 * compute into out (host or device), as FP64 values (complex arrays as interleaved re, im):
 *   SWCL_DBG_COEF   a1 c[n_walk][N_tr][N_I][N/2+1] complex
 *   SWCL_DBG_DELTA  a3 Delta[n_walk][N_ell][N_tr][N_k] (mixed paths: FP32 values widened); only
 *                   when the last forward pass held Delta for every multipole at once (no
 *                   memory-budget chunks, no Limber rows), else SWCL_ERR_STATE
 *   SWCL_DBG_GTAB   a2 w_n pi(l) M_{l,n} per tracer class [n_cls][N_ell][N/2+1] complex
 *   SWCL_DBG_PHASE  e^{-i eta_n ln k_q} [N_k][N/2+1] complex
 *   SWCL_DBG_UNIT   a4 unit-amplitude C [n_walk][N_ell][N_tr][N_tr]
 * *count receives the number of doubles written (out may be NULL to query it). */
#define SWCL_DBG_COEF  1
#define SWCL_DBG_DELTA 2
#define SWCL_DBG_GTAB  3
#define SWCL_DBG_PHASE 4
#define SWCL_DBG_UNIT  5
int swcl_debug_read(swcl_ctx* ctx, int what, double* out, int64_t* count);

/* FFTLog coefficients (a1) without a context and without allocating device memory.
 *
 * The paper has no counterpart to this call; it exists for callers that cannot allocate device
 * memory, e.g. a JAX/XLA process that has pre-reserved the GPU's memory for its own arena, a
 * plugin confined to another framework's workspace, or a loop that must not pay for (or risk
 * the failure of) a cudaMalloc.  It never calls cudaMalloc, cudaFree or any allocating routine.
 *
 * Arguments as for swcl_set_grids / swcl_set_tracers / swcl_set_windows, except:
 *   kind[N_tr], fft_bias[N_tr]      host arrays;
 *   taper_chi, taper_c, W, D, B     device arrays of the current device (taper_*, B may be NULL;
 *                                   D is required);
 *   coef                            device output [n_walk][N_tr][N_I][N/2+1] complex
 *                                   (interleaved re, im) -- the same values swcl_compute_cl
 *                                   produces for the same inputs (SWCL_DBG_COEF);
 *   stream                          cudaStream_t the work is queued on (NULL = legacy stream).
 * Work runs on the current CUDA device.  The twiddle, chi-power and phase tables the kernel reads
 * live in one static device array of SWCL_NOALLOC_SCRATCH_BYTES per device, held by every GPU
 * that loads the library until the process exits.  Requests whose tables exceed it,
 * 16 N + 8 N_tr N + 16 N_tr (N/2+1) bytes (each term rounded up to 256), return
 * SWCL_ERR_OOM_BUDGET; bad sizes or pointers return SWCL_ERR_INVALID_ARG; a failing launch
 * returns SWCL_ERR_CUDA.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.  Every call rewrites
 * the tables it reads, so nothing from an earlier call leaks into a later one, but all calls share
 * the one array: calls that overlap on the GPU (different streams, or host threads) race.
 */
#define SWCL_NOALLOC_SCRATCH_BYTES (4u << 20)
int swcl_fftlog_noalloc(int n_walk, int N_tr, int N_I, int N, double chi_min, double chi_max,
                        const int* kind, const double* fft_bias, const double* taper_chi,
                        const double* taper_c, const double* W, const double* D, const double* B,
                        double* coef, void* stream);

/* Self-test of the bounded waits of the tensor-core kernels (no counterpart in the paper): one
 * thread waits on an mbarrier phase that nothing completes.  The wait gives up after the same
 * poll limit as the kernels' waits and raises the status word, so the call returns
 * SWCL_ERR_TIMEOUT; *cycles (nullable) receives the clock cycles the wait took.  The context
 * stays usable (the status word is cleared). */
int swcl_selftest_wait_timeout(swcl_ctx* ctx, int64_t* cycles);

/* Wait for queued work; returns any deferred device error. */
int swcl_sync(swcl_ctx* ctx);

/* Query a SWCL_Q_* value into *value. */
int swcl_query(swcl_ctx* ctx, int key, int64_t* value);

/* Message of the last failing call on ctx ("" if none; static storage of the context). */
const char* swcl_last_error(swcl_ctx* ctx);

/* Static description of a status code. */
const char* swcl_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* SWIFTCL_H */
