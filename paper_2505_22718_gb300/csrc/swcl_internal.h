// Internal declarations of the swiftcl library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include "../../include/swiftcl.h"

namespace swcl {

struct cplx { double x, y; };

// Bits of the context's device status word (ws_status): a tensor-core kernel gave up a bounded
// wait, or a kernel that writes an output (C, P_bar, amp_bar, W_bar, dC) stored a NaN or Inf.
constexpr int kStatusTimeout = 1;
constexpr int kStatusNonfinite = 2;

// Raises kStatusNonfinite in *status when v is NaN or Inf (status may be null).
__device__ __forceinline__ void flag_nonfinite(int* status, double v) {
  if (status && !isfinite(v)) atomicOr(status, kStatusNonfinite);
}

// Programmatic dependent launch.  A kernel launched with pdl = true (launch_k) may start while
// the kernel before it in the stream is still running: it calls pdl_wait() before it touches any
// memory that an earlier kernel of the step writes (after the wait, every earlier kernel of the
// stream has completed and its writes are visible), and pdl_trigger() early, so that the next
// kernel can be scheduled once every CTA of this one has started.  Both are no-ops in a kernel
// launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
template <typename... KArgs, typename... Args>
cudaError_t launch_k(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                     cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args...);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

// Device buffer with a byte count, owned by the context.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Per-precision operand tables for the tensor-core contraction.
struct TcTables {
  bool ready = false;      // forward operand tables built for the current grids/tracers
  bool adj_ready = false;  // VJP operand tables built
  DevBuf bfwd;      // forward B image [cls][l tile][K-block][plane][NT x 128 B]
  DevBuf bvjp;      // VJP B image [cls][column tile][K-block][plane][128 x 128 B]
  DevBuf phase32;   // float2 phase table [n_h][N_k] (transposed)
  DevBuf phase_lo;  // float2 [n_h][N_k]: phase - phase32 (double-float low parts)
  DevBuf tile_alo;  // [n_qt] first knot touched by each 128-point k tile
  DevBuf knot_qt;   // [N_I][2] first/last k tile touching each knot
  int R = 0;        // knot slots per k tile
};

// a3 on tensor cores (contract_tc.cu): fills ws_delta (float) / ws_cbar for the context
int compute_delta_tc(swcl_ctx* c, int precision);
int contract_adj_tc(swcl_ctx* c, int precision);
// a3 / a5 in basis mode as GEMMs against the constant phase operand (basis_tc.cu)
int basis_prepare(swcl_ctx* c);
int basis_forward(swcl_ctx* c, int l_lo, int n_l);
int basis_adjoint(swcl_ctx* c, int l_lo, int n_l, bool accumulate);
size_t basis_fixed_bytes(const swcl_ctx* c);     // constant operands of basis mode
size_t basis_bytes_per_ell(const swcl_ctx* c);   // per-call operand images per multipole

// The k-interpolation stencil and FFT profiles the kernels use: the N_I knots with 4-point
// Lagrange weights, or (basis mode) r low-rank profiles with weights mu.
struct Stencil {
  const int* j0;        // [N_k] first row of each k point's stencil
  const double* w;      // [n_w][N_k][4] weights
  long w_ts;            // tracer stride of w in doubles (0 = shared)
  int NI;               // stencil rows ("knots") per tracer
  const double* D;      // FFT profile rows [NI][N]
  const double* B;      // per-tracer factor [N_tr][NI][N] or null
};

// Grids and tables of the Limber branch (limber.cu): multipoles l_first .. l_first + n_lim - 1 of
// the master list.  D [N_I][N] and B [N_tr][N_I][N] are the knot profiles as given.
struct LimberArgs {
  const double* k = nullptr;
  const double* knots = nullptr;
  const int* ells = nullptr;
  const double* D = nullptr;
  const double* B = nullptr;
  double lnchi_min = 0, L = 0, lnk_lo = 0, lnk_hi = 0;
  int N = 0, N_k = 0, N_I = 0, N_tr = 0, N_ell = 0, l_first = 0, n_lim = 0;
  int kind[64] = {};
};

// Per-(Limber multipole, chi point) stencils (limber.cu), built once per grid: first k point of
// the P stencil (-1 outside the k range) with weights times (L/N)/chi, first knot with weights;
// and the logarithms of the k grid, the knots and l + 1/2.
struct LimberTable {
  int* pst = nullptr;
  int* kst = nullptr;
  double* pw = nullptr;
  double* kw = nullptr;
  double* lnk = nullptr;
  double* lnknots = nullptr;
  double* lnnu = nullptr;
};

}  // namespace swcl

struct swcl_ctx {
  int device = 0;
  int num_sms = 148;                        // multiprocessors of the device (persistent grids)
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t aux = nullptr;               // second stream for independent VJP kernels
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  size_t budget = 0;      // 0 = unbounded
  size_t held = 0;        // device bytes held
  std::string err;
  int64_t last_launches = 0;

  // grids
  bool have_grids = false;
  int N = 0, n_h = 0, N_k = 0, N_ell = 0, N_I = 0;
  double chi_min = 0, chi_max = 0, L = 0;
  std::vector<int> ells_h;
  std::vector<double> k_h, knots_h;
  swcl::DevBuf d_k, d_ells, d_knots, d_wk2;   // wk2 = (2/pi) w_q k_q^2
  swcl::DevBuf d_interp_j0, d_interp_w;       // [N_k] int, [N_k][4] double
  swcl::DevBuf d_twiddle;                     // FFT twiddles e^{-2 pi i t/N}, t < N  (cplx)
  swcl::DevBuf d_phase;                       // [N_k][n_h] cplx  e^{-i eta_n ln k_q}
  swcl::DevBuf d_knot_qrange;                 // [N_I][2] int: first/last q whose stencil uses knot a

  // tracers
  bool have_tracers = false;
  int N_tr = 0, n_cls = 0;
  std::vector<int> kind_h, cls_of_h;
  std::vector<double> bias_h;
  swcl::DevBuf d_cls_of;                      // [N_tr] int
  swcl::DevBuf d_chipow;                      // [N_tr][N] chi^{s-b} T_chi
  swcl::DevBuf d_psi;                         // [N_tr][n_h] cplx  T_c chi_min^{-i eta}/N
  swcl::DevBuf d_gtab;                        // [n_cls][N_ell][n_h] cplx  w_n pi(l) M_{l,n}
  swcl::DevBuf d_kpow;                        // [N_tr][N_k] k^{t-1-b}
  swcl::TcTables tc[4];
  swcl::DevBuf tc_lw32;                       // [N_k][4] float interpolation weights
  swcl::DevBuf tc_kpow32;                     // [N_tr][N_k] float k^{t-1-b}
  swcl::DevBuf tc_lw_lo, tc_kpow_lo;          // double-float low parts of the two tables above

  // windows / power
  int n_walk = 0;
  bool have_windows = false, have_power = false, have_B = false;
  swcl::DevBuf d_W, d_D, d_B, d_P, d_amp;
  swcl::DevBuf d_prev;        // previous D (and B) for change detection
  swcl::DevBuf d_flag;        // device int flag

  // low-rank knot profiles (lowrank.cu)
  bool lr_dirty = true;       // D/B/grids changed since the last factorisation
  bool lr_disabled = false;   // environment override SWCL_PER_KNOT_FFT=1
  bool lr_basis = false;      // basis mode active
  int lr_rank = 0;            // stencil rows used in basis mode
  int lr_true_rank = 0;
  swcl::DevBuf lr_res, lr_norms, lr_Q, lr_coef, lr_w, lr_j0, lr_ones;

  // basis-mode tensor-core GEMMs (basis_tc.cu)
  bool bt_ready = false;       // constant operands built for the current grids/tracers/profiles
  bool bt_disabled = false;    // environment override SWCL_BASIS_GEMM=0
  int bt_f_mt = 0, bt_f_kb = 0, bt_a_mt = 0, bt_a_kb = 0;
  int bt_nt_fwd = 0, bt_nt_adj = 0;   // autotuned column tiles (0 = not tuned yet)
  int bt_fixed_fwd = 0, bt_fixed_adj = 0;  // tiles fixed by the environment (0 = tune)
  uint32_t bt_pmask = 0x3F;    // compensated products issued (all six unless a study narrows it)
  swcl::DevBuf bt_eimg_f, bt_eimg_a;  // phase images: forward A [q][(n,re/im)], adjoint A [(n,re/im)][q]
  swcl::DevBuf bt_gdf, bt_g32;        // Gamma-ratio table as double-float and FP32
  swcl::DevBuf bt_kmu;                // [N_tr][4][N_k] float kpow * mu
  swcl::DevBuf bt_himg, bt_dimg;      // per-call B images (forward H, adjoint kpow mu Dbar)
  // ragged multipole lists: the GEMM columns of listed multipoles only (basis_tc.cu column_plan)
  swcl::DevBuf bt_cmap_f, bt_cmap_a, bt_lpos, bt_wbase;
  int64_t bt_plan_key[7] = {-1, -1, -1, -1, -1, -1, -1};
  int64_t lists_gen = 0;              // bumped when the walkers' multipole lists may change
  int bt_plan_cols = 0;
  bool bt_delta_clean = false;        // Delta rows of unlisted multipoles hold zeros
  bool bt_compact = false;            // the last column plan kept listed multipoles only

  // ragged ell lists
  bool ragged = false;
  std::vector<int> off_h, idx_h;
  swcl::DevBuf d_off, d_idx;
  int64_t n_out_ell = 0;                      // sum_w n_ell(w)

  // workspaces
  swcl::DevBuf ws_coef;      // [n_walk][N_tr][N_I][n_h] cplx
  swcl::DevBuf ws_delta;     // FP64: [n_walk][N_ell][N_tr][N_k] double; mixed: float
  swcl::DevBuf ws_U;         // [n_walk][N_ell][N_tr][N_tr] double, unit-amplitude C
  swcl::DevBuf ws_C;         // [n_out][N_tr][N_tr] double, device staging for host outputs
  swcl::DevBuf ws_cbar;      // [n_walk][N_tr][N_I][n_h] cplx
  swcl::DevBuf ws_dbar;      // FP64: like ws_delta
  swcl::DevBuf ws_Cbar;      // [n_walk][N_ell][N_tr][N_tr] double, symmetrised, zero off-list
  swcl::DevBuf ws_outP, ws_outA, ws_outW;   // device staging of VJP outputs
  swcl::DevBuf ws_status;    // device status word(s)
  swcl::DevBuf ws_aimg;      // VJP: split Dbar image (tensor-core A operand)
  swcl::DevBuf ws_cpart;     // VJP: per-k-tile knot partial sums of cbar
  swcl::DevBuf ws_pbpart;    // VJP: per-multipole-chunk partial sums of P_bar
  swcl::DevBuf ws_qpart;     // forward: per-k-chunk partial pair sums of the k-quadrature
  swcl::DevBuf ws_jin;       // JVP: windows [1 + n_dir][N_tr][N] (base first), P' [n_dir][N_k], A' [n_dir][N_tr]
  swcl::DevBuf ws_dU;        // JVP: [n_dir][N_ell][N_tr][N_tr] tangent of U
  swcl::DevBuf ws_jout;      // JVP output / Fisher input staging for host arrays
  swcl::DevBuf ws_fz;        // Fisher: whitened perturbations [n_x][N_ell][N_tr][N_tr]
  swcl::DevBuf ws_fsmall;    // Fisher: noise [N_tr], modes [N_ell], F [n_x][n_x], status
  bool u_valid = false;      // ws_U holds U of walker 0 at the current inputs (n_walk = 1)
  int limber_switch = 0;     // multipoles >= this take the Limber branch (0 = none)
  swcl::DevBuf ws_lq;        // Limber scratch: forward partial pair sums, VJP weights and partials
  swcl::DevBuf ws_ltab;      // Limber stencil table (LimberTable)
  bool lt_ready = false;     // ws_ltab matches the grids and the switch
  cudaEvent_t ev_limber = nullptr;
  // swcl_compute_batched with a cotangent: the cotangent is unpacked on the auxiliary stream beside
  // the forward pass, and C is packed there beside the VJP (joined at the end of the VJP)
  bool overlap = false;
  // the kernels of the critical path start with programmatic dependent launch (launch_k) when
  // SWCL_PDL=1 at context creation; off by default (measured no faster inside the step's graph)
  bool pdl = false;
  cudaEvent_t ev_pre = nullptr, ev_unpack = nullptr, ev_pack = nullptr, ev_quad = nullptr;
  // pinned staging for small host inputs: copied on the host, then sent without a wait
  unsigned char* stage = nullptr;
  size_t stage_off = 0;
  cudaEvent_t ev_stage = nullptr;   // after the last copy out of `stage`
  int last_fwd_precision = -1;
  int ell_chunk = 0;         // multipoles per Delta chunk of the last forward pass (N_ell = whole)
  int ell_fft = 0;           // multipoles on the FFTLog path in the last forward pass (Limber after)

  // CUDA graph of the batched call (swcl_compute_batched)
  cudaGraphExec_t graph_exec = nullptr;
  struct GraphKey {
    int precision = -1;
    const void* ptrs[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int64_t alloc_gen = -1;
  } graph_key;
  int64_t alloc_gen = 0;      // bumped whenever a device buffer is (re)allocated or sizes change
  bool capturing = false;
  int64_t graph_launches = 0; // kernels in the captured graph

  // CUDA graph of swcl_step_host: host -> device copies of the step's inputs, the batched
  // kernels, device -> host copies of the results and of the status word
  cudaGraphExec_t hgraph_exec = nullptr;
  struct HostKey {
    int precision = -1;
    const void* ptrs[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int64_t alloc_gen = -1;
  } hgraph_key;
  int64_t hgraph_launches = 0;
  swcl::DevBuf hs_C, hs_Cb, hs_Pb, hs_Ab, hs_Wb;   // device side of the step's arrays
  int* hs_status = nullptr;                        // page-locked copy of the status word
  cudaEvent_t ev_host = nullptr;                   // end of the step, polled by the host
  int* hs_status_dev = nullptr;                    // its device-side address
  // host destinations that swcl_step_host sets for the duration of one capture: C, P_bar and
  // amp_bar go device -> host on the stream that produced them, as soon as they are final
  double* early_C = nullptr;
  double* early_Pb = nullptr;
  double* early_Ab = nullptr;

  // per-kernel timing (swcl_profile_*)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Pending { const char* name; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  cudaEvent_t ev_open = nullptr;
  struct Stat { std::string name; int64_t launches = 0; double ms = 0.0; };
  std::vector<Stat> stats;
};

// ---------------------------------------------------------------- helpers ----
namespace swcl {

int fail(swcl_ctx* c, int code, const std::string& msg);
int cuda_fail(swcl_ctx* c, cudaError_t e, const char* what);
int ensure(swcl_ctx* c, DevBuf& b, size_t bytes);
void release(swcl_ctx* c, DevBuf& b);
bool is_device_ptr(const void* p);
bool is_pinned_host_ptr(const void* p);   // page-locked host memory known to CUDA
// device-side address of page-locked host memory (null when the device cannot address it)
void* host_device_ptr(const void* p);

// Up to eight copies as one kernel (hostio.cu): segment s moves bytes[s] from src[s] to dst[s];
// either side may be page-locked host memory given by its device-side address.
struct CopyList {
  const void* src[8] = {};
  void* dst[8] = {};
  size_t bytes[8] = {};
  int n = 0;
  void add(void* d, const void* s, size_t b) {
    if (d && s && b) { src[n] = s; dst[n] = d; bytes[n] = b; ++n; }
  }
};
cudaError_t launch_copy_list(const CopyList& L, cudaStream_t s);
int copy_in(swcl_ctx* c, DevBuf& dst, const void* src, size_t bytes);
int copy_in_queued(swcl_ctx* c, DevBuf& dst, const void* src, size_t bytes, bool* host_src);
int copy_out(swcl_ctx* c, void* dst, const void* src, size_t bytes);
Stencil stencil(const swcl_ctx* c);
int factor_profiles(swcl_ctx* c);
int expand_basis_coefficients(swcl_ctx* c, void* out, bool df_input);
void prof_begin(swcl_ctx* c);
void prof_end(swcl_ctx* c, const char* name);

// ------------------------------------------------------------ launchers ----
// tables (tables.cu)
cudaError_t launch_fft_twiddles(cplx* tw, int N, cudaStream_t s);
cudaError_t launch_phase_table(cplx* phase, const double* k, int N_k, int n_h, double L,
                               cudaStream_t s);
cudaError_t launch_interp_weights(int* j0, double* w, const double* k, int N_k,
                                  const double* knots, int N_I, cudaStream_t s);
cudaError_t launch_quad_weights(double* wk2, const double* k, int N_k, cudaStream_t s);
cudaError_t launch_gamma_table(cplx* gtab, const int* ells, int N_ell, int n_h, double L,
                               double b, int kind, cudaStream_t s);
cudaError_t launch_tracer_tables(double* chipow, cplx* psi, double* kpow, const double* k,
                                 int N_k, int N, double chi_min, double L, double b, int kind,
                                 const double* taper_chi, const double* taper_c,
                                 cudaStream_t s);

// a1 FFTLog (fft.cu)
cudaError_t launch_fftlog_fwd(cplx* coef, const double* W, const double* chipow,
                              const double* D, const double* B, const cplx* psi,
                              const cplx* twiddle, int n_walk, int N_tr, int N_I, int N,
                              cudaStream_t s);
// same coefficients as double-float pairs (re_hi, im_hi, re_lo, im_lo), the input of the
// tensor-core contraction
cudaError_t launch_fftlog_fwd_df(float4* coef, const double* W, const double* chipow,
                                  const double* D, const double* B, const cplx* psi,
                                  const cplx* twiddle, int n_walk, int N_tr, int N_I, int N,
                                  cudaStream_t s);
// adjoint: W_bar[w][i][m] = chipow_i[m] sum_a D_a[m] B_ia[m] Re sum_n conj(psi_n) cbar_n e^{+2pi i n m/N}
cudaError_t launch_fftlog_adj(double* W_bar, const cplx* cbar, const double* chipow,
                              const double* D, const double* B, const cplx* psi,
                              const cplx* twiddle, int n_walk, int N_tr, int N_I, int N,
                              double* scratch, cudaStream_t s, int* status = nullptr,
                              bool pdl = false);
size_t fftlog_adj_scratch_bytes(int n_walk, int N_tr, int N_I, int N);
bool fftlog_adj_single_launch(int n_walk, int N_tr, int N_I, int N);   // no chunk reduction

// a3 FP64 contraction (contract_fp64.cu)
cudaError_t launch_contract_fp64(double* delta, const cplx* coef, const cplx* phase,
                                 const cplx* gtab, const int* cls_of, const double* kpow,
                                 const int* j0, const double* lw, long lw_ts, int n_walk,
                                 int N_tr, int N_I, int n_h, int N_k, int N_ell, int l_lo,
                                 int n_l, cudaStream_t s);
cudaError_t launch_contract_fp64_adj(cplx* cbar, const double* dbar, const cplx* phase,
                                     const cplx* gtab, const int* cls_of, const double* kpow,
                                     const int* j0, const double* lw, long lw_ts, int n_walk,
                                     int N_tr, int N_I, int n_h, int N_k, int N_ell, int l_lo,
                                     int n_l, bool accumulate, cudaStream_t s);

// a4 k-quadrature and VJP reductions (quad.cu).  Delta and Dbar buffers hold the multipoles
// l_lo .. l_lo + n_l - 1 ([n_walk][n_l][N_tr][N_k]); U and Cbar_full all N_ell.
// scratch: quad_scratch_bytes(n_walk, N_tr, N_k, n_l) of per-k-chunk pair sums
cudaError_t launch_quad_fp64(double* U, const double* delta, const double* P, const double* wk2,
                             int n_walk, int N_tr, int N_k, int N_ell, int l_lo, int n_l,
                             double* scratch, cudaStream_t s);
// listed [n_walk][n_l] (may be null): negative entries mark multipoles a walker does not list,
// whose U is written as zero without reading Delta
cudaError_t launch_quad_f32(double* U, const float* delta, const double* P, const double* wk2,
                            int n_walk, int N_tr, int N_k, int N_ell, int l_lo, int n_l,
                            double* scratch, cudaStream_t s, const int* listed = nullptr);
size_t quad_scratch_bytes(int n_walk, int N_tr, int N_k, int n_l);

// self-test of the bounded waits (selftest.cu)
cudaError_t launch_wait_nothing(int* status, long long* cycles, cudaStream_t s);
cudaError_t launch_scale_pack(double* C, const double* U, const double* amp, const int* off,
                              const int* idx, int n_walk, int N_tr, int N_ell, int64_t n_out,
                              cudaStream_t s, int* status = nullptr);
cudaError_t launch_unpack_sym(double* Cbar_full, const double* Cbar, const int* off,
                              const int* idx, int n_walk, int N_tr, int N_ell, int64_t n_out,
                              cudaStream_t s);
cudaError_t launch_amp_bar(double* amp_bar, const double* Cbar_full, const double* U,
                           const double* amp, int n_walk, int N_tr, int N_ell, cudaStream_t s,
                           int* status = nullptr);
// Dbar for the chunk and its partial sums of P_bar in scratch (indexed by
// the global multipole); launch_pbar_reduce adds all chunks into P_bar [n_walk][N_k]
template <typename T>
cudaError_t launch_delta_bar(T* dbar, const T* delta, const double* Cbar_full, const double* amp,
                             const double* P, const double* wk2, int n_walk, int N_tr, int N_k,
                             int N_ell, int l_lo, int n_l, double* scratch, cudaStream_t s,
                             const int* listed = nullptr,   // listed: as in launch_quad_f32
                             bool pdl = false);
cudaError_t launch_pbar_reduce(double* P_bar, const double* scratch, const double* wk2,
                               int n_walk, int N_k, int N_ell, cudaStream_t s,
                               int* status = nullptr);
size_t delta_bar_scratch_bytes(int n_walk, int N_k, int N_ell);

// Limber branch (limber.cu): the stencil table, then forward rows of U [n_walk][N_ell] (or, with
// the tangents Wt [n_dir][N_tr][N] (may be null) and Pd [n_dir][N_k], forward-mode rows of dU
// [n_dir][N_ell] for the base walker W, P), and the reverse mode adding into Wb (may be null) on
// s_main and into Pb on s_pbar (after q_ready).  scratch: limber_scratch_bytes(a, rows).
size_t limber_table_bytes(const LimberArgs& a);
LimberTable limber_table_view(void* base, const LimberArgs& a);
size_t limber_scratch_bytes(const LimberArgs& a, int n_rows);
cudaError_t launch_limber_table(const LimberTable& t, const LimberArgs& a, cudaStream_t s);
cudaError_t launch_limber_rows(double* U, double* scratch, const LimberArgs& a, const LimberTable& t,
                               const double* W, const double* P, int n_walk, cudaStream_t s);
cudaError_t launch_limber_jvp(double* dU, double* scratch, const LimberArgs& a, const LimberTable& t,
                              const double* W, const double* P, const double* Wt, const double* Pd,
                              int n_dir, cudaStream_t s);
cudaError_t launch_limber_vjp(double* Wb, double* Pb, double* scratch, const LimberArgs& a,
                              const LimberTable& t, const double* W, const double* P,
                              const double* Sfull, const double* amp, int n_walk,
                              cudaStream_t s_main, cudaStream_t s_pbar, cudaEvent_t q_ready,
                              int* status = nullptr);
// U[w][l_lo + ll][i][j] = U[..][j][i] = sum over n_chunk partial pair sums part[w][ll][chunk][pair]
// (quad.cu)
cudaError_t launch_pair_reduce(double* U, const double* part, int n_walk, int N_tr, int N_ell,
                               int l_lo, int n_l, int n_chunk, cudaStream_t s);

// forward mode and Fisher matrix (forecast.cu).  delta holds the base walker and then one
// walker per tangent ([1 + n_dir][n_l][N_tr][N_k]; only the base when !has_w); Pdot [n_dir][N_k].
template <typename T>
cudaError_t launch_quad_jvp(double* dU, const T* delta, const double* P, const double* Pdot,
                            const double* wk2, bool has_w, int n_dir, int N_tr, int N_k,
                            int N_ell, int l_lo, int n_l, cudaStream_t s);
cudaError_t launch_jvp_combine(double* Cdot, const double* dU, const double* U, const double* amp,
                               const double* Adot, int n_dir, int N_tr, int N_ell, cudaStream_t s,
                               int* status = nullptr);
// F [n_x][n_x] from X [n_x][N_ell][N_tr][N_tr], Ct = A A U + diag(noise); Z is scratch of X's size
cudaError_t launch_fisher(double* F, double* Z, const double* X, const double* U,
                          const double* amp, const double* noise, const double* modes,
                          int* status, int n_x, int N_tr, int N_ell, cudaStream_t s);

}  // namespace swcl
