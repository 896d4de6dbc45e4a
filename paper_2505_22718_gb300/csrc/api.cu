// C ABI of the library (include/swiftcl.h): argument checking, device buffers, and the
// sequence of kernels for the forward pass (a1-a4) and the VJP (a5).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <set>
#include <utility>

#include "swcl_internal.h"

using swcl::cplx;
using swcl::DevBuf;

namespace swcl {

int fail(swcl_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(swcl_ctx* c, cudaError_t e, const char* what) {
  return fail(c, SWCL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int ensure(swcl_ctx* c, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.p && b.bytes >= bytes) return SWCL_OK;
  size_t freed = b.p ? b.bytes : 0;
  if (c->budget && c->held - freed + bytes > c->budget)
    return fail(c, SWCL_ERR_OOM_BUDGET,
                "memory budget exceeded: need " + std::to_string(c->held - freed + bytes) +
                    " bytes, budget " + std::to_string(c->budget));
  if (b.p) {
    cudaFree(b.p);
    c->held -= b.bytes;
    b.p = nullptr;
    b.bytes = 0;
  }
  if (c->capturing)
    return fail(c, SWCL_ERR_STATE, "device buffer would grow during graph capture");
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return cuda_fail(c, e, "cudaMalloc");
  }
  b.bytes = bytes;
  c->held += bytes;
  ++c->alloc_gen;
  return SWCL_OK;
}

void release(swcl_ctx* c, DevBuf& b) {
  if (b.p) {
    cudaFree(b.p);
    c->held -= b.bytes;
  }
  b.p = nullptr;
  b.bytes = 0;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void* host_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

bool is_pinned_host_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

int copy_in(swcl_ctx* c, DevBuf& dst, const void* src, size_t bytes) {
  int st = ensure(c, dst, bytes);
  if (st) return st;
  cudaError_t e = cudaMemcpyAsync(dst.p, src, bytes, cudaMemcpyDefault, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync (input)");
  if (!is_device_ptr(src)) {
    e = cudaStreamSynchronize(c->stream);  // the caller may free a host array on return
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  }
  return SWCL_OK;
}

constexpr size_t kStageBytes = 4 << 20;      // pinned staging ring per context
constexpr size_t kStageMax = 1 << 20;        // host inputs up to this size go through it

// Queues a copy without waiting.  A small host array is first copied on the host into the
// context's pinned staging buffer (the caller may reuse it at once); a larger host array sets
// *host_src, and the caller then synchronises the stream once before returning.
int copy_in_queued(swcl_ctx* c, DevBuf& dst, const void* src, size_t bytes, bool* host_src) {
  int st = ensure(c, dst, bytes);
  if (st) return st;
  cudaError_t e;
  if (!is_device_ptr(src) && bytes <= kStageMax && c->stage) {
    if (c->stage_off + bytes > kStageBytes) {
      // every earlier copy out of the staging buffer has finished before it is overwritten
      e = cudaEventSynchronize(c->ev_stage);
      if (e != cudaSuccess) return cuda_fail(c, e, "staging wait");
      c->stage_off = 0;
    }
    unsigned char* p = c->stage + c->stage_off;
    std::memcpy(p, src, bytes);
    e = cudaMemcpyAsync(dst.p, p, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_stage, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync (staged input)");
    c->stage_off += (bytes + 255) & ~size_t(255);
    return SWCL_OK;
  }
  e = cudaMemcpyAsync(dst.p, src, bytes, cudaMemcpyDefault, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync (input)");
  if (!is_device_ptr(src)) *host_src = true;
  return SWCL_OK;
}

int copy_out(swcl_ctx* c, void* dst, const void* src, size_t bytes) {
  if (dst == src || bytes == 0) return SWCL_OK;
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync (output)");
  if (!is_device_ptr(dst)) {
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  }
  return SWCL_OK;
}

static cudaEvent_t take_event(swcl_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void prof_begin(swcl_ctx* c) {
  if (!c->prof || c->capturing) return;
  c->ev_open = take_event(c);
  if (c->ev_open) cudaEventRecord(c->ev_open, c->stream);
}

void prof_end(swcl_ctx* c, const char* name) {
  if (!c->prof || c->capturing || !c->ev_open) return;
  cudaEvent_t b = take_event(c);
  if (!b) return;
  cudaEventRecord(b, c->stream);
  c->pending.push_back({name, c->ev_open, b});
  c->ev_open = nullptr;
}

static int prof_flush(swcl_ctx* c) {
  if (c->pending.empty()) return SWCL_OK;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "profile sync");
  for (auto& p : c->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    swcl_ctx::Stat* st = nullptr;
    for (auto& s : c->stats)
      if (s.name == p.name) st = &s;
    if (!st) {
      c->stats.push_back(swcl_ctx::Stat{p.name, 0, 0.0});
      st = &c->stats.back();
    }
    st->launches += 1;
    st->ms += ms;
    c->ev_pool.push_back(p.a);
    c->ev_pool.push_back(p.b);
  }
  c->pending.clear();
  return SWCL_OK;
}

Stencil stencil(const swcl_ctx* c) {
  Stencil v;
  if (c->lr_basis) {
    v.j0 = (const int*)c->lr_j0.p;
    v.w = (const double*)c->lr_w.p;
    v.w_ts = c->have_B ? (long)c->N_k * 4 : 0;
    v.NI = c->have_B ? 4 : c->lr_true_rank;
    v.D = c->have_B ? (const double*)c->lr_ones.p : (const double*)c->lr_Q.p;
    v.B = c->have_B ? (const double*)c->lr_Q.p : nullptr;
  } else {
    v.j0 = (const int*)c->d_interp_j0.p;
    v.w = (const double*)c->d_interp_w.p;
    v.w_ts = 0;
    v.NI = c->N_I;
    v.D = (const double*)c->d_D.p;
    v.B = c->have_B ? (const double*)c->d_B.p : nullptr;
  }
  return v;
}

}  // namespace swcl

namespace {

__global__ void k_differs(int* flag, const double* a, const double* b, long n) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
    if (a[t] != b[t]) { *flag = 1; return; }
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

#define SWCL_TRY_CUDA(ctx, expr, what)                    \
  do {                                                    \
    cudaError_t _e = (expr);                              \
    if (_e != cudaSuccess) return swcl::cuda_fail(ctx, _e, what); \
  } while (0)

#define SWCL_TRY(expr)            \
  do {                            \
    int _s = (expr);              \
    if (_s != SWCL_OK) return _s; \
  } while (0)

#define SWCL_LAUNCH(ctx, expr, what)  \
  do {                                \
    ++(ctx)->last_launches;           \
    swcl::prof_begin(ctx);            \
    cudaError_t _le = (expr);         \
    swcl::prof_end(ctx, what);        \
    if (_le != cudaSuccess) return swcl::cuda_fail(ctx, _le, what); \
  } while (0)

int64_t out_count(const swcl_ctx* c) {
  return c->ragged ? c->n_out_ell : (int64_t)c->n_walk * c->N_ell;
}

}  // namespace

extern "C" {

const char* swcl_strerror(int s) {
  switch (s) {
    case SWCL_OK: return "ok";
    case SWCL_ERR_INVALID_ARG: return "invalid argument";
    case SWCL_ERR_UNSUPPORTED: return "unsupported";
    case SWCL_ERR_OOM_BUDGET: return "memory budget exceeded";
    case SWCL_ERR_CUDA: return "CUDA error";
    case SWCL_ERR_TIMEOUT: return "device wait timed out";
    case SWCL_ERR_NONFINITE: return "non-finite value";
    case SWCL_ERR_STATE: return "call out of order";
    default: return "unknown status";
  }
}

const char* swcl_last_error(swcl_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int swcl_create(swcl_ctx** out, int device, size_t mem_budget_bytes, void* stream) {
  if (!out) return SWCL_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return SWCL_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return SWCL_ERR_INVALID_ARG;
  DeviceGuard g(device);
  swcl_ctx* c = new swcl_ctx();
  c->device = device;
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      c->num_sms < 1) {
    cudaGetLastError();
    c->num_sms = 148;
  }
  c->budget = mem_budget_bytes;
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return SWCL_ERR_CUDA;
    }
    c->own_stream = true;
  }
  // a second stream and two events fork independent kernels of the VJP off the main stream
  // (the fork and join are recorded into CUDA graphs as branches)
  if (cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_limber, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_stage, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_pre, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_unpack, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_pack, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_quad, cudaEventDisableTiming) != cudaSuccess ||
      cudaHostAlloc((void**)&c->stage, swcl::kStageBytes, cudaHostAllocDefault) != cudaSuccess) {
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return SWCL_ERR_CUDA;
  }
  // SWCL_PER_KNOT_FFT=1 keeps the paper's one FFT per knot (no low-rank profiles)
  if (const char* v = std::getenv("SWCL_PER_KNOT_FFT")) c->lr_disabled = std::atoi(v) != 0;
  if (const char* v = std::getenv("SWCL_PDL")) c->pdl = std::atoi(v) != 0;
  if (const char* v = std::getenv("SWCL_BASIS_GEMM")) c->bt_disabled = std::atoi(v) == 0;
  // the accuracy study of the compensated products: a subset of the six products of the basis
  // GEMMs (bit t = product t in the order (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)); only the sets
  // 0x2F, 0x37, 0x1F, 0x17 and 0x07 exist, at the 96-column two-K-block tile (SWCL_BASIS_TILES
  // 1120,1120); they all miss the accuracy gate
  if (const char* v = std::getenv("SWCL_BASIS_PRODUCTS")) {
    const unsigned m = (unsigned)std::strtoul(v, nullptr, 0);
    if (m == 0x2Fu || m == 0x37u || m == 0x1Fu || m == 0x17u || m == 0x07u) c->bt_pmask = m;
  }
  // fixed basis-GEMM tiles "fwd,adj" (tile codes as reported by SWCL_Q_TILE_*) instead of tuning
  if (const char* v = std::getenv("SWCL_BASIS_TILES")) {
    int f = 0, a = 0;
    if (std::sscanf(v, "%d,%d", &f, &a) == 2) {
      c->bt_fixed_fwd = f;
      c->bt_fixed_adj = a;
    }
  }
  // device status word raised by bounded waits in the tensor-core kernels
  if (swcl::ensure(c, c->ws_status, 16) != SWCL_OK ||
      cudaMemset(c->ws_status.p, 0, 16) != cudaSuccess) {
    cudaGetLastError();
    if (c->own_stream) cudaStreamDestroy(c->stream);
    swcl::release(c, c->ws_status);
    delete c;
    return SWCL_ERR_CUDA;
  }
  *out = c;
  return SWCL_OK;
}

int swcl_destroy(swcl_ctx* c) {
  if (!c) return SWCL_OK;
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  DevBuf* bufs[] = {&c->d_k, &c->d_ells, &c->d_knots, &c->d_wk2, &c->d_interp_j0,
                    &c->d_interp_w, &c->d_twiddle, &c->d_phase, &c->d_knot_qrange,
                    &c->d_cls_of, &c->d_chipow, &c->d_psi, &c->d_gtab, &c->d_kpow, &c->d_W,
                    &c->d_D, &c->d_B, &c->d_P, &c->d_amp, &c->d_off, &c->d_idx, &c->ws_coef,
                    &c->ws_delta, &c->ws_U, &c->ws_C, &c->ws_cbar, &c->ws_dbar, &c->ws_Cbar,
                    &c->ws_outP, &c->ws_outA, &c->ws_outW, &c->ws_status, &c->tc_lw32,
                    &c->tc_kpow32, &c->tc_lw_lo, &c->tc_kpow_lo, &c->ws_aimg, &c->ws_cpart, &c->ws_pbpart, &c->d_prev,
                    &c->d_flag, &c->lr_res, &c->lr_norms, &c->lr_Q, &c->lr_coef, &c->lr_w,
                    &c->lr_j0, &c->lr_ones, &c->bt_eimg_f, &c->bt_eimg_a, &c->bt_gdf,
                    &c->bt_g32, &c->bt_kmu, &c->bt_himg, &c->bt_dimg, &c->ws_qpart, &c->bt_cmap_f,
                    &c->bt_cmap_a, &c->bt_lpos, &c->bt_wbase,
                    &c->ws_jin, &c->ws_dU, &c->ws_jout, &c->ws_fz, &c->ws_fsmall, &c->ws_lq,
                    &c->ws_ltab, &c->hs_C, &c->hs_Cb, &c->hs_Pb, &c->hs_Ab, &c->hs_Wb};
  for (DevBuf* b : bufs) swcl::release(c, *b);
  for (auto& t : c->tc) {
    swcl::release(c, t.bfwd);
    swcl::release(c, t.bvjp);
    swcl::release(c, t.phase32);
    swcl::release(c, t.phase_lo);
    swcl::release(c, t.tile_alo);
    swcl::release(c, t.knot_qt);
  }
  for (auto& p : c->pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->hgraph_exec) cudaGraphExecDestroy(c->hgraph_exec);
  if (c->hs_status) cudaFreeHost(c->hs_status);
  if (c->ev_host) cudaEventDestroy(c->ev_host);
  if (c->aux) cudaStreamDestroy(c->aux);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_limber) cudaEventDestroy(c->ev_limber);
  if (c->ev_stage) cudaEventDestroy(c->ev_stage);
  if (c->ev_pre) cudaEventDestroy(c->ev_pre);
  if (c->ev_unpack) cudaEventDestroy(c->ev_unpack);
  if (c->ev_pack) cudaEventDestroy(c->ev_pack);
  if (c->ev_quad) cudaEventDestroy(c->ev_quad);
  if (c->stage) cudaFreeHost(c->stage);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return SWCL_OK;
}

int swcl_set_grids(swcl_ctx* c, double chi_min, double chi_max, int N, const double* k, int N_k,
                   const int* ells, int N_ell, const double* knots, int N_I) {
  if (!c) return SWCL_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  c->err.clear();
  ++c->alloc_gen;
  if (!(chi_min > 0) || !(chi_max > chi_min) || !std::isfinite(chi_max))
    return swcl::fail(c, SWCL_ERR_INVALID_ARG, "need 0 < chi_min < chi_max");
  if (N < 16 || N > 8192 || (N & (N - 1)))
    return swcl::fail(c, SWCL_ERR_INVALID_ARG, "N must be a power of two in [16, 8192]");
  if (!k || N_k < 2 || !ells || N_ell < 1 || !knots || N_I < 1)
    return swcl::fail(c, SWCL_ERR_INVALID_ARG, "need k (N_k >= 2), ells (N_ell >= 1), knots (N_I >= 1)");
  std::vector<double> kh(N_k), knh(N_I);
  std::vector<int> eh(N_ell);
  SWCL_TRY_CUDA(c, cudaMemcpy(kh.data(), k, sizeof(double) * N_k, cudaMemcpyDefault), "copy k");
  SWCL_TRY_CUDA(c, cudaMemcpy(knh.data(), knots, sizeof(double) * N_I, cudaMemcpyDefault), "copy knots");
  SWCL_TRY_CUDA(c, cudaMemcpy(eh.data(), ells, sizeof(int) * N_ell, cudaMemcpyDefault), "copy ells");
  for (int q = 0; q < N_k; ++q)
    if (!(kh[q] > 0) || !std::isfinite(kh[q]) || (q && !(kh[q] > kh[q - 1])))
      return swcl::fail(c, SWCL_ERR_INVALID_ARG, "k must be finite, positive, strictly increasing");
  for (int a = 0; a < N_I; ++a)
    if (!(knh[a] > 0) || !std::isfinite(knh[a]) || (a && !(knh[a] > knh[a - 1])))
      return swcl::fail(c, SWCL_ERR_INVALID_ARG, "knots must be finite, positive, strictly increasing");
  for (int l = 0; l < N_ell; ++l)
    if (eh[l] < 0 || eh[l] > 100000) return swcl::fail(c, SWCL_ERR_INVALID_ARG, "ell out of range");
  c->have_grids = c->have_tracers = c->have_windows = c->have_power = false;
  ++c->lists_gen;
  c->lr_dirty = true;
  c->lr_basis = false;
  c->ragged = false;
  for (auto& t : c->tc) t.ready = t.adj_ready = false;
  c->bt_ready = false;
  c->N = N;
  c->n_h = N / 2 + 1;
  c->N_k = N_k;
  c->N_ell = N_ell;
  c->N_I = N_I;
  c->chi_min = chi_min;
  c->chi_max = chi_max;
  c->L = std::log(chi_max / chi_min);
  c->k_h = kh;
  c->knots_h = knh;
  c->ells_h = eh;
  c->last_fwd_precision = -1;
  c->u_valid = false;
  SWCL_TRY(swcl::copy_in(c, c->d_k, kh.data(), sizeof(double) * N_k));
  SWCL_TRY(swcl::copy_in(c, c->d_knots, knh.data(), sizeof(double) * N_I));
  SWCL_TRY(swcl::copy_in(c, c->d_ells, eh.data(), sizeof(int) * N_ell));
  SWCL_TRY(swcl::ensure(c, c->d_wk2, sizeof(double) * N_k));
  SWCL_TRY(swcl::ensure(c, c->d_interp_j0, sizeof(int) * N_k));
  SWCL_TRY(swcl::ensure(c, c->d_interp_w, sizeof(double) * 4 * N_k));
  SWCL_TRY(swcl::ensure(c, c->d_twiddle, sizeof(cplx) * N));
  SWCL_TRY(swcl::ensure(c, c->d_phase, sizeof(cplx) * (size_t)N_k * c->n_h));
  c->last_launches = 0;
  SWCL_LAUNCH(c, swcl::launch_fft_twiddles((cplx*)c->d_twiddle.p, N, c->stream), "twiddles");
  SWCL_LAUNCH(c, swcl::launch_phase_table((cplx*)c->d_phase.p, (const double*)c->d_k.p, N_k,
                                          c->n_h, c->L, c->stream), "phase table");
  SWCL_LAUNCH(c, swcl::launch_interp_weights((int*)c->d_interp_j0.p, (double*)c->d_interp_w.p,
                                             (const double*)c->d_k.p, N_k,
                                             (const double*)c->d_knots.p, N_I, c->stream),
              "interp weights");
  SWCL_LAUNCH(c, swcl::launch_quad_weights((double*)c->d_wk2.p, (const double*)c->d_k.p, N_k,
                                           c->stream), "quad weights");
  SWCL_TRY_CUDA(c, cudaStreamSynchronize(c->stream), "set_grids");
  c->have_grids = true;
  c->lt_ready = false;
  return SWCL_OK;
}

int swcl_set_tracers(swcl_ctx* c, int N_tr, const int* kind, const double* fft_bias,
                     const double* taper_chi, const double* taper_c) {
  if (!c) return SWCL_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  c->err.clear();
  ++c->alloc_gen;
  if (!c->have_grids) return swcl::fail(c, SWCL_ERR_STATE, "set_grids first");
  if (N_tr < 1 || N_tr > 64 || !kind || !fft_bias)
    return swcl::fail(c, SWCL_ERR_INVALID_ARG, "need 1 <= N_tr <= 64, kind and fft_bias");
  std::vector<int> kh(N_tr);
  std::vector<double> bh(N_tr);
  SWCL_TRY_CUDA(c, cudaMemcpy(kh.data(), kind, sizeof(int) * N_tr, cudaMemcpyDefault), "copy kind");
  SWCL_TRY_CUDA(c, cudaMemcpy(bh.data(), fft_bias, sizeof(double) * N_tr, cudaMemcpyDefault), "copy bias");
  int lmin = c->ells_h[0];
  for (int l : c->ells_h) lmin = l < lmin ? l : lmin;
  for (int i = 0; i < N_tr; ++i) {
    if (kh[i] < SWCL_DENSITY || kh[i] > SWCL_RSD)
      return swcl::fail(c, SWCL_ERR_INVALID_ARG,
                        "tracer kind must be SWCL_DENSITY, SWCL_LENSING, SWCL_MAGNIFICATION or SWCL_RSD");
    if ((kh[i] == SWCL_LENSING || kh[i] == SWCL_RSD) && lmin < 2)
      return swcl::fail(c, SWCL_ERR_INVALID_ARG, "lensing and RSD tracers need every ell >= 2");
    if (!(bh[i] < 1.0) || !(bh[i] > -(double)lmin - 1.0))
      return swcl::fail(c, SWCL_ERR_INVALID_ARG, "fft_bias must satisfy -ell_min - 1 < b < 1 (Eq. 3.4)");
    // the j_l'' moment is p (p - 1) M_l(p - 2): p - 2 must stay inside the strip of M_l
    if (kh[i] == SWCL_RSD && !(bh[i] > 1.0 - (double)lmin))
      return swcl::fail(c, SWCL_ERR_INVALID_ARG, "RSD tracers need 1 - ell_min < fft_bias < 1 (Eq. 2.10)");
  }
  // classes: distinct (kind, b)
  std::vector<std::pair<int, double>> cls;
  std::vector<int> cls_of(N_tr);
  for (int i = 0; i < N_tr; ++i) {
    int found = -1;
    for (size_t j = 0; j < cls.size(); ++j)
      if (cls[j].first == kh[i] && cls[j].second == bh[i]) found = (int)j;
    if (found < 0) {
      found = (int)cls.size();
      cls.push_back({kh[i], bh[i]});
    }
    cls_of[i] = found;
  }
  c->have_tracers = false;
  ++c->lists_gen;
  for (auto& t : c->tc) t.ready = t.adj_ready = false;
  c->bt_ready = false;
  c->last_fwd_precision = -1;
  c->u_valid = false;
  c->lr_dirty = true;
  c->lr_basis = false;
  c->N_tr = N_tr;
  c->n_cls = (int)cls.size();
  c->kind_h = kh;
  c->bias_h = bh;
  c->cls_of_h = cls_of;
  const int N = c->N, n_h = c->n_h;
  SWCL_TRY(swcl::copy_in(c, c->d_cls_of, cls_of.data(), sizeof(int) * N_tr));
  SWCL_TRY(swcl::ensure(c, c->d_chipow, sizeof(double) * N_tr * N));
  SWCL_TRY(swcl::ensure(c, c->d_psi, sizeof(cplx) * N_tr * n_h));
  SWCL_TRY(swcl::ensure(c, c->d_kpow, sizeof(double) * N_tr * c->N_k));
  SWCL_TRY(swcl::ensure(c, c->d_gtab, sizeof(cplx) * c->n_cls * (size_t)c->N_ell * n_h));
  DevBuf tchi, tcn;
  if (taper_chi) SWCL_TRY(swcl::copy_in(c, tchi, taper_chi, sizeof(double) * N_tr * N));
  if (taper_c) SWCL_TRY(swcl::copy_in(c, tcn, taper_c, sizeof(double) * N_tr * n_h));
  int st = SWCL_OK;
  for (int i = 0; i < N_tr && st == SWCL_OK; ++i) {
    cudaError_t e = swcl::launch_tracer_tables(
        (double*)c->d_chipow.p + (size_t)i * N, (cplx*)c->d_psi.p + (size_t)i * n_h,
        (double*)c->d_kpow.p + (size_t)i * c->N_k, (const double*)c->d_k.p, c->N_k, N,
        c->chi_min, c->L, bh[i], kh[i], taper_chi ? (const double*)tchi.p + (size_t)i * N : nullptr,
        taper_c ? (const double*)tcn.p + (size_t)i * n_h : nullptr, c->stream);
    if (e != cudaSuccess) st = swcl::cuda_fail(c, e, "tracer tables");
  }
  for (int j = 0; j < c->n_cls && st == SWCL_OK; ++j) {
    cudaError_t e = swcl::launch_gamma_table((cplx*)c->d_gtab.p + (size_t)j * c->N_ell * n_h,
                                             (const int*)c->d_ells.p, c->N_ell, n_h, c->L,
                                             cls[j].second, cls[j].first, c->stream);
    if (e != cudaSuccess) st = swcl::cuda_fail(c, e, "gamma table");
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  swcl::release(c, tchi);
  swcl::release(c, tcn);
  if (st) return st;
  if (e != cudaSuccess) return swcl::cuda_fail(c, e, "set_tracers");
  c->have_tracers = true;
  return SWCL_OK;
}

namespace {
// On an early error return, waits for copies already queued from host arrays, which the caller
// may free once the call returns.
struct QueuedHostCopies {
  swcl_ctx* c;
  bool pending = false;
  ~QueuedHostCopies() {
    if (pending) cudaStreamSynchronize(c->stream);
  }
};
}  // namespace

int swcl_set_windows(swcl_ctx* c, int n_walk, const double* W, const double* D, const double* B) {
  if (!c) return SWCL_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  c->err.clear();
  if (!c->have_tracers) return swcl::fail(c, SWCL_ERR_STATE, "set_grids and set_tracers first");
  if (n_walk < 1 || !W) return swcl::fail(c, SWCL_ERR_INVALID_ARG, "need n_walk >= 1 and W");
  if (c->have_power && c->n_walk != n_walk)
    return swcl::fail(c, SWCL_ERR_INVALID_ARG, "n_walk differs from set_power");
  const int N = c->N;
  // host sources are waited for once, at the end of the call
  QueuedHostCopies q{c};
  bool& host_src = q.pending;
  SWCL_TRY(swcl::copy_in_queued(c, c->d_W, W, sizeof(double) * (size_t)n_walk * c->N_tr * N, &host_src));
  // D and B: the knot profiles are re-factorised (low-rank mode) only when their values change
  const size_t dn = (size_t)c->N_I * N, bn = B ? (size_t)c->N_tr * c->N_I * N : 0;
  const bool had_prev = c->have_windows && c->have_B == (B != nullptr) && c->d_D.p &&
                        c->d_prev.p && c->d_prev.bytes >= sizeof(double) * (dn + bn);
  if (had_prev) {
    cudaError_t e = cudaMemcpyAsync(c->d_prev.p, c->d_D.p, sizeof(double) * dn, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && bn)
      e = cudaMemcpyAsync((double*)c->d_prev.p + dn, c->d_B.p, sizeof(double) * bn, cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return swcl::cuda_fail(c, e, "keep previous D");
  }
  if (D) {
    SWCL_TRY(swcl::copy_in_queued(c, c->d_D, D, sizeof(double) * dn, &host_src));
  } else {
    std::vector<double> ones(dn, 1.0);
    SWCL_TRY(swcl::copy_in(c, c->d_D, ones.data(), sizeof(double) * ones.size()));
  }
  if (c->have_B != (B != nullptr) || c->n_walk != n_walk) ++c->alloc_gen;  // new graph needed
  if (c->n_walk != n_walk) ++c->lists_gen;
  c->have_B = B != nullptr;
  if (B) SWCL_TRY(swcl::copy_in_queued(c, c->d_B, B, sizeof(double) * bn, &host_src));
  if (had_prev && !c->lr_dirty) {
    SWCL_TRY(swcl::ensure(c, c->d_flag, sizeof(int)));
    int flag = 0;
    SWCL_TRY_CUDA(c, cudaMemsetAsync(c->d_flag.p, 0, sizeof(int), c->stream), "flag");
    k_differs<<<152, 256, 0, c->stream>>>((int*)c->d_flag.p, (const double*)c->d_D.p,
                                           (const double*)c->d_prev.p, (long)dn);
    if (bn)
      k_differs<<<152, 256, 0, c->stream>>>((int*)c->d_flag.p, (const double*)c->d_B.p,
                                             (const double*)c->d_prev.p + dn, (long)bn);
    SWCL_TRY_CUDA(c, cudaMemcpyAsync(&flag, c->d_flag.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "flag read");
    SWCL_TRY_CUDA(c, cudaStreamSynchronize(c->stream), "flag sync");
    host_src = false;   // the flag read waited for the copies too
    if (flag) c->lr_dirty = true;
  } else {
    c->lr_dirty = true;
  }
  if (host_src) {
    host_src = false;
    SWCL_TRY_CUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  }
  SWCL_TRY(swcl::ensure(c, c->d_prev, sizeof(double) * (dn + bn)));
  c->n_walk = n_walk;
  c->have_windows = true;
  c->last_fwd_precision = -1;
  c->u_valid = false;
  if (c->ragged && (int)c->off_h.size() != n_walk + 1) c->ragged = false;
  return SWCL_OK;
}

int swcl_set_window_samples(swcl_ctx* c, int n_walk, const double* W) {
  if (!c) return SWCL_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  c->err.clear();
  if (!c->have_windows)
    return swcl::fail(c, SWCL_ERR_STATE, "swcl_set_windows first (it sets D, B and n_walk)");
  if (!W || n_walk != c->n_walk)
    return swcl::fail(c, SWCL_ERR_INVALID_ARG, "need W and the n_walk of the last swcl_set_windows");
  QueuedHostCopies q{c};
  SWCL_TRY(swcl::copy_in_queued(c, c->d_W, W, sizeof(double) * (size_t)n_walk * c->N_tr * c->N,
                                &q.pending));
  if (q.pending) {
    q.pending = false;
    SWCL_TRY_CUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  }
  c->last_fwd_precision = -1;
  c->u_valid = false;
  return SWCL_OK;
}

int swcl_set_power(swcl_ctx* c, int n_walk, const double* P, const double* amp) {
  if (!c) return SWCL_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  c->err.clear();
  if (!c->have_tracers) return swcl::fail(c, SWCL_ERR_STATE, "set_grids and set_tracers first");
  if (n_walk < 1 || !P || !amp) return swcl::fail(c, SWCL_ERR_INVALID_ARG, "need n_walk >= 1, P, amp");
  if (c->have_windows && c->n_walk != n_walk)
    return swcl::fail(c, SWCL_ERR_INVALID_ARG, "n_walk differs from set_windows");
  if (c->n_walk != n_walk) {
    ++c->alloc_gen;
    ++c->lists_gen;
  }
  QueuedHostCopies q{c};
  SWCL_TRY(swcl::copy_in_queued(c, c->d_P, P, sizeof(double) * (size_t)n_walk * c->N_k, &q.pending));
  SWCL_TRY(swcl::copy_in_queued(c, c->d_amp, amp, sizeof(double) * (size_t)n_walk * c->N_tr, &q.pending));
  if (q.pending) {
    q.pending = false;
    SWCL_TRY_CUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  }
  c->n_walk = n_walk;
  c->have_power = true;
  c->last_fwd_precision = -1;
  c->u_valid = false;
  return SWCL_OK;
}

int swcl_set_ell_lists(swcl_ctx* c, const int* offsets, const int* ell_idx) {
  if (!c) return SWCL_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  c->err.clear();
  ++c->alloc_gen;
  ++c->lists_gen;
  if (!c->have_windows && !c->have_power)
    return swcl::fail(c, SWCL_ERR_STATE, "set_windows or set_power first (they fix n_walk)");
  if (!offsets) {
    c->ragged = false;
    return SWCL_OK;
  }
  if (!ell_idx) return swcl::fail(c, SWCL_ERR_INVALID_ARG, "ell_idx is NULL");
  std::vector<int> off(c->n_walk + 1);
  SWCL_TRY_CUDA(c, cudaMemcpy(off.data(), offsets, sizeof(int) * off.size(), cudaMemcpyDefault), "copy offsets");
  if (off[0] != 0) return swcl::fail(c, SWCL_ERR_INVALID_ARG, "offsets[0] must be 0");
  for (int w = 0; w < c->n_walk; ++w)
    if (off[w + 1] < off[w]) return swcl::fail(c, SWCL_ERR_INVALID_ARG, "offsets must be nondecreasing");
  std::vector<int> idx(off.back());
  if (!idx.empty())
    SWCL_TRY_CUDA(c, cudaMemcpy(idx.data(), ell_idx, sizeof(int) * idx.size(), cudaMemcpyDefault), "copy ell_idx");
  for (int w = 0; w < c->n_walk; ++w)
    for (int o = off[w]; o < off[w + 1]; ++o) {
      if (idx[o] < 0 || idx[o] >= c->N_ell)
        return swcl::fail(c, SWCL_ERR_INVALID_ARG, "ell_idx entry outside the master list");
      if (o > off[w] && idx[o] <= idx[o - 1])
        return swcl::fail(c, SWCL_ERR_INVALID_ARG, "each walker's ell_idx must be strictly increasing");
    }
  c->off_h = off;
  c->idx_h = idx;
  SWCL_TRY(swcl::copy_in(c, c->d_off, off.data(), sizeof(int) * off.size()));
  SWCL_TRY(swcl::copy_in(c, c->d_idx, idx.empty() ? off.data() : idx.data(),
                         sizeof(int) * (idx.empty() ? 1 : idx.size())));
  c->n_out_ell = off.back();
  c->ragged = true;
  return SWCL_OK;
}

// Reads (and clears) the device status word: raised by the tensor-core kernels on a wait
// timeout, and by the kernels that write C, P_bar, amp_bar, W_bar or dC when a value they store
// is NaN or Inf.  A timeout is reported first.
static int check_status(swcl_ctx* c) {
  if (!c->ws_status.p) return SWCL_OK;
  int h = 0;
  cudaError_t e = cudaMemcpy(&h, c->ws_status.p, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return swcl::cuda_fail(c, e, "status read");
  if (h) {
    cudaMemset(c->ws_status.p, 0, sizeof(int));
    if (h & swcl::kStatusTimeout)
      return swcl::fail(c, SWCL_ERR_TIMEOUT, "a tensor-core kernel gave up waiting on an mbarrier");
    return swcl::fail(c, SWCL_ERR_NONFINITE,
                      "an output (C, P_bar, amp_bar, W_bar or dC) holds a NaN or Inf");
  }
  return SWCL_OK;
}

// Basis mode with split-bf16 products runs a3 and its transpose as GEMMs against the constant
// phase operand (basis_tc.cu); the other forms use the knot-stencil kernels with the basis view.
static bool use_basis_gemm(const swcl_ctx* c, int precision) {
  return precision == SWCL_SPLIT_BF16 && c->lr_basis && !c->bt_disabled;
}

static int check_ready(swcl_ctx* c, int precision) {
  if (!c->have_grids || !c->have_tracers || !c->have_windows || !c->have_power)
    return swcl::fail(c, SWCL_ERR_STATE, "set_grids, set_tracers, set_windows and set_power first");
  if (precision != SWCL_FP64 && precision != SWCL_3XTF32 && precision != SWCL_SPLIT_BF16 &&
      precision != SWCL_TF32X6)
    return swcl::fail(c, SWCL_ERR_INVALID_ARG, "unknown precision");
  return SWCL_OK;
}

// Multipoles per chunk of Delta: all of them, unless the memory budget cannot hold Delta and
// Dbar (and, in basis mode, the per-call GEMM operands) for every multipole at once.  Then the
// forward pass contracts and integrates chunk by chunk, and the VJP recomputes each chunk's
// Delta before its reverse mode.  Returns 0 when not even 8 multipoles fit.
static int plan_ell_chunk(swcl_ctx* c, int precision, int n_need) {
  // n_need: the multipoles that take the FFTLog path (all but the Limber rows)
  if (n_need <= 0) return c->N_ell;
  const int N_ell = c->N_ell;
  const bool fp64 = precision == SWCL_FP64;
  const bool basis = use_basis_gemm(c, precision);
  if (!fp64 && !basis) return N_ell;   // knot-stencil tensor-core forms: every multipole at once
  if (!c->budget) return n_need;
  const swcl::Stencil sv = swcl::stencil(c);
  const size_t nw = c->n_walk, nrow = nw * c->N_tr, ntr2 = (size_t)c->N_tr * c->N_tr;
  size_t per_l = 2 * nrow * c->N_k * (fp64 ? sizeof(double) : sizeof(float)) +
                 swcl::quad_scratch_bytes(c->n_walk, c->N_tr, c->N_k, 1);
  if (basis) per_l += swcl::basis_bytes_per_ell(c);
  // workspace that does not scale with the chunk
  size_t fixed = 2 * sizeof(cplx) * nrow * sv.NI * c->n_h              // coefficients, cbar
                 + 2 * sizeof(double) * nw * N_ell * ntr2               // U, symmetrised cotangent
                 + sizeof(double) * out_count(c) * ntr2                 // output staging
                 + sizeof(double) * nrow * c->N
                 + swcl::fftlog_adj_scratch_bytes(c->n_walk, c->N_tr, sv.NI, c->N)
                 + swcl::delta_bar_scratch_bytes(c->n_walk, c->N_k, N_ell)
                 + sizeof(double) * (nw * c->N_k + nrow);
  if (basis) fixed += swcl::basis_fixed_bytes(c);
  const DevBuf* ws[] = {&c->ws_coef, &c->ws_delta, &c->ws_U, &c->ws_C, &c->ws_cbar, &c->ws_dbar,
                        &c->ws_Cbar, &c->ws_outP, &c->ws_outA, &c->ws_outW, &c->ws_pbpart,
                        &c->ws_qpart, &c->bt_eimg_f, &c->bt_eimg_a, &c->bt_gdf, &c->bt_g32, &c->bt_kmu,
                        &c->bt_himg, &c->bt_dimg};
  size_t ws_now = 0;
  for (const DevBuf* b : ws) ws_now += b->bytes;
  const size_t other = c->held - ws_now;     // tables, inputs
  if (other + fixed + per_l * n_need <= c->budget) return n_need;
  if (other + fixed + per_l * 8 > c->budget) return 0;
  const size_t n = (c->budget - other - fixed) / per_l;
  return (int)std::min<size_t>(n_need, std::max<size_t>(8, n / 8 * 8));
}

// Delta for multipoles [l_lo, l_lo + n_l) into ws_delta ([n_walk][n_l][N_tr][N_k])
static int contract_chunk(swcl_ctx* c, int precision, int l_lo, int n_l) {
  const swcl::Stencil sv = swcl::stencil(c);
  if (!use_basis_gemm(c, precision)) c->bt_delta_clean = false;   // every row rewritten
  if (precision == SWCL_FP64) {
    SWCL_LAUNCH(c, swcl::launch_contract_fp64((double*)c->ws_delta.p, (const cplx*)c->ws_coef.p,
                                              (const cplx*)c->d_phase.p, (const cplx*)c->d_gtab.p,
                                              (const int*)c->d_cls_of.p, (const double*)c->d_kpow.p,
                                              sv.j0, sv.w, sv.w_ts, c->n_walk, c->N_tr, sv.NI,
                                              c->n_h, c->N_k, c->N_ell, l_lo, n_l, c->stream),
                "contract fp64");
    return SWCL_OK;
  }
  if (use_basis_gemm(c, precision)) return swcl::basis_forward(c, l_lo, n_l);
  if (l_lo != 0 || n_l != c->N_ell)
    return swcl::fail(c, SWCL_ERR_OOM_BUDGET, "the knot-stencil tensor-core form needs Delta for every multipole");
  return swcl::compute_delta_tc(c, precision);
}

// The Limber rows of the master list (multipoles >= the switch, a suffix of the ascending list):
// fills a and returns SWCL_OK; a.n_lim = 0 when the branch is off or no multipole reaches it.
static int limber_plan(swcl_ctx* c, int precision, swcl::LimberArgs& a) {
  a = swcl::LimberArgs();
  a.l_first = c->N_ell;
  if (c->limber_switch <= 0) return SWCL_OK;
  int first = c->N_ell;
  for (int i = 0; i < c->N_ell; ++i)
    if (c->ells_h[i] >= c->limber_switch) { first = i; break; }
  if (first == c->N_ell) return SWCL_OK;
  for (int i = 1; i < c->N_ell; ++i)
    if (c->ells_h[i] <= c->ells_h[i - 1])
      return swcl::fail(c, SWCL_ERR_INVALID_ARG, "the Limber branch needs an ascending multipole list");
  for (int i = 0; i < c->N_tr; ++i)
    if (c->kind_h[i] == SWCL_RSD)
      return swcl::fail(c, SWCL_ERR_UNSUPPORTED, "RSD tracers have no Limber form");
  if (precision != SWCL_FP64 && !use_basis_gemm(c, precision))
    return swcl::fail(c, SWCL_ERR_UNSUPPORTED,
                      "the Limber branch needs SWCL_FP64 or the basis-mode SWCL_SPLIT_BF16 form");
  a.k = (const double*)c->d_k.p;
  a.knots = (const double*)c->d_knots.p;
  a.ells = (const int*)c->d_ells.p;
  a.D = (const double*)c->d_D.p;
  a.B = c->have_B ? (const double*)c->d_B.p : nullptr;
  a.lnchi_min = std::log(c->chi_min);
  a.L = c->L;
  a.lnk_lo = std::log(c->k_h.front());
  a.lnk_hi = std::log(c->k_h.back());
  a.N = c->N;
  a.N_k = c->N_k;
  a.N_I = c->N_I;
  a.N_tr = c->N_tr;
  a.N_ell = c->N_ell;
  a.l_first = first;
  a.n_lim = c->N_ell - first;
  for (int i = 0; i < c->N_tr; ++i) a.kind[i] = c->kind_h[i];
  return SWCL_OK;
}

// The stencil table of the current grids and switch (built outside graph capture, once) and
// scratch for n_rows walkers or tangents.
static int limber_prepare(swcl_ctx* c, const swcl::LimberArgs& a, int n_rows, swcl::LimberTable& t) {
  if (!c->lt_ready) {
    if (c->capturing) return swcl::fail(c, SWCL_ERR_STATE, "Limber table built during capture");
    SWCL_TRY(swcl::ensure(c, c->ws_ltab, swcl::limber_table_bytes(a)));
    t = swcl::limber_table_view(c->ws_ltab.p, a);
    SWCL_LAUNCH(c, swcl::launch_limber_table(t, a, c->stream), "limber table");
    c->lt_ready = true;
  }
  t = swcl::limber_table_view(c->ws_ltab.p, a);
  return swcl::ensure(c, c->ws_lq, swcl::limber_scratch_bytes(a, n_rows));
}

int swcl_set_limber(swcl_ctx* c, int ell_switch) {
  if (!c) return SWCL_ERR_INVALID_ARG;
  c->err.clear();
  if (ell_switch < 0) return swcl::fail(c, SWCL_ERR_INVALID_ARG, "ell_switch must be >= 0");
  c->limber_switch = ell_switch;
  c->lt_ready = false;
  c->last_fwd_precision = -1;
  c->u_valid = false;
  ++c->alloc_gen;   // the captured graph of swcl_compute_batched has other kernels now
  return SWCL_OK;
}

int swcl_compute_cl(swcl_ctx* c, int precision, double* C_out) {
  if (!c) return SWCL_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  c->err.clear();
  SWCL_TRY(check_ready(c, precision));
  if (!C_out) return swcl::fail(c, SWCL_ERR_INVALID_ARG, "C_out is NULL");
  if (c->lr_dirty) {
    if (c->capturing) return swcl::fail(c, SWCL_ERR_STATE, "knot profiles changed during capture");
    SWCL_TRY(swcl::factor_profiles(c));
    c->lr_dirty = false;
  }
  c->last_launches = 0;
  const swcl::Stencil sv = swcl::stencil(c);
  const int nw = c->n_walk, N_tr = c->N_tr, N_I = sv.NI, n_h = c->n_h, N = c->N;
  const int N_k = c->N_k, N_ell = c->N_ell;
  const size_t nrow = (size_t)nw * N_tr;
  const bool fp64 = precision == SWCL_FP64;
  swcl::LimberArgs lim;
  SWCL_TRY(limber_plan(c, precision, lim));
  const int n_fft = lim.l_first;   // FFTLog multipoles [0, n_fft), Limber [n_fft, N_ell)
  // the Limber table and scratch first, so that the multipole chunks are planned around them
  swcl::LimberTable lt;
  if (lim.n_lim > 0) SWCL_TRY(limber_prepare(c, lim, nw, lt));
  const int n_lc = plan_ell_chunk(c, precision, n_fft);
  if (n_lc == 0)
    return swcl::fail(c, SWCL_ERR_OOM_BUDGET, "memory budget too small for 8 multipoles of Delta");
  SWCL_TRY(swcl::ensure(c, c->ws_coef, sizeof(cplx) * nrow * N_I * n_h));
  SWCL_TRY(swcl::ensure(c, c->ws_delta, nrow * n_lc * N_k * (fp64 ? sizeof(double) : sizeof(float))));
  SWCL_TRY(swcl::ensure(c, c->ws_U, sizeof(double) * nw * (size_t)N_ell * N_tr * N_tr));
  SWCL_TRY(swcl::ensure(c, c->ws_qpart, swcl::quad_scratch_bytes(nw, N_tr, N_k, n_lc)));
  if (fp64)
    SWCL_LAUNCH(c, swcl::launch_fftlog_fwd((cplx*)c->ws_coef.p, (const double*)c->d_W.p,
                                           (const double*)c->d_chipow.p, sv.D, sv.B,
                                           (const cplx*)c->d_psi.p, (const cplx*)c->d_twiddle.p,
                                           nw, N_tr, N_I, N, c->stream), "fftlog");
  else
    SWCL_LAUNCH(c, swcl::launch_fftlog_fwd_df((float4*)c->ws_coef.p, (const double*)c->d_W.p,
                                               (const double*)c->d_chipow.p, sv.D, sv.B,
                                               (const cplx*)c->d_psi.p, (const cplx*)c->d_twiddle.p,
                                               nw, N_tr, N_I, N, c->stream), "fftlog");
  // In a batched forward + VJP with one multipole chunk and no Limber rows, U feeds only the
  // packing of C and amp_bar, both on the auxiliary stream, while the VJP's Dbar needs Delta
  // alone: the k-quadrature then runs on the auxiliary stream too, beside the reverse mode.
  const bool quad_aside = c->overlap && n_lc >= n_fft && lim.n_lim == 0 && swcl::is_device_ptr(C_out);
  for (int l_lo = 0; l_lo < n_fft; l_lo += n_lc) {
    const int n_l = std::min(n_lc, n_fft - l_lo);
    SWCL_TRY(contract_chunk(c, precision, l_lo, n_l));
    cudaStream_t qs = c->stream;
    if (quad_aside) {
      SWCL_TRY_CUDA(c, cudaEventRecord(c->ev_quad, c->stream), "fork quadrature");
      SWCL_TRY_CUDA(c, cudaStreamWaitEvent(c->aux, c->ev_quad, 0), "fork quadrature");
      qs = c->aux;
    }
    if (fp64)
      SWCL_LAUNCH(c, swcl::launch_quad_fp64((double*)c->ws_U.p, (const double*)c->ws_delta.p,
                                            (const double*)c->d_P.p, (const double*)c->d_wk2.p, nw,
                                            N_tr, N_k, N_ell, l_lo, n_l, (double*)c->ws_qpart.p,
                                            qs), "k-quadrature fp64");
    else
      SWCL_LAUNCH(c, swcl::launch_quad_f32((double*)c->ws_U.p, (const float*)c->ws_delta.p,
                                           (const double*)c->d_P.p, (const double*)c->d_wk2.p, nw,
                                           N_tr, N_k, N_ell, l_lo, n_l, (double*)c->ws_qpart.p,
                                           qs,
                                           use_basis_gemm(c, precision) && c->bt_compact
                                               ? (const int*)c->bt_lpos.p : nullptr),
                  "k-quadrature f32");
    ++c->last_launches;  // the pair-sum reduction
  }
  if (lim.n_lim > 0) {
    SWCL_LAUNCH(c, swcl::launch_limber_rows((double*)c->ws_U.p, (double*)c->ws_lq.p, lim, lt,
                                            (const double*)c->d_W.p, (const double*)c->d_P.p, nw,
                                            c->stream), "limber");
    ++c->last_launches;  // the pair-sum reduction
  }
  c->ell_chunk = n_lc;
  c->ell_fft = n_fft;
  const int64_t n_out = out_count(c);
  const size_t cbytes = sizeof(double) * (size_t)n_out * N_tr * N_tr;
  double* dst = C_out;
  bool dev_out = swcl::is_device_ptr(C_out);
  if (!dev_out) {
    SWCL_TRY(swcl::ensure(c, c->ws_C, cbytes));
    dst = (double*)c->ws_C.p;
  }
  // in a batched forward + VJP the packing runs on the auxiliary stream beside the VJP, which
  // joins it at its end
  cudaStream_t pack_stream = c->stream;
  if (c->overlap && dev_out) {
    SWCL_TRY_CUDA(c, cudaEventRecord(c->ev_pack, c->stream), "fork pack");
    SWCL_TRY_CUDA(c, cudaStreamWaitEvent(c->aux, c->ev_pack, 0), "fork pack");
    pack_stream = c->aux;
  }
  SWCL_LAUNCH(c, swcl::launch_scale_pack(dst, (const double*)c->ws_U.p, (const double*)c->d_amp.p,
                                         c->ragged ? (const int*)c->d_off.p : nullptr,
                                         c->ragged ? (const int*)c->d_idx.p : nullptr, nw, N_tr,
                                         N_ell, n_out, pack_stream, (int*)c->ws_status.p),
              "scale/pack");
  if (c->early_C && dev_out)
    SWCL_TRY_CUDA(c, cudaMemcpyAsync(c->early_C, dst, cbytes, cudaMemcpyDeviceToHost, pack_stream),
                  "C device -> host");
  c->last_fwd_precision = precision;
  c->u_valid = true;
  if (!dev_out) {
    SWCL_TRY(swcl::copy_out(c, C_out, dst, cbytes));
    SWCL_TRY(check_status(c));
  }
  return SWCL_OK;
}

int swcl_vjp(swcl_ctx* c, int precision, const double* C_bar, double* P_bar, double* amp_bar,
             double* W_bar) {
  if (!c) return SWCL_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  c->err.clear();
  SWCL_TRY(check_ready(c, precision));
  if (!C_bar) return swcl::fail(c, SWCL_ERR_INVALID_ARG, "C_bar is NULL");
  if (c->last_fwd_precision != precision)
    return swcl::fail(c, SWCL_ERR_STATE, "call swcl_compute_cl with the same precision first");
  c->last_launches = 0;
  const swcl::Stencil sv = swcl::stencil(c);
  const int nw = c->n_walk, N_tr = c->N_tr, N_I = sv.NI, n_h = c->n_h, N = c->N;
  const int N_k = c->N_k, N_ell = c->N_ell;
  const int64_t n_out = out_count(c);
  const size_t nrow = (size_t)nw * N_tr;
  const bool fp64 = precision == SWCL_FP64;
  const int n_lc = c->ell_chunk;
  swcl::LimberArgs lim;
  SWCL_TRY(limber_plan(c, precision, lim));
  const int n_fft = lim.l_first;   // FFTLog multipoles [0, n_fft), Limber [n_fft, N_ell)
  const bool recompute = n_lc < n_fft;
  swcl::LimberTable lt;
  if (lim.n_lim > 0) SWCL_TRY(limber_prepare(c, lim, nw, lt));
  // cotangent on the device
  const size_t cbytes = sizeof(double) * (size_t)n_out * N_tr * N_tr;
  const double* cb = C_bar;
  if (!swcl::is_device_ptr(C_bar)) {
    SWCL_TRY(swcl::copy_in(c, c->ws_C, C_bar, cbytes));
    cb = (const double*)c->ws_C.p;
  }
  SWCL_TRY(swcl::ensure(c, c->ws_Cbar, sizeof(double) * nw * (size_t)N_ell * N_tr * N_tr));
  SWCL_TRY(swcl::ensure(c, c->ws_dbar, nrow * n_lc * N_k * (fp64 ? sizeof(double) : sizeof(float))));
  SWCL_TRY(swcl::ensure(c, c->ws_cbar, sizeof(cplx) * nrow * N_I * n_h));
  SWCL_TRY(swcl::ensure(c, c->ws_outP, sizeof(double) * nw * (size_t)N_k));
  SWCL_TRY(swcl::ensure(c, c->ws_outA, sizeof(double) * nrow));
  const size_t wbytes = sizeof(double) * nrow * N;
  SWCL_TRY(swcl::ensure(c, c->ws_outW, wbytes + swcl::fftlog_adj_scratch_bytes(nw, N_tr, N_I, N)));
  if (c->overlap) {
    // unpacked on the auxiliary stream during the forward pass (swcl_compute_batched)
    SWCL_TRY_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_unpack, 0), "join unpack");
  } else {
    SWCL_LAUNCH(c, swcl::launch_unpack_sym((double*)c->ws_Cbar.p, cb,
                                           c->ragged ? (const int*)c->d_off.p : nullptr,
                                           c->ragged ? (const int*)c->d_idx.p : nullptr, nw, N_tr,
                                           N_ell, n_out, c->stream), "unpack cotangent");
  }
  SWCL_TRY(swcl::ensure(c, c->ws_pbpart, swcl::delta_bar_scratch_bytes(nw, N_k, N_ell)));
  double* Pb = P_bar && swcl::is_device_ptr(P_bar) ? P_bar : (double*)c->ws_outP.p;
  double* Ab = amp_bar && swcl::is_device_ptr(amp_bar) ? amp_bar : (double*)c->ws_outA.p;
  // amp_bar and the P_bar reduction do not feed the transposed contraction: they run on the
  // auxiliary stream, beside it (not while profiling, which times kernels one by one)
  const bool fork = !c->prof;
  cudaStream_t side = fork ? c->aux : c->stream;
  if (fork) {
    SWCL_TRY_CUDA(c, cudaEventRecord(c->ev_fork, c->stream), "fork");
    SWCL_TRY_CUDA(c, cudaStreamWaitEvent(c->aux, c->ev_fork, 0), "fork");
  }
  SWCL_LAUNCH(c, swcl::launch_amp_bar(Ab, (const double*)c->ws_Cbar.p, (const double*)c->ws_U.p,
                                      (const double*)c->d_amp.p, nw, N_tr, N_ell, side,
                                      (int*)c->ws_status.p),
              "amp_bar");
  for (int l_lo = 0; l_lo < n_fft; l_lo += n_lc) {
    const int n_l = std::min(n_lc, n_fft - l_lo);
    const bool accumulate = l_lo > 0;
    if (recompute) SWCL_TRY(contract_chunk(c, precision, l_lo, n_l));
    if (fp64)
      SWCL_LAUNCH(c, swcl::launch_delta_bar<double>((double*)c->ws_dbar.p,
                                                    (const double*)c->ws_delta.p,
                                                    (const double*)c->ws_Cbar.p,
                                                    (const double*)c->d_amp.p, (const double*)c->d_P.p,
                                                    (const double*)c->d_wk2.p, nw, N_tr, N_k, N_ell,
                                                    l_lo, n_l, (double*)c->ws_pbpart.p, c->stream),
                  "delta_bar fp64");
    else
      SWCL_LAUNCH(c, swcl::launch_delta_bar<float>((float*)c->ws_dbar.p,
                                                   (const float*)c->ws_delta.p,
                                                   (const double*)c->ws_Cbar.p,
                                                   (const double*)c->d_amp.p, (const double*)c->d_P.p,
                                                   (const double*)c->d_wk2.p, nw, N_tr, N_k, N_ell,
                                                   l_lo, n_l, (double*)c->ws_pbpart.p, c->stream,
                                                   use_basis_gemm(c, precision) && c->bt_compact
                                                       ? (const int*)c->bt_lpos.p : nullptr,
                                                   c->pdl && !c->prof),
                  "delta_bar f32");
    if (!W_bar) continue;
    if (fp64) {
      SWCL_LAUNCH(c, swcl::launch_contract_fp64_adj((cplx*)c->ws_cbar.p, (const double*)c->ws_dbar.p,
                                                    (const cplx*)c->d_phase.p,
                                                    (const cplx*)c->d_gtab.p,
                                                    (const int*)c->d_cls_of.p,
                                                    (const double*)c->d_kpow.p,
                                                    sv.j0, sv.w, sv.w_ts, nw, N_tr, N_I,
                                                    n_h, N_k, N_ell, l_lo, n_l, accumulate,
                                                    c->stream), "contract adj fp64");
    } else if (use_basis_gemm(c, precision)) {
      SWCL_TRY(swcl::basis_adjoint(c, l_lo, n_l, accumulate));
    } else {
      SWCL_TRY(swcl::contract_adj_tc(c, precision));   // whole multipole range (no chunks)
    }
  }
  if (fork) {
    // the reduction waits for the last delta_bar chunk (main stream)
    SWCL_TRY_CUDA(c, cudaEventRecord(c->ev_fork, c->stream), "fork");
    SWCL_TRY_CUDA(c, cudaStreamWaitEvent(c->aux, c->ev_fork, 0), "fork");
  }
  SWCL_LAUNCH(c, swcl::launch_pbar_reduce(Pb, (const double*)c->ws_pbpart.p,
                                          (const double*)c->d_wk2.p, nw, N_k, n_fft, side,
                                          (int*)c->ws_status.p),
              "P_bar reduce");
  double* Wb = nullptr;
  if (W_bar) {
    Wb = swcl::is_device_ptr(W_bar) ? W_bar : (double*)c->ws_outW.p;
    double* scratch = (double*)((char*)c->ws_outW.p + wbytes);
    if (n_fft > 0) {
      SWCL_LAUNCH(c, swcl::launch_fftlog_adj(Wb, (const cplx*)c->ws_cbar.p,
                                             (const double*)c->d_chipow.p, sv.D, sv.B,
                                             (const cplx*)c->d_psi.p, (const cplx*)c->d_twiddle.p,
                                             nw, N_tr, N_I, N, scratch, c->stream,
                                             (int*)c->ws_status.p, c->pdl && !c->prof), "fftlog adj");
      if (!swcl::fftlog_adj_single_launch(nw, N_tr, N_I, N)) ++c->last_launches;  // chunk reduction
    } else {
      SWCL_TRY_CUDA(c, cudaMemsetAsync(Wb, 0, wbytes, c->stream), "clear W_bar");
    }
  }
  if (lim.n_lim > 0) {
    // W_bar (main stream, after the FFTLog adjoint) and P_bar (auxiliary stream, after its
    // reduction) gain the Limber rows' terms
    SWCL_LAUNCH(c, swcl::launch_limber_vjp(Wb, Pb, (double*)c->ws_lq.p, lim, lt,
                                           (const double*)c->d_W.p, (const double*)c->d_P.p,
                                           (const double*)c->ws_Cbar.p, (const double*)c->d_amp.p,
                                           nw, c->stream, side, c->ev_limber,
                                           (int*)c->ws_status.p), "limber vjp");
    c->last_launches += W_bar ? 3 : 2;  // W_bar reduction, P_bar gather and reduction
  }
  if (W_bar) SWCL_TRY(swcl::copy_out(c, W_bar, Wb, wbytes));
  // swcl_step_host: P_bar and amp_bar are final here on the side stream; their copies to the host
  // run beside the rest of the reverse mode
  if (c->early_Pb)
    SWCL_TRY_CUDA(c, cudaMemcpyAsync(c->early_Pb, Pb, sizeof(double) * nw * (size_t)N_k,
                                     cudaMemcpyDeviceToHost, side), "P_bar device -> host");
  if (c->early_Ab)
    SWCL_TRY_CUDA(c, cudaMemcpyAsync(c->early_Ab, Ab, sizeof(double) * nrow, cudaMemcpyDeviceToHost,
                                     side), "amp_bar device -> host");
  if (fork) {
    // join: the main stream (and the caller's later work on it) sees the auxiliary kernels
    SWCL_TRY_CUDA(c, cudaEventRecord(c->ev_join, c->aux), "join");
    SWCL_TRY_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_join, 0), "join");
  }
  if (P_bar) SWCL_TRY(swcl::copy_out(c, P_bar, Pb, sizeof(double) * nw * (size_t)N_k));
  if (amp_bar) SWCL_TRY(swcl::copy_out(c, amp_bar, Ab, sizeof(double) * nrow));
  // host outputs made the call synchronous: report a deferred device status now
  if ((P_bar && P_bar != Pb) || (amp_bar && amp_bar != Ab) || (W_bar && W_bar != Wb))
    SWCL_TRY(check_status(c));
  return SWCL_OK;
}

}  // extern "C"

// The kernels of one batched step (forward, and the VJP when C_bar is given) on the context
// stream, device pointers only; swcl_compute_batched and swcl_step_host capture it in graphs.
static int batched_body(swcl_ctx* c, int precision, double* C_out, const double* C_bar,
                        double* P_bar, double* amp_bar, double* W_bar) {
  // the cotangent's unpacking depends on C_bar alone: on the auxiliary stream, beside the
  // forward pass (not while profiling, which times kernels one by one)
  const bool overlap = C_bar && !c->prof;
  if (overlap) {
    const size_t n = (size_t)c->n_walk * c->N_ell * c->N_tr * c->N_tr;
    int st0 = swcl::ensure(c, c->ws_Cbar, sizeof(double) * n);
    if (st0) return st0;
    cudaError_t e = cudaEventRecord(c->ev_pre, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->aux, c->ev_pre, 0);
    if (e == cudaSuccess)
      e = swcl::launch_unpack_sym((double*)c->ws_Cbar.p, C_bar,
                                  c->ragged ? (const int*)c->d_off.p : nullptr,
                                  c->ragged ? (const int*)c->d_idx.p : nullptr, c->n_walk,
                                  c->N_tr, c->N_ell, out_count(c), c->aux);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_unpack, c->aux);
    if (e != cudaSuccess) return swcl::cuda_fail(c, e, "unpack cotangent");
  }
  c->overlap = overlap;
  int st = swcl_compute_cl(c, precision, C_out);
  const int64_t n_fwd = c->last_launches;
  if (st == SWCL_OK && C_bar) {
    st = swcl_vjp(c, precision, C_bar, P_bar, amp_bar, W_bar);
    c->last_launches += n_fwd + (overlap ? 1 : 0);   // forward and unpack kernels too
  }
  c->overlap = false;
  return st;
}

// Captures run() into a graph on the context stream (after one run outside it, which builds
// tables and sizes every buffer); on failure the partial graph is dropped.
template <class Run>
static int capture_graph(swcl_ctx* c, Run run, cudaGraphExec_t* exec, int64_t* gen_out) {
  SWCL_TRY(run());
  *gen_out = c->alloc_gen;
  cudaGraph_t graph = nullptr;
  SWCL_TRY_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  c->capturing = true;
  int st = run();
  c->capturing = false;
  if (st != SWCL_OK) {
    // a failed capture: join the auxiliary stream so that the capture can end, then drop the
    // partial graph and the capture error it leaves behind
    cudaEventRecord(c->ev_join, c->aux);
    cudaStreamWaitEvent(c->stream, c->ev_join, 0);
  }
  cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
  if (st != SWCL_OK) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return st;
  }
  if (e != cudaSuccess) return swcl::cuda_fail(c, e, "end capture");
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    *exec = nullptr;
    return swcl::cuda_fail(c, e, "graph instantiate");
  }
  return SWCL_OK;
}

extern "C" {

int swcl_compute_batched(swcl_ctx* c, int precision, double* C_out, const double* C_bar,
                         double* P_bar, double* amp_bar, double* W_bar) {
  if (!c) return SWCL_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  c->err.clear();
  SWCL_TRY(check_ready(c, precision));
  const void* ptrs[5] = {C_out, C_bar, P_bar, amp_bar, W_bar};
  for (const void* p : ptrs)
    if (p && !swcl::is_device_ptr(p))
      return swcl::fail(c, SWCL_ERR_INVALID_ARG, "swcl_compute_batched takes device pointers only");
  if (!C_out) return swcl::fail(c, SWCL_ERR_INVALID_ARG, "C_out is NULL");
  auto run = [&]() -> int { return batched_body(c, precision, C_out, C_bar, P_bar, amp_bar, W_bar); };
  bool same = c->graph_exec && c->graph_key.precision == precision &&
              c->graph_key.alloc_gen == c->alloc_gen;
  for (int t = 0; t < 5 && same; ++t) same = c->graph_key.ptrs[t] == ptrs[t];
  if (!same) {
    if (c->graph_exec) {
      cudaGraphExecDestroy(c->graph_exec);
      c->graph_exec = nullptr;
    }
    int64_t gen = 0;
    SWCL_TRY(capture_graph(c, run, &c->graph_exec, &gen));
    c->graph_key.precision = precision;
    c->graph_key.alloc_gen = gen;
    for (int t = 0; t < 5; ++t) c->graph_key.ptrs[t] = ptrs[t];
    c->graph_launches = c->last_launches;
  }
  SWCL_TRY_CUDA(c, cudaGraphLaunch(c->graph_exec, c->stream), "graph launch");
  c->last_launches = c->graph_launches;
  return SWCL_OK;
}

int swcl_step_host(swcl_ctx* c, int precision, const double* W, const double* P, const double* amp,
                   const double* C_bar, double* C_out, double* P_bar, double* amp_bar,
                   double* W_bar) {
  if (!c) return SWCL_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  c->err.clear();
  SWCL_TRY(check_ready(c, precision));
  if (!C_out) return swcl::fail(c, SWCL_ERR_INVALID_ARG, "C_out is NULL");
  if ((P == nullptr) != (amp == nullptr))
    return swcl::fail(c, SWCL_ERR_INVALID_ARG, "P and amp go together (both or neither)");
  if (!C_bar && (P_bar || amp_bar || W_bar))
    return swcl::fail(c, SWCL_ERR_INVALID_ARG, "gradients need C_bar");
  const void* ptrs[8] = {W, P, amp, C_bar, C_out, P_bar, amp_bar, W_bar};
  // the pointers of the captured graph were checked when it was captured
  bool known = c->hgraph_exec != nullptr;
  for (int t = 0; t < 8 && known; ++t) known = c->hgraph_key.ptrs[t] == ptrs[t];
  for (const void* p : ptrs)
    if (!known && p && !swcl::is_pinned_host_ptr(p))
      return swcl::fail(c, SWCL_ERR_INVALID_ARG,
                        "swcl_step_host takes page-locked host arrays only (cudaHostAlloc / cudaHostRegister)");
  const size_t nC = (size_t)out_count(c) * c->N_tr * c->N_tr;
  const size_t nW = (size_t)c->n_walk * c->N_tr * c->N, nP = (size_t)c->n_walk * c->N_k;
  const size_t nA = (size_t)c->n_walk * c->N_tr;
  SWCL_TRY(swcl::ensure(c, c->hs_C, sizeof(double) * nC));
  if (C_bar) SWCL_TRY(swcl::ensure(c, c->hs_Cb, sizeof(double) * nC));
  if (P_bar) SWCL_TRY(swcl::ensure(c, c->hs_Pb, sizeof(double) * nP));
  if (amp_bar) SWCL_TRY(swcl::ensure(c, c->hs_Ab, sizeof(double) * nA));
  if (W_bar) SWCL_TRY(swcl::ensure(c, c->hs_Wb, sizeof(double) * nW));
  if (!c->hs_status) {
    SWCL_TRY_CUDA(c, cudaHostAlloc((void**)&c->hs_status, sizeof(int), cudaHostAllocMapped),
                  "cudaHostAlloc (status word)");
    if (cudaHostGetDevicePointer((void**)&c->hs_status_dev, c->hs_status, 0) != cudaSuccess) {
      cudaGetLastError();
      c->hs_status_dev = nullptr;
    }
  }
  // the input buffers exist with these sizes since swcl_set_windows / swcl_set_power
  if (c->d_W.bytes < sizeof(double) * nW || c->d_P.bytes < sizeof(double) * nP ||
      c->d_amp.bytes < sizeof(double) * nA)
    return swcl::fail(c, SWCL_ERR_STATE, "set_windows and set_power for this n_walk first");
  double* dC = (double*)c->hs_C.p;
  double* dCb = C_bar ? (double*)c->hs_Cb.p : nullptr;
  double* dPb = P_bar ? (double*)c->hs_Pb.p : nullptr;
  double* dAb = amp_bar ? (double*)c->hs_Ab.p : nullptr;
  double* dWb = W_bar ? (double*)c->hs_Wb.p : nullptr;
  // The copies run as two kernels that address the host arrays directly, when the device can
  // (page-locked memory mapped into its address space); else as copy nodes.
  // (resolved when the graph is captured)
  const void* dptr[8] = {};
  bool direct = false;
  auto resolve = [&]() {
    direct = c->hs_status_dev != nullptr;
    for (int t = 0; t < 8 && direct; ++t)
      if (ptrs[t]) direct = (dptr[t] = swcl::host_device_ptr(ptrs[t])) != nullptr;
  };
  auto run_direct = [&]() -> int {
    swcl::CopyList in;
    in.add(c->d_W.p, dptr[0], sizeof(double) * nW);
    in.add(c->d_P.p, dptr[1], sizeof(double) * nP);
    in.add(c->d_amp.p, dptr[2], sizeof(double) * nA);
    in.add(dCb, dptr[3], sizeof(double) * nC);
    cudaError_t e = swcl::launch_copy_list(in, c->stream);
    if (e != cudaSuccess) return swcl::cuda_fail(c, e, "step inputs host -> device");
    int st = batched_body(c, precision, dC, dCb, dPb, dAb, dWb);
    if (st) return st;
    c->last_launches += 2;   // the two copy kernels
    swcl::CopyList out;
    out.add(const_cast<void*>(dptr[4]), dC, sizeof(double) * nC);
    out.add(const_cast<void*>(dptr[5]), dPb, sizeof(double) * nP);
    out.add(const_cast<void*>(dptr[6]), dAb, sizeof(double) * nA);
    out.add(const_cast<void*>(dptr[7]), dWb, sizeof(double) * nW);
    out.add(c->hs_status_dev, c->ws_status.p, sizeof(int));
    e = swcl::launch_copy_list(out, c->stream);
    if (e != cudaSuccess) return swcl::cuda_fail(c, e, "step results device -> host");
    return SWCL_OK;
  };
  auto run = [&]() -> int {
    if (direct) return run_direct();
    auto h2d = [&](void* dst, const void* src, size_t bytes) {
      return src ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream) : cudaSuccess;
    };
    auto d2h = [&](void* dst, const void* src, size_t bytes) {
      return dst ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream) : cudaSuccess;
    };
    // the cotangent is first read by its unpacking on the auxiliary stream (batched_body), so
    // its copy goes there and runs beside the window copy and the forward pass
    const bool aside = C_bar && !c->prof;
    cudaError_t e = cudaSuccess;
    if (aside) {
      e = cudaEventRecord(c->ev_fork, c->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(c->aux, c->ev_fork, 0);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(dCb, C_bar, sizeof(double) * nC, cudaMemcpyHostToDevice, c->aux);
    }
    if (e == cudaSuccess) e = h2d(c->d_W.p, W, sizeof(double) * nW);
    if (e == cudaSuccess) e = h2d(c->d_P.p, P, sizeof(double) * nP);
    if (e == cudaSuccess) e = h2d(c->d_amp.p, amp, sizeof(double) * nA);
    if (e == cudaSuccess && !aside) e = h2d(dCb, C_bar, sizeof(double) * nC);
    if (e != cudaSuccess) return swcl::cuda_fail(c, e, "step inputs host -> device");
    // C, P_bar and amp_bar are copied out by the kernels' own streams as soon as they are final
    c->early_C = C_out;
    c->early_Pb = P_bar;
    c->early_Ab = amp_bar;
    int st = batched_body(c, precision, dC, dCb, dPb, dAb, dWb);
    c->early_C = c->early_Pb = c->early_Ab = nullptr;
    if (st) return st;
    e = d2h(W_bar, dWb, sizeof(double) * nW);
    if (e == cudaSuccess) e = d2h(c->hs_status, c->ws_status.p, sizeof(int));
    if (e != cudaSuccess) return swcl::cuda_fail(c, e, "step results device -> host");
    return SWCL_OK;
  };
  bool same = c->hgraph_exec && c->hgraph_key.precision == precision &&
              c->hgraph_key.alloc_gen == c->alloc_gen;
  for (int t = 0; t < 8 && same; ++t) same = c->hgraph_key.ptrs[t] == ptrs[t];
  if (!same) {
    if (c->hgraph_exec) {
      cudaGraphExecDestroy(c->hgraph_exec);
      c->hgraph_exec = nullptr;
    }
    int64_t gen = 0;
    resolve();
    SWCL_TRY(capture_graph(c, run, &c->hgraph_exec, &gen));
    c->hgraph_key.precision = precision;
    c->hgraph_key.alloc_gen = gen;
    for (int t = 0; t < 8; ++t) c->hgraph_key.ptrs[t] = ptrs[t];
    c->hgraph_launches = c->last_launches;
  }
  SWCL_TRY_CUDA(c, cudaGraphLaunch(c->hgraph_exec, c->stream), "graph launch");
  // wait by polling an event: a sampler's step is short (a fraction of a millisecond), and a
  // polling thread sees the end of the graph sooner than one woken from a blocking wait
  if (!c->ev_host)
    SWCL_TRY_CUDA(c, cudaEventCreateWithFlags(&c->ev_host, cudaEventDisableTiming), "event");
  SWCL_TRY_CUDA(c, cudaEventRecord(c->ev_host, c->stream), "event record");
  for (;;) {
    const cudaError_t q = cudaEventQuery(c->ev_host);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return swcl::cuda_fail(c, q, "step wait");
  }
  c->last_launches = c->hgraph_launches;
  c->last_fwd_precision = precision;
  const int h = *c->hs_status;
  if (h) {
    *c->hs_status = 0;
    SWCL_TRY_CUDA(c, cudaMemset(c->ws_status.p, 0, sizeof(int)), "status clear");
    if (h & swcl::kStatusTimeout)
      return swcl::fail(c, SWCL_ERR_TIMEOUT, "a tensor-core kernel gave up waiting on an mbarrier");
    return swcl::fail(c, SWCL_ERR_NONFINITE,
                      "an output (C, P_bar, amp_bar or W_bar) holds a NaN or Inf");
  }
  return SWCL_OK;
}

namespace {

// c->n_walk is n for the lifetime of the scope: the JVP contracts the base walker and one walker
// per tangent window with the ordinary forward kernels
struct WalkScope {
  swcl_ctx* c;
  int old;
  WalkScope(swcl_ctx* c_, int n) : c(c_), old(c_->n_walk) { c->n_walk = n; }
  ~WalkScope() { c->n_walk = old; }
};

// bytes from a host or device array to a device address on the context stream; a host source
// is waited for, so that the caller may reuse it on return
int copy_to(swcl_ctx* c, void* dst, const void* src, size_t bytes, const char* what) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess && !swcl::is_device_ptr(src)) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? SWCL_OK : swcl::cuda_fail(c, e, what);
}

}  // namespace

int swcl_jvp(swcl_ctx* c, int precision, int n_dir, const double* P_dot, const double* amp_dot,
             const double* W_dot, double* C_dot) {
  if (!c) return SWCL_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  c->err.clear();
  SWCL_TRY(check_ready(c, precision));
  if (c->n_walk != 1)
    return swcl::fail(c, SWCL_ERR_UNSUPPORTED,
                      "the JVP is taken at one parameter point: set_windows with n_walk = 1");
  if (n_dir < 1 || n_dir > 256 || !C_dot)
    return swcl::fail(c, SWCL_ERR_INVALID_ARG, "need 1 <= n_dir <= 256 and C_dot");
  if (c->lr_dirty) {
    SWCL_TRY(swcl::factor_profiles(c));
    c->lr_dirty = false;
  }
  c->last_launches = 0;
  const swcl::Stencil sv = swcl::stencil(c);
  const int N_tr = c->N_tr, N_I = sv.NI, n_h = c->n_h, N = c->N, N_k = c->N_k, N_ell = c->N_ell;
  const bool fp64 = precision == SWCL_FP64;
  const bool has_w = W_dot != nullptr;
  const int nw2 = has_w ? 1 + n_dir : 1;
  const size_t wrow = (size_t)N_tr * N, n2 = (size_t)N_tr * N_tr;
  SWCL_TRY(swcl::ensure(c, c->ws_jin, sizeof(double) * (nw2 * wrow + (size_t)n_dir * (N_k + N_tr))));
  double* jW = (double*)c->ws_jin.p;
  double* jP = jW + nw2 * wrow;
  double* jA = jP + (size_t)n_dir * N_k;
  SWCL_TRY(copy_to(c, jW, c->d_W.p, sizeof(double) * wrow, "copy W"));
  if (has_w) SWCL_TRY(copy_to(c, jW + wrow, W_dot, sizeof(double) * n_dir * wrow, "copy W_dot"));
  if (P_dot) SWCL_TRY(copy_to(c, jP, P_dot, sizeof(double) * n_dir * N_k, "copy P_dot"));
  else SWCL_TRY_CUDA(c, cudaMemsetAsync(jP, 0, sizeof(double) * n_dir * N_k, c->stream), "clear P_dot");
  if (amp_dot) SWCL_TRY(copy_to(c, jA, amp_dot, sizeof(double) * n_dir * N_tr, "copy amp_dot"));
  else SWCL_TRY_CUDA(c, cudaMemsetAsync(jA, 0, sizeof(double) * n_dir * N_tr, c->stream), "clear amp_dot");
  SWCL_TRY(swcl::ensure(c, c->ws_U, sizeof(double) * N_ell * n2));
  SWCL_TRY(swcl::ensure(c, c->ws_dU, sizeof(double) * n_dir * N_ell * n2));
  swcl::LimberArgs lim;
  SWCL_TRY(limber_plan(c, precision, lim));
  const int n_fft = lim.l_first;   // FFTLog multipoles [0, n_fft), Limber [n_fft, N_ell)
  swcl::LimberTable lt;
  if (lim.n_lim > 0) SWCL_TRY(limber_prepare(c, lim, n_dir, lt));
  // the forward kernels see 1 + n_dir walkers: the base, then the tangent windows
  c->last_fwd_precision = -1;
  c->u_valid = false;
  {
    WalkScope scope(c, nw2);
    const int n_lc = plan_ell_chunk(c, precision, n_fft);
    if (n_lc == 0)
      return swcl::fail(c, SWCL_ERR_OOM_BUDGET, "memory budget too small for 8 multipoles of Delta");
    c->ell_chunk = n_lc;
    c->ell_fft = n_fft;
    SWCL_TRY(swcl::ensure(c, c->ws_coef, sizeof(cplx) * nw2 * N_tr * N_I * n_h));
    SWCL_TRY(swcl::ensure(c, c->ws_delta, (size_t)nw2 * N_tr * n_lc * N_k * (fp64 ? sizeof(double) : sizeof(float))));
    SWCL_TRY(swcl::ensure(c, c->ws_qpart, swcl::quad_scratch_bytes(1, N_tr, N_k, n_lc)));
    if (fp64)
      SWCL_LAUNCH(c, swcl::launch_fftlog_fwd((cplx*)c->ws_coef.p, jW, (const double*)c->d_chipow.p,
                                             sv.D, sv.B, (const cplx*)c->d_psi.p,
                                             (const cplx*)c->d_twiddle.p, nw2, N_tr, N_I, N,
                                             c->stream), "fftlog");
    else
      SWCL_LAUNCH(c, swcl::launch_fftlog_fwd_df((float4*)c->ws_coef.p, jW, (const double*)c->d_chipow.p,
                                                sv.D, sv.B, (const cplx*)c->d_psi.p,
                                                (const cplx*)c->d_twiddle.p, nw2, N_tr, N_I, N,
                                                c->stream), "fftlog");
    for (int l_lo = 0; l_lo < n_fft; l_lo += n_lc) {
      const int n_l = std::min(n_lc, n_fft - l_lo);
      SWCL_TRY(contract_chunk(c, precision, l_lo, n_l));
      // the base walker's U (first block of Delta), then the tangent pair sums
      if (fp64) {
        SWCL_LAUNCH(c, swcl::launch_quad_fp64((double*)c->ws_U.p, (const double*)c->ws_delta.p,
                                              (const double*)c->d_P.p, (const double*)c->d_wk2.p, 1,
                                              N_tr, N_k, N_ell, l_lo, n_l, (double*)c->ws_qpart.p,
                                              c->stream), "k-quadrature fp64");
        SWCL_LAUNCH(c, swcl::launch_quad_jvp<double>((double*)c->ws_dU.p, (const double*)c->ws_delta.p,
                                                     (const double*)c->d_P.p, jP,
                                                     (const double*)c->d_wk2.p, has_w, n_dir, N_tr,
                                                     N_k, N_ell, l_lo, n_l, c->stream), "jvp quadrature");
      } else {
        SWCL_LAUNCH(c, swcl::launch_quad_f32((double*)c->ws_U.p, (const float*)c->ws_delta.p,
                                             (const double*)c->d_P.p, (const double*)c->d_wk2.p, 1,
                                             N_tr, N_k, N_ell, l_lo, n_l, (double*)c->ws_qpart.p,
                                             c->stream), "k-quadrature f32");
        SWCL_LAUNCH(c, swcl::launch_quad_jvp<float>((double*)c->ws_dU.p, (const float*)c->ws_delta.p,
                                                    (const double*)c->d_P.p, jP,
                                                    (const double*)c->d_wk2.p, has_w, n_dir, N_tr,
                                                    N_k, N_ell, l_lo, n_l, c->stream), "jvp quadrature");
      }
      ++c->last_launches;  // the pair-sum reduction of the base quadrature
    }
  }
  if (lim.n_lim > 0) {
    SWCL_LAUNCH(c, swcl::launch_limber_rows((double*)c->ws_U.p, (double*)c->ws_lq.p, lim, lt, jW,
                                            (const double*)c->d_P.p, 1, c->stream), "limber");
    SWCL_LAUNCH(c, swcl::launch_limber_jvp((double*)c->ws_dU.p, (double*)c->ws_lq.p, lim, lt, jW,
                                           (const double*)c->d_P.p, has_w ? jW + wrow : nullptr, jP,
                                           n_dir, c->stream), "limber jvp");
    c->last_launches += 2;  // the pair-sum reductions
  }
  const size_t cbytes = sizeof(double) * n_dir * N_ell * n2;
  double* dst = C_dot;
  const bool dev_out = swcl::is_device_ptr(C_dot);
  if (!dev_out) {
    SWCL_TRY(swcl::ensure(c, c->ws_jout, cbytes));
    dst = (double*)c->ws_jout.p;
  }
  SWCL_LAUNCH(c, swcl::launch_jvp_combine(dst, (const double*)c->ws_dU.p, (const double*)c->ws_U.p,
                                          (const double*)c->d_amp.p, jA, n_dir, N_tr, N_ell,
                                          c->stream, (int*)c->ws_status.p), "jvp combine");
  c->u_valid = true;
  if (!dev_out) {
    SWCL_TRY(swcl::copy_out(c, C_dot, dst, cbytes));
    SWCL_TRY(check_status(c));
  }
  return SWCL_OK;
}

int swcl_gaussian_fisher(swcl_ctx* c, int n_x, const double* X, const double* noise,
                         const double* modes, double* F) {
  if (!c) return SWCL_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  c->err.clear();
  if (!c->u_valid || c->n_walk != 1)
    return swcl::fail(c, SWCL_ERR_STATE,
                      "call swcl_compute_cl or swcl_jvp at one parameter point (n_walk = 1) first");
  if (n_x < 1 || n_x > 1024 || !X || !modes || !F)
    return swcl::fail(c, SWCL_ERR_INVALID_ARG, "need 1 <= n_x <= 1024, X, modes and F");
  c->last_launches = 0;
  const int N_tr = c->N_tr, N_ell = c->N_ell;
  const size_t n2 = (size_t)N_tr * N_tr;
  std::vector<double> small(N_tr + N_ell, 0.0);
  if (noise)
    SWCL_TRY_CUDA(c, cudaMemcpy(small.data(), noise, sizeof(double) * N_tr, cudaMemcpyDefault), "copy noise");
  SWCL_TRY_CUDA(c, cudaMemcpy(small.data() + N_tr, modes, sizeof(double) * N_ell, cudaMemcpyDefault),
                "copy modes");
  for (int i = 0; i < N_tr + N_ell; ++i)
    if (!(small[i] >= 0.0) || !std::isfinite(small[i]))
      return swcl::fail(c, SWCL_ERR_INVALID_ARG, "noise and modes must be finite and >= 0");
  const size_t fbytes = sizeof(double) * n_x * n_x;
  SWCL_TRY(swcl::ensure(c, c->ws_fsmall, sizeof(double) * (N_tr + N_ell) + fbytes + 16));
  double* d_noise = (double*)c->ws_fsmall.p;
  double* d_modes = d_noise + N_tr;
  double* d_F = d_modes + N_ell;
  int* d_status = (int*)(d_F + (size_t)n_x * n_x);
  SWCL_TRY(copy_to(c, d_noise, small.data(), sizeof(double) * (N_tr + N_ell), "copy noise, modes"));
  const size_t xbytes = sizeof(double) * n_x * N_ell * n2;
  const double* Xd = X;
  if (!swcl::is_device_ptr(X)) {
    SWCL_TRY(swcl::ensure(c, c->ws_jout, xbytes));
    SWCL_TRY(copy_to(c, c->ws_jout.p, X, xbytes, "copy X"));
    Xd = (const double*)c->ws_jout.p;
  }
  SWCL_TRY(swcl::ensure(c, c->ws_fz, xbytes));
  SWCL_TRY_CUDA(c, cudaMemsetAsync(d_status, 0, sizeof(int), c->stream), "clear status");
  SWCL_LAUNCH(c, swcl::launch_fisher(d_F, (double*)c->ws_fz.p, Xd, (const double*)c->ws_U.p,
                                     (const double*)c->d_amp.p, noise ? d_noise : nullptr, d_modes,
                                     d_status, n_x, N_tr, N_ell, c->stream), "fisher");
  ++c->last_launches;  // whitening and Gram kernels
  int bad = 0;
  SWCL_TRY_CUDA(c, cudaMemcpyAsync(&bad, d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
                "read status");
  SWCL_TRY_CUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (bad)
    return swcl::fail(c, SWCL_ERR_INVALID_ARG, "C + noise is not positive definite at some multipole");
  SWCL_TRY(swcl::copy_out(c, F, d_F, fbytes));
  return SWCL_OK;
}

int swcl_profile_enable(swcl_ctx* c, int enable) {
  if (!c) return SWCL_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  if (!enable) {
    int st = swcl::prof_flush(c);
    c->prof = false;
    return st;
  }
  c->prof = true;
  return SWCL_OK;
}

int swcl_profile_reset(swcl_ctx* c) {
  if (!c) return SWCL_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  int st = swcl::prof_flush(c);
  c->stats.clear();
  return st;
}

int swcl_profile_read(swcl_ctx* c, int max_entries, char* names, int64_t* launches, double* ms,
                      int* n_entries) {
  if (!c || max_entries < 0 || !n_entries) return SWCL_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  int st = swcl::prof_flush(c);
  if (st) return st;
  int n = (int)c->stats.size();
  *n_entries = n;
  for (int i = 0; i < n && i < max_entries; ++i) {
    if (names) {
      std::strncpy(names + 32 * i, c->stats[i].name.c_str(), 31);
      names[32 * i + 31] = 0;
    }
    if (launches) launches[i] = c->stats[i].launches;
    if (ms) ms[i] = c->stats[i].ms;
  }
  return SWCL_OK;
}

namespace {
__global__ void k_widen(double* out, const float* in, long n) {
  long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = (double)in[t];
}
__global__ void k_join_df(double* out, const float4* in, long n) {
  long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    const float4 v = in[t];
    out[2 * t] = (double)v.x + (double)v.z;
    out[2 * t + 1] = (double)v.y + (double)v.w;
  }
}
}  // namespace

int swcl_debug_read(swcl_ctx* c, int what, double* out, int64_t* count) {
  if (!c || !count) return SWCL_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  c->err.clear();
  const void* src = nullptr;
  int64_t n = 0;
  bool widen = false, dfpair = false;
  switch (what) {
    case SWCL_DBG_COEF:
      src = c->ws_coef.p; n = 2LL * c->n_walk * c->N_tr * c->N_I * c->n_h;
      dfpair = c->last_fwd_precision > SWCL_FP64;
      if (c->lr_basis) {
        *count = n;
        if (!out) return SWCL_OK;
        if (c->last_fwd_precision < 0) return swcl::fail(c, SWCL_ERR_STATE, "no forward pass yet");
        DevBuf tmp;
        SWCL_TRY(swcl::ensure(c, tmp, sizeof(double) * n));
        int st = swcl::expand_basis_coefficients(c, tmp.p, dfpair);
        if (st == SWCL_OK) st = swcl::copy_out(c, out, tmp.p, sizeof(double) * n);
        cudaStreamSynchronize(c->stream);
        swcl::release(c, tmp);
        return st;
      }
      break;
    case SWCL_DBG_DELTA:
      src = c->ws_delta.p; n = (int64_t)c->n_walk * c->N_ell * c->N_tr * c->N_k;
      widen = c->last_fwd_precision != SWCL_FP64; break;
    case SWCL_DBG_GTAB:
      src = c->d_gtab.p; n = 2LL * c->n_cls * c->N_ell * c->n_h; break;
    case SWCL_DBG_PHASE:
      src = c->d_phase.p; n = 2LL * c->N_k * c->n_h; break;
    case SWCL_DBG_UNIT:
      src = c->ws_U.p; n = (int64_t)c->n_walk * c->N_ell * c->N_tr * c->N_tr; break;
    default:
      return swcl::fail(c, SWCL_ERR_INVALID_ARG, "unknown debug array");
  }
  *count = n;
  if (!out) return SWCL_OK;
  if (!src) return swcl::fail(c, SWCL_ERR_STATE, "array not computed yet");
  if (what == SWCL_DBG_DELTA && c->last_fwd_precision < 0)
    return swcl::fail(c, SWCL_ERR_STATE, "no forward pass yet");
  if (what == SWCL_DBG_DELTA &&
      (c->ell_chunk != c->N_ell || c->ell_fft != c->N_ell ||
       c->ws_delta.bytes < (size_t)n * (c->last_fwd_precision == SWCL_FP64 ? sizeof(double) : sizeof(float))))
    return swcl::fail(c, SWCL_ERR_STATE,
                      "Delta is held in multipole chunks (memory budget or Limber rows): not readable");
  if (dfpair) {
    // double-float pairs (re_hi, im_hi, re_lo, im_lo) -> (re, im)
    DevBuf tmp;
    SWCL_TRY(swcl::ensure(c, tmp, sizeof(double) * n));
    k_join_df<<<(unsigned)((n / 2 + 255) / 256), 256, 0, c->stream>>>((double*)tmp.p, (const float4*)src, n / 2);
    int st = swcl::copy_out(c, out, tmp.p, sizeof(double) * n);
    cudaStreamSynchronize(c->stream);
    swcl::release(c, tmp);
    return st;
  }
  if (widen) {
    DevBuf tmp;
    SWCL_TRY(swcl::ensure(c, tmp, sizeof(double) * n));
    k_widen<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>((double*)tmp.p, (const float*)src, n);
    int st = swcl::copy_out(c, out, tmp.p, sizeof(double) * n);
    cudaStreamSynchronize(c->stream);
    swcl::release(c, tmp);
    return st;
  }
  SWCL_TRY(swcl::copy_out(c, out, src, sizeof(double) * n));
  SWCL_TRY_CUDA(c, cudaStreamSynchronize(c->stream), "debug read");
  return SWCL_OK;
}

int swcl_selftest_wait_timeout(swcl_ctx* c, int64_t* cycles) {
  if (!c) return SWCL_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  c->err.clear();
  SWCL_TRY(swcl::ensure(c, c->d_flag, 16));
  SWCL_TRY_CUDA(c, swcl::launch_wait_nothing((int*)c->ws_status.p, (long long*)c->d_flag.p, c->stream),
                "self-test launch");
  long long h = 0;
  SWCL_TRY_CUDA(c, cudaMemcpyAsync(&h, c->d_flag.p, sizeof(h), cudaMemcpyDeviceToHost, c->stream),
                "self-test read");
  SWCL_TRY_CUDA(c, cudaStreamSynchronize(c->stream), "self-test sync");
  if (cycles) *cycles = h;
  return check_status(c);
}

int swcl_sync(swcl_ctx* c) {
  if (!c) return SWCL_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return swcl::cuda_fail(c, e, "swcl_sync");
  return check_status(c);
}

int swcl_query(swcl_ctx* c, int key, int64_t* value) {
  if (!c || !value) return SWCL_ERR_INVALID_ARG;
  switch (key) {
    case SWCL_Q_WORKSPACE_BYTES: *value = (int64_t)c->held; return SWCL_OK;
    case SWCL_Q_RECOMPUTE: *value = c->ell_chunk > 0 && c->ell_chunk < c->ell_fft ? 1 : 0; return SWCL_OK;
    case SWCL_Q_N_HALF: *value = c->n_h; return SWCL_OK;
    case SWCL_Q_KERNEL_LAUNCHES: *value = c->last_launches; return SWCL_OK;
    case SWCL_Q_PROFILE_RANK: *value = c->lr_basis ? c->lr_true_rank : 0; return SWCL_OK;
    case SWCL_Q_TILE_FWD: *value = c->bt_nt_fwd; return SWCL_OK;
    case SWCL_Q_TILE_ADJ: *value = c->bt_nt_adj; return SWCL_OK;
    default: return swcl::fail(c, SWCL_ERR_INVALID_ARG, "unknown query key");
  }
}

}  // extern "C"
