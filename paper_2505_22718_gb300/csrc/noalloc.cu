// swcl_fftlog_noalloc: the FFTLog step (a1) for callers that cannot allocate device memory.
//
// Some callers can't call cudaMalloc: a JAX or XLA process that has pre-reserved most of the
// GPU's memory for its own arena (cudaMalloc then fails), a plugin that must run inside another
// framework's fixed workspace, or a latency-critical loop where an allocation (and its
// implicit synchronisation) is not acceptable.  This entry point needs no context and allocates
// nothing.  The caller passes the inputs and the output; the per-call tables the FFT kernel reads
// besides them (twiddles, chi powers, output phases) live in one file-scope device array of
// fixed size, which every GPU that loads the library holds until the process exits.
#include <cmath>
#include <mutex>

#include "swcl_internal.h"

namespace {

constexpr size_t kScratchBytes = SWCL_NOALLOC_SCRATCH_BYTES;

// The shared scratch.  Host code must not take its address directly: in host code the name is
// a host-side stand-in, so its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Device address of the scratch on the current device, looked up once per device.  A cached
// address is checked against the runtime's view of it first: after a cudaDeviceReset (or any
// reload of the module on that device) the old address no longer belongs to device memory, and
// it is then looked up again instead of being written through.
bool still_device_memory(void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice;
}

int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return SWCL_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_scratch_addr[dev] && !still_device_memory(g_scratch_addr[dev])) g_scratch_addr[dev] = nullptr;
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return SWCL_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return SWCL_OK;
}

}  // namespace

extern "C" int swcl_fftlog_noalloc(int n_walk, int N_tr, int N_I, int N, double chi_min,
                                   double chi_max, const int* kind, const double* fft_bias,
                                   const double* taper_chi, const double* taper_c,
                                   const double* W, const double* D, const double* B,
                                   double* coef, void* stream) {
  if (n_walk < 1 || N_tr < 1 || N_I < 1 || N < 16 || N > 8192 || (N & (N - 1)))
    return SWCL_ERR_INVALID_ARG;
  if (!(chi_min > 0) || !(chi_max > chi_min) || !std::isfinite(chi_max) || !kind || !fft_bias ||
      !W || !D || !coef)
    return SWCL_ERR_INVALID_ARG;
  for (int i = 0; i < N_tr; ++i) {
    if (kind[i] < SWCL_DENSITY || kind[i] > SWCL_RSD) return SWCL_ERR_INVALID_ARG;
    if (!(fft_bias[i] < 1.0)) return SWCL_ERR_INVALID_ARG;
  }
  const int n_h = N / 2 + 1;
  const size_t tw_b = align256(sizeof(swcl::cplx) * N);
  const size_t cp_b = align256(sizeof(double) * (size_t)N_tr * N);
  const size_t ps_b = align256(sizeof(swcl::cplx) * (size_t)N_tr * n_h);
  if (tw_b + cp_b + ps_b > kScratchBytes) return SWCL_ERR_OOM_BUDGET;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SWCL_ERR_CUDA;
  }
  void* base = nullptr;
  int st = scratch_address(dev, &base);
  if (st != SWCL_OK) return st;
  char* p = static_cast<char*>(base);
  swcl::cplx* twiddle = reinterpret_cast<swcl::cplx*>(p);
  double* chipow = reinterpret_cast<double*>(p + tw_b);
  swcl::cplx* psi = reinterpret_cast<swcl::cplx*>(p + tw_b + cp_b);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double L = std::log(chi_max / chi_min);
  // every table entry is rewritten before the FFT reads it: nothing from an earlier call leaks
  cudaError_t e = swcl::launch_fft_twiddles(twiddle, N, s);
  for (int i = 0; i < N_tr && e == cudaSuccess; ++i)
    e = swcl::launch_tracer_tables(chipow + (size_t)i * N, psi + (size_t)i * n_h, nullptr, nullptr,
                                   0, N, chi_min, L, fft_bias[i], kind[i],
                                   taper_chi ? taper_chi + (size_t)i * N : nullptr,
                                   taper_c ? taper_c + (size_t)i * n_h : nullptr, s);
  if (e == cudaSuccess)
    e = swcl::launch_fftlog_fwd(reinterpret_cast<swcl::cplx*>(coef), W, chipow, D, B, psi, twiddle,
                                n_walk, N_tr, N_I, N, s);
  if (e != cudaSuccess) return SWCL_ERR_CUDA;
  return SWCL_OK;
}
