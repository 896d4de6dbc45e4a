// Copies between page-locked host arrays and device buffers as one kernel, for swcl_step_host:
// the step's inputs (window samples, P, amplitudes, cotangent) in one launch at its start and its
// results (C, P_bar, amp_bar, W_bar, the status word) in one launch at its end.  A CUDA graph
// holds them as two kernel nodes instead of one copy node per array; the kernel reads or writes
// the host arrays directly (page-locked memory is addressable from the device).
#include "swcl_internal.h"

namespace swcl {
namespace {

// segment s of the list: bytes[s] from src[s] to dst[s]; y = segment, x = grid-stride within it,
// in 16-, 8- or 4-byte units as the two addresses and the length allow
__global__ void k_copy_list(CopyList L) {
  const int s = blockIdx.y;
  if (s >= L.n) return;
  const char* src = static_cast<const char*>(L.src[s]);
  char* dst = static_cast<char*>(L.dst[s]);
  const size_t bytes = L.bytes[s];
  const uintptr_t al = reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst) | bytes;
  const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nt = (size_t)gridDim.x * blockDim.x;
  if ((al & 15) == 0) {
    const uint4* a = reinterpret_cast<const uint4*>(src);
    uint4* b = reinterpret_cast<uint4*>(dst);
    for (size_t e = t0; e < bytes / 16; e += nt) b[e] = a[e];
  } else if ((al & 7) == 0) {
    const uint2* a = reinterpret_cast<const uint2*>(src);
    uint2* b = reinterpret_cast<uint2*>(dst);
    for (size_t e = t0; e < bytes / 8; e += nt) b[e] = a[e];
  } else if ((al & 3) == 0) {
    const unsigned* a = reinterpret_cast<const unsigned*>(src);
    unsigned* b = reinterpret_cast<unsigned*>(dst);
    for (size_t e = t0; e < bytes / 4; e += nt) b[e] = a[e];
  } else {
    for (size_t e = t0; e < bytes; e += nt) dst[e] = src[e];
  }
}

}  // namespace

cudaError_t launch_copy_list(const CopyList& L, cudaStream_t s) {
  if (L.n <= 0) return cudaSuccess;
  size_t most = 0;
  for (int i = 0; i < L.n; ++i) most = L.bytes[i] > most ? L.bytes[i] : most;
  // 16 bytes per thread and pass; at most 64 blocks per segment
  const size_t blocks = (most / 16 + 255) / 256;
  const unsigned gx = (unsigned)(blocks < 1 ? 1 : blocks > 64 ? 64 : blocks);
  k_copy_list<<<dim3(gx, (unsigned)L.n), 256, 0, s>>>(L);
  return cudaGetLastError();
}

}  // namespace swcl
