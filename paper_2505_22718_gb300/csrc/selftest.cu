// Self-test of the bounded-wait path the tensor-core kernels share: one thread waits on an
// mbarrier phase that nothing completes.  The wait gives up after the same poll limit as every
// wait in those kernels, raises the abort flag and the context's status word; the host then
// reports SWCL_ERR_TIMEOUT and the context stays usable.  No fault, trap or unbounded loop.
#include "swcl_internal.h"
#include "tc_common.cuh"

namespace swcl {
namespace {

__global__ void k_wait_nothing(int* __restrict__ status, long long* __restrict__ cycles) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x != 0) return;
  tc::mbar_init(tc::smem_u32(&bar), 1);
  abort_flag = 0;
  tc::fence_barrier_init();
  const long long t0 = clock64();
  const bool ok = tc::mbar_wait(tc::smem_u32(&bar), 0, &abort_flag);  // phase 0 never completes
  *cycles = clock64() - t0;
  if (!ok && abort_flag) atomicExch(status, 1);
}

}  // namespace

cudaError_t launch_wait_nothing(int* status, long long* cycles, cudaStream_t s) {
  k_wait_nothing<<<1, 32, 0, s>>>(status, cycles);
  return cudaGetLastError();
}

}  // namespace swcl
