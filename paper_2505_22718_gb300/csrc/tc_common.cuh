// Inline-PTX building blocks for the sm_103a tensor-core kernels: mbarriers, bulk copies,
// tcgen05 (TMEM allocation, MMA, commit, loads) and the operand splits of the compensated
// products.  Shared by contract_tc.cu, contract_tc_adj.cu, basis_tc.cu and selftest.cu.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace swcl {
namespace tc {

constexpr int kMTile = 128;            // rows (k points) per CTA = TMEM lanes
constexpr int kRowBytes = 128;         // bytes of one operand row per K-block and plane
constexpr int kPlaneA = kMTile * kRowBytes;   // 16 KB
constexpr long kSpinLimit = 1L << 18;  // bounded mbarrier waits (about 1 s), then a timeout

// Arithmetic of the compensated products.  The formed A element is an FP32 value; it is split
// exactly into planes (A = a0 + a1 [+ a2]).  The B table is FP64 and split into planes of its
// own.  Products with pa + pb <= max order are accumulated in FP32 in TMEM.
//   Tf32x3:  A 2 tf32 planes, B 2 tf32 planes, products (0,0) (0,1) (1,0)            (~22 bits)
//   Tf32x6:  A 3 tf32 planes, B 3 tf32 planes, products with pa + pb <= 2 (6)       (~33 bits)
//   Bf16x9:  A 3 bf16 planes, B 4 bf16 planes, products with pa + pb <= 3 (9)       (~32 bits)
struct Tf32x3 {
  static constexpr int kPlanesA = 2, kPlanesB = 2;
  static constexpr int kKb = 32;        // K elements per 128-byte row
  static constexpr int kKmma = 8;       // K per MMA instruction
  static constexpr int kProducts = 3;
  static constexpr int kElemBytes = 4;
  static constexpr bool kBf16 = false;
  __host__ __device__ static constexpr int pa(int t) { return t == 2 ? 1 : 0; }
  __host__ __device__ static constexpr int pb(int t) { return t == 1 ? 1 : 0; }
  // instruction descriptor: D f32 (bits 4-5 = 1), A/B tf32 (bits 7-9, 10-12 = 2), K-major A and B
  __host__ __device__ static constexpr uint32_t idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
  }
};

struct Tf32x6 : Tf32x3 {
  static constexpr int kPlanesA = 3, kPlanesB = 3;
  static constexpr int kProducts = 6;
  // (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
  __host__ __device__ static constexpr int pa(int t) { return t == 2 ? 1 : t == 4 ? 1 : t == 5 ? 2 : 0; }
  __host__ __device__ static constexpr int pb(int t) { return t == 1 ? 1 : t == 3 ? 2 : t == 4 ? 1 : 0; }
};

struct Bf16x9 {
  static constexpr int kPlanesA = 3, kPlanesB = 4;
  static constexpr int kKb = 64;
  static constexpr int kKmma = 16;
  static constexpr int kProducts = 9;
  static constexpr int kElemBytes = 2;
  static constexpr bool kBf16 = true;
  // (0,0) (0,1) (1,0) (0,2) (1,1) (2,0) (0,3) (1,2) (2,1)
  __host__ __device__ static constexpr int pa(int t) {
    return t == 2 ? 1 : t == 4 ? 1 : t == 5 ? 2 : t == 7 ? 1 : t == 8 ? 2 : 0;
  }
  __host__ __device__ static constexpr int pb(int t) {
    return t == 1 ? 1 : t == 3 ? 2 : t == 4 ? 1 : t == 6 ? 3 : t == 7 ? 2 : t == 8 ? 1 : 0;
  }
  // D f32, A/B bf16 (bits 7-9, 10-12 = 1)
  __host__ __device__ static constexpr uint32_t idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
  }
};

// Byte offset of element (row r, k) inside one [rows x 128 B] plane of a K-block in the
// canonical K-major layout without swizzle: 8-row x 16-byte core matrices stored as 128
// contiguous bytes, K-adjacent cores 128 B apart (LBO), 8-row groups 1024 B apart (SBO).
__host__ __device__ inline uint32_t core_offset(int r, int kbyte) {
  return (uint32_t)((((r >> 3) * 8 + (kbyte >> 4)) << 7) + ((r & 7) << 4) + (kbyte & 15));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4 (16-29), SBO >> 4 (32-45),
// version 1 (bits 46-47), no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(1024 >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  uint64_t st;
  asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(st) : "r"(bar) : "memory");
  (void)st;
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  uint64_t st;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
               : "=l"(st) : "r"(bar), "r"(bytes) : "memory");
  (void)st;
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}
// Non-blocking test of a phase (never suspends the thread, unlike try_wait)
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}
// Bounded wait: gives up (and raises the CTA's abort flag) after kSpinLimit polls, or as soon
// as another thread of the CTA has raised it.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  for (long it = 0; it < kSpinLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}
// Same, ignoring the abort flag (used to drain work already in flight before teardown).
__device__ __forceinline__ bool mbar_wait_drain(uint32_t bar, uint32_t parity) {
  for (long it = 0; it < kSpinLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// global -> shared bulk copy completing on an mbarrier (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
               ::"r"(dst_slot), "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

template <class P>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                    uint32_t accumulate);
template <>
__device__ __forceinline__ void mma<Tf32x3>(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
}
template <>
__device__ __forceinline__ void mma<Tf32x6>(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  mma<Tf32x3>(d_tmem, adesc, bdesc, idesc, accumulate);
}
template <>
__device__ __forceinline__ void mma<Bf16x9>(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
}

// arrive on `bar` once every tcgen05 operation issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(bar) : "memory");
}

// 32 lanes x 16 columns of 32-bit TMEM words: thread (lane) gets its row's 16 columns
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int t = 0; t < 16; ++t) v[t] = __uint_as_float(r[t]);
}

// Double-float arithmetic (a value carried as hi + lo, |lo| <= ulp(hi)/2) from error-free
// transformations: the product's rounding error from an FMA, the sum's from TwoSum.
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// (a_hi + a_lo)(b_hi + b_lo) - (c_hi + c_lo)(d_hi + d_lo) in double-float (sgn = -1), or + (sgn = 1)
__device__ __forceinline__ void df_dot2(float ah, float al, float bh, float bl, float ch, float cl,
                                        float dh, float dl, float sgn, float& hi, float& lo) {
  float p1, e1, p2, e2;
  two_prod(ah, bh, p1, e1);
  two_prod(ch, dh, p2, e2);
  e1 = fmaf(ah, bl, fmaf(al, bh, e1));
  e2 = fmaf(ch, dl, fmaf(cl, dh, e2));
  float s, es;
  two_sum(p1, sgn * p2, s, es);
  const float l = es + e1 + sgn * e2;
  hi = s + l;
  lo = l - (hi - s);
}
// (s_hi, s_lo) += (a_hi + a_lo)(b_hi + b_lo) in double-float
__device__ __forceinline__ void df_fma(float ah, float al, float bh, float bl, float& sh, float& sl) {
  float p, e;
  two_prod(ah, bh, p, e);
  e = fmaf(ah, bl, fmaf(al, bh, e));
  float t, te;
  two_sum(sh, p, t, te);
  te += sl + e;
  sh = t + te;
  sl = te - (sh - t);
}

// tf32 rounding (to nearest, ties away), kept in a 32-bit float container
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

}  // namespace tc
}  // namespace swcl
