// a3 and its transpose (a5) on the tensor cores in basis mode, where the knot profiles are low
// rank (lowrank.cu): both become GEMMs against one constant operand, the phase table
// E_{q,n} = e^{-i eta_n ln k_q}.
//
// With r basis profiles of FFTLog coefficients F_{w,i,s,n} (Eq. 3.3) and weights
// mu_{i,q,s} = sum_a lambda_{q,a} coef_{i,a,s} (the k-interpolation of Sec. 3.2 carried through the
// basis), Eq. 3.4-3.5 read
//   Delta_i(l, q) = kpow_i[q] sum_s mu_{i,q,s} Re sum_n E_{q,n} H_{w,i,l,s,n},
//   H_{w,i,l,s,n} = F_{w,i,s,n} G_{cls(i)}[l][n],   G = w_n pi_i(l) M_{l,n}.
// Forward GEMM: rows q, columns (w, i, l, s) (s fastest), K = (n, re/im) interleaved:
//   A[q][2n] = Re E, A[q][2n+1] = Im E;  B[j][2n] = Re H, B[j][2n+1] = -Im H.
// The reverse mode of the same expression is
//   Fbar_{w,i,s,n} = sum_l conj(G[l][n]) Y_{w,i,s,l,n},
//   Y_{w,i,s,l,n} = sum_q conj(E_{q,n}) kpow_i[q] mu_{i,q,s} Dbar_i(l, q),
// the adjoint GEMM: rows (n, re/im), columns (w, i, s, l) (l fastest), K = q:
//   A[2n][q] = Re E, A[2n+1][q] = -Im E;  B[j][q] = kpow mu Dbar;
// its epilogue multiplies by conj(G) and sums over l.
//
// Compensated products with FP32 accumulation (the 5th-generation tensor cores take bf16 operands
// here): the constant operand is split once from FP64 into 3 bf16 planes; the forward B operand
// H is formed in double-float arithmetic from double-float F and G and split into 3 planes; the
// adjoint B operand is an FP32 product split exactly into 3 planes.  The 6 products with
// pa + pb <= 2 are issued.  The tensor core accumulates one pipeline stage at a time (KS = 1 or 2
// consecutive 32-deep K-blocks), the leading product and the corrections in separate TMEM slots
// (double-buffered); the drain warps add each stage's partial sums into FP32 registers with
// round-to-nearest.
//
// Warp roles: warp 0 streams both operand images into a shared-memory ring with cp.async.bulk;
// warp 1 owns TMEM and issues tcgen05.mma; the remaining 4 or 8 warps drain TMEM (with 8, two
// warps per 32-lane quarter, each with half of the columns) and run the epilogue.  All waits are bounded; a timeout raises
// the context's status word (SWCL_ERR_TIMEOUT).
#include <algorithm>
#include <cuda_bf16.h>

#include "swcl_internal.h"
#include "tc_common.cuh"

namespace swcl {
namespace {

using namespace tc;

constexpr int kK = 32;                  // K elements (bf16) per 64-byte operand row
constexpr int kRow = 64;                // bytes per operand row and K-block
constexpr int kM = 128;                 // rows per CTA (TMEM lanes)
constexpr int kPlaneM = kM * kRow;      // 8 KB: one plane of the A operand per K-block
// Two variants: DW = 8 drain warps (one CTA per SM, column tiles up to 128) and DW = 4 (tiles
// up to 64, two CTAs per SM: two MMA-issuing threads share the SM's tensor core, which pays when
// one thread alone cannot issue small MMAs as fast as the tensor core runs them).
__host__ __device__ constexpr int threads_for(int DW) { return 64 + 32 * DW; }
constexpr int kMaxNT = 128;
constexpr int kHalf = kMaxNT / 2;       // columns per drain thread at most
constexpr int kMaxStages = 6;

// Both operands 3 bf16 planes (24 significant bits); the products with pa + pb <= 2:
// (0,0) | (0,1) (1,0) (0,2) (1,1) (2,0).  The dropped terms are below 2^-24 of each product, the
// same as the FP32 accumulation in which the sums are formed (measured: the normalised C error of
// the N5K-shaped and large workloads is the same with 10 products as with these 6).
struct A3B3 {
  static constexpr int kPlanesA = 3, kPlanesB = 3, kProducts = 6;
  __host__ __device__ static constexpr int pa(int t) { return t == 2 ? 1 : t == 4 ? 1 : t == 5 ? 2 : 0; }
  __host__ __device__ static constexpr int pb(int t) { return t == 1 ? 1 : t == 3 ? 2 : t == 4 ? 1 : 0; }
};
constexpr int kPlanes = 3;      // planes of every operand image

// D f32, A/B bf16, K-major A and B, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of (row r, byte kb) in one [rows x 64 B] plane, canonical K-major layout without
// swizzle: 8-row x 16-byte core matrices of 128 contiguous bytes, K-adjacent cores 128 B apart
// (LBO), 8-row groups 512 B apart (SBO).
__host__ __device__ inline uint32_t off64(int r, int kbyte) {
  return (uint32_t)((((r >> 3) * 4 + (kbyte >> 4)) << 7) + ((r & 7) << 4) + (kbyte & 15));
}
__device__ __forceinline__ uint64_t desc64(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(512 >> 4) << 32) | (1ull << 46);
}

// 32 lanes x 16 columns of 32-bit TMEM words without waiting: the registers are valid after
// tmem_wait_ld(); reg_fence() keeps their uses behind the wait.
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void reg_fence(uint32_t (&r)[16]) {
#pragma unroll
  for (int t = 0; t < 16; ++t) asm volatile("" : "+r"(r[t]));
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
      ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

// Cluster helpers (the two-SM tile and the split-K tile)
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_addr(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cl_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cl_addr) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cl(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait_cl(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cl(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  for (long it = 0; it < kSpinLimit; ++it) {
    if (mbar_try_wait_cl(bar, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}
// every thread of both CTAs
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// TMEM of both CTAs, allocated and released by one warp in each of them together
__device__ __forceinline__ void tmem_alloc_pair(uint32_t dst_slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;"
               ::"r"(dst_slot), "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void mma_bf16_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                              uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}"
      ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
// arrive on the barrier at cluster address `bar` once every MMA issued so far has completed
__device__ __forceinline__ void mma_commit_pair(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(bar) : "memory");
}

// A stage holds KS consecutive K-blocks (contiguous in both images): KS A-blocks of a1 bytes,
// then KS B-blocks of b1 bytes.
struct Layout {
  uint32_t a1, b1, a_bytes, b_bytes, stage, bar_off, total;
  int stages;
};
template <class P>
__host__ __device__ inline Layout layout(int NT, int stages, int KS) {
  Layout L;
  L.stages = stages;
  L.a1 = P::kPlanesA * kPlaneM;
  L.b1 = P::kPlanesB * NT * kRow;
  L.a_bytes = KS * L.a1;
  L.b_bytes = KS * L.b1;
  L.stage = L.a_bytes + L.b_bytes;
  L.bar_off = stages * L.stage;
  L.total = L.bar_off + 8 * (3 * stages + 1) + 16 + 1024;
  return L;
}

struct GemmShape {
  int n_mt, n_kb, NT, stages;
  uint32_t tmem_cols;
  uint32_t pre_off;     // offset of the epilogue's staged table rows (0: none), k_gemm_basis only
};

// Products issued (bit t = product t of A3B3) and the first correction among them, whose MMA
// overwrites the correction slot of each stage.  All six in production; the other sets exist for
// the accuracy study of the compensated products (SWCL_BASIS_PRODUCTS).
__host__ __device__ constexpr int first_correction(uint32_t pm) {
  return (pm & 2u) ? 1 : (pm & 4u) ? 2 : (pm & 8u) ? 3 : (pm & 16u) ? 4 : 5;
}

// ------------------------------------------------------------------ epilogues ----

// 8-byte asynchronous copy global -> shared; bytes = 0 fills the destination with zeros (src is
// then not read, but stays a valid address)
__device__ __forceinline__ void cp_async8(void* dst, const void* src, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
}
// the drain warps' own barrier (barrier 1; barrier 0 is the CTA's)
__device__ __forceinline__ void drain_bar(int nthreads) {
  asm volatile("bar.sync 1, %0;\n" ::"r"(nthreads) : "memory");
}

// The epilogues read this thread's accumulator column c at acc[c * stride] (shared memory; see
// the drain), in loops that are not unrolled: the kernel runs them once per CTA, so a compact
// body keeps the cold instruction fetch short.

// Forward: Delta[w][l][i][q] = sum_s kmu[i][s][q] Z[q][(w, i, l, s)]
struct EpiFwd {
  float* delta;
  const float* kmu;     // [N_tr][4][N_k]
  const int2* cmap;     // ragged lists: column group -> {w N_tr + i, l}; null: every multipole
  int N_k, N_tr, n_l, r, n_cols;
  static constexpr bool kGamma = false;   // no table rows staged in shared memory
  __device__ __forceinline__ void prefetch(float2*, int, int, int, int, int) const {}
  __device__ __forceinline__ void set_stage(const float2*, int) {}
  // row m, this thread's columns j0 .. j0 + nc - 1 (j0 is a multiple of r)
  __device__ __forceinline__ void operator()(int m, int j0, const float* acc, int stride, int nc) const {
    if (m >= N_k) return;
    if (cmap) {
      ragged(m, j0, acc, stride, nc);
      return;
    }
    // column j = ((w N_tr + i) n_l + l) r + s, walked incrementally
    int s = j0 % r, g = j0 / r;
    int l = g % n_l, wi = g / n_l;
    int i = wi % N_tr, w = wi / N_tr;
    float kmv[4];                     // kmu[i][s][m] of the current tracer
#pragma unroll
    for (int u = 0; u < 4; ++u) kmv[u] = u < r ? __ldg(kmu + ((size_t)i * 4 + u) * N_k + m) : 0.0f;
    float v = 0.0f;
    const int ncols = min(nc, n_cols - j0);
#pragma unroll 4
    for (int c = 0; c < ncols; ++c) {
      const float km = s == 0 ? kmv[0] : s == 1 ? kmv[1] : s == 2 ? kmv[2] : kmv[3];
      v = fmaf(km, acc[c * stride], v);
      if (s == r - 1) {
        delta[(((size_t)w * n_l + l) * N_tr + i) * N_k + m] = v;
        v = 0.0f;
      }
      if (++s == r) {
        s = 0;
        if (++l == n_l) {
          l = 0;
          if (++i == N_tr) { i = 0; ++w; }
#pragma unroll
          for (int u = 0; u < 4; ++u) kmv[u] = u < r ? __ldg(kmu + ((size_t)i * 4 + u) * N_k + m) : 0.0f;
        }
      }
    }
  }
  // Ragged lists: each group of r columns is one (w, i, l) of the column map.  Kept out of line so
  // that the kernels of the common case keep their register allocation.
  __device__ __noinline__ void ragged(int m, int j0, const float* acc, int stride, int nc) const {
    const int ncols = min(nc, n_cols - j0);
    int s = j0 % r, g = j0 / r;
    int i = -1;
    float kmv[4] = {0.f, 0.f, 0.f, 0.f};
    float v = 0.0f;
    for (int c = 0; c < ncols; ++c) {
      if (s == 0 || c == 0) {
        const int2 cm = __ldg(cmap + g);
        const int ni = cm.x % N_tr;
        if (ni != i) {
          i = ni;
#pragma unroll
          for (int u = 0; u < 4; ++u) kmv[u] = u < r ? __ldg(kmu + ((size_t)i * 4 + u) * N_k + m) : 0.0f;
        }
      }
      const float km = s == 0 ? kmv[0] : s == 1 ? kmv[1] : s == 2 ? kmv[2] : kmv[3];
      v = fmaf(km, acc[c * stride], v);
      if (s == r - 1) {
        const int2 cm = __ldg(cmap + g);
        delta[(((size_t)(cm.x / N_tr) * n_l + cm.y) * N_tr + i) * N_k + m] = v;
        v = 0.0f;
      }
      if (++s == r) {
        s = 0;
        ++g;
      }
    }
  }
};

// Adjoint: Fbar[(w, i, s)][n] += sum_l conj(G[l][n]) Y[(n, re/im)][(w, i, s, l)]; the lanes of
// rows 2n (Re Y) and 2n+1 (Im Y) are neighbours and combine with one shuffle.
struct EpiAdj {
  cplx* cbar;           // [n_walk][N_tr][NI][n_h]
  const float2* g32;    // [n_cls][N_ell][n_h]
  const int* cls_of;
  const int2* cmap;     // ragged lists: column -> {(w N_tr + i) r + s, l}; null: every multipole
  int n_h, N_tr, N_ell, l_lo, n_l, r, NI, n_cols;
  // Gamma rows of the tile staged in shared memory during the main loop: gs[c][n - 64 mt] for the
  // tile's columns c = j - gs_j0 (null: read from L2 in the epilogue)
  const float2* gs = nullptr;
  int gs_j0 = 0;
  static constexpr bool kGamma = true;
  __device__ __forceinline__ void set_stage(const float2* p, int j0) { gs = p; gs_j0 = j0; }
  // Issue the copies of the tile's NT x 64 Gamma values (threads tid, tid + nthr, ... of the
  // nthr drain threads, which all call it).  The row offset of each column (its class needs a
  // table load) goes to shared memory first, after dst's NT x 64 values, so that no copy waits
  // on a load.
  __device__ __forceinline__ void prefetch(float2* dst, int mt, int nt, int NT, int tid,
                                           int nthr) const {
    constexpr int kN = kM / 2;
    long long* rowoff = reinterpret_cast<long long*>(dst + (size_t)NT * kN);
    const int n0 = mt * kN, j0 = nt * NT;
    for (int cc = tid; cc < NT; cc += nthr) {
      const int j = j0 + cc;
      long long o = -1;
      if (j < n_cols) {
        int g, l;
        if (cmap) {
          const int2 cm = __ldg(cmap + j);
          g = cm.x;
          l = cm.y;
        } else {
          g = j / n_l;
          l = j - g * n_l;
        }
        o = ((long long)__ldg(cls_of + (g / r) % N_tr) * N_ell + l_lo + l) * n_h;
      }
      rowoff[cc] = o;
    }
    drain_bar(nthr);
    for (int e = tid; e < NT * kN; e += nthr) {
      const long long o = rowoff[e / kN];
      const int n = n0 + e % kN;
      const bool ok = o >= 0 && n < n_h;
      cp_async8(dst + e, ok ? g32 + o + n : g32, ok ? 8 : 0);
    }
  }
  static constexpr uint32_t stage_bytes(int NT) {
    return (uint32_t)(NT * (kM / 2) * sizeof(float2) + NT * sizeof(long long));
  }
  __device__ __forceinline__ void flush(int g, int n, int t, float are, float aim) const {
    const float re = are + __shfl_xor_sync(0xffffffffu, are, 1);
    const float im = aim + __shfl_xor_sync(0xffffffffu, aim, 1);
    if (t == 0 && n < n_h) {
      const int wi = g / r, s = g % r;
      cplx* dst = cbar + ((size_t)wi * NI + s) * n_h + n;
      atomicAdd(&dst->x, (double)re);
      atomicAdd(&dst->y, (double)im);
    }
  }
  __device__ __forceinline__ void operator()(int m, int j0, const float* acc, int stride, int nc) const {
    const int n = m >> 1, t = m & 1;
    const bool live = n < n_h;
    const int nn = live ? n : 0;
    // column j = ((w N_tr + i) r + s) n_l + l, walked incrementally; the same for every lane,
    // so the group changes (shuffles) are warp-uniform.  Gamma values are loaded 16 at a time.
    const int ncols = min(nc, n_cols - j0);
    if (ncols <= 0) return;
    if (cmap) {
      ragged(n, t, live, nn, j0, acc, stride, ncols, (m >> 1) & (kM / 2 - 1));
      return;
    }
    if (gs) {
      staged(n, t, live, j0, acc, stride, ncols, (m >> 1) & (kM / 2 - 1));
      return;
    }
    int l = j0 % n_l, g = j0 / n_l;
    const float2* grow = g32 + ((size_t)__ldg(cls_of + (g / r) % N_tr) * N_ell + l_lo) * n_h + nn;
    float are = 0.0f, aim = 0.0f;
#pragma unroll 1
    for (int c0 = 0; c0 < ncols; c0 += 16) {
      // one batch of loads for columns c0 .. c0 + 15, following the group changes
      float2 G[16];
      int lb = l, gb = g;
      const float2* growb = grow;
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        G[u] = (c0 + u < ncols) ? __ldg(growb + (size_t)lb * n_h) : make_float2(0.f, 0.f);
        if (++lb == n_l) {
          lb = 0;
          ++gb;
          growb = g32 + ((size_t)__ldg(cls_of + (gb / r) % N_tr) * N_ell + l_lo) * n_h + nn;
        }
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        if (c0 + u < ncols) {
          const float y = live ? acc[(c0 + u) * stride] : 0.0f;
          if (t == 0) {
            are = fmaf(G[u].x, y, are);
            aim = fmaf(-G[u].y, y, aim);
          } else {
            are = fmaf(G[u].y, y, are);
            aim = fmaf(G[u].x, y, aim);
          }
          if (++l == n_l) {
            flush(g, n, t, are, aim);
            are = 0.0f;
            aim = 0.0f;
            l = 0;
            ++g;
            grow = g32 + ((size_t)__ldg(cls_of + (g / r) % N_tr) * N_ell + l_lo) * n_h + nn;
          }
        }
      }
    }
    if (l != 0) flush(g, n, t, are, aim);
  }
  // Every multipole, Gamma from the staged rows (nl = n - 64 mt)
  __device__ __noinline__ void staged(int n, int t, bool live, int j0, const float* acc,
                                      int stride, int ncols, int nl) const {
    int l = j0 % n_l, g = j0 / n_l;
    const float2* gcol = gs + (size_t)(j0 - gs_j0) * (kM / 2) + nl;
    float are = 0.0f, aim = 0.0f;
#pragma unroll 4
    for (int cc = 0; cc < ncols; ++cc) {
      const float2 G = gcol[(size_t)cc * (kM / 2)];
      const float y = live ? acc[cc * stride] : 0.0f;
      // t = 0 (Re row): (Gx, -Gy); t = 1 (Im row): (Gy, Gx)
      are = fmaf(t ? G.y : G.x, y, are);
      aim = fmaf(t ? G.x : -G.y, y, aim);
      if (++l == n_l) {
        flush(g, n, t, are, aim);
        are = 0.0f;
        aim = 0.0f;
        l = 0;
        ++g;
      }
    }
    if (l != 0) flush(g, n, t, are, aim);
  }
  // The same with the column map: a group (w, i, s) is a run of columns with equal map.x, which
  // is the same for every lane (the group changes and their shuffles stay warp-uniform).
  __device__ __noinline__ void ragged(int n, int t, bool live, int nn, int j0, const float* acc,
                                      int stride, int ncols, int nl) const {
    int g = __ldg(&cmap[j0].x);
    float are = 0.0f, aim = 0.0f;
#pragma unroll 1
    for (int c0 = 0; c0 < ncols; c0 += 16) {
      float2 G[16];
      int gg[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        gg[u] = -1;
        G[u] = make_float2(0.f, 0.f);
        if (c0 + u < ncols) {
          const int2 cm = __ldg(cmap + j0 + c0 + u);
          gg[u] = cm.x;
          G[u] = gs ? gs[(size_t)(j0 + c0 + u - gs_j0) * (kM / 2) + nl]
                    : __ldg(g32 + ((size_t)__ldg(cls_of + (cm.x / r) % N_tr) * N_ell + l_lo + cm.y) * n_h + nn);
        }
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        if (c0 + u < ncols) {
          if (gg[u] != g) {
            flush(g, n, t, are, aim);
            are = 0.0f;
            aim = 0.0f;
            g = gg[u];
          }
          const float y = live ? acc[(c0 + u) * stride] : 0.0f;
          if (t == 0) {
            are = fmaf(G[u].x, y, are);
            aim = fmaf(-G[u].y, y, aim);
          } else {
            are = fmaf(G[u].y, y, are);
            aim = fmaf(G[u].x, y, aim);
          }
        }
      }
    }
    flush(g, n, t, are, aim);
  }
};

// ------------------------------------------------------------------- GEMM ----

// CH: 16-column chunks per drain thread at most (3 for tiles up to 96 columns with 8 drain
// warps, 4 otherwise); it sizes the accumulator registers.
// MG: one accumulator slot per TMEM buffer instead of two.  Each stage issues its correction
// products first and the leading products last, so the slot holds the small corrections when
// the leading terms arrive: the leading sum is rounded as often as in its own slot, and the
// correction bits below the FP32 resolution of the sum are the ones that would be lost in the
// drain's addition anyway.  Half the TMEM per tile allows tiles up to 240 columns.
//
// SK = 2: split K in two.  A cluster of two CTAs computes one tile, each over its half of the
// stages (the first CTA the first half); each drains its partial sums into registers as usual and
// stages them in its shared memory; the first CTA then adds the second's through distributed
// shared memory (two FP32 terms: the same sum in any order) and runs the epilogue.  Launched with
// a cluster dimension of 2 (cudaLaunchKernelEx), grid = 2 x tiles.
template <class P, class Epi, int DW, int CH, int KS, uint32_t PM = 0x3Fu, bool MG = false, int SK = 1>
__global__ void __launch_bounds__(threads_for(DW), DW == 4 ? 2 : 1)
k_gemm_basis(const uint8_t* __restrict__ aimg, const uint8_t* __restrict__ bimg, GemmShape sh,
             Epi epi, int* __restrict__ status) {
  pdl_trigger();   // the next kernel of the step may be scheduled
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // n_kb counts the stages' worth of K (KS K-blocks each, the last one possibly short); with a
  // split, this CTA's stages are kb_lo .. kb_lo + n_kb - 1 of the n_all stages of the tile
  const int NT = sh.NT, S = sh.stages, n_kb1 = sh.n_kb, n_all = (n_kb1 + KS - 1) / KS;
  const int rank = SK == 2 ? (int)cluster_ctarank() : 0;
  const int half_kb = (n_all + 1) / 2;
  const int kb_lo = SK == 2 ? rank * half_kb : 0;
  const int n_kb = SK == 2 ? (rank == 0 ? half_kb : n_all - half_kb) : n_all;
  const int tile = SK == 2 ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const Layout L = layout<P>(NT, S, KS);
  // Barriers per stage: ready[s] completes when the stage's copies have landed (transaction
  // count only); full[s] when the copy warp has seen ready[s] AND the drain warps have emptied
  // the TMEM buffer the stage accumulates into (1 + DW arrivals: one per drain warp, since
  // 32 DW single-thread arrivals would serialise on the barrier word); mmadone[s] when the
  // stage's MMAs are done (one commit), which frees the stage for the copy warp and the
  // accumulator for the drain warps.  The MMA thread waits once and commits once per stage:
  // a single thread issues tcgen05.mma only about as fast as the tensor core executes a
  // 128 x 96 x 16 product, so its own time between MMAs is the critical resource, and two
  // K-blocks per stage halve the round trips.
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + L.bar_off);
  uint64_t* full = bars;
  uint64_t* mmadone = bars + S;
  uint64_t* ready = bars + 2 * S;
  uint64_t* done = bars + 3 * S;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * S + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = tile % sh.n_mt;
  const int nt = tile / sh.n_mt;
  const int stride = (NT + 31) & ~31;   // TMEM columns per accumulator slot

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&full[s]), 1 + DW);     // the copy warp + one arrival per drain warp
      mbar_init(smem_u32(&mmadone[s]), 1);
      mbar_init(smem_u32(&ready[s]), 1);
    }
    mbar_init(smem_u32(done), 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), sh.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // barriers and TMEM are set up; the operands and outputs belong to the kernels before
  pdl_wait();

  bool drain_ok = false;   // the split-K reduction: this drain warp's partial sums are valid
  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------- copies ----
      // Issues the copies of K-block `next` as soon as its stage is free and forwards landed
      // K-blocks (ready -> full) in order.  Both conditions are polled without suspending
      // (test_wait): a thread suspended on "stage free" would hold back the forward of a landed
      // K-block until the tensor core had finished the previous one, a bubble per K-block.
      const uint8_t* asrc = aimg + ((size_t)mt * n_kb1 + (size_t)kb_lo * KS) * L.a1;
      const uint8_t* bsrc = bimg + ((size_t)nt * n_kb1 + (size_t)kb_lo * KS) * L.b1;
      int next = 0, fwd = 0;
      long idle = 0;
      while (fwd < n_kb) {
        bool progress = false;
        if (next < n_kb) {
          const int s = next % S, r = next / S;
          if (r == 0 || mbar_test_wait(smem_u32(&mmadone[s]), (r - 1) & 1)) {
            uint8_t* st = base + s * L.stage;
            const int nk = min(KS, n_kb1 - (kb_lo + next) * KS);      // K-blocks in this stage
            mbar_arrive_tx(smem_u32(&ready[s]), nk * (L.a1 + L.b1));
            bulk_g2s(smem_u32(st), asrc + (size_t)next * KS * L.a1, nk * L.a1, smem_u32(&ready[s]));
            bulk_g2s(smem_u32(st + L.a_bytes), bsrc + (size_t)next * KS * L.b1, nk * L.b1,
                     smem_u32(&ready[s]));
            ++next;
            progress = true;
          }
        }
        if (fwd < next && mbar_test_wait(smem_u32(&ready[fwd % S]), (fwd / S) & 1)) {
          mbar_arrive(smem_u32(&full[fwd % S]));
          ++fwd;
          progress = true;
        }
        if (progress) {
          idle = 0;
        } else if (++idle > (kSpinLimit << 6) || *abort_flag) {   // non-suspending polls
          *abort_flag = 1;
          break;
        }
      }
      // copies still in flight (issued, not forwarded) land before the CTA exits
      for (int kb = fwd; kb < next; ++kb) mbar_wait_drain(smem_u32(&ready[kb % S]), (kb / S) & 1);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------------- MMA ----
      const uint32_t idesc = idesc_bf16(kM, NT);
      const uint32_t b_plane = NT * kRow;
      for (int kb = 0; kb < n_kb; ++kb) {
        const int s = kb % S, r = kb / S, b = kb & 1;
        if (!mbar_wait(smem_u32(&full[s]), r & 1, abort_flag)) break;
        tc_fence_after();
        const uint32_t a0 = smem_u32(base + s * L.stage);
        const int nk = min(KS, n_kb1 - (kb_lo + kb) * KS);
        if constexpr (MG) {
          const uint32_t d = tmem + (uint32_t)(b * stride);
          // corrections first (the first of them overwrites the slot), the leading products last
#pragma unroll
          for (int t = 1; t <= P::kProducts; ++t) {
            const int tt = t % P::kProducts;
#pragma unroll
            for (int h = 0; h < KS; ++h) {
              if (h >= nk) break;
              const uint64_t da = desc64(a0 + h * L.a1), db = desc64(a0 + L.a_bytes + h * L.b1);
#pragma unroll
              for (int j = 0; j < kK / 16; ++j) {
                const uint64_t ad = da + (uint64_t)((P::pa(tt) * kPlaneM + j * 256) >> 4);
                const uint64_t bd = db + (uint64_t)((P::pb(tt) * b_plane + j * 256) >> 4);
                const bool first = (t == 1) && (h == 0) && (j == 0);
                mma_bf16(d, ad, bd, idesc, first ? 0u : 1u);
              }
            }
          }
        } else {
          const uint32_t d_main = tmem + (uint32_t)((2 * b) * stride);
          const uint32_t d_corr = tmem + (uint32_t)((2 * b + 1) * stride);
#pragma unroll
          for (int h = 0; h < KS; ++h) {
            if (h >= nk) break;
            const uint64_t da = desc64(a0 + h * L.a1), db = desc64(a0 + L.a_bytes + h * L.b1);
#pragma unroll
            for (int j = 0; j < kK / 16; ++j) {
#pragma unroll
              for (int t = 0; t < P::kProducts; ++t) {
                if (!((PM >> t) & 1u)) continue;
                // descriptor start addresses advance in 16-byte units
                const uint64_t ad = da + (uint64_t)((P::pa(t) * kPlaneM + j * 256) >> 4);
                const uint64_t bd = db + (uint64_t)((P::pb(t) * b_plane + j * 256) >> 4);
                const bool lead = (t == 0);
                const bool first = (h == 0) && (j == 0) && (lead || t == first_correction(PM));
                mma_bf16(lead ? d_main : d_corr, ad, bd, idesc, first ? 0u : 1u);
              }
            }
          }
        }
        mma_commit(smem_u32(&mmadone[s]));
      }
      // every issued MMA has completed before TMEM is released
      mma_commit(smem_u32(done));
      mbar_wait_drain(smem_u32(done), 0);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ drain ----
    const int quarter = warp & 3;        // TMEM lanes 32*quarter .. +31 for this warp
    const int half = DW == 8 ? (warp - 2) >> 2 : 0;   // column half (DW = 8)
    const int row = quarter * 32 + lane;
    const int nch = NT / 16;
    const int nch0 = DW == 8 ? (nch + 1) / 2 : nch;
    const int c_begin = half ? nch0 : 0;
    const int my = half ? nch - nch0 : nch0;   // 16-column chunks of this thread (<= 4)
    float acc[CH * 16];
#pragma unroll
    for (int t = 0; t < CH * 16; ++t) acc[t] = 0.0f;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    // the epilogue's table rows: copies issued now, waited for after the main loop
    float2* gstage = nullptr;
    if constexpr (Epi::kGamma) {
      if (sh.pre_off) {
        gstage = reinterpret_cast<float2*>(base + sh.pre_off);
        epi.prefetch(gstage, mt, nt, NT, tid - 64, 32 * DW);
      }
    }
    // the first two K-blocks find their accumulator buffers empty
    if (lane == 0) {
      mbar_arrive(smem_u32(&full[0]));
      if (n_kb > 1) mbar_arrive(smem_u32(&full[1 % S]));
    }
    bool ok = true;
    for (int kb = 0; kb < n_kb && ok; ++kb) {
      const int b = kb & 1;
      // warp-uniform exit: every lane leaves the loop together (the loop has warp barriers)
      const bool got = mbar_wait(smem_u32(&mmadone[kb % S]), (kb / S) & 1, abort_flag);
      if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
      tc_fence_after();
      const uint32_t slot_m = lane_base + (MG ? b : 2 * b) * stride + c_begin * 16;
      const uint32_t slot_c = lane_base + (2 * b + 1) * stride + c_begin * 16;
      if constexpr (MG) {
        // one slot: up to four chunks in flight per wait (two with eight chunks per thread)
        constexpr int kF = CH > 4 ? 2 : 4;
#pragma unroll
        for (int g = 0; g < CH; g += kF) {
          uint32_t m[kF][16];
#pragma unroll
          for (int u = 0; u < kF; ++u)
            if (g + u < my) tmem_ld16_async(slot_m + (g + u) * 16, m[u]);
          tmem_wait_ld();
#pragma unroll
          for (int u = 0; u < kF; ++u) {
            if (g + u < my) {
              reg_fence(m[u]);
#pragma unroll
              for (int t = 0; t < 16; ++t) acc[(g + u) * 16 + t] += __uint_as_float(m[u][t]);
            }
          }
        }
      } else if constexpr (CH <= 3) {
        // up to three chunks: every load of the K-block in flight behind one wait
        uint32_t m0[16], r0[16], m1[16], r1[16], m2[16], r2[16];
        tmem_ld16_async(slot_m, m0);
        tmem_ld16_async(slot_c, r0);
        if (my > 1) {
          tmem_ld16_async(slot_m + 16, m1);
          tmem_ld16_async(slot_c + 16, r1);
        }
        if (my > 2) {
          tmem_ld16_async(slot_m + 32, m2);
          tmem_ld16_async(slot_c + 32, r2);
        }
        tmem_wait_ld();
        reg_fence(m0);
        reg_fence(r0);
#pragma unroll
        for (int t = 0; t < 16; ++t) acc[t] += __uint_as_float(m0[t]) + __uint_as_float(r0[t]);
        if (my > 1) {
          reg_fence(m1);
          reg_fence(r1);
#pragma unroll
          for (int t = 0; t < 16; ++t) acc[16 + t] += __uint_as_float(m1[t]) + __uint_as_float(r1[t]);
        }
        if (my > 2) {
          reg_fence(m2);
          reg_fence(r2);
#pragma unroll
          for (int t = 0; t < 16; ++t) acc[32 + t] += __uint_as_float(m2[t]) + __uint_as_float(r2[t]);
        }
      } else {
        // four chunks: two in flight per wait
#pragma unroll
        for (int g = 0; g < CH; g += 2) {
          uint32_t m0[16], r0[16], m1[16], r1[16];
          tmem_ld16_async(slot_m + g * 16, m0);
          tmem_ld16_async(slot_c + g * 16, r0);
          tmem_ld16_async(slot_m + (g + 1) * 16, m1);
          tmem_ld16_async(slot_c + (g + 1) * 16, r1);
          tmem_wait_ld();
          reg_fence(m0);
          reg_fence(r0);
          reg_fence(m1);
          reg_fence(r1);
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            acc[g * 16 + t] += __uint_as_float(m0[t]) + __uint_as_float(r0[t]);
            acc[(g + 1) * 16 + t] += __uint_as_float(m1[t]) + __uint_as_float(r1[t]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      // buffer b is free for K-block kb + 2: every lane of the warp has finished its loads
      if (lane == 0 && kb + 2 < n_kb) mbar_arrive(smem_u32(&full[(kb + 2) % S]));
    }
    // every drain thread's staged copies have landed and are visible to the others (every drain
    // warp reaches this barrier once, whether its loop completed or stopped early)
    if (gstage) {
      cp_async_commit_wait_all();
      drain_bar(32 * DW);
    }
    // every lane of a drain warp reaches the epilogue (its shuffles need the full warp)
    const bool all_ok = __all_sync(0xffffffffu, ok) && !*abort_flag;
    if (all_ok) {
      // the stages are idle now (every MMA has completed, every copy has landed): the
      // accumulators go to shared memory, column-major over the drain threads, and the epilogue
      // reads them from there in a loop that is not unrolled
      const int dt = tid - 64;                       // drain thread 0 .. 32 DW - 1
      float* ep = reinterpret_cast<float*>(base);
#pragma unroll
      for (int c = 0; c < CH * 16; ++c)
        if (c < my * 16) ep[c * (32 * DW) + dt] = acc[c];
      if constexpr (SK == 1) {
        Epi e = epi;
        e.set_stage(gstage, nt * NT);
        e(mt * kM + row, nt * NT + c_begin * 16, ep + dt, 32 * DW, my * 16);
      }
    }
    if constexpr (SK == 2) drain_ok = all_ok;
  }
  if constexpr (SK == 2) {
    // both CTAs' partial sums are staged (every thread of the cluster takes part)
    cluster_sync_all();
    if (rank == 0 && warp >= 2) {
      const uint32_t peer_abort = cluster_addr(smem_u32((const void*)abort_flag), 1);
      int pa;
      asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(pa) : "r"(peer_abort) : "memory");
      const bool go = __all_sync(0xffffffffu, drain_ok && pa == 0);
      if (go) {
        const int quarter = warp & 3, half = (warp - 2) >> 2, row = quarter * 32 + lane;
        const int nch = NT / 16, nch0 = (nch + 1) / 2;
        const int c_begin = half ? nch0 : 0, my = half ? nch - nch0 : nch0;
        const int dt = tid - 64;
        float* ep = reinterpret_cast<float*>(base);
        const uint32_t rep = cluster_addr(smem_u32(ep), 1);
        for (int c0 = 0; c0 < my * 16; c0 += 8) {
          float v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            asm volatile("ld.shared::cluster.f32 %0, [%1];"
                         : "=f"(v[u]) : "r"(rep + 4u * (uint32_t)((c0 + u) * (32 * DW) + dt)) : "memory");
#pragma unroll
          for (int u = 0; u < 8; ++u) ep[(c0 + u) * (32 * DW) + dt] += v[u];
        }
        Epi e = epi;
        e.set_stage(nullptr, nt * NT);
        e(mt * kM + row, nt * NT + c_begin * 16, ep + dt, 32 * DW, my * 16);
      } else if (lane == 0) {
        *abort_flag = 1;
      }
    }
    // the second CTA's shared memory is read until here
    cluster_sync_all();
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicExch(status, 1);
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, sh.tmem_cols);
  }
}

// Persistent form of the two-K-block GEMM (tile code bit 12): one CTA per SM walks the tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...  The barriers, the TMEM allocation and the stage ring
// stay live across tiles: the stage counter g runs over all of the CTA's stages, so the copy warp
// fetches the next tile's first stages while the drain warps run the epilogue of the previous
// tile, and the MMA thread starts the next tile as soon as two accumulator buffers are free.  The
// epilogue stages its accumulators in a region of its own (not in the stage ring, which is being
// refilled).  Arithmetic per tile as in k_gemm_basis<..., KS = 2>.
template <class P>
__host__ __device__ inline Layout layout_persist(int NT, int stages, int CH) {
  Layout L = layout<P>(NT, stages, 2);
  const uint32_t ep_bytes = (uint32_t)CH * 16 * 256 * sizeof(float);
  L.bar_off = stages * L.stage + ep_bytes;
  L.total = L.bar_off + 8 * (3 * stages + 1) + 16 + 1024;
  return L;
}

template <class P, class Epi, int CH>
__global__ void __launch_bounds__(threads_for(8), 1)
k_gemm_persist(const uint8_t* __restrict__ aimg, const uint8_t* __restrict__ bimg, GemmShape sh,
               int n_tiles, Epi epi, int* __restrict__ status) {
  constexpr int DW = 8, KS = 2;
  pdl_trigger();   // the next kernel of the step may be scheduled
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int NT = sh.NT, S = sh.stages, n_kb1 = sh.n_kb, n_kb = (n_kb1 + KS - 1) / KS;
  const Layout L = layout_persist<P>(NT, S, CH);
  // barriers as in k_gemm_basis: full[s] (copies landed and the TMEM buffer drained: the copy
  // warp + one arrival per drain warp), mmadone[s] (one commit), ready[s] (transaction count)
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + L.bar_off);
  uint64_t* full = bars;
  uint64_t* mmadone = bars + S;
  uint64_t* ready = bars + 2 * S;
  uint64_t* done = bars + 3 * S;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * S + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* ep = reinterpret_cast<float*>(base + S * L.stage);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_my = blockIdx.x < n_tiles ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int T = n_my * n_kb;             // this CTA's stages over all its tiles
  const int stride = (NT + 31) & ~31;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&full[s]), 1 + DW);
      mbar_init(smem_u32(&mmadone[s]), 1);
      mbar_init(smem_u32(&ready[s]), 1);
    }
    mbar_init(smem_u32(done), 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), sh.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // barriers and TMEM are set up; the operands and outputs belong to the kernels before
  pdl_wait();

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------- copies ----
      int next = 0, fwd = 0;
      long idle = 0;
      while (fwd < T) {
        bool progress = false;
        if (next < T) {
          const int s = next % S, r = next / S;
          if (r == 0 || mbar_test_wait(smem_u32(&mmadone[s]), (r - 1) & 1)) {
            const int tile = blockIdx.x + (next / n_kb) * gridDim.x, kb = next % n_kb;
            const int mt = tile % sh.n_mt, nt = tile / sh.n_mt;
            uint8_t* st = base + s * L.stage;
            const int nk = min(KS, n_kb1 - kb * KS);
            mbar_arrive_tx(smem_u32(&ready[s]), nk * (L.a1 + L.b1));
            bulk_g2s(smem_u32(st), aimg + ((size_t)mt * n_kb1 + kb * KS) * L.a1, nk * L.a1,
                     smem_u32(&ready[s]));
            bulk_g2s(smem_u32(st + L.a_bytes), bimg + ((size_t)nt * n_kb1 + kb * KS) * L.b1,
                     nk * L.b1, smem_u32(&ready[s]));
            ++next;
            progress = true;
          }
        }
        if (fwd < next && mbar_test_wait(smem_u32(&ready[fwd % S]), (fwd / S) & 1)) {
          mbar_arrive(smem_u32(&full[fwd % S]));
          ++fwd;
          progress = true;
        }
        if (progress) {
          idle = 0;
        } else if (++idle > (kSpinLimit << 6) || *abort_flag) {
          *abort_flag = 1;
          break;
        }
      }
      for (int g = fwd; g < next; ++g) mbar_wait_drain(smem_u32(&ready[g % S]), (g / S) & 1);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------------- MMA ----
      const uint32_t idesc = idesc_bf16(kM, NT);
      const uint32_t b_plane = NT * kRow;
      for (int g = 0; g < T; ++g) {
        const int s = g % S, r = g / S, b = g & 1, kb = g % n_kb;
        if (!mbar_wait(smem_u32(&full[s]), r & 1, abort_flag)) break;
        tc_fence_after();
        const uint32_t a0 = smem_u32(base + s * L.stage);
        const uint32_t d_main = tmem + (uint32_t)((2 * b) * stride);
        const uint32_t d_corr = tmem + (uint32_t)((2 * b + 1) * stride);
        const int nk = min(KS, n_kb1 - kb * KS);
#pragma unroll
        for (int h = 0; h < KS; ++h) {
          if (h >= nk) break;
          const uint64_t da = desc64(a0 + h * L.a1), db = desc64(a0 + L.a_bytes + h * L.b1);
#pragma unroll
          for (int j = 0; j < kK / 16; ++j) {
#pragma unroll
            for (int t = 0; t < P::kProducts; ++t) {
              const uint64_t ad = da + (uint64_t)((P::pa(t) * kPlaneM + j * 256) >> 4);
              const uint64_t bd = db + (uint64_t)((P::pb(t) * b_plane + j * 256) >> 4);
              const bool lead = (t == 0);
              const bool first = (h == 0) && (j == 0) && (t <= 1);
              mma_bf16(lead ? d_main : d_corr, ad, bd, idesc, first ? 0u : 1u);
            }
          }
        }
        mma_commit(smem_u32(&mmadone[s]));
      }
      mma_commit(smem_u32(done));
      mbar_wait_drain(smem_u32(done), 0);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ drain ----
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row = quarter * 32 + lane;
    const int nch = NT / 16;
    const int nch0 = (nch + 1) / 2;
    const int c_begin = half ? nch0 : 0;
    const int my = half ? nch - nch0 : nch0;
    const int dt = tid - 64;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    if (lane == 0) {
      mbar_arrive(smem_u32(&full[0]));
      if (T > 1) mbar_arrive(smem_u32(&full[1 % S]));
    }
    bool ok = true;
    for (int it = 0; it < n_my && ok; ++it) {
      const int tile = blockIdx.x + it * gridDim.x;
      const int mt = tile % sh.n_mt, nt = tile / sh.n_mt;
      float acc[CH * 16];
#pragma unroll
      for (int t = 0; t < CH * 16; ++t) acc[t] = 0.0f;
      for (int kb = 0; kb < n_kb; ++kb) {
        const int g = it * n_kb + kb, b = g & 1;
        const bool got = mbar_wait(smem_u32(&mmadone[g % S]), (g / S) & 1, abort_flag);
        if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
        tc_fence_after();
        const uint32_t slot_m = lane_base + (2 * b) * stride + c_begin * 16;
        const uint32_t slot_c = lane_base + (2 * b + 1) * stride + c_begin * 16;
        uint32_t m0[16], r0[16], m1[16], r1[16], m2[16], r2[16];
        tmem_ld16_async(slot_m, m0);
        tmem_ld16_async(slot_c, r0);
        if (my > 1) {
          tmem_ld16_async(slot_m + 16, m1);
          tmem_ld16_async(slot_c + 16, r1);
        }
        if (my > 2) {
          tmem_ld16_async(slot_m + 32, m2);
          tmem_ld16_async(slot_c + 32, r2);
        }
        tmem_wait_ld();
        reg_fence(m0);
        reg_fence(r0);
#pragma unroll
        for (int t = 0; t < 16; ++t) acc[t] += __uint_as_float(m0[t]) + __uint_as_float(r0[t]);
        if (my > 1) {
          reg_fence(m1);
          reg_fence(r1);
#pragma unroll
          for (int t = 0; t < 16; ++t) acc[16 + t] += __uint_as_float(m1[t]) + __uint_as_float(r1[t]);
        }
        if (my > 2) {
          reg_fence(m2);
          reg_fence(r2);
#pragma unroll
          for (int t = 0; t < 16; ++t) acc[32 + t] += __uint_as_float(m2[t]) + __uint_as_float(r2[t]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0 && g + 2 < T) mbar_arrive(smem_u32(&full[(g + 2) % S]));
      }
      if (!(__all_sync(0xffffffffu, ok) && !*abort_flag)) break;
      // the epilogue of this tile: the MMAs of the next one run meanwhile
#pragma unroll
      for (int c = 0; c < CH * 16; ++c)
        if (c < my * 16) ep[c * (32 * DW) + dt] = acc[c];
      epi(mt * kM + row, nt * NT + c_begin * 16, ep + dt, 32 * DW, my * 16);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicExch(status, 1);
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, sh.tmem_cols);
  }
}

// Persistent form with epilogue warps (tile-code bits 10 + 12 + 16, k_gemm_persist_ep).  As
// k_gemm_persist, one CTA per SM walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...  with
// the barriers, TMEM and stage ring live across tiles, but the epilogue has four warps of its
// own: at the end of a tile the drain warps write their sums into a row-major hand-off region
// (pitch NT + 1 words: conflict-free in both directions) and go on draining the next tile, while
// the epilogue warps (one row and all NT columns per thread) run the epilogue from there.  The
// epilogue of tile t thus runs beside the main loop of tile t + 1.  Barriers of the hand-off:
// epi_full (one arrival per drain warp) and epi_free (one per epilogue warp).  The epilogue's
// table rows come from L2 (no staging).
constexpr int kEpiWarps = 4;   // one per TMEM lane quarter, all of a row's columns
__host__ __device__ constexpr int threads_persist_ep() { return 64 + 32 * 8 + 32 * kEpiWarps; }

template <class P>
__host__ __device__ inline Layout layout_persist_ep(int NT, int stages) {
  Layout L = layout<P>(NT, stages, 2);
  const uint32_t hb_bytes = (uint32_t)kM * (NT + 1) * sizeof(float);
  L.bar_off = (stages * L.stage + hb_bytes + 7) & ~7u;
  L.total = L.bar_off + 8 * (3 * stages + 3) + 16 + 1024;
  return L;
}

template <class P, class Epi, int CH>
__global__ void __launch_bounds__(threads_persist_ep(), 1)
k_gemm_persist_ep(const uint8_t* __restrict__ aimg, const uint8_t* __restrict__ bimg, GemmShape sh,
                  int n_tiles, Epi epi, int* __restrict__ status) {
  constexpr int DW = 8, KS = 2;
  pdl_trigger();   // the next kernel of the step may be scheduled
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int NT = sh.NT, S = sh.stages, n_kb1 = sh.n_kb, n_kb = (n_kb1 + KS - 1) / KS;
  const Layout L = layout_persist_ep<P>(NT, S);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + L.bar_off);
  uint64_t* full = bars;
  uint64_t* mmadone = bars + S;
  uint64_t* ready = bars + 2 * S;
  uint64_t* done = bars + 3 * S;
  uint64_t* epi_full = bars + 3 * S + 1;
  uint64_t* epi_free = bars + 3 * S + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * S + 3);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* hb = reinterpret_cast<float*>(base + S * L.stage);   // [kM][NT + 1]
  const int hp = NT + 1;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_my = blockIdx.x < n_tiles ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int T = n_my * n_kb;
  const int stride = (NT + 31) & ~31;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&full[s]), 1 + DW);
      mbar_init(smem_u32(&mmadone[s]), 1);
      mbar_init(smem_u32(&ready[s]), 1);
    }
    mbar_init(smem_u32(done), 1);
    mbar_init(smem_u32(epi_full), DW);
    mbar_init(smem_u32(epi_free), kEpiWarps);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), sh.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // barriers and TMEM are set up; the operands and outputs belong to the kernels before
  pdl_wait();

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------- copies ----
      int next = 0, fwd = 0;
      long idle = 0;
      while (fwd < T) {
        bool progress = false;
        if (next < T) {
          const int s = next % S, r = next / S;
          if (r == 0 || mbar_test_wait(smem_u32(&mmadone[s]), (r - 1) & 1)) {
            const int tile = blockIdx.x + (next / n_kb) * gridDim.x, kb = next % n_kb;
            const int mt = tile % sh.n_mt, nt = tile / sh.n_mt;
            uint8_t* st = base + s * L.stage;
            const int nk = min(KS, n_kb1 - kb * KS);
            mbar_arrive_tx(smem_u32(&ready[s]), nk * (L.a1 + L.b1));
            bulk_g2s(smem_u32(st), aimg + ((size_t)mt * n_kb1 + kb * KS) * L.a1, nk * L.a1,
                     smem_u32(&ready[s]));
            bulk_g2s(smem_u32(st + L.a_bytes), bimg + ((size_t)nt * n_kb1 + kb * KS) * L.b1,
                     nk * L.b1, smem_u32(&ready[s]));
            ++next;
            progress = true;
          }
        }
        if (fwd < next && mbar_test_wait(smem_u32(&ready[fwd % S]), (fwd / S) & 1)) {
          mbar_arrive(smem_u32(&full[fwd % S]));
          ++fwd;
          progress = true;
        }
        if (progress) {
          idle = 0;
        } else if (++idle > (kSpinLimit << 6) || *abort_flag) {
          *abort_flag = 1;
          break;
        }
      }
      for (int g = fwd; g < next; ++g) mbar_wait_drain(smem_u32(&ready[g % S]), (g / S) & 1);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------------- MMA ----
      const uint32_t idesc = idesc_bf16(kM, NT);
      const uint32_t b_plane = NT * kRow;
      for (int g = 0; g < T; ++g) {
        const int s = g % S, r = g / S, b = g & 1, kb = g % n_kb;
        if (!mbar_wait(smem_u32(&full[s]), r & 1, abort_flag)) break;
        tc_fence_after();
        const uint32_t a0 = smem_u32(base + s * L.stage);
        const uint32_t d_main = tmem + (uint32_t)((2 * b) * stride);
        const uint32_t d_corr = tmem + (uint32_t)((2 * b + 1) * stride);
        const int nk = min(KS, n_kb1 - kb * KS);
#pragma unroll
        for (int h = 0; h < KS; ++h) {
          if (h >= nk) break;
          const uint64_t da = desc64(a0 + h * L.a1), db = desc64(a0 + L.a_bytes + h * L.b1);
#pragma unroll
          for (int j = 0; j < kK / 16; ++j) {
#pragma unroll
            for (int t = 0; t < P::kProducts; ++t) {
              const uint64_t ad = da + (uint64_t)((P::pa(t) * kPlaneM + j * 256) >> 4);
              const uint64_t bd = db + (uint64_t)((P::pb(t) * b_plane + j * 256) >> 4);
              const bool first = (h == 0) && (j == 0) && (t <= 1);
              mma_bf16(t == 0 ? d_main : d_corr, ad, bd, idesc, first ? 0u : 1u);
            }
          }
        }
        mma_commit(smem_u32(&mmadone[s]));
      }
      mma_commit(smem_u32(done));
      mbar_wait_drain(smem_u32(done), 0);
    }
    __syncwarp();
  } else if (warp < 2 + DW) {
    // ------------------------------------------------------------ drain ----
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row = quarter * 32 + lane;
    const int nch = NT / 16;
    const int nch0 = (nch + 1) / 2;
    const int c_begin = half ? nch0 : 0;
    const int my = half ? nch - nch0 : nch0;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    if (lane == 0) {
      mbar_arrive(smem_u32(&full[0]));
      if (T > 1) mbar_arrive(smem_u32(&full[1 % S]));
    }
    bool ok = true;
    for (int it = 0; it < n_my && ok; ++it) {
      float acc[CH * 16];
#pragma unroll
      for (int t = 0; t < CH * 16; ++t) acc[t] = 0.0f;
      for (int kb = 0; kb < n_kb; ++kb) {
        const int g = it * n_kb + kb, b = g & 1;
        const bool got = mbar_wait(smem_u32(&mmadone[g % S]), (g / S) & 1, abort_flag);
        if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
        tc_fence_after();
        const uint32_t slot_m = lane_base + (2 * b) * stride + c_begin * 16;
        const uint32_t slot_c = lane_base + (2 * b + 1) * stride + c_begin * 16;
        // one 16-column chunk (leading and correction slots) in flight per wait: the registers
        // are shared with the epilogue warps
#pragma unroll
        for (int cc = 0; cc < CH; ++cc) {
          if (cc < my) {
            uint32_t m0[16], r0[16];
            tmem_ld16_async(slot_m + cc * 16, m0);
            tmem_ld16_async(slot_c + cc * 16, r0);
            tmem_wait_ld();
            reg_fence(m0);
            reg_fence(r0);
#pragma unroll
            for (int t = 0; t < 16; ++t) acc[cc * 16 + t] += __uint_as_float(m0[t]) + __uint_as_float(r0[t]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0 && g + 2 < T) mbar_arrive(smem_u32(&full[(g + 2) % S]));
      }
      if (!ok) break;
      // hand the tile's sums to the epilogue warps once they have read the previous tile's
      if (it > 0) {
        const bool fr = mbar_wait(smem_u32(epi_free), (it - 1) & 1, abort_flag);
        if (!__all_sync(0xffffffffu, fr)) { ok = false; break; }
      }
      float* hr = hb + (size_t)row * hp + c_begin * 16;
#pragma unroll
      for (int c = 0; c < CH * 16; ++c)
        if (c < my * 16) hr[c] = acc[c];
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(epi_full));
    }
  } else {
    // ---------------------------------------------------------- epilogue ----
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const int c0 = 0, nc = NT;
    for (int it = 0; it < n_my; ++it) {
      const bool got = mbar_wait(smem_u32(epi_full), it & 1, abort_flag);
      if (!__all_sync(0xffffffffu, got)) break;
      const int tile = blockIdx.x + it * gridDim.x;
      const int mt = tile % sh.n_mt, nt = tile / sh.n_mt;
      Epi e = epi;
      e.set_stage(nullptr, nt * NT);
      e(mt * kM + row, nt * NT + c0, hb + (size_t)row * hp + c0, 1, nc);
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(epi_free));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicExch(status, 1);
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, sh.tmem_cols);
  }
}

// ------------------------------------------------------- two-SM tile (cta_group::2) ----

// A cluster of two CTAs on two SMs computes one 256 x NT tile with tcgen05.mma.cta_group::2:
// each MMA instruction, issued by one thread of the first CTA, multiplies 256 rows of A (128 in
// each CTA's shared memory) by NT columns of B (NT / 2 in each CTA's shared memory) into both
// CTAs' TMEM (each holds its own 128 rows x NT columns).  Against the one-SM tile of the same
// width this halves the MMA instructions and the B bytes each SM copies per K-block, so a stage
// is smaller and three of them fit.
//
// Handshakes: each CTA copies its own halves and relays "landed" to the first CTA's full[s]
// (a remote arrive); the drain warps of both CTAs relay "buffer drained" there too, so full[s]
// takes 2 (1 + DW) arrivals.  The MMA thread commits each stage to mmadone[s] in both CTAs (one
// commit per barrier; a commit tracks every MMA the thread issued before it).  Waits on barriers
// that the other CTA or the tensor core signals use acquire at cluster scope.


// Grid: 2 CTAs per (row-tile pair, column tile); sh.n_mt is the number of 128-row tiles (the A
// image holds an even count, the last one zero when n_mt is odd), sh.NT the tile's columns; the
// B image is laid out in half tiles of NT / 2 columns ([2 nt + rank][kb][planes][NT / 2 x 64 B]).
template <class P, class Epi, int CH>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(threads_for(8), 1)
k_gemm_2sm(const uint8_t* __restrict__ aimg, const uint8_t* __restrict__ bimg, GemmShape sh,
           Epi epi, int* __restrict__ status) {
  constexpr int DW = 8, KS = 2;
  pdl_trigger();   // the next kernel of the step may be scheduled
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int NT = sh.NT, H = NT / 2, S = sh.stages, n_kb1 = sh.n_kb, n_kb = (n_kb1 + KS - 1) / KS;
  const Layout L = layout<P>(H, S, KS);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + L.bar_off);
  uint64_t* full = bars;              // used in CTA 0 only
  uint64_t* mmadone = bars + S;
  uint64_t* ready = bars + 2 * S;
  uint64_t* done = bars + 3 * S;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * S + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = cluster_ctarank();
  const int n_mt2 = (sh.n_mt + 1) / 2;
  const int pair = blockIdx.x >> 1;
  const int mt = 2 * (pair % n_mt2) + (int)rank;   // this CTA's 128-row tile of A
  const int nt = pair / n_mt2;                      // the pair's column tile
  const int stride = (NT + 31) & ~31;
  const uint32_t full0 = cluster_addr(smem_u32(&full[0]), 0);   // CTA 0's full[0]

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&full[s]), 2 * (1 + DW));
      mbar_init(smem_u32(&mmadone[s]), 1);
      mbar_init(smem_u32(&ready[s]), 1);
    }
    mbar_init(smem_u32(done), 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc_pair(smem_u32(tmem_slot), sh.tmem_cols);
  tc_fence_before();
  cluster_sync_all();   // barriers of both CTAs initialised, TMEM of both allocated
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // barriers and TMEM are set up; the operands and outputs belong to the kernels before
  pdl_wait();
  if (rank == 1 && tid == 0) {
    // the MMA thread addresses both CTAs' accumulators through CTA 0's TMEM address
    uint32_t lead;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(lead) : "r"(cluster_addr(smem_u32(tmem_slot), 0)) : "memory");
    if (lead != tmem) *abort_flag = 1;
  }

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------- copies ----
      const uint8_t* asrc = aimg + (size_t)mt * n_kb1 * L.a1;
      const uint8_t* bsrc = bimg + (size_t)(2 * nt + (int)rank) * n_kb1 * L.b1;
      int next = 0, fwd = 0;
      long idle = 0;
      while (fwd < n_kb) {
        bool progress = false;
        if (next < n_kb) {
          const int s = next % S, r = next / S;
          if (r == 0 || mbar_test_wait_cl(smem_u32(&mmadone[s]), (r - 1) & 1)) {
            uint8_t* st = base + s * L.stage;
            const int nk = min(KS, n_kb1 - next * KS);
            mbar_arrive_tx(smem_u32(&ready[s]), nk * (L.a1 + L.b1));
            bulk_g2s(smem_u32(st), asrc + (size_t)next * KS * L.a1, nk * L.a1, smem_u32(&ready[s]));
            bulk_g2s(smem_u32(st + L.a_bytes), bsrc + (size_t)next * KS * L.b1, nk * L.b1,
                     smem_u32(&ready[s]));
            ++next;
            progress = true;
          }
        }
        if (fwd < next && mbar_test_wait(smem_u32(&ready[fwd % S]), (fwd / S) & 1)) {
          mbar_arrive_remote(full0 + 8u * (uint32_t)(fwd % S));
          ++fwd;
          progress = true;
        }
        if (progress) {
          idle = 0;
        } else if (++idle > (kSpinLimit << 6) || *abort_flag) {
          *abort_flag = 1;
          break;
        }
      }
      for (int kb = fwd; kb < next; ++kb) mbar_wait_drain(smem_u32(&ready[kb % S]), (kb / S) & 1);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      // ------------------------------------------------------------- MMA ----
      const uint32_t idesc = idesc_bf16(2 * kM, NT);
      const uint32_t b_plane = H * kRow;
      const uint32_t peer_done0 = cluster_addr(smem_u32(&mmadone[0]), 1);
      for (int kb = 0; kb < n_kb; ++kb) {
        const int s = kb % S, r = kb / S, b = kb & 1;
        if (!mbar_wait_cl(smem_u32(&full[s]), r & 1, abort_flag)) break;
        tc_fence_after();
        const uint32_t a0 = smem_u32(base + s * L.stage);
        const uint32_t d_main = tmem + (uint32_t)((2 * b) * stride);
        const uint32_t d_corr = tmem + (uint32_t)((2 * b + 1) * stride);
        const int nk = min(KS, n_kb1 - kb * KS);
#pragma unroll
        for (int h = 0; h < KS; ++h) {
          if (h >= nk) break;
          const uint64_t da = desc64(a0 + h * L.a1), db = desc64(a0 + L.a_bytes + h * L.b1);
#pragma unroll
          for (int j = 0; j < kK / 16; ++j) {
#pragma unroll
            for (int t = 0; t < P::kProducts; ++t) {
              const uint64_t ad = da + (uint64_t)((P::pa(t) * kPlaneM + j * 256) >> 4);
              const uint64_t bd = db + (uint64_t)((P::pb(t) * b_plane + j * 256) >> 4);
              const bool lead = (t == 0);
              const bool first = (h == 0) && (j == 0) && (t <= 1);
              mma_bf16_pair(lead ? d_main : d_corr, ad, bd, idesc, first ? 0u : 1u);
            }
          }
        }
        mma_commit_pair(smem_u32(&mmadone[s]));
        mma_commit_pair(peer_done0 + 8u * (uint32_t)s);
      }
      mma_commit_pair(smem_u32(done));
      mbar_wait_drain(smem_u32(done), 0);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ drain ----
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row = quarter * 32 + lane;
    const int nch = NT / 16;
    const int nch0 = (nch + 1) / 2;
    const int c_begin = half ? nch0 : 0;
    const int my = half ? nch - nch0 : nch0;
    float acc[CH * 16];
#pragma unroll
    for (int t = 0; t < CH * 16; ++t) acc[t] = 0.0f;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    float2* gstage = nullptr;
    if constexpr (Epi::kGamma) {
      if (sh.pre_off) {
        gstage = reinterpret_cast<float2*>(base + sh.pre_off);
        epi.prefetch(gstage, mt, nt, NT, tid - 64, 32 * DW);
      }
    }
    if (lane == 0) {
      mbar_arrive_remote(full0);
      if (n_kb > 1) mbar_arrive_remote(full0 + 8u * (uint32_t)(1 % S));
    }
    bool ok = true;
    for (int kb = 0; kb < n_kb && ok; ++kb) {
      const int b = kb & 1;
      const bool got = mbar_wait_cl(smem_u32(&mmadone[kb % S]), (kb / S) & 1, abort_flag);
      if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
      tc_fence_after();
      const uint32_t slot_m = lane_base + (2 * b) * stride + c_begin * 16;
      const uint32_t slot_c = lane_base + (2 * b + 1) * stride + c_begin * 16;
      if constexpr (CH <= 3) {
        uint32_t m0[16], r0[16], m1[16], r1[16], m2[16], r2[16];
        tmem_ld16_async(slot_m, m0);
        tmem_ld16_async(slot_c, r0);
        if (my > 1) {
          tmem_ld16_async(slot_m + 16, m1);
          tmem_ld16_async(slot_c + 16, r1);
        }
        if (my > 2) {
          tmem_ld16_async(slot_m + 32, m2);
          tmem_ld16_async(slot_c + 32, r2);
        }
        tmem_wait_ld();
        reg_fence(m0);
        reg_fence(r0);
#pragma unroll
        for (int t = 0; t < 16; ++t) acc[t] += __uint_as_float(m0[t]) + __uint_as_float(r0[t]);
        if (my > 1) {
          reg_fence(m1);
          reg_fence(r1);
#pragma unroll
          for (int t = 0; t < 16; ++t) acc[16 + t] += __uint_as_float(m1[t]) + __uint_as_float(r1[t]);
        }
        if (my > 2) {
          reg_fence(m2);
          reg_fence(r2);
#pragma unroll
          for (int t = 0; t < 16; ++t) acc[32 + t] += __uint_as_float(m2[t]) + __uint_as_float(r2[t]);
        }
      } else {
#pragma unroll
        for (int g = 0; g < CH; g += 2) {
          uint32_t m0[16], r0[16], m1[16], r1[16];
          tmem_ld16_async(slot_m + g * 16, m0);
          tmem_ld16_async(slot_c + g * 16, r0);
          tmem_ld16_async(slot_m + (g + 1) * 16, m1);
          tmem_ld16_async(slot_c + (g + 1) * 16, r1);
          tmem_wait_ld();
          reg_fence(m0);
          reg_fence(r0);
          reg_fence(m1);
          reg_fence(r1);
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            acc[g * 16 + t] += __uint_as_float(m0[t]) + __uint_as_float(r0[t]);
            acc[(g + 1) * 16 + t] += __uint_as_float(m1[t]) + __uint_as_float(r1[t]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0 && kb + 2 < n_kb) mbar_arrive_remote(full0 + 8u * (uint32_t)((kb + 2) % S));
    }
    if (gstage) {
      cp_async_commit_wait_all();
      drain_bar(32 * DW);
    }
    const bool all_ok = __all_sync(0xffffffffu, ok) && !*abort_flag;
    if (all_ok) {
      const int dt = tid - 64;
      float* ep = reinterpret_cast<float*>(base);
#pragma unroll
      for (int c = 0; c < CH * 16; ++c)
        if (c < my * 16) ep[c * (32 * DW) + dt] = acc[c];
      Epi e = epi;
      e.set_stage(gstage, nt * NT);
      e(mt * kM + row, nt * NT + c_begin * 16, ep + dt, 32 * DW, my * 16);
    }
  }
  tc_fence_before();
  // both CTAs are past their last TMEM access and CTA 0's MMAs have completed
  cluster_sync_all();
  if (tid == 0 && *abort_flag) atomicExch(status, 1);
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_pair(tmem, sh.tmem_cols);
  }
}

// -------------------------------------------------------------- operand images ----

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// FP64 value -> n bf16 planes, each the rounded remainder of the previous ones
template <int NP>
__device__ __forceinline__ void split_f64(double x, __nv_bfloat16 (&p)[NP]) {
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    p[k] = __float2bfloat16_rn((float)x);
    x -= (double)bf(p[k]);
  }
}
// double-float (hi + lo) -> 3 bf16 planes (the remainder of each plane rounded into the next)
__device__ __forceinline__ void split_df(float hi, float lo, __nv_bfloat16 (&p)[3]) {
  p[0] = __float2bfloat16_rn(hi);
  float r = (hi - bf(p[0])) + lo;
  p[1] = __float2bfloat16_rn(r);
  p[2] = __float2bfloat16_rn(r - bf(p[1]));
}
// FP32 -> 3 bf16 planes (exact)
__device__ __forceinline__ void split_f32(float x, __nv_bfloat16 (&p)[3]) {
  p[0] = __float2bfloat16_rn(x);
  const float r = x - bf(p[0]);
  p[1] = __float2bfloat16_rn(r);
  p[2] = __float2bfloat16_rn(r - bf(p[1]));
}

template <int NP>
__device__ __forceinline__ void store_planes(uint8_t* dst, uint32_t plane_bytes, uint32_t off,
                                             const __nv_bfloat16 (&v)[8][NP]) {
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    __align__(16) __nv_bfloat16 o[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) o[u] = v[u][p];
    *reinterpret_cast<uint4*>(dst + (size_t)p * plane_bytes + off) = *reinterpret_cast<const uint4*>(o);
  }
}

// Forward A image [mt][kb][3 planes][128 rows x 64 B]: (q, 2n + t) = Re/Im E_{q,n}
__global__ void k_eimg_fwd(uint8_t* __restrict__ img, const cplx* __restrict__ phase, int N_k,
                           int n_h, int n_mt, int n_kb) {
  const long total = (long)n_mt * n_kb * kM * 4;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    long t = e;
    const int ch = (int)(t % 4); t /= 4;
    const int row = (int)(t % kM); t /= kM;
    const int kb = (int)(t % n_kb); t /= n_kb;
    const int mt = (int)t;
    const int q = mt * kM + row;
    __nv_bfloat16 v[8][kPlanes];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int n = (kb * kK + ch * 8) / 2 + u;
      cplx E = {0.0, 0.0};
      if (q < N_k && n < n_h) E = phase[(size_t)q * n_h + n];
      split_f64<kPlanes>(E.x, v[2 * u]);
      split_f64<kPlanes>(E.y, v[2 * u + 1]);
    }
    store_planes<kPlanes>(img + ((size_t)mt * n_kb + kb) * kPlanes * kPlaneM, kPlaneM,
                          off64(row, ch * 16), v);
  }
}

// Adjoint A image [mt][kb][3 planes][128 rows x 64 B]: (2n + t, q) = Re E_{q,n}, -Im E_{q,n}
__global__ void k_eimg_adj(uint8_t* __restrict__ img, const cplx* __restrict__ phase, int N_k,
                           int n_h, int n_mt, int n_kb) {
  const long total = (long)n_mt * n_kb * kM * 4;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    long t = e;
    const int row = (int)(t % kM); t /= kM;
    const int ch = (int)(t % 4); t /= 4;
    const int kb = (int)(t % n_kb); t /= n_kb;
    const int mt = (int)t;
    const int m = mt * kM + row;
    const int n = m >> 1;
    __nv_bfloat16 v[8][kPlanes];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = kb * kK + ch * 8 + u;
      double x = 0.0;
      if (q < N_k && n < n_h) {
        const cplx E = phase[(size_t)q * n_h + n];
        x = (m & 1) ? -E.y : E.x;
      }
      split_f64<kPlanes>(x, v[u]);
    }
    store_planes<kPlanes>(img + ((size_t)mt * n_kb + kb) * kPlanes * kPlaneM, kPlaneM,
                          off64(row, ch * 16), v);
  }
}

// double-float copy (re_hi, im_hi, re_lo, im_lo) and FP32 copy of the Gamma-ratio table
__global__ void k_gtab_split(float4* __restrict__ gdf, float2* __restrict__ g32,
                             const cplx* __restrict__ gtab, long n) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const cplx g = gtab[e];
    const float rh = (float)g.x, ih = (float)g.y;
    gdf[e] = make_float4(rh, ih, (float)(g.x - (double)rh), (float)(g.y - (double)ih));
    g32[e] = make_float2(rh, ih);
  }
}

// kmu[i][s][q] = kpow_i[q] mu_{p(i), q, s}  (p = i with per-tracer profiles, else 0)
__global__ void k_kmu(float* __restrict__ kmu, const double* __restrict__ kpow,
                      const double* __restrict__ mu, int N_tr, int N_k, int r, int per_tracer) {
  const long total = (long)N_tr * 4 * N_k;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int q = (int)(e % N_k);
    const int s = (int)((e / N_k) % 4);
    const int i = (int)(e / (4L * N_k));
    const int p = per_tracer ? i : 0;
    kmu[e] = s < r ? (float)(kpow[(size_t)i * N_k + q] * mu[((size_t)p * N_k + q) * 4 + s]) : 0.0f;
  }
}


// Forward B image [nt][kb][3 planes][NT rows x 64 B]: row j = (w, i, l, s) (s fastest),
// (j, 2n) = Re H, (j, 2n+1) = -Im H, H = F_{w,i,s,n} G_{cls(i)}[l_lo + l][n] in double-float.
// Grid (n_kb, n_nt), NT * 4 threads: thread (row, ch) writes 16 bytes of each plane (four n).
// at most 40 registers (no spills): four blocks of 384 threads (96-column tiles) per SM
__global__ void __maxnreg__(40) k_himg(uint8_t* __restrict__ img, const float4* __restrict__ F,
                       const float4* __restrict__ gdf, const int* __restrict__ cls_of,
                       const int2* __restrict__ cmap, int N_tr, int N_ell, int n_h, int l_lo,
                       int n_l, int r, int NI, int n_cols, int NT, int n_kb) {
  pdl_trigger();
  const int kb = blockIdx.x, nt = blockIdx.y;
  const int row = threadIdx.x >> 2, ch = threadIdx.x & 3;
  const int j = nt * NT + row;
  __nv_bfloat16 v[8][kPlanes];
  const bool live = j < n_cols;
  int s = 0, l = 0, wi = 0, i = 0;
  if (live) {
    s = j % r;
    const int g = j / r;
    if (cmap) {
      const int2 cm = cmap[g];
      wi = cm.x;
      l = cm.y;
    } else {
      l = g % n_l;
      wi = g / n_l;
    }
    i = wi % N_tr;
  }
  const float4* Fr = F + ((size_t)wi * NI + s) * n_h;
  const float4* Gr = gdf + ((size_t)(live ? cls_of[i] : 0) * N_ell + l_lo + l) * n_h;
  const int n0 = (kb * kK + ch * 8) / 2;
  // the Gamma table and the column maps are the grid's; F comes from the FFTLog before
  float4 gv[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) gv[u] = (live && n0 + u < n_h) ? Gr[n0 + u] : make_float4(0.f, 0.f, 0.f, 0.f);
  pdl_wait();
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int n = n0 + u;
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    if (live && n < n_h) {
      const float4 f = Fr[n], g = gv[u];
      // Re = fr gr - fi gi, Im = fr gi + fi gr
      df_dot2(f.x, f.z, g.x, g.z, f.y, f.w, g.y, g.w, -1.0f, rh, rl);
      df_dot2(f.x, f.z, g.y, g.w, f.y, f.w, g.x, g.z, 1.0f, ih, il);
    }
    split_df(rh, rl, v[2 * u]);
    split_df(-ih, -il, v[2 * u + 1]);
  }
  store_planes<kPlanes>(img + ((size_t)nt * n_kb + kb) * kPlanes * NT * kRow, NT * kRow,
                        off64(row, ch * 16), v);
}

// Adjoint B image [nt][kb][3 planes][NT rows x 64 B]: row j = (w, i, s, l) (l fastest),
// (j, q) = kmu[i][s][q] Dbar[w][l][i][q].  Grid (n_kb, n_nt), NT * 4 threads: thread (row, ch)
// writes eight q; vec4: N_k % 4 == 0, so that the rows of Dbar and kmu hold 16-byte aligned
// groups of four.
// at most 32 registers (no spills): five blocks of 384 threads per SM
__global__ void __maxnreg__(32) k_dimg(uint8_t* __restrict__ img, const float* __restrict__ dbar,
                       const float* __restrict__ kmu, const int2* __restrict__ cmap, int N_tr,
                       int N_k, int n_l, int r, int n_cols, int NT, int n_kb, int vec4,
                       double* __restrict__ zero, long n_zero) {
  pdl_trigger();
  const int kb = blockIdx.x, nt = blockIdx.y;
  const int row = threadIdx.x >> 2, ch = threadIdx.x & 3;
  const int j = nt * NT + row;
  const bool live = j < n_cols;
  int l = 0, s = 0, i = 0, w = 0;
  if (live) {
    int g;
    if (cmap) {
      const int2 cm = cmap[j];
      g = cm.x;
      l = cm.y;
    } else {
      l = j % n_l;
      g = j / n_l;
    }
    s = g % r;
    const int wi = g / r;
    i = wi % N_tr;
    w = wi / N_tr;
  }
  const float* drow = dbar + (((size_t)w * n_l + l) * N_tr + i) * N_k;
  const float* krow = kmu + ((size_t)i * 4 + s) * N_k;
  const int q0 = kb * kK + ch * 8;
  // Dbar comes from the kernel before; zero[0 .. n_zero) (the adjoint GEMM's accumulator, which
  // the adjoint of the step before read last) is cleared here for the GEMM that follows
  pdl_wait();
  if (zero) {
    const long nthr = (long)gridDim.x * gridDim.y * blockDim.x;
    const long t0 = ((long)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x;
    for (long e = t0; e < n_zero; e += nthr) zero[e] = 0.0;
  }
  float x[8];
  if (vec4 && live && q0 + 8 <= N_k) {
    const float4 d0 = *reinterpret_cast<const float4*>(drow + q0);
    const float4 d1 = *reinterpret_cast<const float4*>(drow + q0 + 4);
    const float4 k0 = *reinterpret_cast<const float4*>(krow + q0);
    const float4 k1 = *reinterpret_cast<const float4*>(krow + q0 + 4);
    x[0] = k0.x * d0.x; x[1] = k0.y * d0.y; x[2] = k0.z * d0.z; x[3] = k0.w * d0.w;
    x[4] = k1.x * d1.x; x[5] = k1.y * d1.y; x[6] = k1.z * d1.z; x[7] = k1.w * d1.w;
  } else {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = q0 + u;
      x[u] = (live && q < N_k) ? krow[q] * drow[q] : 0.0f;
    }
  }
  __nv_bfloat16 v[8][3];
#pragma unroll
  for (int u = 0; u < 8; ++u) split_f32(x[u], v[u]);
  store_planes<kPlanes>(img + ((size_t)nt * n_kb + kb) * kPlanes * NT * kRow, NT * kRow,
                        off64(row, ch * 16), v);
}

unsigned grid_for(long total) {
  return (unsigned)std::max<long>(1, std::min<long>((total + 255) / 256, 152L * 32));
}

// Tile configuration code: column tile NT in bits 0-7, bit 8 = the two-CTAs-per-SM variant.
constexpr int kPair = 256;
// bit 10 = two K-blocks per pipeline stage: one barrier round trip, commit and drain per 64 of K
constexpr int kDeep = 1024;
// bit 12 (with bit 10) = the persistent two-K-block GEMM (k_gemm_persist), tiles up to 96 columns
constexpr int kPersist = 4096;
// bit 16 (with bits 10 and 12) = the persistent GEMM with epilogue warps (k_gemm_persist_ep)
constexpr int kPersistEp = 65536;
// bit 13 (with bit 10) = the two-SM tile (k_gemm_2sm): 256 rows x NT columns per CTA pair,
// NT in {64, 96, 128}; bit 11 with it = stage the adjoint epilogue's table rows in shared memory
// even where that leaves room for two pipeline stages only
constexpr int kTwoSM = 8192;
constexpr int kTableFirst = 2048;
// bit 14 = one accumulator slot per TMEM buffer (k_gemm_basis<..., MG = true>): column tiles up to
// kMaxNTWide; tiles wider than 128 take one K-block per stage except 160 with bit 10
constexpr int kMerged = 16384;
constexpr int kMaxNTWide = 240;
// bit 15 (with bit 14, one K-block per stage, 160 columns or more) = K split over a cluster of
// two CTAs (k_gemm_basis<..., SK = 2>): twice the CTAs of the wide tiles for few walkers
constexpr int kSplitK = 32768;

// columns per tile of the B operand image: a two-SM tile's image holds half tiles
inline int img_cols(int code) { return (code & kTwoSM) ? (code & 255) / 2 : (code & 255); }
inline int img_tiles(int code, int n_nt) { return (code & kTwoSM) ? 2 * n_nt : n_nt; }

// extra: bytes of table rows the epilogue stages in shared memory during the main loop; they are
// added only where they fit beside the stage count the tile has without them, and only in the
// one-CTA-per-SM non-persistent form
template <class P>
int shape_for(swcl_ctx* c, int code, int n_mt, int n_kb, GemmShape& sh, uint32_t& smem,
              uint32_t extra = 0) {
  const int NT = code & 255;
  const bool pair = code & kPair;
  const int KS = (code & kDeep) ? 2 : 1;
  const uint32_t cap = pair ? 113 * 1024 : 227 * 1024;
  int stages = kMaxStages;
  const bool persist = code & kPersist;
  const bool two_sm = code & kTwoSM;
  if (persist && (!(code & kDeep) || NT > 96))
    return fail(c, SWCL_ERR_INVALID_ARG, "persistent GEMM tiles: two K-blocks per stage, <= 96 columns");
  if (two_sm && (!(code & kDeep) || persist || pair || NT % 32 || NT < 64 || NT > 128))
    return fail(c, SWCL_ERR_INVALID_ARG, "two-SM GEMM tiles: two K-blocks per stage, 64, 96 or 128 columns");
  if ((code & kTableFirst) && !two_sm)
    return fail(c, SWCL_ERR_INVALID_ARG, "GEMM tile code: bit 11 needs the two-SM tile");
  const bool merged = code & kMerged;
  if (merged && (persist || two_sm || NT % 16 || NT < 64 || NT > kMaxNTWide ||
                 (NT > 160 && KS == 2) || (pair && (KS != 1 || NT % 32 || NT > 128))))
    return fail(c, SWCL_ERR_INVALID_ARG,
                "one-slot GEMM tiles: 64..240 columns (<= 160 with two K-blocks; 64, 96 or 128 "
                "with one K-block at two CTAs per SM)");
  if (!merged && NT > kMaxNT)
    return fail(c, SWCL_ERR_INVALID_ARG, "GEMM tiles wider than 128 columns need bit 14");
  const bool splitk = code & kSplitK;
  if (splitk && (!merged || KS != 1 || NT < 160 || n_kb < 2))
    return fail(c, SWCL_ERR_INVALID_ARG, "split-K GEMM tiles: bit 14, one K-block per stage, >= 160 columns");
  const bool persist_ep = code & kPersistEp;
  if (persist_ep && !persist)
    return fail(c, SWCL_ERR_INVALID_ARG, "GEMM tile code: bit 16 needs bits 10 and 12");
  auto lay = [&](int st) {
    return persist_ep ? layout_persist_ep<P>(NT, st)
         : persist ? layout_persist<P>(NT, st, 3) : layout<P>(two_sm ? NT / 2 : NT, st, KS);
  };
  // the table rows the epilogue stages sit after the barriers
  auto with_extra = [&](const Layout& L) {
    return ((L.bar_off + 8 * (3 * L.stages + 1) + 16 + 127) & ~127u) + extra + 1024;
  };
  Layout L = lay(stages);
  while (stages > 2 && L.total > cap) L = lay(--stages);
  if (extra && (code & kTableFirst))
    while (stages > 2 && with_extra(L) > cap) L = lay(--stages);
  if (L.total > cap) return fail(c, SWCL_ERR_UNSUPPORTED, "basis GEMM tile does not fit shared memory");
  const int stride = (NT + 31) & ~31;
  uint32_t cols = 32;
  while (cols < (uint32_t)((merged ? 2 : 4) * stride)) cols <<= 1;
  if (cols > 512) return fail(c, SWCL_ERR_UNSUPPORTED, "basis GEMM tile does not fit TMEM");
  // the epilogue stages the accumulators of the 256 drain threads in the stage ring
  if (!persist && !pair && L.stages * L.stage < (uint32_t)(16 * ((NT / 16 + 1) / 2) * 256 * 4))
    return fail(c, SWCL_ERR_UNSUPPORTED, "basis GEMM tile: stage ring smaller than the epilogue");
  sh = GemmShape{n_mt, n_kb, NT, stages, cols, 0};
  smem = L.total;
  if (extra && !persist && !pair && !splitk && with_extra(L) <= cap) {
    sh.pre_off = (L.bar_off + 8 * (3 * stages + 1) + 16 + 127) & ~127u;
    smem = with_extra(L);
  }
  return SWCL_OK;
}

template <class P, class Epi, int DW, int CH, int KS, uint32_t PM = 0x3Fu, bool MG = false>
cudaError_t launch_variant(swcl_ctx* c, const uint8_t* a, const uint8_t* b, const GemmShape& sh,
                           uint32_t smem, int n_nt, const Epi& epi) {
  cudaError_t e = cudaFuncSetAttribute(k_gemm_basis<P, Epi, DW, CH, KS, PM, MG>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return launch_k(c->pdl && !c->prof, k_gemm_basis<P, Epi, DW, CH, KS, PM, MG>, dim3((unsigned)(sh.n_mt * n_nt)),
                  dim3(threads_for(DW)), smem, c->stream, a, b, sh, epi, (int*)c->ws_status.p);
}

// The product subsets of the accuracy study, at the 96-column two-K-block tile only.
template <class P, class Epi>
cudaError_t launch_subset(swcl_ctx* c, uint32_t pm, const uint8_t* a, const uint8_t* b,
                          const GemmShape& sh, uint32_t smem, int n_nt, const Epi& epi) {
  switch (pm) {
    case 0x2Fu: return launch_variant<P, Epi, 8, 3, 2, 0x2Fu>(c, a, b, sh, smem, n_nt, epi);
    case 0x37u: return launch_variant<P, Epi, 8, 3, 2, 0x37u>(c, a, b, sh, smem, n_nt, epi);
    case 0x1Fu: return launch_variant<P, Epi, 8, 3, 2, 0x1Fu>(c, a, b, sh, smem, n_nt, epi);
    case 0x17u: return launch_variant<P, Epi, 8, 3, 2, 0x17u>(c, a, b, sh, smem, n_nt, epi);
    case 0x07u: return launch_variant<P, Epi, 8, 3, 2, 0x07u>(c, a, b, sh, smem, n_nt, epi);
    default: return cudaErrorInvalidValue;
  }
}

template <class P, class Epi>
cudaError_t launch_persist_ep(swcl_ctx* c, const uint8_t* a, const uint8_t* b, const GemmShape& sh,
                              uint32_t smem, int n_nt, const Epi& epi) {
  cudaError_t e = cudaFuncSetAttribute(k_gemm_persist_ep<P, Epi, 3>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int n_tiles = sh.n_mt * n_nt;
  const int grid = std::min(n_tiles, std::max(1, c->num_sms));
  return launch_k(c->pdl && !c->prof, k_gemm_persist_ep<P, Epi, 3>, dim3((unsigned)grid), dim3(threads_persist_ep()),
                  smem, c->stream, a, b, sh, n_tiles, epi, (int*)c->ws_status.p);
}

template <class P, class Epi>
cudaError_t launch_persist(swcl_ctx* c, const uint8_t* a, const uint8_t* b, const GemmShape& sh,
                           uint32_t smem, int n_nt, const Epi& epi) {
  cudaError_t e = cudaFuncSetAttribute(k_gemm_persist<P, Epi, 3>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int n_tiles = sh.n_mt * n_nt;
  const int grid = std::min(n_tiles, std::max(1, c->num_sms));
  return launch_k(c->pdl && !c->prof, k_gemm_persist<P, Epi, 3>, dim3((unsigned)grid), dim3(threads_for(8)), smem,
                  c->stream, a, b, sh, n_tiles, epi, (int*)c->ws_status.p);
}

// one K-block per stage, one accumulator slot, 8 chunks per drain thread, K split over a
// cluster of two CTAs
template <class P, class Epi>
cudaError_t launch_splitk(swcl_ctx* c, const uint8_t* a, const uint8_t* b, const GemmShape& sh,
                          uint32_t smem, int n_nt, const Epi& epi) {
  auto kern = k_gemm_basis<P, Epi, 8, 8, 1, 0x3Fu, true, 2>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * sh.n_mt * n_nt));
  cfg.blockDim = dim3(threads_for(8));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c->stream;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = c->pdl && !c->prof ? 2 : 1;
  e = cudaLaunchKernelEx(&cfg, kern, a, b, sh, epi, (int*)c->ws_status.p);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

template <class P, class Epi, int CH>
cudaError_t launch_2sm(swcl_ctx* c, const uint8_t* a, const uint8_t* b, const GemmShape& sh,
                       uint32_t smem, int n_nt, const Epi& epi) {
  cudaError_t e = cudaFuncSetAttribute(k_gemm_2sm<P, Epi, CH>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int n_mt2 = (sh.n_mt + 1) / 2;
  return launch_k(c->pdl && !c->prof, k_gemm_2sm<P, Epi, CH>, dim3((unsigned)(2 * n_mt2 * n_nt)), dim3(threads_for(8)),
                  smem, c->stream, a, b, sh, epi, (int*)c->ws_status.p);
}

template <class P, class Epi>
cudaError_t launch_gemm(swcl_ctx* c, int code, const uint8_t* a, const uint8_t* b,
                        const GemmShape& sh, uint32_t smem, int n_nt, const Epi& epi) {
  const int nch = sh.NT / 16;
  if (c->bt_pmask != 0x3Fu) {
    if (code != (96 | kDeep)) return cudaErrorInvalidValue;   // study subsets: tile 1120 only
    return launch_subset<P, Epi>(c, c->bt_pmask, a, b, sh, smem, n_nt, epi);
  }
  if (code & kTwoSM)
    return (nch + 1) / 2 <= 3 ? launch_2sm<P, Epi, 3>(c, a, b, sh, smem, n_nt, epi)
                              : launch_2sm<P, Epi, 4>(c, a, b, sh, smem, n_nt, epi);
  if (code & kSplitK) return launch_splitk<P, Epi>(c, a, b, sh, smem, n_nt, epi);
  if ((code & kMerged) && (code & kPair))   // two CTAs per SM, four drain warps: whole rows
    return nch <= 4 ? launch_variant<P, Epi, 4, 4, 1, 0x3Fu, true>(c, a, b, sh, smem, n_nt, epi)
         : nch <= 6 ? launch_variant<P, Epi, 4, 6, 1, 0x3Fu, true>(c, a, b, sh, smem, n_nt, epi)
                    : launch_variant<P, Epi, 4, 8, 1, 0x3Fu, true>(c, a, b, sh, smem, n_nt, epi);
  if (code & kMerged) {
    const int ch = (nch + 1) / 2;
    if (!(code & kDeep)) return launch_variant<P, Epi, 8, 8, 1, 0x3Fu, true>(c, a, b, sh, smem, n_nt, epi);
    return ch <= 3 ? launch_variant<P, Epi, 8, 3, 2, 0x3Fu, true>(c, a, b, sh, smem, n_nt, epi)
         : ch <= 4 ? launch_variant<P, Epi, 8, 4, 2, 0x3Fu, true>(c, a, b, sh, smem, n_nt, epi)
                   : launch_variant<P, Epi, 8, 8, 2, 0x3Fu, true>(c, a, b, sh, smem, n_nt, epi);
  }
  if (code & kPersistEp) return launch_persist_ep<P, Epi>(c, a, b, sh, smem, n_nt, epi);
  if (code & kPersist) return launch_persist<P, Epi>(c, a, b, sh, smem, n_nt, epi);
  if (code & kPair)   // four drain warps: every chunk of a row in one thread
    return nch <= 3 ? launch_variant<P, Epi, 4, 3, 1>(c, a, b, sh, smem, n_nt, epi)
                    : launch_variant<P, Epi, 4, 4, 1>(c, a, b, sh, smem, n_nt, epi);
  if (code & kDeep)
    return (nch + 1) / 2 <= 3 ? launch_variant<P, Epi, 8, 3, 2>(c, a, b, sh, smem, n_nt, epi)
                              : launch_variant<P, Epi, 8, 4, 2>(c, a, b, sh, smem, n_nt, epi);
  return (nch + 1) / 2 <= 3 ? launch_variant<P, Epi, 8, 3, 1>(c, a, b, sh, smem, n_nt, epi)
                            : launch_variant<P, Epi, 8, 4, 1>(c, a, b, sh, smem, n_nt, epi);
}

// Candidate tile codes: column tiles that are multiples of 16; in forward tiles each drain
// thread's column range (whole 16-column chunks; split in two halves with eight drain warps)
// holds whole groups of r basis columns.
std::vector<int> tile_candidates(int r, bool need_groups, bool tuned_only = false) {
  std::vector<int> v;
  // one-slot tiles: two K-blocks per stage up to 160 columns, one beyond.  Tuned in the adjoint
  // only: in the forward their C error (4.4e-5 of the oracle at N5K shape, against 3.1e-5 with
  // two slots) took a mixed-precision JVP over its gate
  for (int nt = 64; nt <= kMaxNTWide && !(tuned_only && need_groups); nt += 16) {
    const int half0 = 16 * ((nt / 16 + 1) / 2);
    if (need_groups && (nt % r != 0 || half0 % r != 0)) continue;
    if (nt <= 160 && nt % 32 == 0) v.push_back(nt | kDeep | kMerged);
    if (nt >= 160 && (nt % 32 == 0 || nt == 208 || nt == 240)) {
      v.push_back(nt | kMerged);
      if (need_groups) v.push_back(nt | kMerged | kSplitK);   // forward
    }
    if (nt <= 128 && nt % 32 == 0) v.push_back(nt | kMerged | kPair);   // two CTAs per SM
  }
  // two-SM tiles, in the adjoint also with the table rows staged at two stages: selectable, not
  // tuned (measured no faster than the one-SM tiles of the same width)
  for (int nt = 64; nt <= kMaxNT && !tuned_only; nt += 32) {
    const int half0 = 16 * ((nt / 16 + 1) / 2);
    if (!need_groups || (nt % r == 0 && half0 % r == 0)) {
      v.push_back(nt | kDeep | kTwoSM);
      if (!need_groups) v.push_back(nt | kDeep | kTwoSM | kTableFirst);
    }
  }
  if (!tuned_only) {
    for (int nt = 32; nt <= kMaxNT; nt += 16) {
      const int half0 = 16 * ((nt / 16 + 1) / 2);
      if (!need_groups || (nt % r == 0 && half0 % r == 0)) v.push_back(nt);
    }
    for (int nt = 32; nt <= 64; nt += 16)
      if (!need_groups || nt % r == 0) v.push_back(nt | kPair);
  }
  for (int nt = 64; nt <= kMaxNT; nt += 32) {
    const int half0 = 16 * ((nt / 16 + 1) / 2);
    if (!need_groups || (nt % r == 0 && half0 % r == 0)) {
      v.push_back(nt | kDeep);
      if (nt <= 96) {
        v.push_back(nt | kDeep | kPersist);
        v.push_back(nt | kDeep | kPersist | kPersistEp);
      }
    }
  }
  return v;
}

int basis_rank(swcl_ctx* c) { return c->lr_true_rank; }

bool valid_tile(int code, const std::vector<int>& cands) {
  return std::find(cands.begin(), cands.end(), code) != cands.end();
}

}  // namespace

size_t basis_fixed_bytes(const swcl_ctx* c) {
  // row tiles rounded up to an even count, as in basis_prepare
  const size_t f_mt = (((c->N_k + kM - 1) / kM) + 1) & ~1, f_kb = (2 * c->n_h + kK - 1) / kK;
  const size_t a_mt = (((2 * c->n_h + kM - 1) / kM) + 1) & ~1, a_kb = (c->N_k + kK - 1) / kK;
  const size_t ng = (size_t)c->n_cls * c->N_ell * c->n_h;
  return (f_mt * f_kb + a_mt * a_kb) * kPlanes * kPlaneM + ng * (sizeof(float4) + sizeof(float2)) +
         sizeof(float) * (size_t)c->N_tr * 4 * c->N_k +
         (size_t)kMaxNTWide * (f_kb + a_kb) * kPlanes * kRow;   // column padding of the last tile
}

size_t basis_bytes_per_ell(const swcl_ctx* c) {
  const size_t f_kb = (2 * c->n_h + kK - 1) / kK, a_kb = (c->N_k + kK - 1) / kK;
  return (size_t)c->n_walk * c->N_tr * std::max(1, c->lr_true_rank) * (f_kb + a_kb) * kPlanes * kRow;
}

// Constant operands of basis mode: the two phase images, the FP32/double-float Gamma tables and
// kpow * mu.  Rebuilt whenever the grids, tracers or knot profiles change.
int basis_prepare(swcl_ctx* c) {
  if (c->bt_ready) return SWCL_OK;
  const int N_k = c->N_k, n_h = c->n_h;
  const int r = basis_rank(c);
  int st;
  c->bt_f_mt = (N_k + kM - 1) / kM;
  c->bt_f_kb = (2 * n_h + kK - 1) / kK;
  c->bt_a_mt = (2 * n_h + kM - 1) / kM;
  c->bt_a_kb = (N_k + kK - 1) / kK;
  // the images hold an even number of row tiles (the last one zero when the count is odd), so
  // that the two-SM tiles take rows in pairs of tiles
  const int f_mt2 = (c->bt_f_mt + 1) & ~1, a_mt2 = (c->bt_a_mt + 1) & ~1;
  const size_t ef = (size_t)f_mt2 * c->bt_f_kb * kPlanes * kPlaneM;
  const size_t ea = (size_t)a_mt2 * c->bt_a_kb * kPlanes * kPlaneM;
  if ((st = ensure(c, c->bt_eimg_f, ef))) return st;
  if ((st = ensure(c, c->bt_eimg_a, ea))) return st;
  const long ng = (long)c->n_cls * c->N_ell * n_h;
  if ((st = ensure(c, c->bt_gdf, sizeof(float4) * ng))) return st;
  if ((st = ensure(c, c->bt_g32, sizeof(float2) * ng))) return st;
  if ((st = ensure(c, c->bt_kmu, sizeof(float) * (size_t)c->N_tr * 4 * N_k))) return st;
  long tot = (long)f_mt2 * c->bt_f_kb * kM * 4;
  k_eimg_fwd<<<grid_for(tot), 256, 0, c->stream>>>((uint8_t*)c->bt_eimg_f.p, (const cplx*)c->d_phase.p,
                                                   N_k, n_h, f_mt2, c->bt_f_kb);
  tot = (long)a_mt2 * c->bt_a_kb * kM * 4;
  k_eimg_adj<<<grid_for(tot), 256, 0, c->stream>>>((uint8_t*)c->bt_eimg_a.p, (const cplx*)c->d_phase.p,
                                                   N_k, n_h, a_mt2, c->bt_a_kb);
  k_gtab_split<<<grid_for(ng), 256, 0, c->stream>>>((float4*)c->bt_gdf.p, (float2*)c->bt_g32.p,
                                                    (const cplx*)c->d_gtab.p, ng);
  k_kmu<<<grid_for((long)c->N_tr * 4 * N_k), 256, 0, c->stream>>>(
      (float*)c->bt_kmu.p, (const double*)c->d_kpow.p, (const double*)c->lr_w.p, c->N_tr, N_k, r,
      c->have_B ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "basis operand tables");
  c->bt_nt_fwd = c->bt_fixed_fwd;
  c->bt_nt_adj = c->bt_fixed_adj;
  c->bt_ready = true;
  return SWCL_OK;
}

namespace {

// Columns of the two basis GEMMs for the multipoles [l_lo, l_lo + n_l).  Without ragged lists (or
// when the multipoles run in several chunks) every (walker, tracer, multipole, profile) is a
// column.  With ragged lists covered by one chunk, only the multipoles each walker lists are:
// forward columns (w, i, listed l, s), adjoint columns (w, i, s, listed l), with the maps
//   cmap_f[group of r columns] = {w N_tr + i, l},   cmap_a[column] = {(w N_tr + i) r + s, l},
//   lpos[w][l] = position of l in walker w's list (-1 if unlisted),  wbase[w] = {first column,
//   listed count},
// built on the host once per configuration (outside graph capture).  Delta rows of unlisted
// multipoles are then never written by the forward GEMM: they are cleared once, so that the
// reductions over all multipoles (U, P_bar) read zeros there.
struct ColPlan {
  int n_cols = 0;
  const int2* cmap_f = nullptr;
  const int2* cmap_a = nullptr;
  const int* lpos = nullptr;
  const int2* wbase = nullptr;
};

int column_plan(swcl_ctx* c, int l_lo, int n_l, ColPlan& p) {
  const int r = basis_rank(c);
  p = ColPlan();
  const bool compact = c->ragged && (int)c->off_h.size() == c->n_walk + 1 && l_lo == 0 &&
                       n_l == c->N_ell;
  c->bt_compact = compact;
  if (!compact) {
    p.n_cols = c->n_walk * c->N_tr * n_l * r;
    c->bt_delta_clean = false;   // every row of Delta is written
    return SWCL_OK;
  }
  const int nw = c->n_walk, N_tr = c->N_tr;
  const int64_t n_listed = c->off_h.back();
  int st;
  if ((st = ensure(c, c->bt_cmap_f, sizeof(int2) * std::max<int64_t>(1, n_listed * N_tr)))) return st;
  if ((st = ensure(c, c->bt_cmap_a, sizeof(int2) * std::max<int64_t>(1, n_listed * N_tr * r)))) return st;
  if ((st = ensure(c, c->bt_lpos, sizeof(int) * (size_t)nw * n_l))) return st;
  if ((st = ensure(c, c->bt_wbase, sizeof(int2) * (size_t)nw))) return st;
  const int64_t key[7] = {c->lists_gen, nw, N_tr, n_l, r, (int64_t)(uintptr_t)c->ws_delta.p,
                          (int64_t)c->ws_delta.bytes};
  if (!std::equal(key, key + 7, c->bt_plan_key)) {
    if (c->capturing) return fail(c, SWCL_ERR_STATE, "GEMM column plan built during capture");
    std::vector<int2> cf, ca, wb(nw);
    std::vector<int> lp((size_t)nw * n_l, -1);
    cf.reserve(n_listed * N_tr);
    ca.reserve(n_listed * N_tr * r);
    int col = 0;
    for (int w = 0; w < nw; ++w) {
      const int o0 = c->off_h[w], m = c->off_h[w + 1] - o0;
      wb[w] = make_int2(col, m);
      for (int u = 0; u < m; ++u) lp[(size_t)w * n_l + c->idx_h[o0 + u]] = u;
      for (int i = 0; i < N_tr; ++i)
        for (int u = 0; u < m; ++u) cf.push_back(make_int2(w * N_tr + i, c->idx_h[o0 + u]));
      for (int i = 0; i < N_tr; ++i)
        for (int s = 0; s < r; ++s)
          for (int u = 0; u < m; ++u) ca.push_back(make_int2((w * N_tr + i) * r + s, c->idx_h[o0 + u]));
      col += N_tr * m * r;
    }
    if (!cf.empty()) {
      if ((st = copy_in(c, c->bt_cmap_f, cf.data(), sizeof(int2) * cf.size()))) return st;
      if ((st = copy_in(c, c->bt_cmap_a, ca.data(), sizeof(int2) * ca.size()))) return st;
    }
    if ((st = copy_in(c, c->bt_lpos, lp.data(), sizeof(int) * lp.size()))) return st;
    if ((st = copy_in(c, c->bt_wbase, wb.data(), sizeof(int2) * wb.size()))) return st;
    std::copy(key, key + 7, c->bt_plan_key);
    c->bt_plan_cols = col;
    c->bt_delta_clean = false;
  }
  if (!c->bt_delta_clean) {
    cudaError_t e = cudaMemsetAsync(c->ws_delta.p, 0, c->ws_delta.bytes, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "clear Delta");
    c->bt_delta_clean = true;
  }
  p.n_cols = c->bt_plan_cols;
  p.cmap_f = (const int2*)c->bt_cmap_f.p;
  p.cmap_a = (const int2*)c->bt_cmap_a.p;
  p.lpos = (const int*)c->bt_lpos.p;
  p.wbase = (const int2*)c->bt_wbase.p;
  return SWCL_OK;
}

int build_h(swcl_ctx* c, const ColPlan& cp, int NT, int n_nt, int l_lo, int n_l) {
  const Stencil sv = stencil(c);
  const int r = basis_rank(c);
  const int n_cols = cp.n_cols;
  int st = ensure(c, c->bt_himg, (size_t)n_nt * c->bt_f_kb * kPlanes * NT * kRow);
  if (st) return st;
  cudaError_t e = launch_k(c->pdl && !c->prof, k_himg, dim3((unsigned)c->bt_f_kb, (unsigned)n_nt), dim3(NT * 4),
                           0, c->stream, (uint8_t*)c->bt_himg.p, (const float4*)c->ws_coef.p,
                           (const float4*)c->bt_gdf.p, (const int*)c->d_cls_of.p, cp.cmap_f,
                           c->N_tr, c->N_ell, c->n_h, l_lo, n_l, r, sv.NI, n_cols, NT, c->bt_f_kb);
  return e == cudaSuccess ? SWCL_OK : cuda_fail(c, e, "basis forward operand");
}

int build_d(swcl_ctx* c, const ColPlan& cp, int NT, int n_nt, int n_l, double* zero = nullptr,
            long n_zero = 0) {
  const int r = basis_rank(c);
  const int n_cols = cp.n_cols;
  int st = ensure(c, c->bt_dimg, (size_t)n_nt * c->bt_a_kb * kPlanes * NT * kRow);
  if (st) return st;
  cudaError_t e = launch_k(c->pdl && !c->prof, k_dimg, dim3((unsigned)c->bt_a_kb, (unsigned)n_nt), dim3(NT * 4),
                           0, c->stream, (uint8_t*)c->bt_dimg.p, (const float*)c->ws_dbar.p,
                           (const float*)c->bt_kmu.p, cp.cmap_a, c->N_tr, c->N_k, n_l, r, n_cols,
                           NT, c->bt_a_kb, c->N_k % 4 == 0 ? 1 : 0, zero, n_zero);
  return e == cudaSuccess ? SWCL_OK : cuda_fail(c, e, "basis adjoint operand");
}

// one counted (and, when profiling, timed) launch
template <class F>
int counted(swcl_ctx* c, const char* name, F f) {
  ++c->last_launches;
  prof_begin(c);
  const int st = f();
  prof_end(c, name);
  return st;
}

// Times each candidate tile (operand build excluded) and keeps the fastest.
template <class Run>
int autotune(swcl_ctx* c, const std::vector<int>& cands, Run run, int& best) {
  // each candidate: operand build + one warm-up launch, then three timed launches
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
    return fail(c, SWCL_ERR_CUDA, "autotune events");
  float best_ms = 1e30f;
  best = cands.front();
  int st = SWCL_OK;
  for (int code : cands) {
    if ((st = run(code, true))) break;
    cudaEventRecord(a, c->stream);
    for (int rep = 0; rep < 3 && st == SWCL_OK; ++rep) st = run(code, false);
    cudaEventRecord(b, c->stream);
    if (st) break;
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best_ms) { best_ms = ms; best = code; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return st;
}

}  // namespace

// Delta (FP32, [n_walk][n_l][N_tr][N_k]) for multipoles [l_lo, l_lo + n_l) from the basis
// coefficients in ws_coef (double-float).
int basis_forward(swcl_ctx* c, int l_lo, int n_l) {
  int st = basis_prepare(c);
  if (st) return st;
  const int r = basis_rank(c);
  ColPlan cp;
  if ((st = column_plan(c, l_lo, n_l, cp))) return st;
  const int n_cols = cp.n_cols;
  if (n_cols == 0) return SWCL_OK;   // no walker lists a multipole of this chunk
  auto run = [&](int code, bool build) -> int {
    const int NT = code & 255;
    const int n_nt = (n_cols + NT - 1) / NT;
    if (build && (st = build_h(c, cp, img_cols(code), img_tiles(code, n_nt), l_lo, n_l))) return st;
    GemmShape sh;
    uint32_t smem;
    if ((st = shape_for<A3B3>(c, code, c->bt_f_mt, c->bt_f_kb, sh, smem))) return st;
    EpiFwd epi{(float*)c->ws_delta.p, (const float*)c->bt_kmu.p, cp.cmap_f, c->N_k, c->N_tr, n_l, r,
               n_cols};
    cudaError_t e = launch_gemm<A3B3>(c, code, (const uint8_t*)c->bt_eimg_f.p,
                                      (const uint8_t*)c->bt_himg.p, sh, smem, n_nt, epi);
    return e == cudaSuccess ? SWCL_OK : cuda_fail(c, e, "basis forward GEMM");
  };
  if (c->bt_nt_fwd && !valid_tile(c->bt_nt_fwd, tile_candidates(r, true)))
    return fail(c, SWCL_ERR_INVALID_ARG, "SWCL_BASIS_TILES: not a forward tile for this rank");
  if (c->bt_nt_fwd == 0) {
    if (c->capturing) c->bt_nt_fwd = 96 % r == 0 ? 96 : 64;
    else if ((st = autotune(c, tile_candidates(r, true, true), run, c->bt_nt_fwd))) return st;
  }
  const int code = c->bt_nt_fwd, NT = code & 255;
  const int n_nt = (n_cols + NT - 1) / NT;
  if ((st = counted(c, "basis operand fwd", [&] {
         return build_h(c, cp, img_cols(code), img_tiles(code, n_nt), l_lo, n_l);
       })))
    return st;
  return counted(c, "basis gemm fwd", [&] { return run(code, false); });
}

// ws_cbar (FP64 complex, [n_walk][N_tr][NI][n_h], zeroed here) from ws_dbar (FP32,
// [n_walk][n_l][N_tr][N_k]) for multipoles [l_lo, l_lo + n_l); accumulate = keep ws_cbar.
int basis_adjoint(swcl_ctx* c, int l_lo, int n_l, bool accumulate) {
  int st = basis_prepare(c);
  if (st) return st;
  const Stencil sv = stencil(c);
  const int r = basis_rank(c);
  ColPlan cp;
  if ((st = column_plan(c, l_lo, n_l, cp))) return st;
  const int n_cols = cp.n_cols;
  const size_t cbytes = sizeof(cplx) * (size_t)c->n_walk * c->N_tr * sv.NI * c->n_h;
  if (n_cols == 0) {   // no walker lists a multipole of this chunk
    cudaError_t e = accumulate ? cudaSuccess : cudaMemsetAsync(c->ws_cbar.p, 0, cbytes, c->stream);
    return e == cudaSuccess ? SWCL_OK : cuda_fail(c, e, "clear cbar");
  }
  auto run = [&](int code, bool build) -> int {
    const int NT = code & 255;
    const int n_nt = (n_cols + NT - 1) / NT;
    if (build && (st = build_d(c, cp, img_cols(code), img_tiles(code, n_nt), n_l))) return st;
    GemmShape sh;
    uint32_t smem;
    if ((st = shape_for<A3B3>(c, code, c->bt_a_mt, c->bt_a_kb, sh, smem,
                              EpiAdj::stage_bytes(code & 255))))
      return st;
    EpiAdj epi{(cplx*)c->ws_cbar.p, (const float2*)c->bt_g32.p, (const int*)c->d_cls_of.p,
               cp.cmap_a, c->n_h, c->N_tr, c->N_ell, l_lo, n_l, r, sv.NI, n_cols};
    cudaError_t e = launch_gemm<A3B3>(c, code, (const uint8_t*)c->bt_eimg_a.p,
                                      (const uint8_t*)c->bt_dimg.p, sh, smem, n_nt, epi);
    return e == cudaSuccess ? SWCL_OK : cuda_fail(c, e, "basis adjoint GEMM");
  };
  if (c->bt_nt_adj && !valid_tile(c->bt_nt_adj, tile_candidates(r, false)))
    return fail(c, SWCL_ERR_INVALID_ARG, "SWCL_BASIS_TILES: not an adjoint tile");
  if (c->bt_nt_adj == 0) {
    if (c->capturing) {
      c->bt_nt_adj = 96;
    } else {
      // the tuning launches accumulate into ws_cbar, which is cleared below
      if ((st = autotune(c, tile_candidates(r, false, true), run, c->bt_nt_adj))) return st;
      if (accumulate) return fail(c, SWCL_ERR_STATE, "basis adjoint tuned inside an accumulation");
    }
  }
  // the adjoint image's builder clears the GEMM's accumulator (one launch less than a memset
  // between them, which would also break the programmatic launch of the GEMM)
  double* zero = accumulate ? nullptr : (double*)c->ws_cbar.p;
  const long n_zero = (long)(cbytes / sizeof(double));
  const int code = c->bt_nt_adj, NT = code & 255;
  const int n_nt = (n_cols + NT - 1) / NT;
  if ((st = counted(c, "basis operand adj", [&] {
         return build_d(c, cp, img_cols(code), img_tiles(code, n_nt), n_l, zero, n_zero);
       })))
    return st;
  return counted(c, "basis gemm adj", [&] { return run(code, false); });
}

}  // namespace swcl
