// a3 on the 5th-generation tensor cores (tcgen05, sm_103a): the contraction with k-interpolation
//   Delta_i(l, q) = kpow_i[q] * sum_K A_i[q][K] B_cls(i)[K][l]
// as one real GEMM per (walker, tracer, 128-row k tile, multipole tile), K = 2 (N/2 + 1) with the
// complex index interleaved (K = 2n: real part, 2n+1: imaginary part):
//   A[q][2n] + i A[q][2n+1] = (sum_r lw[q][r] c_{i, j0[q]+r, n}) e^{-i eta_n ln k_q},
//   B[2n][l] = Re(w_n pi(l) M_{l,n}),  B[2n+1][l] = -Im(w_n pi(l) M_{l,n}).
// Compensated products with FP32 accumulation in TMEM (Tf32x3, Tf32x6, Bf16x9 in tc_common.cuh).
// The coefficients arrive as double-float pairs (hi + lo), so their rounding, which is the same
// for every k point and would not average out in the k-sum, stays below 2^-44; the interpolation
// and phase product run in FP32 (errors that vary from k point to k point) and the FP32 result
// is split exactly into tf32/bf16 planes.  Warp roles: warps 0-7 form A in shared memory (interpolation, phase,
// split) and drain the accumulator; thread 0 also streams the pre-split B image with
// cp.async.bulk and, once all warps have handed over a K-block, issues its tcgen05.mma
// instructions; warp 0 owns the TMEM allocation.  All waits are
// bounded; a timeout raises a status word the host reports as SWCL_ERR_TIMEOUT.
#include <algorithm>

#include "swcl_internal.h"
#include "tc_common.cuh"

namespace swcl {
namespace {

using namespace tc;

constexpr int kProducers = 256;
constexpr int kThreadsTc = kProducers;   // two warpgroups: the full register file is available

constexpr uint32_t kCoefSmem = 16 * 1024;   // staged knot coefficients of one K-block

struct SmemLayout {
  int stages;
  uint32_t stage_bytes, a_bytes, b_plane_bytes, coef_off, bar_off, total;
};

template <class P>
__host__ __device__ inline SmemLayout smem_layout(int NT, int stages) {
  SmemLayout s;
  s.stages = stages;
  s.a_bytes = P::kPlanesA * kPlaneA;
  s.b_plane_bytes = NT * kRowBytes;
  s.stage_bytes = s.a_bytes + P::kPlanesB * s.b_plane_bytes;
  s.coef_off = stages * s.stage_bytes;
  s.bar_off = s.coef_off + kCoefSmem;
  s.total = s.bar_off + 8 * (3 * stages + 5) + 16 + 1024;  // barriers, tmem slot, abort, align
  return s;
}

// Exact split of FP32 values into planes: tf32 keeps 11 significant bits, so three tf32 planes
// (or three bf16 planes of 8 bits) hold all 24 bits of an FP32 value; two tf32 planes keep 22.
template <class P>
__device__ __forceinline__ void store_split(uint8_t* a_stage, uint32_t off, const float* v) {
  if constexpr (!P::kBf16) {
    float4 p0, p1, p2;
    float* a0 = &p0.x; float* a1 = &p1.x; float* a2 = &p2.x;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float x = v[t];
      a0[t] = tf32_rna(x);
      const float r1 = x - a0[t];
      a1[t] = tf32_rna(r1);
      a2[t] = r1 - a1[t];
    }
    *reinterpret_cast<float4*>(a_stage + off) = p0;
    *reinterpret_cast<float4*>(a_stage + kPlaneA + off) = p1;
    if constexpr (P::kPlanesA == 3) *reinterpret_cast<float4*>(a_stage + 2 * kPlaneA + off) = p2;
  } else {
    __align__(16) __nv_bfloat16 p0[8], p1[8], p2[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const float x = v[t];
      p0[t] = __float2bfloat16_rn(x);
      const float r1 = x - __bfloat162float(p0[t]);
      p1[t] = __float2bfloat16_rn(r1);
      p2[t] = __float2bfloat16_rn(r1 - __bfloat162float(p1[t]));
    }
    *reinterpret_cast<uint4*>(a_stage + off) = *reinterpret_cast<const uint4*>(p0);
    *reinterpret_cast<uint4*>(a_stage + kPlaneA + off) = *reinterpret_cast<const uint4*>(p1);
    *reinterpret_cast<uint4*>(a_stage + 2 * kPlaneA + off) = *reinterpret_cast<const uint4*>(p2);
  }
}

template <class P>
__global__ void __launch_bounds__(kThreadsTc, 1)
k_contract_tc(float* __restrict__ delta, const float4* __restrict__ coefdf,
              const float2* __restrict__ phaseT, const uint8_t* __restrict__ bimg,
              const int* __restrict__ cls_of, const float* __restrict__ kpow32,
              const int* __restrict__ j0, const float* __restrict__ lw32, long lw_ts, int N_tr,
              int N_I, int n_h, int N_k, int N_ell, int NT, int n_lt, int n_qt, int n_kb,
              int stages, uint32_t tmem_cols, int* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const SmemLayout L = smem_layout<P>(NT, stages);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + L.bar_off);
  // afull[s] = bars[s], bfull[s] = bars[S + s], empty[s] = bars[2S + s],
  // accfull[b] = bars[3S + b], accempty[b] = bars[3S + 2 + b], done = bars[3S + 4]
  const int S = stages;
  uint64_t* accfull = bars + 3 * S;
  uint64_t* accempty = bars + 3 * S + 2;
  uint64_t* done = bars + 3 * S + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * S + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  int bid = blockIdx.x;
  const int lt = bid % n_lt; bid /= n_lt;
  const int qt = bid % n_qt; bid /= n_qt;
  const int wi = bid;                      // walker * N_tr + tracer
  const int i = wi % N_tr;
  const int w = wi / N_tr;
  const int q0 = qt * kMTile;
  const int l0 = lt * NT;
  const int cls = cls_of[i];
  const int stride = (NT + 31) & ~31;      // TMEM columns per accumulator slot

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&bars[s]), kProducers);   // afull: one arrival per producer thread
      mbar_init(smem_u32(&bars[S + s]), 1);        // bfull: expect_tx arrival of thread 0
      mbar_init(smem_u32(&bars[2 * S + s]), 1);    // empty: MMA commit
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&accfull[b]), 1);          // MMA commit of one K-block
      mbar_init(smem_u32(&accempty[b]), kProducers); // drained by every producer thread
    }
    mbar_init(smem_u32(done), 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(tmem_slot), tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int CPK = P::kKb / 2;               // complex coefficients per K-block
  const int CPC = CPK / 8;                  // complex coefficients per 16-byte chunk
  const uint32_t b_bytes = P::kPlanesB * L.b_plane_bytes;
  const uint8_t* bsrc = bimg + (size_t)(cls * n_lt + lt) * n_kb * b_bytes;

  {
    // ------------------------------------------------------------ producers ----
    // Each thread also owns one accumulator row (k point) and half of the multipole columns:
    // after every K-block it adds the tensor core's short partial sums (one K-block each,
    // leading product and corrections in separate TMEM slots) into FP32 registers with
    // round-to-nearest, so no long running sum is ever accumulated inside the tensor core.
    const int quarter = warp & 3, half = warp >> 2;
    const int row_acc = quarter * 32 + lane;
    const int nchunks = NT / 16;
    const int c_begin = half ? (nchunks + 1) / 2 : 0;
    const int my_chunks = half ? nchunks - (nchunks + 1) / 2 : (nchunks + 1) / 2;  // <= 4
    float acc[64];
#pragma unroll
    for (int t = 0; t < 64; ++t) acc[t] = 0.0f;
    int last_round[4] = {-1, -1, -1, -1};   // thread 0: last round whose B copy was issued
    const float4* cf = coefdf + (size_t)wi * N_I * n_h;

    // Formation: thread tid forms row prow (fixed) and the 16-byte chunks phalf, phalf+2, ...
    const int prow = tid & (kMTile - 1);
    const int phalf = tid >> 7;
    const int pq = q0 + prow;
    const bool plive = pq < N_k;
    int jq = 0, rmax = 0;
    float wr[4] = {0.f, 0.f, 0.f, 0.f};
    if (plive) {
      jq = j0[pq];
      const float4 wq = *reinterpret_cast<const float4*>(lw32 + (size_t)i * lw_ts + (size_t)pq * 4);
      wr[0] = wq.x; wr[1] = wq.y; wr[2] = wq.z; wr[3] = wq.w;
      rmax = min(4, N_I - jq);
    }
    // The knots this tile touches are staged in shared memory once per K-block (every row of a
    // warp reads the same few knots); the loads of K-block kb+1 (knots and phases) are issued
    // into registers right after K-block kb is handed to the tensor core.  A tile spanning too many knots reads them from global memory.
    const int a_lo = j0[q0];
    const int a_hi = min(N_I - 1, j0[min(q0 + kMTile, N_k) - 1] + 3);
    const int span = a_hi - a_lo + 1;
    const bool staged = span * CPK * 16 <= (int)kCoefSmem;
    float4* Cs = reinterpret_cast<float4*>(base + L.coef_off);
    float4 cpre[4];
    float2 epre[4 * 4];
    auto prefetch = [&](int kbn) {
      if (staged) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = tid + kProducers * u;
          cpre[u] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (e < span * CPK) {
            const int kn = e / CPK, off = e - kn * CPK;
            const int n = kbn * CPK + off;
            if (n < n_h) cpre[u] = cf[(size_t)(a_lo + kn) * n_h + n];
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int cc = 0; cc < CPC; ++cc) {
          const int n = kbn * CPK + (phalf + 2 * c) * CPC + cc;
          epre[c * CPC + cc] = (plive && n < n_h) ? phaseT[(size_t)n * N_k + pq] : make_float2(0.f, 0.f);
        }
    };
    prefetch(0);

    auto drain = [&](int kd) -> bool {
      const int b = kd & 1;
      if (!mbar_wait(smem_u32(&accfull[b]), (kd >> 1) & 1, abort_flag)) return false;
      tc_fence_after();
      const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (c < my_chunks) {
          float m[16], r[16];
          tmem_ld16(lane_base + (2 * b) * stride + (c_begin + c) * 16, m);
          tmem_ld16(lane_base + (2 * b + 1) * stride + (c_begin + c) * 16, r);
#pragma unroll
          for (int t = 0; t < 16; ++t) acc[c * 16 + t] += m[t] + r[t];
        }
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&accempty[b]));
      return true;
    };

    // tcgen05.mma for K-block kb, issued by thread 0 once all producers have handed it over
    auto issue = [&](int kb) -> bool {
      const int s = kb % S;
      const int r = kb / S;
      const int b = kb & 1;
      if (kb >= 2 && !mbar_wait(smem_u32(&accempty[b]), ((kb >> 1) - 1) & 1, abort_flag)) return false;
      if (!mbar_wait(smem_u32(&bars[s]), r & 1, abort_flag)) return false;
      if (!mbar_wait(smem_u32(&bars[S + s]), r & 1, abort_flag)) return false;
      tc_fence_after();
      const uint32_t idesc = P::idesc(kMTile, NT);
      const uint32_t a0 = smem_u32(base + s * L.stage_bytes);
      const uint32_t b0 = a0 + L.a_bytes;
      const uint32_t d_main = tmem + (uint32_t)((2 * b) * stride);
      const uint32_t d_corr = tmem + (uint32_t)((2 * b + 1) * stride);
#pragma unroll
      for (int j = 0; j < P::kKb / P::kKmma; ++j) {
#pragma unroll
        for (int t = 0; t < P::kProducts; ++t) {
          const uint64_t ad = make_desc(a0 + P::pa(t) * kPlaneA + j * 256);
          const uint64_t bd = make_desc(b0 + P::pb(t) * L.b_plane_bytes + j * 256);
          // leading product into the main slot, corrections into the correction slot; the
          // first MMA of a K-block into a slot overwrites it
          const bool lead = (t == 0);
          const bool first = (j == 0) && (lead || t == 1);
          mma<P>(lead ? d_main : d_corr, ad, bd, idesc, first ? 0u : 1u);
        }
      }
      mma_commit(smem_u32(&bars[2 * S + s]));
      mma_commit(smem_u32(&accfull[b]));
      return true;
    };

    // After a failed (timed-out) wait a thread skips all remaining work but still executes every
    // named barrier of the loop, so no thread is left waiting on a barrier that cannot complete.
    bool ok = true;
    for (int kb = 0; kb < n_kb; ++kb) {
      const int s = kb % S;
      const int r = kb / S;
      uint8_t* st = base + s * L.stage_bytes;
      if (staged) {
        // every producer has finished reading the previous K-block's knots
        asm volatile("bar.sync 1, %0;" ::"r"(kProducers) : "memory");
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = tid + kProducers * u;
          if (ok && e < span * CPK) Cs[e] = cpre[u];
        }
        asm volatile("bar.sync 1, %0;" ::"r"(kProducers) : "memory");
      }
      if (!ok) continue;
      if (r > 0 && !mbar_wait(smem_u32(&bars[2 * S + s]), (r - 1) & 1, abort_flag)) { ok = false; continue; }
      if (tid == 0) {
        mbar_arrive_tx(smem_u32(&bars[S + s]), b_bytes);
        bulk_g2s(smem_u32(st + L.a_bytes), bsrc + (size_t)kb * b_bytes, b_bytes,
                 smem_u32(&bars[S + s]));
        last_round[s] = r;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int chunk = phalf + 2 * c;     // 0..7: 16-byte column of the 128-byte row
        float v[2 * 4];
#pragma unroll
        for (int t = 0; t < 2 * CPC; ++t) v[t] = 0.0f;
        if (plive) {
#pragma unroll
          for (int cc = 0; cc < CPC; ++cc) {
            const int nl = chunk * CPC + cc;
            const int n = kb * CPK + nl;
            if (n < n_h) {
              // sum_r lw_r (c_hi + c_lo): low parts first, then the high parts
              float4 cv[4];
#pragma unroll
              for (int rr = 0; rr < 4; ++rr) {
                if (rr < rmax)
                  cv[rr] = staged ? Cs[(jq - a_lo + rr) * CPK + nl] : cf[(size_t)(jq + rr) * n_h + n];
                else
                  cv[rr] = make_float4(0.f, 0.f, 0.f, 0.f);
              }
              float xr = 0.0f, xi = 0.0f;
#pragma unroll
              for (int rr = 0; rr < 4; ++rr) {
                xr = fmaf(wr[rr], cv[rr].z, xr);
                xi = fmaf(wr[rr], cv[rr].w, xi);
              }
#pragma unroll
              for (int rr = 0; rr < 4; ++rr) {
                xr = fmaf(wr[rr], cv[rr].x, xr);
                xi = fmaf(wr[rr], cv[rr].y, xi);
              }
              const float2 e = epre[c * CPC + cc];
              v[2 * cc] = fmaf(xr, e.x, -xi * e.y);
              v[2 * cc + 1] = fmaf(xr, e.y, xi * e.x);
            }
          }
        }
        store_split<P>(st, core_offset(prow, chunk * 16), v);
      }
      fence_proxy_async();
      mbar_arrive(smem_u32(&bars[s]));
      if (tid == 0 && !issue(kb)) ok = false;
      // next K-block's knots and phases: in flight during the drain and the barrier waits
      if (kb + 1 < n_kb) prefetch(kb + 1);
      if (kb >= 1 && !drain(kb - 1)) ok = false;
    }
    if (ok) ok = drain(n_kb - 1);
    // ----------------------------------------------------------- epilogue ----
    const int q = q0 + row_acc;
    if (ok && q < N_k) {
      const float kp = kpow32[(size_t)i * N_k + q];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (c < my_chunks) {
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const int l = l0 + (c_begin + c) * 16 + t;
            if (l < N_ell) delta[(((size_t)w * N_ell + l) * N_tr + i) * N_k + q] = kp * acc[c * 16 + t];
          }
        }
      }
    }
    if (tid == 0) {
      // every issued MMA has completed before TMEM is released
      mma_commit(smem_u32(done));
      mbar_wait_drain(smem_u32(done), 0);
      if (*abort_flag) {
        // bulk copies still in flight after an abort land before the CTA exits
        for (int s = 0; s < S; ++s)
          if (last_round[s] >= 0) mbar_wait_drain(smem_u32(&bars[S + s]), last_round[s] & 1);
        atomicExch(status, 1);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, tmem_cols);
  }
}

// ------------------------------------------------------------- operand prep ----

// B image: [cls][lt][kb][plane][NT rows x 128 B] of w_n pi(l) M_{l,n} (K-major in n), split
// from FP64 into kPlanesB planes (b = b0 + b1 + ..., each plane the rounded remainder).
template <class P>
__global__ void k_build_bimg(uint8_t* __restrict__ img, const cplx* __restrict__ gtab, int n_cls,
                             int N_ell, int n_h, int NT, int n_lt, int n_kb) {
  const long per_kb = (long)NT * P::kKb;                   // elements of one plane
  const long total = (long)n_cls * n_lt * n_kb * per_kb;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    long t = e;
    const int k = (int)(t % P::kKb); t /= P::kKb;
    const int lr = (int)(t % NT); t /= NT;
    const int kb = (int)(t % n_kb); t /= n_kb;
    const int lt = (int)(t % n_lt); t /= n_lt;
    const int c = (int)t;
    const int K = kb * P::kKb + k;
    const int n = K >> 1;
    const int l = lt * NT + lr;
    double val = 0.0;
    if (l < N_ell && n < n_h) {
      const cplx g = gtab[((size_t)c * N_ell + l) * n_h + n];
      val = (K & 1) ? -g.y : g.x;
    }
    uint8_t* dst = img + ((((size_t)c * n_lt + lt) * n_kb + kb) * P::kPlanesB) * NT * kRowBytes;
    const uint32_t off = core_offset(lr, k * P::kElemBytes);
    double rem = val;
#pragma unroll
    for (int p = 0; p < P::kPlanesB; ++p) {
      if constexpr (!P::kBf16) {
        const float b = tf32_rna((float)rem);
        *reinterpret_cast<float*>(dst + p * NT * kRowBytes + off) = b;
        rem -= (double)b;
      } else {
        const __nv_bfloat16 b = __double2bfloat16(rem);
        *reinterpret_cast<__nv_bfloat16*>(dst + p * NT * kRowBytes + off) = b;
        rem -= (double)__bfloat162float(b);
      }
    }
  }
}

// phaseT[n][q] = (float2) phase[q][n], and the double-float low parts phase - phaseT
__global__ void k_phase_t(float2* __restrict__ out, float2* __restrict__ out_lo,
                          const cplx* __restrict__ phase, int N_k, int n_h) {
  __shared__ float2 tile[32][33], tlo[32][33];
  const int n0 = blockIdx.x * 32, q0 = blockIdx.y * 32;
  for (int t = threadIdx.y; t < 32; t += blockDim.y) {
    const int q = q0 + t, n = n0 + threadIdx.x;
    if (q < N_k && n < n_h) {
      const cplx v = phase[(size_t)q * n_h + n];
      const float2 h = make_float2((float)v.x, (float)v.y);
      tile[t][threadIdx.x] = h;
      tlo[t][threadIdx.x] = make_float2((float)(v.x - (double)h.x), (float)(v.y - (double)h.y));
    }
  }
  __syncthreads();
  for (int t = threadIdx.y; t < 32; t += blockDim.y) {
    const int n = n0 + t, q = q0 + threadIdx.x;
    if (q < N_k && n < n_h) {
      out[(size_t)n * N_k + q] = tile[threadIdx.x][t];
      out_lo[(size_t)n * N_k + q] = tlo[threadIdx.x][t];
    }
  }
}

// FP64 -> double-float (hi = rounded value, lo = the remainder rounded)
__global__ void k_to_f32(float* __restrict__ out, float* __restrict__ out_lo,
                         const double* __restrict__ in, long n) {
  long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    const float h = (float)in[t];
    out[t] = h;
    out_lo[t] = (float)(in[t] - (double)h);
  }
}

template <class P>
int prepare_tables(swcl_ctx* c, int precision, int& NT, int& n_lt, int& n_kb) {
  TcTables& T = c->tc[precision];
  const int n_h = c->n_h;
  // multipole tile: the whole list when it fits, else the widest tile whose stages fit 227 KB
  // four TMEM accumulator slots (two K-blocks in flight, leading product and corrections each)
  // of up to 128 columns fill the 512 columns of TMEM
  const int nt_max = 128;
  NT = std::min(nt_max, ((c->N_ell + 15) / 16) * 16);
  n_lt = (c->N_ell + NT - 1) / NT;
  n_kb = (2 * n_h + P::kKb - 1) / P::kKb;
  if (T.ready) return SWCL_OK;
  const size_t bimg = (size_t)c->n_cls * n_lt * n_kb * P::kPlanesB * NT * kRowBytes;
  int st = ensure(c, T.bfwd, bimg);
  if (st) return st;
  st = ensure(c, T.phase32, sizeof(float2) * (size_t)c->N_k * n_h);
  if (st) return st;
  st = ensure(c, T.phase_lo, sizeof(float2) * (size_t)c->N_k * n_h);
  if (st) return st;
  const Stencil sv = stencil(c);
  const long n_lw = 4L * c->N_k * (sv.w_ts ? c->N_tr : 1);
  st = ensure(c, c->tc_lw32, sizeof(float) * n_lw);
  if (st) return st;
  st = ensure(c, c->tc_lw_lo, sizeof(float) * n_lw);
  if (st) return st;
  st = ensure(c, c->tc_kpow32, sizeof(float) * (size_t)c->N_tr * c->N_k);
  if (st) return st;
  st = ensure(c, c->tc_kpow_lo, sizeof(float) * (size_t)c->N_tr * c->N_k);
  if (st) return st;
  const long per = (long)c->n_cls * n_lt * n_kb * NT * P::kKb;
  k_build_bimg<P><<<(unsigned)std::min<long>((per + 255) / 256, 152L * 64), 256, 0, c->stream>>>(
      (uint8_t*)T.bfwd.p, (const cplx*)c->d_gtab.p, c->n_cls, c->N_ell, n_h, NT, n_lt, n_kb);
  dim3 gt((n_h + 31) / 32, (c->N_k + 31) / 32), bt(32, 8);
  k_phase_t<<<gt, bt, 0, c->stream>>>((float2*)T.phase32.p, (float2*)T.phase_lo.p,
                                      (const cplx*)c->d_phase.p, c->N_k, n_h);
  k_to_f32<<<(unsigned)((n_lw + 255) / 256), 256, 0, c->stream>>>((float*)c->tc_lw32.p,
                                                                 (float*)c->tc_lw_lo.p, sv.w, n_lw);
  long nk = (long)c->N_tr * c->N_k;
  k_to_f32<<<(unsigned)((nk + 255) / 256), 256, 0, c->stream>>>((float*)c->tc_kpow32.p,
                                                               (float*)c->tc_kpow_lo.p,
                                                               (const double*)c->d_kpow.p, nk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "tensor-core operand tables");
  T.ready = true;
  return SWCL_OK;
}

template <class P>
int run_forward(swcl_ctx* c, int precision) {
  const Stencil sv = stencil(c);
  int NT, n_lt, n_kb;
  int st = prepare_tables<P>(c, precision, NT, n_lt, n_kb);
  if (st) return st;
  int stages = 4;
  SmemLayout L = smem_layout<P>(NT, stages);
  while (stages > 2 && L.total > 227 * 1024) L = smem_layout<P>(NT, --stages);
  if (L.total > 227 * 1024) return fail(c, SWCL_ERR_UNSUPPORTED, "tensor-core tile does not fit shared memory");
  // several accumulators (rotating over K-blocks) when TMEM has room: the tensor core's FP32
  // accumulation error grows with the number of MMAs added into one accumulator
  const int acc_stride = (NT + 31) & ~31;
  uint32_t tmem_cols = 32;
  while (tmem_cols < (uint32_t)(4 * acc_stride)) tmem_cols <<= 1;
  const int n_qt = (c->N_k + kMTile - 1) / kMTile;
  const long grid = (long)c->n_walk * c->N_tr * n_qt * n_lt;
  cudaError_t e = cudaFuncSetAttribute(k_contract_tc<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)L.total);
  if (e != cudaSuccess) return cuda_fail(c, e, "contract tc attribute");
  prof_begin(c);
  ++c->last_launches;
  k_contract_tc<P><<<(unsigned)grid, kThreadsTc, L.total, c->stream>>>(
      (float*)c->ws_delta.p, (const float4*)c->ws_coef.p, (const float2*)c->tc[precision].phase32.p,
      (const uint8_t*)c->tc[precision].bfwd.p, (const int*)c->d_cls_of.p,
      (const float*)c->tc_kpow32.p, sv.j0, (const float*)c->tc_lw32.p, sv.w_ts, c->N_tr, sv.NI,
      c->n_h, c->N_k, c->N_ell, NT, n_lt, n_qt, n_kb, stages, tmem_cols,
      (int*)c->ws_status.p);
  e = cudaGetLastError();
  prof_end(c, "contract tc");
  if (e != cudaSuccess) return cuda_fail(c, e, "contract tc launch");
  return SWCL_OK;
}

}  // namespace

int compute_delta_tc(swcl_ctx* c, int precision) {
  if (precision == SWCL_3XTF32) return run_forward<Tf32x3>(c, precision);
  if (precision == SWCL_TF32X6) return run_forward<Tf32x6>(c, precision);
  if (precision == SWCL_SPLIT_BF16) return run_forward<Bf16x9>(c, precision);
  return fail(c, SWCL_ERR_INVALID_ARG, "not a tensor-core precision");
}

}  // namespace swcl
