// a5 on the tensor cores: the transposed contraction of the VJP,
//   Xbar_{q,n}  = kpow_i[q] sum_l Dbar_i(l, q) conj(w_n pi(l) M_{l,n}),
//   cbar_q,n    = Xbar_{q,n} conj(e^{-i eta_n ln k_q}),
//   cbar_{a,n}  = sum_q lambda_{q,a} cbar_q,n          (transpose of the k-interpolation),
// as one real GEMM per (walker, tracer, 128-row k tile, 128-column tile of (n, re/im)) with
// K = multipoles.  Both operands are pre-split images streamed by cp.async.bulk (A: Dbar, B: the
// Gamma table transposed); the tensor core accumulates one K-block at a time into double-buffered
// TMEM slots that the other warps drain into FP32 registers, as in the forward kernel.  The
// epilogue applies k^{t-1-b} and the phase and reduces over the tile's k points into per-knot
// partial sums (staged in shared memory), all in double-float arithmetic: the phase rotates
// quickly with k at large n, so these k-sums cancel strongly, and single FP32 roundings of the
// phase, the weights or the running sum would reach the gradient W_bar through the inverse
// transform (Eq. 3.2).  The partials are written as FP64; a second kernel adds the partials of
// neighbouring tiles deterministically.
#include <algorithm>
#include <vector>

#include "swcl_internal.h"
#include "tc_common.cuh"

namespace swcl {
namespace {

using namespace tc;

constexpr int kWarps = 8;
constexpr int kThr = kWarps * 32 + 32;
constexpr int kCT = 128;   // output columns per CTA (64 complex coefficients)

struct AdjLayout {
  uint32_t a_bytes, b_bytes, stage_bytes, bar_off, total;
};

template <class P>
__host__ __device__ inline AdjLayout adj_layout(int stages) {
  AdjLayout L;
  L.a_bytes = P::kPlanesA * kPlaneA;
  L.b_bytes = P::kPlanesB * kCT * kRowBytes;
  L.stage_bytes = L.a_bytes + L.b_bytes;
  L.bar_off = stages * L.stage_bytes;
  L.total = L.bar_off + 8 * (2 * stages + 5) + 16 + 1024;
  return L;
}

template <class P>
__global__ void __launch_bounds__(kThr, 1)
k_contract_tc_adj(cplx* __restrict__ cpart, const uint8_t* __restrict__ aimg,
                  const uint8_t* __restrict__ bimgT, const int* __restrict__ cls_of,
                  const float* __restrict__ kpow32, const float* __restrict__ kpow_lo,
                  const int* __restrict__ j0, const float* __restrict__ lw32,
                  const float* __restrict__ lw_lo, long lw_ts, const float2* __restrict__ phaseT,
                  const float2* __restrict__ phase_lo, const int* __restrict__ tile_alo, int N_tr,
                  int N_I, int n_h, int N_k, int n_ct,
                  int n_qt, int n_kb, int R, int stages, uint32_t tmem_cols,
                  int* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const AdjLayout L = adj_layout<P>(stages);
  const int S = stages;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + L.bar_off);
  uint64_t* full = bars;              // [S] operands landed (tx)
  uint64_t* empty = bars + S;         // [S] MMA done with the stage
  uint64_t* accfull = bars + 2 * S;   // [2]
  uint64_t* accempty = bars + 2 * S + 2;
  uint64_t* done = bars + 2 * S + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  int bid = blockIdx.x;
  const int ct = bid % n_ct; bid /= n_ct;
  const int qt = bid % n_qt; bid /= n_qt;
  const int wi = bid;
  const int i = wi % N_tr;
  const int q0 = qt * kMTile;
  const int cls = cls_of[i];
  constexpr int stride = kCT;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&accfull[b]), 1);
      mbar_init(smem_u32(&accempty[b]), kWarps * 32);
    }
    mbar_init(smem_u32(done), 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == kWarps) tmem_alloc(smem_u32(tmem_slot), tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint8_t* asrc = aimg + (size_t)(wi * n_qt + qt) * n_kb * L.a_bytes;
  const uint8_t* bsrc = bimgT + (size_t)(cls * n_ct + ct) * n_kb * L.b_bytes;

  if (warp < kWarps) {
    const int quarter = warp & 3, half = warp >> 2;
    const int row_acc = quarter * 32 + lane;
    const int c_begin = half * 4;            // 8 chunks of 16 columns; 4 per half
    float acc[64];
#pragma unroll
    for (int t = 0; t < 64; ++t) acc[t] = 0.0f;
    int last_round[4] = {-1, -1, -1, -1};

    auto drain = [&](int kd) -> bool {
      const int b = kd & 1;
      if (!mbar_wait(smem_u32(&accfull[b]), (kd >> 1) & 1, abort_flag)) return false;
      tc_fence_after();
      const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float m[16], r[16];
        tmem_ld16(lane_base + (2 * b) * stride + (c_begin + c) * 16, m);
        tmem_ld16(lane_base + (2 * b + 1) * stride + (c_begin + c) * 16, r);
#pragma unroll
        for (int t = 0; t < 16; ++t) acc[c * 16 + t] += m[t] + r[t];
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&accempty[b]));
      return true;
    };

    bool ok = true;
    for (int kb = 0; kb < n_kb && ok; ++kb) {
      const int s = kb % S;
      const int r = kb / S;
      uint8_t* st = base + s * L.stage_bytes;
      if (r > 0 && !mbar_wait(smem_u32(&empty[s]), (r - 1) & 1, abort_flag)) { ok = false; break; }
      if (tid == 0) {
        mbar_arrive_tx(smem_u32(&full[s]), L.a_bytes + L.b_bytes);
        bulk_g2s(smem_u32(st), asrc + (size_t)kb * L.a_bytes, L.a_bytes, smem_u32(&full[s]));
        bulk_g2s(smem_u32(st + L.a_bytes), bsrc + (size_t)kb * L.b_bytes, L.b_bytes, smem_u32(&full[s]));
        last_round[s] = r;
      }
      if (kb >= 1 && !drain(kb - 1)) ok = false;
    }
    if (ok) ok = drain(n_kb - 1);
    if (tid == 0 && *abort_flag) {
      for (int s = 0; s < S; ++s)
        if (last_round[s] >= 0) mbar_wait_drain(smem_u32(&full[s]), last_round[s] & 1);
      atomicExch(status, 1);
    }
    // ---------------------------------------------------------------- epilogue ----
    // all MMAs are complete (last drain) and every stage has been consumed: reuse stage memory.
    // V[m][r] = X conj(E) as double-float (re_hi, im_hi, re_lo, im_lo); tlw/tlwl the row's
    // Lagrange weights (hi, lo)
    constexpr int VS = kMTile + 1;                                    // padded row stride
    float4* V = reinterpret_cast<float4*>(base);                       // [64 columns][VS]
    int* tj0 = reinterpret_cast<int*>(base + 64 * VS * sizeof(float4));
    float4* tlw = reinterpret_cast<float4*>(tj0 + kMTile);
    float4* tlwl = tlw + kMTile;
    asm volatile("bar.sync 1, %0;" ::"r"(kWarps * 32) : "memory");
    {
      const int q = q0 + row_acc;
      const bool live = ok && q < N_k;
      const float kp = live ? kpow32[(size_t)i * N_k + q] : 0.0f;
      const float kpl = live ? kpow_lo[(size_t)i * N_k + q] : 0.0f;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
#pragma unroll
        for (int t = 0; t < 16; t += 2) {
          const int m = (c_begin + c) * 8 + t / 2;        // local complex column
          const int n = ct * (kCT / 2) + m;
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (live && n < n_h) {
            // X = k^{t-1-b} acc exactly as double-float, then X conj(E) in double-float
            float xr, xrl, xi, xil;
            two_prod(kp, acc[c * 16 + t], xr, xrl);
            two_prod(kp, acc[c * 16 + t + 1], xi, xil);
            xrl = fmaf(kpl, acc[c * 16 + t], xrl);
            xil = fmaf(kpl, acc[c * 16 + t + 1], xil);
            const float2 e = phaseT[(size_t)n * N_k + q];
            const float2 el = phase_lo[(size_t)n * N_k + q];
            // Re = xr er + xi ei,  Im = xi er - xr ei
            df_dot2(xr, xrl, e.x, el.x, xi, xil, e.y, el.y, 1.0f, v.x, v.z);
            df_dot2(xi, xil, e.x, el.x, xr, xrl, e.y, el.y, -1.0f, v.y, v.w);
          }
          V[m * VS + row_acc] = v;
        }
      }
      if (half == 0) {
        tj0[row_acc] = q < N_k ? j0[q] : 0x7fffffff;
        const size_t lo = (size_t)i * lw_ts + (size_t)q * 4;
        tlw[row_acc] = q < N_k ? *reinterpret_cast<const float4*>(lw32 + lo) : make_float4(0.f, 0.f, 0.f, 0.f);
        tlwl[row_acc] = q < N_k ? *reinterpret_cast<const float4*>(lw_lo + lo) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    asm volatile("bar.sync 1, %0;" ::"r"(kWarps * 32) : "memory");
    if (ok) {
      const int a_lo = tile_alo[qt];
      const int q_last = min(q0 + kMTile, N_k) - 1;
      const int a_hi = min(N_I - 1, tj0[q_last - q0] + 3);
      const int nk = a_hi - a_lo + 1;
      cplx* out = cpart + (size_t)(wi * n_qt + qt) * R * n_h;
      // four consecutive knots per item: the rows whose stencil holds any of them are walked
      // once, each row's V and weights are read once, and the four knots accumulate in
      // independent double-float sums (a warp's 32 items share the knots, so the branches on the
      // stencil offset are warp-uniform)
      const int ngrp = (nk + 3) / 4;
      for (int item = tid; item < ngrp * 64; item += kWarps * 32) {
        const int gq = item / 64, m = item - gq * 64;
        const int a0 = a_lo + 4 * gq;
        const int n = ct * (kCT / 2) + m;
        if (n >= n_h) continue;
        float sr[4], srl[4], si[4], sil[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) sr[u] = srl[u] = si[u] = sil[u] = 0.f;
        // first row whose stencil can hold knot a0 (j0 >= a0 - 3; j0 is nondecreasing in q)
        int lo = 0, hi = kMTile;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (tj0[mid] < a0 - 3) lo = mid + 1; else hi = mid;
        }
        for (int r = lo; r < kMTile; ++r) {
          const int jr = tj0[r];
          if (jr > a0 + 3) break;
          const float4 lw = tlw[r], lwl = tlwl[r];
          const float4 v = V[m * VS + r];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int d = a0 + u - jr;
            if (d >= 0 && d <= 3) {
              const float l = d == 0 ? lw.x : d == 1 ? lw.y : d == 2 ? lw.z : lw.w;
              const float ll = d == 0 ? lwl.x : d == 1 ? lwl.y : d == 2 ? lwl.z : lwl.w;
              df_fma(l, ll, v.x, v.z, sr[u], srl[u]);
              df_fma(l, ll, v.y, v.w, si[u], sil[u]);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (a0 + u <= a_hi)
            out[(size_t)(4 * gq + u) * n_h + n] =
                cplx{(double)sr[u] + (double)srl[u], (double)si[u] + (double)sil[u]};
      }
    }
  } else if (lane == 0) {
    // ---------------------------------------------------------------- MMA ----
    const uint32_t idesc = P::idesc(kMTile, kCT);
    for (int kb = 0; kb < n_kb; ++kb) {
      const int s = kb % S;
      const int r = kb / S;
      const int b = kb & 1;
      if (kb >= 2 && !mbar_wait(smem_u32(&accempty[b]), ((kb >> 1) - 1) & 1, abort_flag)) break;
      if (!mbar_wait(smem_u32(&full[s]), r & 1, abort_flag)) break;
      tc_fence_after();
      const uint32_t a0 = smem_u32(base + s * L.stage_bytes);
      const uint32_t b0 = a0 + L.a_bytes;
      const uint32_t d_main = tmem + (uint32_t)((2 * b) * stride);
      const uint32_t d_corr = tmem + (uint32_t)((2 * b + 1) * stride);
#pragma unroll
      for (int j = 0; j < P::kKb / P::kKmma; ++j) {
#pragma unroll
        for (int t = 0; t < P::kProducts; ++t) {
          const uint64_t ad = make_desc(a0 + P::pa(t) * kPlaneA + j * 256);
          const uint64_t bd = make_desc(b0 + P::pb(t) * kCT * kRowBytes + j * 256);
          const bool lead = (t == 0);
          const bool first = (j == 0) && (lead || t == 1);
          mma<P>(lead ? d_main : d_corr, ad, bd, idesc, first ? 0u : 1u);
        }
      }
      mma_commit(smem_u32(&empty[s]));
      mma_commit(smem_u32(&accfull[b]));
    }
    mma_commit(smem_u32(done));
    mbar_wait_drain(smem_u32(done), 0);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kWarps) {
    tc_fence_after();
    tmem_dealloc(tmem, tmem_cols);
  }
}

// A image of the VJP GEMM: [wi][qt][kb][planeA][128 rows x 128 B], element (row, k) =
// Dbar[w][l = kb*kKb + k][i][q0 + row], split exactly into planes (FP32 values).
template <class P>
__global__ void k_dbar_img(uint8_t* __restrict__ img, const float* __restrict__ dbar, int n_wi,
                           int N_tr, int N_ell, int N_k, int n_qt, int n_kb) {
  constexpr int EPC = 16 / P::kElemBytes;          // elements per 16-byte chunk
  constexpr int CPR = P::kKb / EPC;                // chunks per row (8)
  const long total = (long)n_wi * n_qt * n_kb * kMTile * CPR;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    long t = e;
    const int row = (int)(t % kMTile); t /= kMTile;     // rows fastest: coalesced reads over q
    const int ch = (int)(t % CPR); t /= CPR;
    const int kb = (int)(t % n_kb); t /= n_kb;
    const int qt = (int)(t % n_qt); t /= n_qt;
    const int wi = (int)t;
    const int w = wi / N_tr, i = wi % N_tr;
    const int q = qt * kMTile + row;
    float v[8];
#pragma unroll
    for (int u = 0; u < EPC; ++u) {
      const int l = kb * P::kKb + ch * EPC + u;
      v[u] = (q < N_k && l < N_ell) ? dbar[(((size_t)w * N_ell + l) * N_tr + i) * N_k + q] : 0.0f;
    }
    uint8_t* dst = img + (((size_t)wi * n_qt + qt) * n_kb + kb) * P::kPlanesA * kPlaneA;
    const uint32_t off = core_offset(row, ch * 16);
    if constexpr (!P::kBf16) {
      float4 p0, p1, p2;
      float* a0 = &p0.x; float* a1 = &p1.x; float* a2 = &p2.x;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a0[u] = tf32_rna(v[u]);
        const float r1 = v[u] - a0[u];
        a1[u] = tf32_rna(r1);
        a2[u] = r1 - a1[u];
      }
      *reinterpret_cast<float4*>(dst + off) = p0;
      *reinterpret_cast<float4*>(dst + kPlaneA + off) = p1;
      if constexpr (P::kPlanesA == 3) *reinterpret_cast<float4*>(dst + 2 * kPlaneA + off) = p2;
    } else {
      __align__(16) __nv_bfloat16 p0[8], p1[8], p2[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        p0[u] = __float2bfloat16_rn(v[u]);
        const float r1 = v[u] - __bfloat162float(p0[u]);
        p1[u] = __float2bfloat16_rn(r1);
        p2[u] = __float2bfloat16_rn(r1 - __bfloat162float(p1[u]));
      }
      *reinterpret_cast<uint4*>(dst + off) = *reinterpret_cast<const uint4*>(p0);
      *reinterpret_cast<uint4*>(dst + kPlaneA + off) = *reinterpret_cast<const uint4*>(p1);
      *reinterpret_cast<uint4*>(dst + 2 * kPlaneA + off) = *reinterpret_cast<const uint4*>(p2);
    }
  }
}

// B image of the VJP GEMM: [cls][ct][kb][planeB][128 rows x 128 B], row = output column
// col = 2n + reim, element k = multipole: Re G[l][n] (reim 0) or -Im G[l][n] (reim 1).
template <class P>
__global__ void k_build_bimgT(uint8_t* __restrict__ img, const cplx* __restrict__ gtab, int n_cls,
                              int N_ell, int n_h, int n_ct, int n_kb) {
  const long total = (long)n_cls * n_ct * n_kb * kCT * P::kKb;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    long t = e;
    const int k = (int)(t % P::kKb); t /= P::kKb;
    const int row = (int)(t % kCT); t /= kCT;
    const int kb = (int)(t % n_kb); t /= n_kb;
    const int ct = (int)(t % n_ct); t /= n_ct;
    const int c = (int)t;
    const int col = ct * kCT + row;
    const int n = col >> 1;
    const int l = kb * P::kKb + k;
    double val = 0.0;
    if (l < N_ell && n < n_h) {
      const cplx g = gtab[((size_t)c * N_ell + l) * n_h + n];
      val = (col & 1) ? -g.y : g.x;
    }
    uint8_t* dst = img + (((size_t)c * n_ct + ct) * n_kb + kb) * P::kPlanesB * kCT * kRowBytes;
    const uint32_t off = core_offset(row, k * P::kElemBytes);
    double rem = val;
#pragma unroll
    for (int p = 0; p < P::kPlanesB; ++p) {
      if constexpr (!P::kBf16) {
        const float b = tf32_rna((float)rem);
        *reinterpret_cast<float*>(dst + p * kCT * kRowBytes + off) = b;
        rem -= (double)b;
      } else {
        const __nv_bfloat16 b = __double2bfloat16(rem);
        *reinterpret_cast<__nv_bfloat16*>(dst + p * kCT * kRowBytes + off) = b;
        rem -= (double)__bfloat162float(b);
      }
    }
  }
}

// cbar[wi][a][n] = sum over the k tiles whose knot range holds a of the tile partials.
__global__ void k_knot_reduce(cplx* __restrict__ cbar, const cplx* __restrict__ cpart,
                              const int* __restrict__ tile_alo, const int* __restrict__ knot_qt,
                              int n_wi, int N_I, int n_h, int n_qt, int R) {
  const long total = (long)n_wi * N_I * n_h;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int n = (int)(e % n_h);
    const int a = (int)((e / n_h) % N_I);
    const int wi = (int)(e / ((long)n_h * N_I));
    double sr = 0.0, si = 0.0;
    for (int qt = knot_qt[2 * a]; qt <= knot_qt[2 * a + 1]; ++qt) {
      const int ka = a - tile_alo[qt];
      if (ka < 0 || ka >= R) continue;
      const cplx v = cpart[((size_t)(wi * n_qt + qt) * R + ka) * n_h + n];
      sr += (double)v.x;
      si += (double)v.y;
    }
    cbar[e] = {sr, si};
  }
}

template <class P>
int run_adjoint(swcl_ctx* c, int precision) {
  TcTables& T = c->tc[precision];
  const Stencil sv = stencil(c);
  const int N_tr = c->N_tr, n_h = c->n_h, N_k = c->N_k, N_ell = c->N_ell, N_I = sv.NI;
  const int n_qt = (N_k + kMTile - 1) / kMTile;
  const int n_ct = (2 * n_h + kCT - 1) / kCT;
  const int n_kb = (N_ell + P::kKb - 1) / P::kKb;
  const int n_wi = c->n_walk * N_tr;
  int st;
  if (!T.adj_ready) {
    // knot ranges of the k tiles (j0 is nondecreasing in q)
    std::vector<int> j0(N_k);
    cudaError_t e = cudaMemcpy(j0.data(), sv.j0, sizeof(int) * N_k, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "read interpolation stencils");
    std::vector<int> alo(n_qt), kq(2 * N_I);
    int R = 1;
    for (int a = 0; a < N_I; ++a) { kq[2 * a] = n_qt; kq[2 * a + 1] = -1; }
    for (int qt = 0; qt < n_qt; ++qt) {
      const int qa = qt * kMTile, qb = std::min(N_k, qa + kMTile) - 1;
      alo[qt] = j0[qa];
      const int ahi = std::min(N_I - 1, j0[qb] + 3);
      R = std::max(R, ahi - alo[qt] + 1);
      for (int a = alo[qt]; a <= ahi; ++a) {
        kq[2 * a] = std::min(kq[2 * a], qt);
        kq[2 * a + 1] = std::max(kq[2 * a + 1], qt);
      }
    }
    T.R = R;
    if ((st = copy_in(c, T.tile_alo, alo.data(), sizeof(int) * n_qt))) return st;
    if ((st = copy_in(c, T.knot_qt, kq.data(), sizeof(int) * 2 * N_I))) return st;
    const size_t bt = (size_t)c->n_cls * n_ct * n_kb * P::kPlanesB * kCT * kRowBytes;
    if ((st = ensure(c, T.bvjp, bt))) return st;
    const long per = (long)c->n_cls * n_ct * n_kb * kCT * P::kKb;
    k_build_bimgT<P><<<(unsigned)std::min<long>((per + 255) / 256, 152L * 64), 256, 0, c->stream>>>(
        (uint8_t*)T.bvjp.p, (const cplx*)c->d_gtab.p, c->n_cls, N_ell, n_h, n_ct, n_kb);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "VJP operand table");
    T.adj_ready = true;
  }
  const size_t abytes = (size_t)n_wi * n_qt * n_kb * P::kPlanesA * kPlaneA;
  if ((st = ensure(c, c->ws_aimg, abytes))) return st;
  if ((st = ensure(c, c->ws_cpart, sizeof(cplx) * (size_t)n_wi * n_qt * T.R * n_h))) return st;
  {
    constexpr int EPC = 16 / P::kElemBytes;
    const long tot = (long)n_wi * n_qt * n_kb * kMTile * (P::kKb / EPC);
    prof_begin(c);
    ++c->last_launches;
    k_dbar_img<P><<<(unsigned)std::min<long>((tot + 255) / 256, 152L * 64), 256, 0, c->stream>>>(
        (uint8_t*)c->ws_aimg.p, (const float*)c->ws_dbar.p, n_wi, N_tr, N_ell, N_k, n_qt, n_kb);
    cudaError_t e = cudaGetLastError();
    prof_end(c, "dbar split");
    if (e != cudaSuccess) return cuda_fail(c, e, "dbar split");
  }
  int stages = 4;
  AdjLayout L = adj_layout<P>(stages);
  while (stages > 2 && L.total > 227 * 1024) L = adj_layout<P>(--stages);
  if (L.total > 227 * 1024) return fail(c, SWCL_ERR_UNSUPPORTED, "VJP tile does not fit shared memory");
  if (L.total < (uint32_t)(64 * (kMTile + 1) * sizeof(float4) + kMTile * (sizeof(int) + 2 * sizeof(float4)) + 1024))
    return fail(c, SWCL_ERR_UNSUPPORTED, "VJP epilogue staging does not fit");
  cudaError_t e = cudaFuncSetAttribute(k_contract_tc_adj<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)L.total);
  if (e != cudaSuccess) return cuda_fail(c, e, "contract adj attribute");
  const long grid = (long)n_wi * n_qt * n_ct;
  prof_begin(c);
  ++c->last_launches;
  k_contract_tc_adj<P><<<(unsigned)grid, kThr, L.total, c->stream>>>(
      (cplx*)c->ws_cpart.p, (const uint8_t*)c->ws_aimg.p, (const uint8_t*)T.bvjp.p,
      (const int*)c->d_cls_of.p, (const float*)c->tc_kpow32.p, (const float*)c->tc_kpow_lo.p, sv.j0,
      (const float*)c->tc_lw32.p, (const float*)c->tc_lw_lo.p, sv.w_ts, (const float2*)T.phase32.p,
      (const float2*)T.phase_lo.p, (const int*)T.tile_alo.p, N_tr, N_I,
      n_h, N_k, n_ct, n_qt, n_kb, T.R, stages, 4 * kCT, (int*)c->ws_status.p);
  e = cudaGetLastError();
  prof_end(c, "contract adj tc");
  if (e != cudaSuccess) return cuda_fail(c, e, "contract adj tc launch");
  const long tot = (long)n_wi * N_I * n_h;
  prof_begin(c);
  ++c->last_launches;
  k_knot_reduce<<<(unsigned)std::min<long>((tot + 255) / 256, 152L * 64), 256, 0, c->stream>>>(
      (cplx*)c->ws_cbar.p, (const cplx*)c->ws_cpart.p, (const int*)T.tile_alo.p,
      (const int*)T.knot_qt.p, n_wi, N_I, n_h, n_qt, T.R);
  e = cudaGetLastError();
  prof_end(c, "knot reduce");
  if (e != cudaSuccess) return cuda_fail(c, e, "knot reduce");
  return SWCL_OK;
}

}  // namespace

int contract_adj_tc(swcl_ctx* c, int precision) {
  if (!c->tc[precision].ready) return fail(c, SWCL_ERR_STATE, "forward tables missing");
  if (precision == SWCL_3XTF32) return run_adjoint<Tf32x3>(c, precision);
  if (precision == SWCL_TF32X6) return run_adjoint<Tf32x6>(c, precision);
  if (precision == SWCL_SPLIT_BF16) return run_adjoint<Bf16x9>(c, precision);
  return fail(c, SWCL_ERR_INVALID_ARG, "not a tensor-core precision");
}

}  // namespace swcl
