// tc32w.cuh -- the FP32-form contraction T = A * B^T on the bf16 tensor
// cores, 128 x 128 output tiles (arithmetic in tc32.cuh): three bf16 terms
// per element, the six term pairs of order t + u <= 2, FP32 accumulation in
// tensor memory over K chunks of 512 and round-to-nearest FP32 sums across
// chunks in registers.
//
// A 64-column tile streams 18 KB of operands per 16-deep K step for 0.79 M
// products, which leaves the product bound by the L2-to-SM traffic; a
// 128-column tile brings 24 KB for 1.57 M products.  To fit two accumulator
// buffers of a 128-column tile into the 512 TMEM columns, the orders share
// accumulators: order 0 (A_0 B_0) has its own 128 columns, orders 1 and 2
// (five pairs, each at most 2^-8 of order 0) sum into a second 128; a buffer
// is 256 columns, buffer b at 256 b, and the MMAs of chunk c + 1 run while
// the epilogue drains chunk c.  Per K step: one MMA of N = 128 into the
// order-0 columns and five into the others.
//
// Warp 0 loads (TMA; A and B in 128-row boxes), warp 1 issues the MMAs, warps 2-9 drain
// (two per TMEM lane quarter, 64 columns each).  Problems, segments and
// tensor maps are the shared records (ozaki_types.cuh); tiles are numbered
// with 128-column tiles (add_tiles with bn = 128).  Every wait is bounded; a
// wait that runs out sets abort, the CTA waits (bounded) for its copies in
// flight, frees TMEM and reports through err.
#pragma once
#include <cuda_bf16.h>

#include "ozaki_types.cuh"
#include "tc_ptx.cuh"
#include "tc32.cuh"

namespace iscsi {

constexpr int T3W_BN = 128;
constexpr int T3W_STAGES = 8;
constexpr int T3W_B_SLICE_BYTES = T3W_BN * T3_BK * 2;  // 4096
constexpr int T3W_STAGE_BYTES = T3_S * (T3_A_SLICE_BYTES + T3W_B_SLICE_BYTES);
constexpr int T3W_SMEM_BYTES = T3W_STAGES * T3W_STAGE_BYTES + 1024;
constexpr int T3W_BUF_COLS = 2 * T3W_BN;  // order 0, then orders 1-2
constexpr int T3W_TMEM_COLS = 512;        // two buffers
constexpr int T3W_EPI_WARPS = 8;
constexpr int T3W_EPI_COLS = T3W_BN / (T3W_EPI_WARPS / 4);  // 64
constexpr int T3W_THREADS = 64 + 32 * T3W_EPI_WARPS;

__global__ void __launch_bounds__(T3W_THREADS, 1)
    k_tc32w_gemm(const OzProblem* __restrict__ probs, int nprobs, const OzSeg* __restrict__ segs,
                 const OzMaps* __restrict__ maps, float* tbase, float* const* __restrict__ tbases,
                 int* __restrict__ err) {
  extern __shared__ unsigned char t3w_smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)t3w_smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t s_stage0 = tc::smem_u32(smem);
  __shared__ uint64_t full_b[T3W_STAGES], empty_b[T3W_STAGES], chunk_b[2], free_b[2], drain_b;
  __shared__ uint32_t tmem_s;
  __shared__ volatile int abort_s;
  __shared__ OzSeg seg_s[OZ_MAX_SEGS];
  __shared__ int segid_s[OZ_MAX_SEGS];
  __shared__ int step0_s[OZ_MAX_SEGS + 1];
  __shared__ int nseg_s;

  int tile = blockIdx.x;
  int lo = 0, hi = nprobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (probs[mid].tile_begin <= tile) lo = mid;
    else hi = mid - 1;
  }
  const OzProblem P = probs[lo];
  float* const Tp = P.t_rel ? (tbases ? tbases[P.tb] : tbase) + P.t : reinterpret_cast<float*>(P.t);
  const int tl = tile - P.tile_begin;
  const int m0 = (tl / P.tiles_n) * T3_BM, n0 = (tl % P.tiles_n) * T3W_BN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int SPC = T3_CHUNK_STEPS;

  if (threadIdx.x == 0) {
    for (int s = 0; s < T3W_STAGES; ++s) {
      tc::mbar_init(tc::smem_u32(&full_b[s]), 1);
      tc::mbar_init(tc::smem_u32(&empty_b[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(tc::smem_u32(&chunk_b[b]), 1);
      tc::mbar_init(tc::smem_u32(&free_b[b]), 32 * T3W_EPI_WARPS);
    }
    tc::mbar_init(tc::smem_u32(&drain_b), 1);
    abort_s = 0;
    int ns = 0, steps = 0;
    for (int g = 0; g < P.seg_count && ns < OZ_MAX_SEGS; ++g) {
      OzSeg sg = segs[P.seg_begin + g];
      if (n0 >= sg.nrows_b || sg.K <= 0) continue;
      seg_s[ns] = sg;
      segid_s[ns] = P.seg_begin + g;
      step0_s[ns] = steps;
      steps += sg.K / T3_BK;
      ++ns;
    }
    step0_s[ns] = steps;
    nseg_s = ns;
    tc::fence_mbar_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tc::smem_u32(&tmem_s), T3W_TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_s;
  const int nseg = nseg_s;
  const int total = step0_s[nseg];
  const int nchunks = (total + SPC - 1) / SPC;

  // a wait that runs out records where (oz_wait_code) and stops every role
  auto wait = [&](uint64_t* bar, uint32_t parity, int site, int detail) -> bool {
    return oz_wait_bounded(bar, parity, site, detail, &abort_s, OZ_SPIN);
  };

  if (warp == 0) {
    // ---------------- producer (TMA): all terms of A and of B per K step
    if (lane == 0) {
      int seg = -1, seg_end = 0, seg_begin = 0;
      const CUtensorMap *ma = nullptr, *mb = nullptr;
      int ax = 0, ay = 0, bx = 0, by = 0;
      int issued = 0;
      for (int g = 0; g < total; ++g) {
        const int st = g % T3W_STAGES;
        if (g >= T3W_STAGES && !wait(&empty_b[st], ((g / T3W_STAGES) - 1) & 1, OZ_SITE_EMPTY, g)) break;
        while (g >= seg_end) {
          ++seg;
          seg_begin = step0_s[seg];
          seg_end = step0_s[seg + 1];
          const OzSeg& S = seg_s[seg];
          ma = &maps[segid_s[seg]].a;
          mb = &maps[segid_s[seg]].bw;
          ax = S.a_k0;
          ay = S.a_row0 + m0;
          bx = S.b_k0;
          by = S.b_row0 + n0;
        }
        const int k0 = (g - seg_begin) * T3_BK;
        const uint32_t fb = tc::smem_u32(&full_b[st]);
        const uint32_t sa = s_stage0 + st * T3W_STAGE_BYTES;
        tc::mbar_arrive_expect_tx(fb, T3W_STAGE_BYTES);
        tc::tma_load_3d(sa, ma, ax + k0, ay, 0, fb);
        tc::tma_load_3d(sa + T3_S * T3_A_SLICE_BYTES, mb, bx + k0, by, 0, fb);
        issued = g + 1;
      }
      for (int g = issued - T3W_STAGES > 0 ? issued - T3W_STAGES : 0; g < issued; ++g)
        tc::mbar_wait_bounded(tc::smem_u32(&full_b[g % T3W_STAGES]), (g / T3W_STAGES) & 1, OZ_SPIN);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t N128 = tc::idesc_bf16_f32(T3_BM, T3W_BN);
      for (int g = 0; g < total; ++g) {
        const int st = g % T3W_STAGES;
        const int ch = g / SPC, kin = g % SPC, b = ch & 1;
        if (kin == 0 && ch >= 2 && !wait(&free_b[b], ((ch >> 1) - 1) & 1, OZ_SITE_FREE, ch)) break;
        if (!wait(&full_b[st], (g / T3W_STAGES) & 1, OZ_SITE_FULL, g)) break;
        tc::fence_after_sync();
        const uint32_t sa = s_stage0 + st * T3W_STAGE_BYTES;
        const uint32_t sb = sa + T3_S * T3_A_SLICE_BYTES;
        auto A = [&](int t) { return tc::smem_desc_sw32(sa + t * T3_A_SLICE_BYTES); };
        auto B = [&](int u) { return tc::smem_desc_sw32(sb + u * T3W_B_SLICE_BYTES); };
        const uint32_t D0 = tmem + (uint32_t)(b * T3W_BUF_COLS), D1 = D0 + T3W_BN;
        const uint32_t first = kin == 0 ? 0u : 1u;  // the first step of a chunk restarts the buffer
        tc::mma_bf16(D0, A(0), B(0), N128, first);
        tc::mma_bf16(D1, A(0), B(1), N128, first);
        tc::mma_bf16(D1, A(1), B(0), N128, 1u);
        tc::mma_bf16(D1, A(0), B(2), N128, 1u);
        tc::mma_bf16(D1, A(1), B(1), N128, 1u);
        tc::mma_bf16(D1, A(2), B(0), N128, 1u);
        tc::mma_commit(tc::smem_u32(&empty_b[st]));
        if (kin == SPC - 1 || g == total - 1) tc::mma_commit(tc::smem_u32(&chunk_b[b]));
      }
      if (abort_s) {
        tc::mma_commit(tc::smem_u32(&drain_b));
        tc::mbar_wait_bounded(tc::smem_u32(&drain_b), 0, OZ_SPIN);
      }
    }
  } else {
    // ---------------- epilogue: warps 2-9; lane quarter = warp % 4, column half = (warp - 2) / 4
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const int gm = m0 + row;
    const int cbase = ((warp - 2) >> 2) * T3W_EPI_COLS;
    const uint32_t lane_base = ((uint32_t)(quarter * 32) << 16) + (uint32_t)cbase;
    float sums[T3W_EPI_COLS];
#pragma unroll
    for (int j = 0; j < T3W_EPI_COLS; ++j) sums[j] = 0.0f;
    bool ok = true;
    for (int ch = 0; ch < nchunks && ok; ++ch) {
      const int b = ch & 1;
      ok = wait(&chunk_b[b], (ch >> 1) & 1, OZ_SITE_CHUNK, ch);
      if (!__all_sync(0xffffffffu, ok)) {  // tcgen05.ld is warp-collective
        ok = false;
        break;
      }
      tc::fence_after_sync();
      const uint32_t D = tmem + lane_base + (uint32_t)(b * T3W_BUF_COLS);
#pragma unroll
      for (int c0 = 0; c0 < T3W_EPI_COLS; c0 += 8) {
        uint32_t r0[8], r1[8];
        tc::tmem_ld8(D + c0, r0);
        tc::tmem_ld8(D + T3W_BN + c0, r1);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j) sums[c0 + j] += __uint_as_float(r0[j]) + __uint_as_float(r1[j]);
      }
      tc::fence_before_sync();
      tc::mbar_arrive(tc::smem_u32(&free_b[b]));
    }
    if (ok && gm < P.M) {
#pragma unroll
      for (int j = 0; j < T3W_EPI_COLS; ++j) {
        const int gn = n0 + cbase + j;
        if (gn < P.N) {
          float* dst = Tp + (long long)gm * P.ldt + gn;
          *dst = P.accumulate ? *dst + sums[j] : sums[j];
        }
      }
    }
  }
  __syncthreads();
  if (abort_s && threadIdx.x == 0) atomicCAS(err, 0, abort_s + (int)min(blockIdx.x, 4095u) * OZ_WAIT_CTA);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, T3W_TMEM_COLS);
  }
}

}  // namespace iscsi
