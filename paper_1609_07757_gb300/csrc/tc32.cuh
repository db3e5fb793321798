// tc32.cuh -- FP32-accuracy contraction T = A * B^T on the bf16 tensor cores,
// the arithmetic of the FP32 form of the sigma step.
//
// Every operand element x (FP32 or FP64) is split into three bf16 terms
//   x_0 = bf16(x),  x_1 = bf16(x - x_0),  x_2 = bf16(x - x_0 - x_1)
// (each rounding keeps 8 significant bits, the residuals are exact in the
// input type, so |x - x_0 - x_1 - x_2| <= 2^-27 |x|).  The product keeps the
// six term pairs of order t + u <= 2,
//   T = sum_k sum_{t+u<=2} A_t B_u + O(2^-24 sum_k |A||B|),
// accumulated in FP32 in tensor memory over K chunks of 512 and across
// chunks in FP32 registers with round-to-nearest (the tensor core's own
// FP32 accumulation is not round-to-nearest, so it only ever sums one chunk).
//
// TMEM holds order L at columns 192 b + 64 L of accumulator buffer b (two
// buffers, alternating per chunk, so the MMAs of chunk c+1 run while the
// epilogue drains chunk c).  A_t x (B_0 .. B_{2-t}) is one MMA of N = 64 (3-t):
// three MMAs per K step of 16.  Loads, MMA issue and the epilogue are split
// over warps as in the FP64 kernel (ozaki.cuh); segments and problems use the
// same records (OzProblem / OzSeg / OzMaps; the exponent fields are unused).
#pragma once
#include <cuda_bf16.h>

#include "ozaki_types.cuh"
#include "tc_ptx.cuh"

namespace iscsi {

constexpr int T3_S = 3;             // bf16 terms per element
constexpr int T3_BM = 128, T3_BN = 64, T3_BK = 16;
constexpr int T3_STAGES = 8;
constexpr int T3_A_SLICE_BYTES = T3_BM * T3_BK * 2;  // 4096
constexpr int T3_B_SLICE_BYTES = T3_BN * T3_BK * 2;  // 2048
constexpr int T3_STAGE_BYTES = T3_S * (T3_A_SLICE_BYTES + T3_B_SLICE_BYTES);
constexpr int T3_SMEM_BYTES = T3_STAGES * T3_STAGE_BYTES + 1024;
constexpr int T3_CHUNK_STEPS = 32;  // K = 512 per tensor-memory chunk
constexpr int T3_BUF_COLS = T3_S * T3_BN;  // 192 columns per accumulator buffer
constexpr int T3_TMEM_COLS = 512;          // 2 buffers (384 columns) used
constexpr int T3_THREADS = 192;            // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue

// the three bf16 terms of x, slice s at out[s * slice_stride]
template <typename V>
__device__ __forceinline__ void t3_store_terms(V x, __nv_bfloat16* out, long long slice_stride) {
  __nv_bfloat16 h0 = __float2bfloat16_rn((float)x);
  V r = x - (V)__bfloat162float(h0);
  __nv_bfloat16 h1 = __float2bfloat16_rn((float)r);
  r -= (V)__bfloat162float(h1);
  __nv_bfloat16 h2 = __float2bfloat16_rn((float)r);
  out[0] = h0;
  out[slice_stride] = h1;
  out[2 * slice_stride] = h2;
}

// terms of X into out[s][row][k] (row stride ldo, rows_pad rows, zero padded).
// Source column of k: colmap[k] (-1: zero) if colmap, else k (zero beyond cols).
template <typename V>
__global__ void k_t3_slice(const V* __restrict__ X, int rows, int cols, long long ld, int trans,
                           const int* __restrict__ colmap, __nv_bfloat16* __restrict__ out, long long slice_stride,
                           int ldo, int rows_pad) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long total = (long long)rows_pad * ldo;
  if (t >= total) return;
  int r = (int)(t / ldo), k = (int)(t % ldo);
  int src = colmap ? colmap[k] : (k < cols ? k : -1);
  V x = (V)0;
  if (r < rows && src >= 0) x = trans ? X[(long long)src * ld + r] : X[(long long)r * ld + src];
  t3_store_terms<V>(x, out + t, slice_stride);
}

// Per CTA one 128 x 64 tile of T (FP32, ldt), over all segments of its
// problem.  With CL = 2, clusters of two CTAs on adjacent column tiles of one
// row block share the A operand by multicast, as in k_oz_gemm (ozaki.cuh).
// Every wait is bounded; a wait that runs out sets abort, the CTA waits
// (bounded) for its copies in flight, frees TMEM and reports via err.
template <int CL>
__global__ void __launch_bounds__(T3_THREADS, 1)
    k_tc32_gemm(const OzProblem* __restrict__ probs, int nprobs, const OzSeg* __restrict__ segs,
                const OzMaps* __restrict__ maps, float* tbase, float* const* __restrict__ tbases,
                int* __restrict__ err) {
  static_assert(CL == 1 || CL == 2, "clusters of one or two CTAs");
  extern __shared__ unsigned char t3_smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)t3_smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t s_stage0 = tc::smem_u32(smem);
  __shared__ uint64_t full_b[T3_STAGES], empty_b[T3_STAGES], chunk_b[2], free_b[2], drain_b;
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
  const int m0 = (tl / P.tiles_n) * T3_BM, n0 = (tl % P.tiles_n) * T3_BN;
  const int n0_pair = ((tl % P.tiles_n) & ~(CL - 1)) * T3_BN;  // first column of the cluster
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int SPC = T3_CHUNK_STEPS;

  if (threadIdx.x == 0) {
    for (int s = 0; s < T3_STAGES; ++s) {
      tc::mbar_init(tc::smem_u32(&full_b[s]), 1);
      tc::mbar_init(tc::smem_u32(&empty_b[s]), CL);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(tc::smem_u32(&chunk_b[b]), 1);
      tc::mbar_init(tc::smem_u32(&free_b[b]), 128);
    }
    tc::mbar_init(tc::smem_u32(&drain_b), 1);
    abort_s = 0;
    int ns = 0, steps = 0;
    for (int g = 0; g < P.seg_count && ns < OZ_MAX_SEGS; ++g) {
      OzSeg sg = segs[P.seg_begin + g];
      if (n0_pair >= sg.nrows_b || sg.K <= 0) continue;
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
    tc::tmem_alloc(tc::smem_u32(&tmem_s), T3_TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  if (CL == 2) tc::cluster_sync();  // the partner's barriers exist before any multicast
  tc::fence_after_sync();
  const uint32_t tmem = tmem_s;
  const int nseg = nseg_s;
  const int total = step0_s[nseg];
  const int nchunks = (total + SPC - 1) / SPC;

  auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
    uint32_t a = tc::smem_u32(bar);
    for (long long i = 0; i < OZ_SPIN; ++i) {
      if (tc::mbar_try_wait(a, parity)) return true;
      if ((i & 1023) == 1023 && abort_s) return false;
    }
    abort_s = 1;
    return false;
  };

  if (warp == 0) {
    // ---------------- producer (TMA): all terms of A and of B per K step
    if (lane == 0) {
      int seg = -1, seg_end = 0, seg_begin = 0;
      const CUtensorMap *ma = nullptr, *mah = nullptr, *mb = nullptr;
      int ax = 0, ay = 0, bx = 0, by = 0;
      int issued = 0;
      const int rank = CL == 2 ? (int)tc::cluster_rank() : 0;
      for (int g = 0; g < total; ++g) {
        const int st = g % T3_STAGES;
        if (g >= T3_STAGES && !wait(&empty_b[st], ((g / T3_STAGES) - 1) & 1)) break;
        while (g >= seg_end) {
          ++seg;
          seg_begin = step0_s[seg];
          seg_end = step0_s[seg + 1];
          const OzSeg& S = seg_s[seg];
          ma = &maps[segid_s[seg]].a;
          mah = &maps[segid_s[seg]].ah;
          mb = &maps[segid_s[seg]].b;
          ax = S.a_k0;
          ay = S.a_row0 + m0;
          bx = S.b_k0;
          by = S.b_row0 + n0;
        }
        const int k0 = (g - seg_begin) * T3_BK;
        const uint32_t fb = tc::smem_u32(&full_b[st]);
        const uint32_t sa = s_stage0 + st * T3_STAGE_BYTES;
        tc::mbar_arrive_expect_tx(fb, T3_STAGE_BYTES);
        if (CL == 1) {
          tc::tma_load_3d(sa, ma, ax + k0, ay, 0, fb);
        } else {
          // this CTA's half of the rows of each A term, to both CTAs
#pragma unroll
          for (int t = 0; t < T3_S; ++t)
            tc::tma_load_3d_mc(sa + t * T3_A_SLICE_BYTES + rank * (T3_A_SLICE_BYTES / 2), mah, ax + k0,
                               ay + rank * (T3_BM / 2), t, fb, (uint16_t)0x3);
        }
        tc::tma_load_3d(sa + T3_S * T3_A_SLICE_BYTES, mb, bx + k0, by, 0, fb);
        issued = g + 1;
      }
      for (int g = issued - T3_STAGES > 0 ? issued - T3_STAGES : 0; g < issued; ++g)
        tc::mbar_wait_bounded(tc::smem_u32(&full_b[g % T3_STAGES]), (g / T3_STAGES) & 1, OZ_SPIN);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t N64 = tc::idesc_bf16_f32(T3_BM, 64), N128 = tc::idesc_bf16_f32(T3_BM, 128),
                         N192 = tc::idesc_bf16_f32(T3_BM, 192);
      for (int g = 0; g < total; ++g) {
        const int st = g % T3_STAGES;
        const int ch = g / SPC, kin = g % SPC, b = ch & 1;
        if (kin == 0 && ch >= 2 && !wait(&free_b[b], ((ch >> 1) - 1) & 1)) break;
        if (!wait(&full_b[st], (g / T3_STAGES) & 1)) break;
        tc::fence_after_sync();
        const uint32_t sa = s_stage0 + st * T3_STAGE_BYTES;
        const uint32_t sb = sa + T3_S * T3_A_SLICE_BYTES;
        const uint32_t D = tmem + (uint32_t)(b * T3_BUF_COLS);
        // A_t x (B_0 .. B_{2-t}) into orders t .. 2; the first MMA of a chunk
        // covers all three orders and restarts the buffer
        tc::mma_bf16(D, tc::smem_desc_sw32(sa), tc::smem_desc_sw32(sb), N192, kin == 0 ? 0u : 1u);
        tc::mma_bf16(D + 64, tc::smem_desc_sw32(sa + T3_A_SLICE_BYTES), tc::smem_desc_sw32(sb), N128, 1u);
        tc::mma_bf16(D + 128, tc::smem_desc_sw32(sa + 2 * T3_A_SLICE_BYTES), tc::smem_desc_sw32(sb), N64, 1u);
        if (CL == 2)
          tc::mma_commit_mc(tc::smem_u32(&empty_b[st]), (uint16_t)0x3);  // both CTAs read this stage
        else
          tc::mma_commit(tc::smem_u32(&empty_b[st]));
        if (kin == SPC - 1 || g == total - 1) tc::mma_commit(tc::smem_u32(&chunk_b[b]));
      }
      if (abort_s) {
        tc::mma_commit(tc::smem_u32(&drain_b));
        tc::mbar_wait_bounded(tc::smem_u32(&drain_b), 0, OZ_SPIN);
      }
    }
  } else {
    // ---------------- epilogue: warps 2-5, TMEM lane quarter = warp % 4
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const int gm = m0 + row;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    float sums[T3_BN];
#pragma unroll
    for (int j = 0; j < T3_BN; ++j) sums[j] = 0.0f;
    bool ok = true;
    for (int ch = 0; ch < nchunks && ok; ++ch) {
      const int b = ch & 1;
      ok = wait(&chunk_b[b], (ch >> 1) & 1);
      if (!__all_sync(0xffffffffu, ok)) {  // tcgen05.ld is warp-collective
        ok = false;
        break;
      }
      tc::fence_after_sync();
      const uint32_t D = tmem + lane_base + (uint32_t)(b * T3_BUF_COLS);
#pragma unroll
      for (int c0 = 0; c0 < T3_BN; c0 += 8) {
        uint32_t r0[8], r1[8], r2[8];
        tc::tmem_ld8(D + c0, r0);
        tc::tmem_ld8(D + 64 + c0, r1);
        tc::tmem_ld8(D + 128 + c0, r2);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j)
          sums[c0 + j] += __uint_as_float(r0[j]) + (__uint_as_float(r1[j]) + __uint_as_float(r2[j]));
      }
      tc::fence_before_sync();
      tc::mbar_arrive(tc::smem_u32(&free_b[b]));
    }
    if (ok && gm < P.M) {
      // segments whose B has fewer valid rows contribute zeros beyond them
#pragma unroll
      for (int j = 0; j < T3_BN; ++j) {
        const int gn = n0 + j;
        if (gn < P.N) {
          float* dst = Tp + (long long)gm * P.ldt + gn;
          *dst = P.accumulate ? *dst + sums[j] : sums[j];
        }
      }
    }
  }
  __syncthreads();
  if (abort_s && threadIdx.x == 0) atomicExch(err, 1);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, T3_TMEM_COLS);
  }
  // no CTA leaves while its partner's copies or MMA commits may still reach it
  if (CL == 2) tc::cluster_sync();
}

}  // namespace iscsi
