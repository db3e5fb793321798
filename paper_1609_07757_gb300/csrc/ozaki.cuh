// ozaki.cuh -- FP64-accurate contraction T = A * B^T on the bf16 tensor cores.
//
// GB300 runs FP64 at ~1.2 TFLOP/s but bf16 MMA at ~2 PFLOP/s, so the FP64
// opposite-spin contraction is computed from exact bf16 slices (an error-free
// splitting in the manner of Ozaki's scheme for accurate matrix products):
//
//   each row of A (and of B, stored K-major as [N][K]) is scaled by a power of
//   two 2^-e so that |x| < 1, then cut into S = 7 slices of 7 bits:
//     x = 2^-7 sum_t a_t 2^-7t,  a_t integers, |a_0| <= 128, |a_t| <= 64;
//   slice t is stored as the bf16 value a_t 2^-7t (exact: <= 8 significant bits);
//   the product sum_k x_k y_k = 2^-14 sum_L 2^-7L I_L with
//     I_L = sum_k sum_{t+u=L} a_t b_u  (integers);
//   one k contributes at most 2 * 2^7 2^6 + (L-1) 2^12 = (L+3) 2^12 to I_L
//   (4 * 2^12 for L = 0), so over a K chunk of 512 every |I_L| <= 7 * 2^21
//   < 2^24 for L <= 4 and the FP32 tensor-memory accumulator of each of
//   these levels holds it exactly;
//   levels L = 0..4 are flushed after every chunk into an exact int64 running
//   sum S = sum_L 2^7(4-L) I_L; levels 5..6 (weight <= 2^-35 of the leading
//   one) accumulate in one FP32 tail over the whole K; levels >= 7 are dropped.
//   T = 2^(e_a + e_b - 14) (S 2^-28 + tail).  The tensor core's FP32
//   accumulation is exact for the integer-valued levels but biased (it does
//   not round to nearest) for the tail, so the tail carries only levels whose
//   weight makes that bias negligible over the whole K.  Relative error
//   ~2^-48 of sum_k |x_k||y_k| (slice truncation, dropped levels, tail).
//
// Tile: 128 rows of A x 64 rows of B per CTA, K step 16, OZ_STAGES-deep TMA ring.
// TMEM holds level L at columns 64L .. 64L+63 (L = 0..6), so the products
// A_t x (B_0 .. B_{6-t}) of one A slice land on consecutive levels and go out
// as one MMA of N = 64 (7 - t) columns (split at 256): 10 MMAs per K step
// instead of 28, each A slice read from shared memory once or twice.
#pragma once
#include <cuda_bf16.h>

#include "ozaki_digits.cuh"
#include "ozaki_types.cuh"
#include "tc_ptx.cuh"

namespace iscsi {

// row exponent e with max_k |X(r,k)| * 2^-e < 1 (0 for an all-zero row);
// X(r,k) = X[r*ld + k], or X[k*ld + r] when trans
__global__ void k_oz_row_exp(const double* __restrict__ X, int rows, int cols, long long ld, int trans,
                             int* __restrict__ e) {
  int r = blockIdx.x;
  int m = 0;
  for (int k = threadIdx.x; k < cols; k += blockDim.x)
    m = max(m, oz_exp_field(trans ? X[(long long)k * ld + r] : X[(long long)r * ld + k]));
  m = __reduce_max_sync(0xffffffffu, m);
  __shared__ int sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    int x = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) x = max(x, sm[i]);
    e[r] = x > 0 ? x - 1022 : 0;  // max |x| = f 2^e, f in [0.5, 1)
  }
}

// slices of X into out[s][row][k] (row stride ldo, rows_pad rows, zero padded).
// Source column of k: colmap[k] (-1: zero) if colmap, else k (zero beyond cols).
__global__ void k_oz_slice(const double* __restrict__ X, int rows, int cols, long long ld, int trans,
                           const int* __restrict__ colmap, const int* __restrict__ e,
                           __nv_bfloat16* __restrict__ out, long long slice_stride, int ldo, int rows_pad) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long total = (long long)rows_pad * ldo;
  if (t >= total) return;
  int r = (int)(t / ldo), k = (int)(t % ldo);
  int src = colmap ? colmap[k] : (k < cols ? k : -1);
  double x = 0.0;
  int ex = 0;
  if (r < rows && src >= 0) {
    x = trans ? X[(long long)src * ld + r] : X[(long long)r * ld + src];
    ex = e[r];
  }
  int a[OZ_S];
  oz_digits(x, ex, a);
  oz_store_digits(a, out + t, slice_stride);
}

// Warp-specialised product kernel.  Per CTA one 128 x 64 output tile:
//   warp 0     (one lane) loads K steps into an OZ_STAGES-deep ring: two TMA boxes
//              (all slices of A, all slices of B) per step, completion as
//              transaction bytes on full[stage],
//   warp 1     (one lane) waits full[stage], issues the MMAs of the step,
//              releases the stage through tcgen05.commit -> empty[stage] and,
//              at the end of a K chunk, signals chunk_done,
//   warps 2+   drain the exact levels of each chunk from TMEM into int64
//              sums held in registers (one output row per thread; with 8
//              epilogue warps, warps w and w+4 share TMEM lane quarter w % 4
//              and take half of the columns each), finish each segment and
//              release the accumulators (acc_free) for the next chunk.
// Every wait is bounded; a wait that runs out sets abort (all roles stop),
// the kernel waits (bounded) for its copies in flight, frees TMEM and
// reports through err.
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_oz_gemm(const OzProblem* __restrict__ probs, int nprobs, const OzSeg* __restrict__ segs,
              const OzMaps* __restrict__ maps, double* tbase, double* const* __restrict__ tbases,
              int* __restrict__ err) {
  extern __shared__ unsigned char oz_smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t s_stage0 = tc::smem_u32(smem);
  __shared__ uint64_t full_b[OZ_STAGES], empty_b[OZ_STAGES], chunk_b, free_b, drain_b;
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
  double* const Tp = P.t_rel ? (tbases ? tbases[P.tb] : tbase) + P.t : reinterpret_cast<double*>(P.t);
  const int tl = tile - P.tile_begin;
  const int m0 = (tl / P.tiles_n) * OZ_BM, n0 = (tl % P.tiles_n) * OZ_BN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int SPC = OZ_CHUNK / OZ_BK;  // steps per chunk

  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      tc::mbar_init(tc::smem_u32(&full_b[s]), 1);
      tc::mbar_init(tc::smem_u32(&empty_b[s]), 1);
    }
    tc::mbar_init(tc::smem_u32(&chunk_b), 1);
    tc::mbar_init(tc::smem_u32(&free_b), 32 * OZ_EPI_WARPS);
    tc::mbar_init(tc::smem_u32(&drain_b), 1);
    abort_s = 0;
    int ns = 0, steps = 0;
    for (int g = 0; g < P.seg_count && ns < OZ_MAX_SEGS; ++g) {
      OzSeg sg = segs[P.seg_begin + g];
      if (n0 >= sg.nrows_b || sg.K <= 0) continue;
      seg_s[ns] = sg;
      segid_s[ns] = P.seg_begin + g;
      step0_s[ns] = steps;
      steps += sg.K / OZ_BK;
      ++ns;
    }
    step0_s[ns] = steps;
    nseg_s = ns;
    tc::fence_mbar_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tc::smem_u32(&tmem_s), OZ_TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_s;
  const int nseg = nseg_s;
  const int total = step0_s[nseg];

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
    // ---------------- producer (TMA)
    if (lane == 0) {
      int seg = -1, seg_end = 0, seg_begin = 0;
      const CUtensorMap *ma = nullptr, *mb = nullptr;
      int ax = 0, ay = 0, bx = 0, by = 0;
      int issued = 0;
      for (int g = 0; g < total; ++g) {
        const int st = g % OZ_STAGES;
        if (g >= OZ_STAGES && !wait(&empty_b[st], ((g / OZ_STAGES) - 1) & 1)) break;
        while (g >= seg_end) {
          ++seg;
          seg_begin = step0_s[seg];
          seg_end = step0_s[seg + 1];
          const OzSeg& S = seg_s[seg];
          ma = &maps[segid_s[seg]].a;
          mb = &maps[segid_s[seg]].b;
          ax = S.a_k0;
          ay = S.a_row0 + m0;
          bx = S.b_k0;
          by = S.b_row0 + n0;
        }
        const int k0 = (g - seg_begin) * OZ_BK;
        const uint32_t fb = tc::smem_u32(&full_b[st]);
        const uint32_t sa = s_stage0 + st * OZ_STAGE_BYTES;
        tc::mbar_arrive_expect_tx(fb, OZ_STAGE_BYTES);
        tc::tma_load_3d(sa, ma, ax + k0, ay, 0, fb);
        tc::tma_load_3d(sa + OZ_S * OZ_A_SLICE_BYTES, mb, bx + k0, by, 0, fb);
        issued = g + 1;
      }
      // copies still in flight (only after an abort) must land before the
      // CTA's shared memory is released: wait for the last phase of each stage
      for (int g = issued - OZ_STAGES > 0 ? issued - OZ_STAGES : 0; g < issued; ++g)
        tc::mbar_wait_bounded(tc::smem_u32(&full_b[g % OZ_STAGES]), (g / OZ_STAGES) & 1, OZ_SPIN);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t N64 = tc::idesc_bf16_f32(OZ_BM, 64), N128 = tc::idesc_bf16_f32(OZ_BM, 128),
                         N192 = tc::idesc_bf16_f32(OZ_BM, 192), N256 = tc::idesc_bf16_f32(OZ_BM, 256);
      constexpr uint32_t TAIL = OZ_EXACT * OZ_BN;  // level 5 (level 6 follows at +64)
      int seg = 0, seg_begin = 0, seg_end = nseg > 0 ? step0_s[1] : 0;
      int chunk = 0;  // chunks completed so far
      for (int g = 0; g < total; ++g) {
        const int st = g % OZ_STAGES;
        while (g >= seg_end) {
          ++seg;
          seg_begin = seg_end;
          seg_end = step0_s[seg + 1];
        }
        const int local = g - seg_begin;
        const int kin = local % SPC;
        if (!wait(&full_b[st], (g / OZ_STAGES) & 1)) break;
        tc::fence_after_sync();
        const uint32_t sa = s_stage0 + st * OZ_STAGE_BYTES;
        const uint32_t sb = sa + OZ_S * OZ_A_SLICE_BYTES;
        auto A = [&](int t) { return tc::smem_desc_sw32(sa + t * OZ_A_SLICE_BYTES); };
        auto B = [&](int u) { return tc::smem_desc_sw32(sb + u * OZ_B_SLICE_BYTES); };
        const bool new_seg = local == 0;
        const bool new_chunk = kin == 0;
        if (!new_chunk) {
          // A_t x (B_0 .. B_{6-t}) into levels t .. 6
          tc::mma_bf16(tmem + 0, A(0), B(0), N256, 1u);
          tc::mma_bf16(tmem + 256, A(0), B(4), N192, 1u);
          tc::mma_bf16(tmem + 64, A(1), B(0), N256, 1u);
          tc::mma_bf16(tmem + 320, A(1), B(4), N128, 1u);
          tc::mma_bf16(tmem + 128, A(2), B(0), N256, 1u);
          tc::mma_bf16(tmem + 384, A(2), B(4), N64, 1u);
          tc::mma_bf16(tmem + 192, A(3), B(0), N256, 1u);
          tc::mma_bf16(tmem + 256, A(4), B(0), N192, 1u);
          tc::mma_bf16(tmem + 320, A(5), B(0), N128, 1u);
          tc::mma_bf16(tmem + 384, A(6), B(0), N64, 1u);
        } else {
          // first step of a chunk: the tail levels (5, 6) run across the
          // chunks of a segment and go first, unless a new segment starts
          // and the epilogue still reads them; the exact levels restart
          // once the epilogue has drained the previous chunk
          if (new_seg && chunk > 0 && !wait(&free_b, (chunk - 1) & 1)) break;
#pragma unroll
          for (int t = 0; t < OZ_EXACT; ++t)
            tc::mma_bf16(tmem + TAIL, A(t), B(OZ_EXACT - t), N128, (new_seg && t == 0) ? 0u : 1u);
          tc::mma_bf16(tmem + TAIL, A(5), B(0), N128, 1u);
          tc::mma_bf16(tmem + TAIL + 64, A(6), B(0), N64, 1u);
          if (!new_seg && chunk > 0 && !wait(&free_b, (chunk - 1) & 1)) break;
          tc::mma_bf16(tmem + 0, A(0), B(0), N256, 0u);
          tc::mma_bf16(tmem + 256, A(0), B(4), N64, 0u);
          tc::mma_bf16(tmem + 64, A(1), B(0), N256, 1u);
          tc::mma_bf16(tmem + 128, A(2), B(0), N192, 1u);
          tc::mma_bf16(tmem + 192, A(3), B(0), N128, 1u);
          tc::mma_bf16(tmem + 256, A(4), B(0), N64, 1u);
        }
        tc::mma_commit(tc::smem_u32(&empty_b[st]));
        if (kin == SPC - 1 || local == seg_end - seg_begin - 1) {
          tc::mma_commit(tc::smem_u32(&chunk_b));
          ++chunk;
        }
      }
      if (abort_s) {
        // let MMAs already issued finish before TMEM is released (bounded)
        tc::mma_commit(tc::smem_u32(&drain_b));
        tc::mbar_wait_bounded(tc::smem_u32(&drain_b), 0, OZ_SPIN);
      }
    }
  } else {
    // ---------------- epilogue: TMEM lane quarter = warp % 4
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const int gm = m0 + row;
    const int cbase = OZ_EPI_WARPS == 4 ? 0 : ((warp - 2) >> 2) * OZ_EPI_COLS;  // first column of this warp
    const uint32_t lane_base = ((uint32_t)(quarter * 32) << 16) + (uint32_t)cbase;
    long long sums[OZ_EPI_COLS];
#pragma unroll
    for (int j = 0; j < OZ_EPI_COLS; ++j) sums[j] = 0;
    int chunk = 0, done_segs = 0;
    for (int s = 0; s < nseg && !abort_s; ++s) {
      const int steps = step0_s[s + 1] - step0_s[s];
      const int nch = (steps + SPC - 1) / SPC;
      const OzSeg& S = seg_s[s];
      for (int ch = 0; ch < nch; ++ch, ++chunk) {
        // warp-uniform decision: tcgen05.ld below is warp-collective
        bool ok = wait(&chunk_b, chunk & 1);
        if (!__all_sync(0xffffffffu, ok)) break;
        tc::fence_after_sync();
#pragma unroll
        for (int c0 = 0; c0 < OZ_EPI_COLS; c0 += 8) {
          uint32_t r0[8], r1[8], r2[8], r3[8], r4[8];
          tc::tmem_ld8(tmem + lane_base + 0 * OZ_BN + c0, r0);
          tc::tmem_ld8(tmem + lane_base + 1 * OZ_BN + c0, r1);
          tc::tmem_ld8(tmem + lane_base + 2 * OZ_BN + c0, r2);
          tc::tmem_ld8(tmem + lane_base + 3 * OZ_BN + c0, r3);
          tc::tmem_ld8(tmem + lane_base + 4 * OZ_BN + c0, r4);
          tc::tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            // level L holds 2^-7L I_L exactly; recover the integers
            int i0 = __float2int_rn(__uint_as_float(r0[j]));
            int i1 = __float2int_rn(__uint_as_float(r1[j]) * 128.0f);
            int i2 = __float2int_rn(__uint_as_float(r2[j]) * 16384.0f);
            int i3 = __float2int_rn(__uint_as_float(r3[j]) * 2097152.0f);
            int i4 = __float2int_rn(__uint_as_float(r4[j]) * 268435456.0f);
            sums[c0 + j] += ((long long)i0 << 28) + ((long long)i1 << 21) + ((long long)i2 << 14) +
                            ((long long)i3 << 7) + (long long)i4;
          }
        }
        if (ch == nch - 1) {
          // this segment's result: 2^(ea+eb-14) (S 2^-28 + tail), into T
          const int ea = gm < P.M ? S.a_exp[gm] : 0;
#pragma unroll
          for (int c0 = 0; c0 < OZ_EPI_COLS; c0 += 8) {
            uint32_t r5[8], r6[8];
            tc::tmem_ld8(tmem + lane_base + OZ_EXACT * OZ_BN + c0, r5);
            tc::tmem_ld8(tmem + lane_base + (OZ_EXACT + 1) * OZ_BN + c0, r6);
            tc::tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int gn = n0 + cbase + c0 + j;
              if (gm < P.M && gn < P.N && gn < S.nrows_b) {
                double v = (double)sums[c0 + j] * 3.7252902984619141e-09 /* 2^-28 */ +
                           ((double)__uint_as_float(r5[j]) + (double)__uint_as_float(r6[j]));
                v = ldexp(v, ea + S.b_exp[gn] - 14);
                double* dst = Tp + (long long)gm * P.ldt + gn;
                *dst = (P.accumulate || done_segs > 0) ? *dst + v : v;
              }
              sums[c0 + j] = 0;
            }
          }
          ++done_segs;
        }
        tc::fence_before_sync();
        tc::mbar_arrive(tc::smem_u32(&free_b));
      }
    }
    if (nseg == 0 && !P.accumulate && gm < P.M) {
      // no segment reaches this tile: its block of T is zero
      for (int j = 0; j < OZ_EPI_COLS; ++j) {
        const int gn = n0 + cbase + j;
        if (gn < P.N) Tp[(long long)gm * P.ldt + gn] = 0.0;
      }
    }
  }
  __syncthreads();
  if (abort_s && threadIdx.x == 0) atomicExch(err, 1);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, OZ_TMEM_COLS);
  }
}

}  // namespace iscsi
