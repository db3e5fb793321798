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
//   over a K chunk of 256 every |I_L| <= 256 (L+3) 2^12 <= 2^24, so the FP32
//   tensor-memory accumulator of each level is exact;
//   levels L = 0..4 are flushed after every chunk into an exact int64 running
//   sum S = sum_L 2^7(4-L) I_L; levels 5..6 (weight <= 2^-35 of the leading
//   one) accumulate in one FP32 tail over the whole K; levels >= 7 are dropped.
//   T = 2^(e_a + e_b - 14) (S 2^-28 + tail).  The tensor core's FP32
//   accumulation is exact for the integer-valued levels but biased (it does
//   not round to nearest) for the tail, so the tail carries only levels whose
//   weight makes that bias negligible over the whole K.  Relative error
//   ~2^-48 of sum_k |x_k||y_k| (slice truncation, dropped levels, tail).
//
// Tile: 128 rows of A x 64 rows of B per CTA, K step 16 (one MMA), 3-stage
// cp.async pipeline; one thread issues the 28 MMAs of a K step; 6 TMEM
// accumulators of 64 columns (levels 0..4 and the tail).
#pragma once
#include <cuda_bf16.h>

#include "ozaki_types.cuh"
#include "tc_ptx.cuh"

namespace iscsi {

// Slicing in integer arithmetic (GB300's FP64 units are slow): with |v| < 2^e,
// N = round(v 2^(49-e)) is read off the FP64 bit pattern, then cut into
// balanced base-128 digits, least significant first: N = sum_t a_t 2^(7(6-t)),
// |a_t| <= 64 for t >= 1 and |a_0| <= 128, i.e. v 2^-e = 2^-7 sum_t a_t 2^-7t
// up to the rounding of N (<= 2^-50).
__device__ __forceinline__ void oz_digits(double v, int e, int (&a)[OZ_S]) {
  long long bits = __double_as_longlong(v);
  int E = (int)((bits >> 52) & 0x7FF);
  long long N = 0;
  if (E != 0) {  // zeros and subnormals give N = 0 (far below the slice resolution)
    long long m = (bits & 0xFFFFFFFFFFFFFll) | (1ll << 52);
    int sh = (E - 1075) + 49 - e;  // v = m 2^(E-1075); N = m 2^sh, sh <= -4 when |v| < 2^e
    if (sh >= 0) N = m << (sh > 10 ? 10 : sh);
    else if (sh > -63) N = (m + (1ll << (-sh - 1))) >> (-sh);
    if (bits < 0) N = -N;
  }
#pragma unroll
  for (int t = OZ_S - 1; t >= 1; --t) {
    int r = (int)(N & 127);
    if (r >= 64) r -= 128;
    a[t] = r;
    N = (N - r) >> 7;
  }
  a[0] = (int)N;
}

__device__ __forceinline__ void oz_store_digits(const int (&a)[OZ_S], __nv_bfloat16* out, long long slice_stride) {
  const float scale[OZ_S] = {1.0f, 0.0078125f, 6.103515625e-05f, 4.76837158203125e-07f, 3.7252902984619141e-09f,
                             2.9103830456733704e-11f, 2.2737367544323206e-13f};  // 2^-7t, exact
#pragma unroll
  for (int s = 0; s < OZ_S; ++s) out[s * slice_stride] = __float2bfloat16_rn(__int2float_rn(a[s]) * scale[s]);
}

// exponent field of |x|: frexp exponent = field - 1022 for normal x (0 for zero)
__device__ __forceinline__ int oz_exp_field(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

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

// [rows x 16] bf16 slice tile, K-major, into core-matrix layout:
// offset(r, kc) = ((r/8)*2 + kc)*128 + (r%8)*16; LBO = 128 B, SBO = 256 B
__device__ __forceinline__ void oz_load_unit(uint32_t sbase, const __nv_bfloat16* src_row0, int ld, int unit) {
  int lane = threadIdx.x & 31;
  int r = unit * 16 + (lane >> 4) * 8 + (lane & 7);
  int kc = (lane >> 3) & 1;
  const __nv_bfloat16* src = src_row0 + (long long)r * ld + kc * 8;
  uint32_t dst = sbase + (uint32_t)(((r >> 3) * 2 + kc) * 128 + (r & 7) * 16);
  tc::cp_async16(dst, src);
}

// one K step (16) of all slices of both operands; a, b point at (row 0 of the
// tile, k0) of slice 0
__device__ __forceinline__ void oz_load_stage(uint32_t sstage, const __nv_bfloat16* a, long long a_slice, int lda,
                                              const __nv_bfloat16* b, long long b_slice, int ldb) {
  // 84 units of 32 chunks: A 7 slices x 8 units, B 7 slices x 4 units
  int warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < OZ_S * 12 / (OZ_THREADS / 32); ++i) {
    int u = warp + i * (OZ_THREADS / 32);
    if (u < OZ_S * 8) {
      int s = u >> 3, unit = u & 7;
      oz_load_unit(sstage + s * OZ_A_SLICE_BYTES, a + s * a_slice, lda, unit);
    } else {
      int v = u - OZ_S * 8;
      int s = v >> 2, unit = v & 3;
      oz_load_unit(sstage + OZ_S * OZ_A_SLICE_BYTES + s * OZ_B_SLICE_BYTES, b + s * b_slice, ldb, unit);
    }
  }
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_oz_gemm(const OzProblem* __restrict__ probs, int nprobs, const OzSeg* __restrict__ segs, double* tbase,
              int* __restrict__ err) {
  extern __shared__ unsigned char oz_smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  uint32_t s_stage0 = tc::smem_u32(smem);
  long long* sums = reinterpret_cast<long long*>(smem + OZ_STAGES * OZ_STAGE_BYTES);  // [BN][BM]
  __shared__ uint64_t mbar[OZ_STAGES];
  __shared__ uint32_t tmem_s;
  __shared__ int abort_s;
  __shared__ OzSeg seg_s[OZ_MAX_SEGS];
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
  double* const Tp = P.t_rel ? tbase + P.t : reinterpret_cast<double*>(P.t);
  int tl = tile - P.tile_begin;
  int m0 = (tl / P.tiles_n) * OZ_BM, n0 = (tl % P.tiles_n) * OZ_BN;
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) tc::mbar_init(tc::smem_u32(&mbar[s]), 1);
    abort_s = 0;
    // the segments that reach this tile, and their first global K step
    int ns = 0, steps = 0;
    for (int g = 0; g < P.seg_count && ns < OZ_MAX_SEGS; ++g) {
      OzSeg sg = segs[P.seg_begin + g];
      if (n0 >= sg.nrows_b || sg.K <= 0) continue;
      seg_s[ns] = sg;
      step0_s[ns] = steps;
      steps += sg.K / OZ_BK;
      ++ns;
    }
    step0_s[ns] = steps;
    nseg_s = ns;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tc::smem_u32(&tmem_s), OZ_TMEM_COLS);
    tc::tmem_relinquish();
  }
  for (int i = threadIdx.x; i < OZ_BM * OZ_BN; i += OZ_THREADS) sums[i] = 0;
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_s;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(OZ_BM, OZ_BN);
  const int nseg = nseg_s;
  const int total = step0_s[nseg];
  const int row = warp * 32 + lane;
  const int gm = m0 + row;

  // register copy of the segment being loaded (loads advance in step order)
  int ld_seg = -1, ld_end = 0, ld_begin = 0;
  const __nv_bfloat16 *la = nullptr, *lb = nullptr;
  long long las = 0, lbs = 0;
  int llda = 0, lldb = 0;
  auto load_step = [&](int g, int stage) {
    while (g >= ld_end) {
      ++ld_seg;
      ld_begin = step0_s[ld_seg];
      ld_end = step0_s[ld_seg + 1];
      const OzSeg& S = seg_s[ld_seg];
      llda = S.lda;
      lldb = S.ldb;
      las = S.a_slice;
      lbs = S.b_slice;
      la = S.as + (long long)m0 * llda;
      lb = S.bs + (long long)n0 * lldb;
    }
    int k0 = (g - ld_begin) * OZ_BK;
    oz_load_stage(s_stage0 + stage * OZ_STAGE_BYTES, la + k0, las, llda, lb + k0, lbs, lldb);
  };
  // segment of the step being computed
  int c_seg = 0, c_begin = 0, c_end = nseg > 0 ? step0_s[1] : 0;

  for (int s = 0; s < OZ_STAGES; ++s) {
    if (s < total) load_step(s, s);
    tc::cp_async_commit();
  }
  bool aborted = false;
  int done_segs = 0;
  for (int g = 0; g < total; ++g) {
    int st = g % OZ_STAGES;
    // step g is commit group g (prologue: 0..S-1, then one group per g >= 1)
    if (g == 0) tc::cp_async_wait<OZ_STAGES - 1>();
    else tc::cp_async_wait<OZ_STAGES - 2>();
    tc::fence_proxy_async();
    __syncthreads();
    while (g >= c_end) {
      ++c_seg;
      c_begin = c_end;
      c_end = step0_s[c_seg + 1];
    }
    const int sgi = c_seg;
    int local = g - c_begin;
    int seg_steps = c_end - c_begin;
    int kin = local % (OZ_CHUNK / OZ_BK);
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
      uint32_t sa = s_stage0 + st * OZ_STAGE_BYTES;
      uint32_t sb = sa + OZ_S * OZ_A_SLICE_BYTES;
#pragma unroll
      for (int L = 0; L < OZ_S; ++L) {
        uint32_t acc_col = (uint32_t)((L < OZ_EXACT ? L : OZ_EXACT) * OZ_BN);
#pragma unroll
        for (int t = 0; t <= L; ++t) {
          int u = L - t;
          uint64_t ad = tc::smem_desc(sa + t * OZ_A_SLICE_BYTES, 128, 256);
          uint64_t bd = tc::smem_desc(sb + u * OZ_B_SLICE_BYTES, 128, 256);
          uint32_t accum;
          if (L < OZ_EXACT) accum = (kin == 0 && t == 0) ? 0u : 1u;
          else accum = (local == 0 && L == OZ_EXACT && t == 0) ? 0u : 1u;
          tc::mma_bf16(tmem + acc_col, ad, bd, idesc, accum);
        }
      }
      tc::mma_commit(tc::smem_u32(&mbar[st]));
    }
    // refill the stage of step g-1 once its MMAs completed
    if (g >= 1 && g - 1 + OZ_STAGES < total) {
      int ps = (g - 1) % OZ_STAGES;
      if (!tc::mbar_wait_bounded(tc::smem_u32(&mbar[ps]), ((g - 1) / OZ_STAGES) & 1, OZ_SPIN)) abort_s = 1;
      else load_step(g - 1 + OZ_STAGES, ps);
    }
    if (g >= 1) tc::cp_async_commit();
    bool seg_end = (local == seg_steps - 1);
    bool chunk_end = (kin == OZ_CHUNK / OZ_BK - 1) || seg_end;
    if (chunk_end) {
      // all MMAs so far done -> flush the exact levels into the int64 sums
      if (!tc::mbar_wait_bounded(tc::smem_u32(&mbar[st]), (g / OZ_STAGES) & 1, OZ_SPIN)) abort_s = 1;
      __syncthreads();  // abort_s is uniform below (tcgen05.ld is warp-collective)
      if (!abort_s) {
        tc::fence_after_sync();
        const OzSeg& S = seg_s[sgi];
        int ea = (seg_end && gm < P.M) ? S.a_exp[gm] : 0;
#pragma unroll 1
        for (int c0 = 0; c0 < OZ_BN; c0 += 16) {
          uint32_t r0[16], r1[16], r2[16], r3[16], r4[16];
          tc::tmem_ld16(tmem + lane_base + 0 * OZ_BN + c0, r0);
          tc::tmem_ld16(tmem + lane_base + 1 * OZ_BN + c0, r1);
          tc::tmem_ld16(tmem + lane_base + 2 * OZ_BN + c0, r2);
          tc::tmem_ld16(tmem + lane_base + 3 * OZ_BN + c0, r3);
          tc::tmem_ld16(tmem + lane_base + 4 * OZ_BN + c0, r4);
          tc::tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            // level L holds 2^-7L I_L exactly; recover the integers
            int i0 = __float2int_rn(__uint_as_float(r0[j]));
            int i1 = __float2int_rn(__uint_as_float(r1[j]) * 128.0f);
            int i2 = __float2int_rn(__uint_as_float(r2[j]) * 16384.0f);
            int i3 = __float2int_rn(__uint_as_float(r3[j]) * 2097152.0f);
            int i4 = __float2int_rn(__uint_as_float(r4[j]) * 268435456.0f);
            long long v = ((long long)i0 << 28) + ((long long)i1 << 21) + ((long long)i2 << 14) +
                          ((long long)i3 << 7) + (long long)i4;
            sums[(c0 + j) * OZ_BM + row] += v;
          }
          if (seg_end) {
            // this segment's result: 2^(ea+eb-14) (S 2^-28 + tail), into T
            uint32_t rt[16];
            tc::tmem_ld16(tmem + lane_base + OZ_EXACT * OZ_BN + c0, rt);
            tc::tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              int gn = n0 + c0 + j;
              long long sv = sums[(c0 + j) * OZ_BM + row];
              sums[(c0 + j) * OZ_BM + row] = 0;
              if (gm < P.M && gn < P.N && gn < S.nrows_b) {
                double v = (double)sv * 3.7252902984619141e-09 /* 2^-28 */ + (double)__uint_as_float(rt[j]);
                v = ldexp(v, ea + S.b_exp[gn] - 14);
                double* dst = Tp + (long long)gm * P.ldt + gn;
                *dst = (P.accumulate || done_segs > 0) ? *dst + v : v;
              }
            }
          }
        }
        tc::fence_before_sync();
      }
      if (seg_end) ++done_segs;
    }
    __syncthreads();
    if (abort_s) {
      aborted = true;
      break;
    }
  }
  tc::cp_async_wait<0>();
  __syncthreads();
  if (aborted || abort_s) {
    if (threadIdx.x == 0) atomicExch(err, 1);
  } else if (nseg == 0 && !P.accumulate) {
    // no segment reaches this tile: its block of T is zero
    if (gm < P.M)
      for (int j = 0; j < OZ_BN; ++j) {
        int gn = n0 + j;
        if (gn < P.N) Tp[(long long)gm * P.ldt + gn] = 0.0;
      }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, OZ_TMEM_COLS);
  }
}

}  // namespace iscsi
