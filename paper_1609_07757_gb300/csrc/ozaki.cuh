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
// Tile: 128 rows of A x 64 rows of B, K step 16, OZ_STAGES-deep operand ring.
// TMEM holds level L at columns 64L .. 64L+63 (L = 0..6), so the products
// A_t x (B_u .. B_{6-t}) of one A slice land on consecutive levels and go out
// as one MMA of N = 64 (7 - t - u) columns (split at 256): 10 MMAs per K step
// instead of 28, each A slice read from shared memory once or twice.
//
// Screening: a block of 128 rows x 16 K of a tiled operand whose values all
// vanish (screened units) is never loaded or multiplied, and a block whose
// largest value lies below the row scale by 7 t bits has zero leading slices
// 0 .. t-1 whose products are skipped (ozaki_types.cuh, OzSeg).
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

// Tiled slices of an FP64 matrix, one thread per tiled row r and 8-wide K
// chunk (8 threads of consecutive rows write one 128-byte run per slice).
// X(row, k) = X[row * ld + k], or X[k * ld + row] when trans; tiled row r
// holds source row rowmap[r] (-1: zeros) if rowmap, else r (zeros beyond
// rows); tiled column k holds source column colmap[k] (-1: zeros) if colmap,
// else k (zeros beyond cols); e: exponent per source row.  out: RT-row tiles
// (RT = OZ_BM or OZ_BN) of kst k steps, rows_pad rows.  live (zero-filled by
// the caller, or null): per block the live slices, 7 - the first slice with a
// nonzero digit.
__global__ void k_oz_slice_tiled(const double* __restrict__ X, int rows, int cols, long long ld, int trans,
                                 const int* __restrict__ rowmap, const int* __restrict__ colmap,
                                 const int* __restrict__ e, __nv_bfloat16* __restrict__ out, int RT, int rows_pad,
                                 int kst, int* __restrict__ live) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int nkc = 2 * kst;
  const bool act = t < (long long)rows_pad * nkc;
  const long long grp = t >> 3;
  const int r = act ? (int)((grp / nkc) * 8 + (t & 7)) : 0;
  const int kc = act ? (int)(grp % nkc) : 0;
  int fz = OZ_S;  // first slice with a nonzero digit among this thread's 8 values
  long long blk = 0;
  if (act) {
    const int src = rowmap ? rowmap[r] : (r < rows ? r : -1);
    const int ex = src >= 0 ? e[src] : 0;
    uint32_t pk[OZ_S][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = kc * 8 + j;
      const int c = colmap ? colmap[k] : (k < cols ? k : -1);
      double x = 0.0;
      if (src >= 0 && c >= 0) x = trans ? X[(long long)c * ld + src] : X[(long long)src * ld + c];
      int a[OZ_S];
      oz_digits(x, ex, a);
#pragma unroll
      for (int sl = 0; sl < OZ_S; ++sl) {
        if (a[sl] != 0 && sl < fz) fz = sl;
        const uint32_t b = oz_digit_bits(a[sl], sl);
        if (j & 1) pk[sl][j >> 1] |= b << 16;
        else pk[sl][j >> 1] = b;
      }
    }
    blk = ((long long)(r / RT) * kst + (kc >> 1));
    __nv_bfloat16* base = out + blk * (OZ_S * RT * OZ_BK) + oz_tiled_elem(r % RT, kc * 8);
#pragma unroll
    for (int sl = 0; sl < OZ_S; ++sl)
      *reinterpret_cast<uint4*>(base + sl * RT * OZ_BK) = make_uint4(pk[sl][0], pk[sl][1], pk[sl][2], pk[sl][3]);
  }
  if (live) {
    // the 8 threads of a group share one block: reduce, then one atomic
    int m = fz;
    m = min(m, __shfl_xor_sync(0xffffffffu, m, 4));
    m = min(m, __shfl_xor_sync(0xffffffffu, m, 2));
    m = min(m, __shfl_xor_sync(0xffffffffu, m, 1));
    if (act && (t & 7) == 0 && m < OZ_S) atomicMax(live + blk, OZ_S - m);
  }
}

// One segment as seen by one output tile, held in registers (the asm
// statements' memory clobbers would otherwise reload its fields every step):
// the tile's first A and B blocks of the segment (tiled) and its rows of the
// live maps.
struct OzSegView {
  const __nv_bfloat16* a;  // tiled: block (row tile, first k step) of A, else null
  const __nv_bfloat16* b;
  const int* alive;        // live slices per k step of the tile's A / B blocks, or null
  const int* blive;
};
__device__ __forceinline__ OzSegView oz_view(const OzSeg& S, int mt, int nt) {
  OzSegView v;
  const long long ab = (long long)(S.a_rt0 + mt) * S.a_kst + S.a_ks0;
  const long long bb = (long long)(S.b_rt0 + nt) * S.b_kst + S.b_ks0;
  v.a = S.a_tiled ? S.a_tiled + ab * OZ_TA_BLOCK : nullptr;
  v.b = S.b_tiled ? S.b_tiled + bb * OZ_TB_BLOCK : nullptr;
  v.alive = S.a_live ? S.a_live + ab : nullptr;
  v.blive = S.b_live ? S.b_live + bb : nullptr;
  return v;
}

// live slices of step ks as the first live slice of each operand (tA, uB);
// the step is skipped when no product A_t B_u with t >= tA, u >= uB, t + u <= 6
// remains
__device__ __forceinline__ bool oz_step(const OzSegView& V, int ks, int& tA, int& uB) {
  tA = V.alive ? OZ_S - __ldg(V.alive + ks) : 0;
  uB = V.blive ? OZ_S - __ldg(V.blive + ks) : 0;
  return tA + uB <= OZ_S - 1;
}

// Per stage the producer leaves the step's description for the MMA thread:
// the first live slice of A (bits 0-2) and of B (bits 3-5) and flags.
constexpr uint32_t OZ_INFO_TILED = 1u << 6;        // tiled operands (no-swizzle layout), else TMA boxes
constexpr uint32_t OZ_INFO_CHUNK = 1u << 7;        // first step of a chunk
constexpr uint32_t OZ_INFO_SEG = 1u << 8;          // first step of a segment (of an item)
constexpr uint32_t OZ_INFO_END = 1u << 9;          // no step: the CTA's work is done
// Bits 16-31 hold the low 16 bits of the stage's sequence number (the CTA's
// running step count).  The MMA thread takes a description only when its stamp
// is the step it expects: the end marker's barrier phase completes on a plain
// arrival right after the word is written, and a reader that saw the phase
// before the word (stale description of the stage's previous step) issued
// that stage as a data step and then waited for a step that never came.
__device__ __forceinline__ uint32_t oz_info_seq(int g) { return ((uint32_t)g & 0xFFFFu) << 16; }

// W x W transpose (W a power of two up to 32) within each group of W lanes:
// lane i of a group holds row i of the group's block on entry and column i on
// return (butterfly exchanges over lane distances W/2, ..., 1).  The epilogue
// holds one output row per thread; after this, each store instruction writes
// runs of W consecutive doubles instead of 32 scattered 8-byte words.
template <int W>
__device__ __forceinline__ void oz_lane_transpose(double (&a)[W], int lane) {
#pragma unroll
  for (int s = W / 2; s >= 1; s >>= 1) {
    const bool hi = (lane & s) != 0;
#pragma unroll
    for (int j = 0; j < W; ++j) {
      if (j & s) continue;
      const double recv = __shfl_xor_sync(0xffffffffu, hi ? a[j] : a[j ^ s], s);
      if (hi) a[j] = recv;
      else a[j ^ s] = recv;
    }
  }
}

// Accumulators restart without a separate clearing pass: the MMA thread keeps
// a mask of the levels written since their last drain, and the first MMA that
// writes a level uses accumulate = 0 (a run of levels whose written state
// differs is split).  Levels that receive no product before they are drained
// are cleared by one MMA of zero operands.
constexpr uint32_t OZ_EXACT_MASK = (1u << OZ_EXACT) - 1;
constexpr uint32_t OZ_TAIL_MASK = ((1u << OZ_S) - 1) & ~OZ_EXACT_MASK;
constexpr uint32_t OZ_ID0 = tc::idesc_bf16_f32(OZ_BM, 0);  // N = 64 nl: add nl << 20 (N >> 3 at bit 17)

// levels [L, L + nl) from A slice t and B slices L - t .. (dA, dB: descriptors
// of slice 0 of the stage; slice t of A starts 4096 bytes, 256 in the
// descriptor's address field, after slice t - 1, slice u of B 2048, 128)
__device__ __forceinline__ void oz_run(uint32_t tmem, uint32_t& wmask, uint64_t dA, uint64_t dB, int t, int L,
                                       int nl) {
  const int e = L + nl;
  while (L < e) {
    const uint32_t w = (wmask >> L) & 1u;
    int k = L + 1;
    while (k < e && ((wmask >> k) & 1u) == w) ++k;
    tc::mma_bf16(tmem + (uint32_t)(OZ_BN * L), dA + (uint64_t)(256 * t), dB + (uint64_t)(128 * (L - t)),
                 OZ_ID0 + ((uint32_t)(k - L) << 20), w);
    wmask |= ((1u << (k - L)) - 1u) << L;
    L = k;
  }
}

// the MMAs of one K step whose levels tA .. 6 are all written already: A_t x
// B_u for t >= tA, t + u <= 6, accumulating, one MMA per run of at most four
// consecutive levels of one A slice (constant code per tA)
template <int TA, typename Mid>
__device__ __forceinline__ void oz_issue_live(uint32_t tmem, uint64_t dA, uint64_t dB, Mid&& mid) {
  int n = 0;
#pragma unroll
  for (int t = TA; t < OZ_S; ++t)
#pragma unroll
    for (int L = t; L < OZ_S; L += 4) {
      tc::mma_bf16(tmem + (uint32_t)(OZ_BN * L), dA + (uint64_t)(256 * t), dB + (uint64_t)(128 * (L - t)),
                   OZ_ID0 + ((uint32_t)(OZ_S - L < 4 ? OZ_S - L : 4) << 20), 1u);
      if (++n == 2 || (TA == OZ_S - 1 && n == 1)) mid();  // the lookahead runs among the step's MMAs
    }
}

// the MMAs of one K step in general: A_t x B_u for t >= tA, u >= uB,
// t + u <= 6 into level L = t + u (TMEM columns 64 L), runs of at most four
// levels split where the written state changes.  which: 0 every level, 1 the
// tail levels (>= OZ_EXACT) only, 2 the exact levels only.
__device__ __forceinline__ void oz_issue_general(uint32_t tmem, uint32_t& wmask, uint64_t dA, uint64_t dB, int tA,
                                              int uB, int which) {
#pragma unroll 1
  for (int t = tA; t <= OZ_S - 1 - uB; ++t) {
    const int hi = which == 2 ? OZ_EXACT - 1 : OZ_S - 1;
    int lo = t + uB;
    if (which == 1 && lo < OZ_EXACT) lo = OZ_EXACT;
    for (int L = lo; L <= hi; L += 4) oz_run(tmem, wmask, dA, dB, t, L, hi - L + 1 < 4 ? hi - L + 1 : 4);
  }
}

// one K step: constant code when every level it writes is written already;
// mid() runs once, among the step's first MMAs
template <typename Mid>
__device__ __forceinline__ void oz_issue_step(uint32_t tmem, uint32_t& wmask, uint64_t dA, uint64_t dB, int tA,
                                              int uB, Mid&& mid) {
  const uint32_t need = (OZ_EXACT_MASK | OZ_TAIL_MASK) & ~((1u << (tA + uB)) - 1u);
  if (uB == 0 && (wmask & need) == need) {
    switch (tA) {
      case 0: oz_issue_live<0>(tmem, dA, dB, mid); return;
      case 1: oz_issue_live<1>(tmem, dA, dB, mid); return;
      case 2: oz_issue_live<2>(tmem, dA, dB, mid); return;
      case 3: oz_issue_live<3>(tmem, dA, dB, mid); return;
      case 4: oz_issue_live<4>(tmem, dA, dB, mid); return;
      case 5: oz_issue_live<5>(tmem, dA, dB, mid); return;
      default: oz_issue_live<6>(tmem, dA, dB, mid); return;
    }
  }
  mid();
  oz_issue_general(tmem, wmask, dA, dB, tA, uB, 0);
}

// the levels of `levels` not written since their last drain are cleared
// (one MMA of zero operands each), so the epilogue reads zero there
__device__ __forceinline__ void oz_clear_unwritten(uint32_t tmem, uint32_t& wmask, uint32_t levels, uint64_t dzA,
                                                   uint64_t dzB) {
  uint32_t m = levels & ~wmask;
  while (m) {
    const int L = __ffs(m) - 1;
    tc::mma_bf16(tmem + (uint32_t)(OZ_BN * L), dzA, dzB, OZ_ID0 + (1u << 20), 0u);
    m &= m - 1;
  }
  wmask |= levels;
}

// Persistent warp-specialised product kernel: CTA b runs the work items
// [cta_start[b], cta_start[b + 1]) of a host-built schedule in order (output
// tiles of 128 x 64, whole or as split-K parts; see OzItem).  Per CTA:
//   warp 0     (one lane) loads the live slices of every issued K step into an
//              OZ_STAGES-deep ring (tiled segments: one bulk copy per operand;
//              others: two TMA boxes), completion as transaction bytes on
//              full[stage];
//   warp 1     (one lane) waits full[stage], reads the step's description
//              that the producer left with it, issues the step's MMAs (the
//              first write of a level after its drain does not accumulate),
//              releases the stage through tcgen05.commit -> empty[stage] and
//              closes every 32 issued steps of a segment (a K chunk, over
//              which the exact levels cannot overflow) with chunk_b; before
//              the exact-level MMAs of a chunk it waits for the drain of the
//              previous one (free_b), issuing the tail-level MMAs first
//              when the previous chunk belongs to the same segment;
//   warps 2-9  per chunk drain the exact levels into
//              int64 sums (one output row per thread; warps w and w + 4
//              share TMEM lane quarter w % 4 and take half of the columns
//              each), release the accumulators (free_b)
//              and, after a segment's last chunk, form its FP64 result
//              2^(ea + eb - 14) (S 2^-28 + tail) and add it into T or into the
//              item's split-K slot.
// Every wait is bounded; a wait that runs out sets abort (all roles stop),
// the kernel waits (bounded) for its copies in flight, frees TMEM and
// reports through err.
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_oz_gemm(const OzProblem* __restrict__ probs, const OzSeg* __restrict__ segs, const OzMaps* __restrict__ maps,
              const OzItem* __restrict__ items, const int* __restrict__ cta_start, double* tbase,
              double* const* __restrict__ tbases, double* __restrict__ ws, int* __restrict__ ws_cnt,
              int* __restrict__ err) {
  extern __shared__ unsigned char oz_smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t s_stage0 = tc::smem_u32(smem);
  __shared__ uint64_t full_b[OZ_STAGES], empty_b[OZ_STAGES], chunk_b, free_b, drain_b, epi_b;
  __shared__ uint32_t tmem_s;
  __shared__ volatile int abort_s;
  __shared__ int last_s;
  __shared__ uint32_t info_s[OZ_STAGES];  // the step each stage holds (producer -> MMA thread)

  const int it0 = cta_start[blockIdx.x], it1 = cta_start[blockIdx.x + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int SPC = OZ_CHUNK / OZ_BK;  // issued steps per chunk

  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      tc::mbar_init(tc::smem_u32(&full_b[s]), 1);
      tc::mbar_init(tc::smem_u32(&empty_b[s]), 1);
    }
    tc::mbar_init(tc::smem_u32(&chunk_b), 1);
    tc::mbar_init(tc::smem_u32(&free_b), 32 * OZ_EPI_WARPS);
    tc::mbar_init(tc::smem_u32(&drain_b), 1);
    tc::mbar_init(tc::smem_u32(&epi_b), 32 * OZ_EPI_WARPS);
    abort_s = 0;
    tc::fence_mbar_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tc::smem_u32(&tmem_s), OZ_TMEM_COLS);
    tc::tmem_relinquish();
  }
  if (warp >= 2) {
    // zero operands of the clearing MMAs, visible to the tensor core
    uint4* z = reinterpret_cast<uint4*>(smem + OZ_STAGES * OZ_STAGE_BYTES);
    for (int i = threadIdx.x - 64; i < OZ_ZERO_BYTES / 16; i += 32 * OZ_EPI_WARPS) z[i] = make_uint4(0u, 0u, 0u, 0u);
    tc::fence_proxy_async();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_s;

  // a wait that runs out records where (oz_wait_code) and stops every role
  auto wait = [&](uint64_t* bar, uint32_t parity, int site, int detail) -> bool {
    return oz_wait_bounded(bar, parity, site, detail, &abort_s, OZ_SPIN);
  };

  if (warp == 0) {
    // ---------------- producer
    if (lane == 0) {
      int g = 0;
      bool ok = true;
      for (int it = it0; it < it1 && ok; ++it) {
        const OzItem I = items[it];
        const OzProblem& P = probs[I.prob];
        const int m0 = I.mt * OZ_BM, n0 = I.nt * OZ_BN;
        int cstep = 0;
        for (int gs = 0; gs < P.seg_count && ok; ++gs) {
          const OzSeg& S = segs[P.seg_begin + gs];
          const int nst = S.K / OZ_BK;
          const int lo = I.s0 - cstep > 0 ? I.s0 - cstep : 0, hi = I.s1 - cstep < nst ? I.s1 - cstep : nst;
          cstep += nst;
          if (lo >= hi || n0 >= S.nrows_b) continue;
          const OzSegView V = oz_view(S, I.mt, I.nt);
          const CUtensorMap* ma = &maps[P.seg_begin + gs].a;
          const CUtensorMap* mb = &maps[P.seg_begin + gs].b;
          const int ax = S.a_k0, ay = S.a_row0 + m0, bx = S.b_k0, by = S.b_row0 + n0;
          int j = 0;  // issued steps of this segment in this item
          for (int ks = lo; ks < hi; ++ks) {
            int tA, uB;
            if (!oz_step(V, ks, tA, uB)) continue;
            const int st = g % OZ_STAGES;
            if (g >= OZ_STAGES && !wait(&empty_b[st], ((g / OZ_STAGES) - 1) & 1, OZ_SITE_EMPTY, it)) {
              ok = false;
              break;
            }
            info_s[st] = oz_info_seq(g) | (uint32_t)tA | ((uint32_t)uB << 3) | (V.a ? OZ_INFO_TILED : 0u) |
                         (j % SPC == 0 ? OZ_INFO_CHUNK : 0u) | (j == 0 ? OZ_INFO_SEG : 0u);
            ++j;
            const uint32_t fb = tc::smem_u32(&full_b[st]);
            const uint32_t sa = s_stage0 + st * OZ_STAGE_BYTES;
            const uint32_t sb = sa + OZ_S * OZ_A_SLICE_BYTES;
            if (V.a) {
              const int m = OZ_S - tA - uB;  // live slices of each operand
              const uint32_t abytes = (uint32_t)m * OZ_A_SLICE_BYTES, bbytes = (uint32_t)m * OZ_B_SLICE_BYTES;
              tc::mbar_arrive_expect_tx(fb, abytes + bbytes);
              tc::bulk_load(sa + tA * OZ_A_SLICE_BYTES, V.a + (long long)ks * OZ_TA_BLOCK + tA * (OZ_BM * OZ_BK),
                            abytes, fb);
              tc::bulk_load(sb + uB * OZ_B_SLICE_BYTES, V.b + (long long)ks * OZ_TB_BLOCK + uB * (OZ_BN * OZ_BK),
                            bbytes, fb);
            } else {
              tc::mbar_arrive_expect_tx(fb, OZ_STAGE_BYTES);
              tc::tma_load_3d(sa, ma, ax + ks * OZ_BK, ay, 0, fb);
              tc::tma_load_3d(sb, mb, bx + ks * OZ_BK, by, 0, fb);
            }
            ++g;
          }
        }
      }
      if (ok) {
        // the end marker: a stage without data
        const int st = g % OZ_STAGES;
        if (g < OZ_STAGES || wait(&empty_b[st], ((g / OZ_STAGES) - 1) & 1, OZ_SITE_EMPTY_END, g)) {
          info_s[st] = oz_info_seq(g) | OZ_INFO_END;
          __threadfence_block();
          tc::mbar_arrive(tc::smem_u32(&full_b[st]));
          ++g;
        }
      }
      // copies still in flight (only after an abort) must land before the
      // CTA's shared memory is released: wait for the last phase of each stage
      for (int q = g - OZ_STAGES > 0 ? g - OZ_STAGES : 0; q < g; ++q)
        tc::mbar_wait_bounded(tc::smem_u32(&full_b[q % OZ_STAGES]), (q / OZ_STAGES) & 1, OZ_SPIN);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: the producer's stage descriptions drive it.
    // Any shared-memory access of this thread waits behind the tensor core's
    // operand reads (~140 cycles), long enough to empty the MMA queue, so the
    // next stage's readiness test and description and the release of the
    // previous stage are issued among the current step's MMAs (lookahead).
    if (lane == 0) {
      const uint32_t sz = s_stage0 + OZ_STAGES * OZ_STAGE_BYTES;  // zero operands
      const uint64_t dzA = tc::smem_desc(sz, 128, 256), dzB = tc::smem_desc(sz + OZ_A_SLICE_BYTES, 128, 256);
      int g = 0, chunk = 0;
      bool open = false;   // MMAs issued since the last chunk commit
      uint32_t wmask = 0;  // levels written since their last drain
      volatile uint32_t* vinfo = info_s;
      // the description of step `step` from its stage, once its stamp says so
      // (bounded re-reads)
      auto take = [&](int stage, int step, uint32_t& out) -> bool {
        const uint32_t want = oz_info_seq(step);
        for (long long i = 0; i < OZ_SPIN; ++i) {
          const uint32_t v = vinfo[stage];
          if ((v & 0xFFFF0000u) == want) {
            out = v;
            return true;
          }
          if ((i & 1023) == 1023 && abort_s) return false;
        }
        atomicCAS((int*)&abort_s, 0, oz_wait_code(OZ_SITE_INFO, step));
        return false;
      };
      uint32_t info = 0;
      bool ok = wait(&full_b[0], 0, OZ_SITE_FULL, 0);
      if (ok) {
        tc::fence_after_sync();
        ok = take(0, 0, info);
      }
      while (ok) {
        const int st = g % OZ_STAGES;
        if (open && (info & (OZ_INFO_CHUNK | OZ_INFO_END))) {
          // the previous chunk is complete (with its segment's tail levels
          // when a new segment follows or the work ends)
          oz_clear_unwritten(tmem, wmask,
                             (info & (OZ_INFO_SEG | OZ_INFO_END)) ? (OZ_EXACT_MASK | OZ_TAIL_MASK) : OZ_EXACT_MASK,
                             dzA, dzB);
          tc::mma_commit(tc::smem_u32(&chunk_b));
          ++chunk;
          open = false;
        }
        if (info & OZ_INFO_END) break;
        const int tA = (int)(info & 7u), uB = (int)((info >> 3) & 7u);
        const uint32_t sa = s_stage0 + st * OZ_STAGE_BYTES;
        const uint32_t sb = sa + OZ_S * OZ_A_SLICE_BYTES;
        const bool tiled = (info & OZ_INFO_TILED) != 0;
        const uint64_t dA = tiled ? tc::smem_desc(sa, 128, 256) : tc::smem_desc_sw32(sa);
        const uint64_t dB = tiled ? tc::smem_desc(sb, 128, 256) : tc::smem_desc_sw32(sb);
        const int gn = g + 1, stn = gn % OZ_STAGES;
        const uint32_t pn = (uint32_t)(gn / OZ_STAGES) & 1u;
        uint32_t ready = 0, info_n = 0;
        auto mid = [&]() {
          // the previous stage is released once the MMAs issued so far are done
          if (g > 0) tc::mma_commit(tc::smem_u32(&empty_b[(g - 1) % OZ_STAGES]));
          ready = tc::mbar_test_wait(tc::smem_u32(&full_b[stn]), pn);
          info_n = vinfo[stn];  // used when ready (read after the acquiring test) and stamped gn
          if ((info_n & 0xFFFF0000u) != oz_info_seq(gn)) ready = 0;
        };
        if (info & OZ_INFO_CHUNK) {
          // the exact levels restart once the epilogue has drained the
          // previous chunk; the tail levels run across the chunks of a
          // segment and go first, unless the segment starts here and the
          // epilogue still reads the previous segment's tail
          const bool seg = (info & OZ_INFO_SEG) != 0;
          mid();
          if (!seg) oz_issue_general(tmem, wmask, dA, dB, tA, uB, 1);
          if (!wait(&free_b, chunk & 1, OZ_SITE_FREE, chunk)) break;
          tc::fence_after_sync();
          wmask &= seg ? 0u : ~OZ_EXACT_MASK;
          oz_issue_general(tmem, wmask, dA, dB, tA, uB, seg ? 0 : 2);
        } else {
          oz_issue_step(tmem, wmask, dA, dB, tA, uB, mid);
        }
        open = true;
        g = gn;
        if (!ready) {
          if (!wait(&full_b[stn], pn, OZ_SITE_FULL, gn)) break;
          if (!take(stn, gn, info_n)) break;
        }
        tc::fence_after_sync();
        info = info_n;
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
    const int cbase = ((warp - 2) >> 2) * OZ_EPI_COLS;  // first column of this warp
    const uint32_t lane_base = ((uint32_t)(quarter * 32) << 16) + (uint32_t)cbase;
    // the accumulators are free from the start (the MMA thread's first
    // writes overwrite them)
    tc::mbar_arrive(tc::smem_u32(&free_b));
    long long sums[OZ_EPI_COLS];
    // the segment's tail levels wait in TMEM's spare columns (OZ_S * OZ_BN on)
    // between the drain and the finalization, not in registers
    const uint32_t tail_base = tmem + lane_base + OZ_S * OZ_BN;
#pragma unroll
    for (int j = 0; j < OZ_EPI_COLS; ++j) sums[j] = 0;
    int chunk = 0, epi_phase = 0;
    bool ok = true;
    // all epilogue threads meet (bounded, unlike a named barrier, so an abort cannot hang it)
    auto epi_sync = [&]() -> bool {
      tc::mbar_arrive(tc::smem_u32(&epi_b));
      const int ph = epi_phase++;
      return wait(&epi_b, ph & 1, OZ_SITE_EPI_SYNC, ph);
    };
    for (int it = it0; it < it1 && ok; ++it) {
      const OzItem I = items[it];
      const OzProblem& P = probs[I.prob];
      const int m0 = I.mt * OZ_BM, n0 = I.nt * OZ_BN;
      const int gm = m0 + row;
      double* const Tp = P.t_rel ? (tbases ? tbases[P.tb] : tbase) + P.t : reinterpret_cast<double*>(P.t);
      // destination of this item's sum: T itself, or the part's block of the split-K slot
      double* const part_base = I.nparts > 1 ? ws + ((long long)I.slot + I.part) * (OZ_BM * OZ_BN) : nullptr;
      bool wrote = false;
      int cstep = 0;
      for (int gs = 0; gs < P.seg_count && ok; ++gs) {
        const OzSeg& S = segs[P.seg_begin + gs];
        const int nst = S.K / OZ_BK;
        const int lo = I.s0 - cstep > 0 ? I.s0 - cstep : 0, hi = I.s1 - cstep < nst ? I.s1 - cstep : nst;
        cstep += nst;
        if (lo >= hi || n0 >= S.nrows_b) continue;
        // issued steps of this segment (the lanes split the steps)
        const OzSegView V = oz_view(S, I.mt, I.nt);
        int niss = 0;
        for (int ks = lo + lane; ks < hi; ks += 32) {
          int tA, uB;
          niss += oz_step(V, ks, tA, uB) ? 1 : 0;
        }
        niss = __reduce_add_sync(0xffffffffu, niss);
        const int nch = (niss + SPC - 1) / SPC;
        for (int ch = 0; ch < nch; ++ch, ++chunk) {
          // warp-uniform decision: tcgen05.ld below is warp-collective
          const bool w_ok = wait(&chunk_b, chunk & 1, OZ_SITE_CHUNK, chunk);
          if (!__all_sync(0xffffffffu, w_ok)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const bool last = ch == nch - 1;
#pragma unroll
          for (int c0 = 0; c0 < OZ_EPI_COLS; c0 += 4) {
            uint32_t r0[4], r1[4], r2[4], r3[4], r4[4];
            tc::tmem_ld4(tmem + lane_base + 0 * OZ_BN + c0, r0);
            tc::tmem_ld4(tmem + lane_base + 1 * OZ_BN + c0, r1);
            tc::tmem_ld4(tmem + lane_base + 2 * OZ_BN + c0, r2);
            tc::tmem_ld4(tmem + lane_base + 3 * OZ_BN + c0, r3);
            tc::tmem_ld4(tmem + lane_base + 4 * OZ_BN + c0, r4);
            tc::tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 4; ++j) {
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
          if (last) {
            // the segment's tail levels (read after the exact ones: fewer live registers)
#pragma unroll
            for (int c0 = 0; c0 < OZ_EPI_COLS; c0 += 8) {
              uint32_t r5[8], r6[8];
              tc::tmem_ld8(tmem + lane_base + OZ_EXACT * OZ_BN + c0, r5);
              tc::tmem_ld8(tmem + lane_base + (OZ_EXACT + 1) * OZ_BN + c0, r6);
              tc::tmem_wait_ld();
#pragma unroll
              for (int j = 0; j < 8; ++j) r5[j] = __float_as_uint(__uint_as_float(r5[j]) + __uint_as_float(r6[j]));
              tc::tmem_st8(tail_base + c0, r5);
            }
            tc::tmem_wait_st();
          }
          tc::fence_before_sync();
          tc::mbar_arrive(tc::smem_u32(&free_b));
          if (last) {
            // this segment's result 2^(ea+eb-14) (S 2^-28 + tail), after the
            // accumulators are released (the MMAs of the next chunk run
            // meanwhile).  Everything read from global memory is loaded into
            // registers first, eight columns at a time: the stores below could
            // alias it, and a chain of dependent reloads would cost far longer
            // than the chunks of MMAs it overlaps.  A split tile's part block
            // is column-major (the 32 rows of a warp are one contiguous run per
            // column), so the part's writes and the combining reads coalesce.
            const int Mp = P.M, Np = P.N, nrb = S.nrows_b;
            const long long ldt = P.ldt;
            const bool addT = P.accumulate || wrote;
            const int* __restrict__ bexp = S.b_exp;
            const int ea = gm < Mp ? __ldg(S.a_exp + gm) : 0;
            double* const rowT = part_base ? part_base + cbase * OZ_BM + row : Tp + (long long)gm * ldt;
#pragma unroll
            for (int c0 = 0; c0 < OZ_EPI_COLS; c0 += 8) {
              uint32_t tl[8];
              tc::tmem_ld8(tail_base + c0, tl);
              int eb[8];
              double old[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int gn = n0 + cbase + c0 + j;
                const bool in = gm < Mp && gn < Np && gn < nrb;
                eb[j] = in ? __ldg(bexp + gn) : 0;
                old[j] = 0.0;
                if (part_base) {
                  if (wrote) old[j] = rowT[(c0 + j) * OZ_BM];
                } else if (in && addT) {
                  old[j] = rowT[gn];
                }
              }
              tc::tmem_wait_ld();
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int gn = n0 + cbase + c0 + j;
                const bool in = gm < Mp && gn < Np && gn < nrb;
                double v = 0.0;
                if (in) {
                  // S 2^-28 + tail, the tail rounded to S's unit (2^-43 of the
                  // largest single product: below the slices' own error)
                  const long long q =
                      sums[c0 + j] + __float2ll_rn(__uint_as_float(tl[j]) * 268435456.0f /* 2^28 */);
                  v = oz_i64_scaled(q, ea + eb[j] - 14 - 28);
                }
                if (part_base) rowT[(c0 + j) * OZ_BM] = old[j] + v;
                else if (in) rowT[gn] = old[j] + v;
                sums[c0 + j] = 0;
              }
            }
            wrote = true;
          }
        }
      }
      if (!ok) break;
      if (!wrote) {
        // no step of this item survived: its part (or tile) is zero
        for (int j = 0; j < OZ_EPI_COLS; ++j) {
          const int gn = n0 + cbase + j;
          if (part_base) part_base[(cbase + j) * OZ_BM + row] = 0.0;
          else if (!P.accumulate && gm < P.M && gn < P.N) Tp[(long long)gm * P.ldt + gn] = 0.0;
        }
      }
      if (part_base) {
        // split K: the last part to finish adds all parts in order into T
        __threadfence();
        if (!epi_sync()) break;
        if (threadIdx.x == 64) last_s = atomicAdd(ws_cnt + I.cnt, 1) == I.nparts - 1;
        if (!epi_sync()) break;
        // every thread reads last_s before any reaches the next item's first epi_sync
        if (last_s) {
          // parts summed in part order (the result does not depend on which
          // part finished last), eight columns at a time, then turned across
          // the lane octets for row-major runs in T
          __threadfence();
          const double* slot = ws + (long long)I.slot * (OZ_BM * OZ_BN);
          const int rb = m0 + quarter * 32 + (lane & ~7);
#pragma unroll
          for (int c0 = 0; c0 < OZ_EPI_COLS; c0 += 8) {
            double v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = 0.0;
#pragma unroll 2
            for (int q = 0; q < I.nparts; ++q) {
              const double* src = slot + (long long)q * (OZ_BM * OZ_BN) + (cbase + c0) * OZ_BM + row;
#pragma unroll
              for (int j = 0; j < 8; ++j) v[j] += __ldcg(src + j * OZ_BM);
            }
            oz_lane_transpose<8>(v, lane);  // v[k]: row rb + k, column gnt
            const int gnt = n0 + cbase + c0 + (lane & 7);
            const bool cin = gnt < P.N;
            double old[8];
#pragma unroll
            for (int k = 0; k < 8; ++k)
              old[k] = P.accumulate && cin && rb + k < P.M ? Tp[(long long)(rb + k) * P.ldt + gnt] : 0.0;
#pragma unroll
            for (int k = 0; k < 8; ++k)
              if (cin && rb + k < P.M) Tp[(long long)(rb + k) * P.ldt + gnt] = old[k] + v[k];
          }
          if (threadIdx.x == 64) ws_cnt[I.cnt] = 0;  // ready for the next launch
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
    tc::tmem_dealloc(tmem, OZ_TMEM_COLS);
  }
}

}  // namespace iscsi
