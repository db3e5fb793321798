// ozaki_types.cuh -- constants and work-list records of the tensor-core
// FP64-accurate contraction (kernels in ozaki.cuh).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "tc_ptx.cuh"

namespace iscsi {

constexpr int OZ_S = 7;            // slices per operand
constexpr int OZ_BITS = 7;         // bits per slice
constexpr int OZ_EXACT = 5;        // levels flushed exactly per chunk
constexpr int OZ_BM = 128;         // rows of A per tile
constexpr int OZ_BN = 64;          // rows of B per tile
constexpr int OZ_BK = 16;          // K per stage (one MMA)
constexpr int OZ_STAGES = 5;       // 215 KB of operand ring (4: 2-3 % slower)
constexpr int OZ_CHUNK = 512;      // K per exact flush
constexpr int OZ_EPI_WARPS = 8;    // two per TMEM lane quarter, half the columns each: the
                                   // exact levels drain twice as fast (the MMA warp waits for
                                   // that drain at every chunk); 4: -7 %, 16: -1 % (register spills)
constexpr int OZ_EPI_COLS = OZ_BN / (OZ_EPI_WARPS / 4);
constexpr int OZ_THREADS = 64 + 32 * OZ_EPI_WARPS;  // warp 0 loads (TMA), warp 1 issues MMAs, the rest drain TMEM
constexpr int OZ_A_SLICE_BYTES = OZ_BM * OZ_BK * 2;   // 4096
constexpr int OZ_B_SLICE_BYTES = OZ_BN * OZ_BK * 2;   // 2048
constexpr int OZ_STAGE_BYTES = OZ_S * (OZ_A_SLICE_BYTES + OZ_B_SLICE_BYTES);
constexpr int OZ_ZERO_BYTES = OZ_A_SLICE_BYTES + OZ_B_SLICE_BYTES;  // zero operands (clearing MMAs)
constexpr int OZ_SMEM_BYTES = OZ_STAGES * OZ_STAGE_BYTES + OZ_ZERO_BYTES + 1024;
constexpr int OZ_TMEM_COLS = 512;  // 7 levels x 64 columns used
constexpr long long OZ_SPIN = 1ll << 24;
// Where a bounded wait of the contraction kernels ran out, as the error word
// they leave: bits 0-2 the wait (OZ_SITE_*), bits 3-18 the role's position
// (item, stage or chunk count, low 16 bits), bits 19-30 the CTA.
constexpr int OZ_SITE_EMPTY = 1;      // producer: a stage's release (the item in the CTA's list)
constexpr int OZ_SITE_EMPTY_END = 2;  // producer: the stage of the end marker (stages filled)
constexpr int OZ_SITE_FULL = 3;       // MMA thread: a stage's data (stages consumed)
constexpr int OZ_SITE_FREE = 4;       // MMA thread: the accumulators' drain (chunks closed)
constexpr int OZ_SITE_CHUNK = 5;      // epilogue: a chunk's products (chunks drained)
constexpr int OZ_SITE_EPI_SYNC = 6;   // epilogue: the split-K meeting (meetings passed)
constexpr int OZ_SITE_INFO = 7;       // MMA thread: a stage's description (stages consumed)
constexpr int OZ_WAIT_CTA = 1 << 19;
__host__ __device__ constexpr int oz_wait_code(int site, int detail) { return site | ((detail & 0xFFFF) << 3); }

// The bounded wait of the contraction kernels: polls the phase of `parity` at
// most `limit` times; every 1024 polls it looks at the CTA's abort word, and a
// wait that runs out stores its code there (the first one wins), so that every
// role stops and the kernel reports through its error word.
__device__ __forceinline__ bool oz_wait_bounded(uint64_t* bar, uint32_t parity, int site, int detail,
                                                volatile int* abort_word, long long limit) {
  const uint32_t a = tc::smem_u32(bar);
  for (long long i = 0; i < limit; ++i) {
    if (tc::mbar_try_wait(a, parity)) return true;
    if ((i & 1023) == 1023 && *abort_word) return false;
  }
  atomicCAS((int*)abort_word, 0, oz_wait_code(site, detail));
  return false;
}

constexpr int OZ_MAX_SEGS = 8;
constexpr int OZ_BW_ROWS = 128;    // rows of B per 128-column tile; B arrays are padded to this

// Tiled operand arrays (the FP64-accurate contraction's own layout).  An
// array of R-row tiles (R = OZ_BM for an A operand, OZ_BN for a B operand) and
// K steps of 16 is stored block by block, block (row tile rt, k step ks) at
// element (rt * kst + ks) * OZ_S * R * 16, so that all slices of one tile and
// K step are one contiguous run that a single bulk copy brings into shared
// memory.  Inside a block, slice s starts at s * R * 16 and element (r, k)
// sits in the tensor core's no-swizzle K-major layout of 8-row x 16-byte core
// matrices: core matrix (r / 8, k / 8) at 128 bytes * (2 (r / 8) + k / 8),
// row r % 8 at 16 bytes within it (descriptor: K-adjacent core matrices 128
// bytes apart, row groups 256 bytes apart).  Consecutive slices of a B block
// then read as one operand of 64 (levels) rows, which the MMA's N extent
// spans.
constexpr int OZ_TA_BLOCK = OZ_S * OZ_BM * OZ_BK;  // elements of one A block (28 KB)
constexpr int OZ_TB_BLOCK = OZ_S * OZ_BN * OZ_BK;  // elements of one B block (14 KB)
__host__ __device__ constexpr int oz_tiled_elem(int r, int k) {
  return (((r >> 3) << 1) + ((k & 15) >> 3)) * 64 + ((r & 7) << 3) + (k & 7);
}

// One operand pair of a product: A[M][K] and B[N][K].  Two sources:
//  * tiled (a_tiled != nullptr): both operands are tiled arrays; the segment
//    starts at row tile a_rt0 / b_rt0 and k step a_ks0 / b_ks0 of its arrays,
//    whose rows hold kst k steps each; a_live / b_live (or null: all live)
//    give per block the number of live slices, 7 - (the first slice with a
//    nonzero digit anywhere in the block): 0 marks a block whose values all
//    vanish (screened units, zero rows), and the products of its leading
//    zero slices are skipped;
//  * TMA (a_tiled == nullptr): K-major slice arrays [S][rows][ld] read through
//    the tensor maps of the segment (OzMaps), block (a_row0, a_k0) of A's and
//    (b_row0, b_k0) of B's; k offsets are multiples of 16; arrays are zero
//    padded so that tiles need no bounds checks (A rows to a multiple of 128,
//    B rows to 64, K to 16).
// Rows of B at or beyond nrows_b contribute nothing (tiles wholly beyond are
// skipped).
struct OzSeg {
  const int* a_exp;  // row exponents of A (index = problem row)
  const int* b_exp;  // row exponents of B (index = problem column)
  int a_row0, a_k0, b_row0, b_k0;
  int K;             // multiple of 16
  int nrows_b;       // valid rows of B
  const __nv_bfloat16* a_tiled;
  const __nv_bfloat16* b_tiled;
  const int* a_live;
  const int* b_live;
  int a_kst, b_kst;
  int a_rt0, a_ks0, b_rt0, b_ks0;
};

// TMA descriptors of a segment's two slice arrays: dims (ld, rows, S), box
// (16, 128 or 64, S), 32-byte swizzle.  Kept in global memory beside the
// segment list (one entry per segment; unused for tiled segments).
struct OzMaps {
  CUtensorMap a, b;
  CUtensorMap bw;  // B in boxes of 16 x OZ_BW_ROWS rows x all slices (128-column tiles, tc32w.cuh)
};

// T[M][N] (FP64, ldt) (+)= sum over segments of A_seg B_seg^T; T is the
// device pointer t, or base + t when t_rel, base being the launch's tbase
// argument or, in a launch over several contexts, tbases[tb] (so problem
// lists survive new output vectors)
struct OzProblem {
  long long t;
  int t_rel;
  int tb;
  long long ldt;
  int M, N;
  int seg_begin, seg_count;
  int tiles_n, tile_begin;
  int accumulate;  // 1: add to T, 0: overwrite with the first segment
};

// One work item of the persistent contraction: the output tile (mt, nt) of
// problem prob over the K steps [s0, s1) of its segments taken in order.  A
// tile cut into nparts > 1 items (split K) leaves part p's FP64 result in
// workspace block slot + p (128 x 64 doubles each, column-major); the part that raises
// counter cnt to nparts adds the blocks in part order into T and resets it.
struct OzItem {
  int prob, mt, nt;
  int s0, s1;
  int part, nparts, slot, cnt;
};

}  // namespace iscsi
