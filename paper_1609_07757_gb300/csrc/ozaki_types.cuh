// ozaki_types.cuh -- constants and work-list records of the tensor-core
// FP64-accurate contraction (kernels in ozaki.cuh).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

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
constexpr int OZ_SMEM_BYTES = OZ_STAGES * OZ_STAGE_BYTES + 1024;
constexpr int OZ_TMEM_COLS = 512;  // 7 levels x 64 columns used
constexpr long long OZ_SPIN = 1ll << 24;

constexpr int OZ_MAX_SEGS = 8;
constexpr int OZ_BW_ROWS = 128;    // rows of B per 128-column tile; B arrays are padded to this

// One operand pair of a product: A[M][K] and B[N][K], both read through TMA
// from K-major slice arrays [S][rows][ld] (bf16).  The segment's block starts
// at (a_row0, a_k0) in A's array and (b_row0, b_k0) in B's; k offsets are
// multiples of 16.  Slice arrays are zero padded so that tiles need no bounds
// checks: A rows to the tile multiple of 128, B rows to the multiple of 64, K
// to a multiple of 16.  Rows of B at or beyond nrows_b contribute nothing
// (tiles wholly beyond are skipped).
struct OzSeg {
  const int* a_exp;  // row exponents of A (index = problem row)
  const int* b_exp;  // row exponents of B (index = problem column)
  int a_row0, a_k0, b_row0, b_k0;
  int K;             // multiple of 16
  int nrows_b;       // valid rows of B
};

// TMA descriptors of a segment's two slice arrays: dims (ld, rows, S), box
// (16, 128 or 64, S), 32-byte swizzle.  Kept in global memory beside the
// segment list (one entry per segment).
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

}  // namespace iscsi
