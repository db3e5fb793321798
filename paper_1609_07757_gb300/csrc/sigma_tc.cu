// sigma_tc.cu -- the FP64 sigma step's contractions on the tensor cores
// (tcgen05), with FP64 accuracy from exact bf16 slices (ozaki.cuh).
//
// Opposite spin, per sigma call and column level class c:
//   k_oz_lift_tiled : per column (X,Y,v), Ct^T[(X,Y,v)][(q,s)] = s s c[X u q, Y u s]
//                     gathered through the contraction/addition tables, the
//                     column's exponent, and its 7 exact bf16 slices (the B
//                     operand, tiled: ozaki_types.cuh)
//   k_oz_gemm       : T_c = G[:M_c, :K_c] Ct_c for all classes, one persistent
//                     launch (schedule: oz_schedule.cu)
// Same spin, per excitation-level block a of the CI vector (rows = alpha
// strings of level a, columns = the allowed beta prefix):
//   sigma_a += sum_a' M_alpha[a, a'] C_a'   (A = M_alpha slices, B = C_a'^T)
//            + C_a M_beta^T                 (A = C_a slices, B = M_beta slices)
// as one multi-segment product per block; blocks with at most 16 rows or
// columns stay on the FP64 thin kernels of sigma.cu.
// G's, M_alpha's and M_beta's slices are built once per context (first use),
// with a live-slice map per block: blocks of screened (zero) units are never
// loaded, and leading zero slices are not multiplied.
//
// The FP32 form (tc32.cuh) runs the same two contractions with three bf16
// terms per element and FP32 accumulation (k_tc32w_gemm): no exponents, no
// exact levels; its operands come from the FP32 copy of the CI vector.
#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "ozaki.cuh"
#include "tc32.cuh"
#include "tc32w.cuh"
#include "tma_map.h"

namespace iscsi {

struct TcClass {
  int mrows;        // rows of T_c
  int ncols;        // hole pairs x vectors
  int krows;        // K of the class
  int kpad;         // krows rounded up to 16
  int npad;         // ncols rounded up to 64
  int hp_start;     // first hole pair of the class in hp_inv
  long long bs_off; // element offset of the class's slices in the B buffer (slice 0)
  long long exp_off;
  long long tot;    // ncols * kpad (elements gathered)
  int wpc;          // warps per column in the tiled lift (1, 2, 4 or 8; the block's 8 warps)
};

struct TcTable {
  int nclass;
  int nvec;
  TcClass c[2 * kMaxElec];
  long long start[2 * kMaxElec + 1];  // flattened (col, k) element offsets
  int col_start[2 * kMaxElec + 1];    // first column of each class over all classes
  int blk_start[2 * kMaxElec + 1];    // first block of each class in the tiled lift (8 / wpc columns each)
};

static inline int round_up(int x, int m) { return (x + m - 1) / m * m; }


// A column (X, Y, v) of Ct^T: its lift entries for every orbital (a+_q |X> and
// a+_s |Y>: target string and sign, and the target alpha string's offset and
// allowed beta count) are staged in shared memory first, so an element (q, s)
// costs the pair table and c.
struct OzLiftCol {
  int a[kMaxOrb], b[kMaxOrb], lim[kMaxOrb];
  long long off[kMaxOrb];
};

// the same entries laid out for n orbitals (off[n], then a[n], b[n], lim[n]),
// as the tiled lift stages them in dynamic shared memory
struct OzLiftView {
  long long* off;
  int *a, *b, *lim;
};
__device__ __forceinline__ OzLiftView oz_lift_view(unsigned char* base, int n) {
  OzLiftView v;
  v.off = reinterpret_cast<long long*>(base);
  v.a = reinterpret_cast<int*>(base + 8 * n);
  v.b = v.a + n;
  v.lim = v.b + n;
  return v;
}
__host__ __device__ constexpr int oz_lift_col_bytes(int n) { return (20 * n + 7) / 8 * 8; }

template <typename V, typename Tab>
__device__ __forceinline__ V oz_lift_value(const Tab& L, const TcClass& C, int k,
                                           const int* __restrict__ pair_split, const V* __restrict__ cv) {
  if (k >= C.krows) return (V)0;
  const int qs = __ldg(pair_split + k);
  const int q = qs >> 16, s = qs & 0xFFFF;
  const int ea = L.a[q], eb = L.b[s];
  if (ea < 0 || eb < 0) return (V)0;
  const int Bp = eb >> 1;
  if (Bp >= L.lim[q]) return (V)0;
  const V x = cv[L.off[q] + Bp];
  return ((ea ^ eb) & 1) ? -x : x;
}

// the column (X, Y, v) of block blockIdx.x: class, local column, staged lift entries
__device__ __forceinline__ int oz_stage_column(const TcTable& tt, int n, int nholeA, int nholeB,
                                               const int* __restrict__ hp_inv, const int* __restrict__ liftA,
                                               const int* __restrict__ liftB, const int8_t* __restrict__ alevel,
                                               const int* __restrict__ nballow, const long long* __restrict__ off,
                                               OzLiftCol& L, int& col, int& vv) {
  int cl = 0;
  while ((int)blockIdx.x >= tt.col_start[cl + 1]) ++cl;
  const TcClass& C = tt.c[cl];
  col = (int)blockIdx.x - tt.col_start[cl];
  const int hp = col / tt.nvec;
  vv = col - hp * tt.nvec;
  const int xy = hp_inv[C.hp_start + hp];
  const int X = xy / nholeB, Y = xy - (xy / nholeB) * nholeB;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const int ea = liftA[q * nholeA + X];
    L.a[q] = ea;
    L.b[q] = liftB[q * nholeB + Y];
    if (ea >= 0) {
      const int A = ea >> 1;
      L.off[q] = off[A];
      L.lim[q] = nballow[alevel[A]];
    }
  }
  __syncthreads();
  return cl;
}

// The lifted column (X, Y, v) of class c, cut into tiled slices: a column is
// walked by C.wpc warps of the block's eight (each a share of the K range, in
// 8-wide chunks per lane: eight independent gathers in flight), which first
// find the column's exponent (frexp of the largest |x|, 0 for an all-zero
// column; the warps' maxima meet in shared memory), then cut each chunk into
// exact slices and write every slice's chunk as one 16-byte store.  A lane's
// first kLiftKeep chunks stay in registers between the two passes (all of a
// full-CI n = 60 column); chunks beyond them are gathered again.  Long columns
// take eight warps (one warp per column left most SMs with a few warps
// waiting on gathers), short ones one (8 columns per block: a K of 256 is 32
// chunks, one per lane).  Columns beyond the class stay zero.
constexpr int kLiftThreads = 256;
constexpr int kLiftKeep = 2;
__host__ __device__ constexpr int oz_lift_wpc(int kpad) {
  // 8-wide chunks of the column, at least 48 per warp
  return kpad / 8 >= 384 ? 8 : kpad / 8 >= 192 ? 4 : kpad / 8 >= 96 ? 2 : 1;
}
__global__ void __launch_bounds__(kLiftThreads) k_oz_lift_tiled(TcTable tt, int n, int nholeA, int nholeB,
                                                       const int* __restrict__ pair_split,
                                                       const int* __restrict__ hp_inv, const int* __restrict__ liftA,
                                                       const int* __restrict__ liftB, const int8_t* __restrict__ alevel,
                                                       const int* __restrict__ nballow,
                                                       const long long* __restrict__ off, const double* __restrict__ c,
                                                       long long ndet, int* __restrict__ exps,
                                                       __nv_bfloat16* __restrict__ bs) {
  // the staged lift tables of the block's columns (dynamic: n entries for as
  // many columns as the launch's largest columns-per-block needs, so that
  // long columns leave the SM's L1 to the gathers and short ones leave room
  // for more blocks)
  extern __shared__ __align__(16) unsigned char lift_tabs[];
  __shared__ int mx[8];
  int cl = 0;
  while ((int)blockIdx.x >= tt.blk_start[cl + 1]) ++cl;
  const TcClass& C = tt.c[cl];
  const int wpc = C.wpc, cpb = 8 / wpc;  // warps per column, columns per block
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wc = warp / wpc, wk = warp % wpc;  // column in the block, share of K
  const int col = ((int)blockIdx.x - tt.blk_start[cl]) * cpb + wc;
  const bool live = col < C.ncols;  // no early return: the block meets below
  const OzLiftView L = oz_lift_view(lift_tabs + wc * oz_lift_col_bytes(n), n);
  const int hp = live ? col / tt.nvec : 0, vv = live ? col - hp * tt.nvec : 0;
  if (live) {
    const int xy = hp_inv[C.hp_start + hp];
    const int X = xy / nholeB, Y = xy - (xy / nholeB) * nholeB;
    for (int q = wk * 32 + lane; q < n; q += 32 * wpc) {
      const int ea = liftA[q * nholeA + X];
      L.a[q] = ea;
      L.b[q] = liftB[q * nholeB + Y];
      if (ea >= 0) {
        const int A = ea >> 1;
        L.off[q] = off[A];
        L.lim[q] = nballow[alevel[A]];
      }
    }
  }
  __syncthreads();
  const double* cv = c + (long long)vv * ndet;
  const int kst = C.kpad / OZ_BK;
  const int kc0 = wk * 32 + lane, kstride = 32 * wpc, nch = 2 * kst;
  double keep[kLiftKeep][8];
  int m = 0;
  if (live) {
#pragma unroll
    for (int i = 0; i < kLiftKeep; ++i) {
      const int kc = kc0 + i * kstride;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        keep[i][j] = kc < nch ? oz_lift_value<double>(L, C, kc * 8 + j, pair_split, cv) : 0.0;
        m = max(m, oz_exp_field(keep[i][j]));
      }
    }
    for (int kc = kc0 + kLiftKeep * kstride; kc < nch; kc += kstride) {
#pragma unroll
      for (int j = 0; j < 8; ++j) m = max(m, oz_exp_field(oz_lift_value<double>(L, C, kc * 8 + j, pair_split, cv)));
    }
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if (lane == 0) mx[warp] = m;
  __syncthreads();
  if (!live) return;
  for (int w = 0; w < wpc; ++w) m = max(m, mx[wc * wpc + w]);
  const int ex = m > 0 ? m - 1022 : 0;
  if (wk == 0 && lane == 0) exps[C.exp_off + col] = ex;
  __nv_bfloat16* tile0 = bs + C.bs_off + (long long)(col / OZ_BN) * kst * OZ_TB_BLOCK;
  // exact slices of one chunk, each slice's 8 values as one 16-byte store
  auto cut = [&](const double (&x)[8], int kc) {
    uint32_t pk[OZ_S][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      int a[OZ_S];
      oz_digits(x[j], ex, a);
#pragma unroll
      for (int sl = 0; sl < OZ_S; ++sl) {
        const uint32_t b = oz_digit_bits(a[sl], sl);
        if (j & 1) pk[sl][j >> 1] |= b << 16;
        else pk[sl][j >> 1] = b;
      }
    }
    __nv_bfloat16* base = tile0 + (long long)(kc >> 1) * OZ_TB_BLOCK + oz_tiled_elem(col % OZ_BN, kc * 8);
#pragma unroll
    for (int sl = 0; sl < OZ_S; ++sl)
      *reinterpret_cast<uint4*>(base + sl * OZ_BN * OZ_BK) = make_uint4(pk[sl][0], pk[sl][1], pk[sl][2], pk[sl][3]);
  };
#pragma unroll
  for (int i = 0; i < kLiftKeep; ++i)
    if (kc0 + i * kstride < nch) cut(keep[i], kc0 + i * kstride);
  for (int kc = kc0 + kLiftKeep * kstride; kc < nch; kc += kstride) {
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = oz_lift_value<double>(L, C, kc * 8 + j, pair_split, cv);
    cut(x, kc);
  }
}

// FP32 form: Ct^T gathered from the FP32 vector and split into three bf16
// terms, one block per column with its lift entries staged as above
__global__ void __launch_bounds__(256) k_t3_lift(TcTable tt, int n, int nholeA, int nholeB,
                                                 const int* __restrict__ pair_split, const int* __restrict__ hp_inv,
                                                 const int* __restrict__ liftA, const int* __restrict__ liftB,
                                                 const int8_t* __restrict__ alevel, const int* __restrict__ nballow,
                                                 const long long* __restrict__ off, const float* __restrict__ c,
                                                 long long ndet, __nv_bfloat16* __restrict__ bs) {
  __shared__ OzLiftCol L;
  int col, vv;
  const TcClass& C = tt.c[oz_stage_column(tt, n, nholeA, nholeB, hp_inv, liftA, liftB, alevel, nballow, off, L, col, vv)];
  const float* cv = c + (long long)vv * ndet;
  __nv_bfloat16* row = bs + C.bs_off + (long long)col * C.kpad;
  const long long stride = (long long)C.npad * C.kpad;
  for (int k = threadIdx.x; k < C.kpad; k += blockDim.x)
    t3_store_terms<float>(oz_lift_value<float>(L, C, k, pair_split, cv), row + k, stride);
}

static int tc_attr() {
  static bool done = false;
  if (!done) {
    ISCSI_CUDA(cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM_BYTES));
    ISCSI_CUDA(cudaFuncSetAttribute(k_tc32w_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, T3W_SMEM_BYTES));
    done = true;
  }
  return kOk;
}

static int tc_err_buf(Context& ctx) {
  if (ctx.oz_err.p) return kOk;
  ISCSI_TRY(ctx.oz_err.alloc(sizeof(int)));
  ISCSI_CUDA(cudaMemsetAsync(ctx.oz_err.p, 0, sizeof(int), stream()));
  return kOk;
}

// tiled slices (ozaki_types.cuh) of a row-major (or transposed) FP64 matrix
// with per-source-row exponents: rows_pad tiled rows (a multiple of RT) of
// kpad columns (a multiple of 16), tiled row r holding source row rowmap[r]
// (or r), tiled column k source column colmap[k] (or k); live (or null):
// the live slices of every block, recomputed here
static int slice_tiled(const double* X, int rows, int cols, long long ld, int trans, const int* rowmap,
                       const int* colmap, int RT, int rows_pad, int kpad, int* exps, __nv_bfloat16* out, int* live,
                       cudaStream_t st) {
  if (rows > 0) {
    k_oz_row_exp<<<rows, 256, 0, st>>>(X, rows, cols, ld, trans, exps); ISCSI_COUNT_LAUNCH();
  }
  const int kst = kpad / OZ_BK;
  if (live) ISCSI_CUDA(cudaMemsetAsync(live, 0, sizeof(int) * (size_t)(rows_pad / RT) * kst, st));
  const long long threads = (long long)rows_pad * 2 * kst;
  if (threads > 0) {
    k_oz_slice_tiled<<<launch_blocks(threads, 256), 256, 0, st>>>(X, rows, cols, ld, trans, rowmap, colmap, exps, out,
                                                                  RT, rows_pad, kst, live); ISCSI_COUNT_LAUNCH();
  }
  ISCSI_CUDA(cudaGetLastError());
  return kOk;
}

// device live map -> host copy (the schedule's cost model; synchronises)
static int live_to_host(const DevBuf& d, size_t n, std::vector<int>& h) {
  h.resize(n);
  if (n) ISCSI_CUDA(cudaMemcpy(h.data(), d.p, sizeof(int) * n, cudaMemcpyDeviceToHost));
  return kOk;
}

static int tc_prepare_g(Context& ctx) {
  if (ctx.oz_gs.p) return kOk;
  cudaStream_t st = stream();
  ISCSI_TRY(tc_attr());
  ISCSI_TRY(tc_err_buf(ctx));
  int np = ctx.npairs;
  ctx.oz_mpad = round_up(np, OZ_BM);
  ctx.oz_kpad = round_up(np, OZ_BK);
  long long slice = (long long)ctx.oz_mpad * ctx.oz_kpad;
  const size_t nblk = (size_t)(ctx.oz_mpad / OZ_BM) * (ctx.oz_kpad / OZ_BK);
  ISCSI_TRY(ctx.oz_gs.alloc(sizeof(__nv_bfloat16) * slice * OZ_S));
  ISCSI_TRY(ctx.oz_gexp.alloc(sizeof(int) * np));
  ISCSI_TRY(ctx.oz_glive.alloc(sizeof(int) * nblk));
  ISCSI_TRY(slice_tiled(ctx.G64.as<double>(), np, np, np, 0, nullptr, nullptr, OZ_BM, ctx.oz_mpad, ctx.oz_kpad,
                        ctx.oz_gexp.as<int>(), ctx.oz_gs.as<__nv_bfloat16>(), ctx.oz_glive.as<int>(), st));
  return live_to_host(ctx.oz_glive, nblk, ctx.oz_glive_h);
}

// a tiled operand: the array (block (0, 0)), its k steps per row tile, the
// segment's first row tile and k step, live map (device, host) or none
struct TiledOp {
  const __nv_bfloat16* base;
  int kst, rt0, ks0;
  const int* live;
  const int* live_h;
};

// segment of a job over two tiled operands
static int add_seg_tiled(OzJob& job, const TiledOp& A, const int* a_exp, const TiledOp& B, const int* b_exp, int K,
                         int nrows_b) {
  OzSeg sg;
  std::memset(&sg, 0, sizeof(sg));
  sg.a_exp = a_exp;
  sg.b_exp = b_exp;
  sg.K = K;
  sg.nrows_b = nrows_b;
  sg.a_tiled = A.base;
  sg.b_tiled = B.base;
  sg.a_live = A.live;
  sg.b_live = B.live;
  sg.a_kst = A.kst;
  sg.b_kst = B.kst;
  sg.a_rt0 = A.rt0;
  sg.a_ks0 = A.ks0;
  sg.b_rt0 = B.rt0;
  sg.b_ks0 = B.ks0;
  OzMaps m;
  std::memset(&m, 0, sizeof(m));
  OzSegHost h;
  h.a_live = A.live_h;
  h.b_live = B.live_h;
  job.segs.push_back(sg);
  job.maps.push_back(m);
  job.sh.push_back(h);
  return kOk;
}

// segment of a job: block (a_row0, a_k0) of A times block (b_row0, b_k0) of B
static int add_seg(OzJob& job, const SliceArray& A, int a_row0, int a_k0, const int* a_exp, const SliceArray& B,
                   int b_row0, int b_k0, const int* b_exp, int K, int nrows_b, int nslice = OZ_S) {
  OzSeg sg;
  std::memset(&sg, 0, sizeof(sg));
  sg.a_exp = a_exp;
  sg.b_exp = b_exp;
  sg.a_row0 = a_row0;
  sg.a_k0 = a_k0;
  sg.b_row0 = b_row0;
  sg.b_k0 = b_k0;
  sg.K = K;
  sg.nrows_b = nrows_b;
  OzMaps m;
  std::memset(&m, 0, sizeof(m));
  if (oz_encode_map(&m.a, A.base, A.ld, A.rows, nslice, A.slice, OZ_BM) ||
      oz_encode_map(&m.b, B.base, B.ld, B.rows, nslice, B.slice, OZ_BN) ||
      oz_encode_map(&m.bw, B.base, B.ld, B.rows, nslice, B.slice, OZ_BW_ROWS)) {
    set_error("tensor-core sigma: TMA descriptor rejected");
    return kErrCuda;
  }
  job.segs.push_back(sg);
  job.maps.push_back(m);
  job.sh.push_back(OzSegHost());
  return kOk;
}

// the job's lists on the device; persistent (FP64-accurate) jobs also get
// their schedule
static int upload_job(OzJob& job, cudaStream_t st, bool persistent = true) {
  ++job.version;
  ISCSI_TRY(job.d_probs.grow(sizeof(OzProblem) * std::max<size_t>(1, job.probs.size())));
  ISCSI_TRY(job.d_segs.grow(sizeof(OzSeg) * std::max<size_t>(1, job.segs.size())));
  ISCSI_TRY(job.d_maps.grow(sizeof(OzMaps) * std::max<size_t>(1, job.maps.size())));
  if (!job.maps.empty())
    ISCSI_CUDA(cudaMemcpyAsync(job.d_maps.p, job.maps.data(), sizeof(OzMaps) * job.maps.size(),
                               cudaMemcpyHostToDevice, st));
  if (!job.probs.empty())
    ISCSI_CUDA(cudaMemcpyAsync(job.d_probs.p, job.probs.data(), sizeof(OzProblem) * job.probs.size(),
                               cudaMemcpyHostToDevice, st));
  if (!job.segs.empty())
    ISCSI_CUDA(cudaMemcpyAsync(job.d_segs.p, job.segs.data(), sizeof(OzSeg) * job.segs.size(), cudaMemcpyHostToDevice,
                               st));
  ISCSI_CUDA(cudaStreamSynchronize(st));  // the host vectors must outlive the copies
  if (persistent) ISCSI_TRY(oz_plan_build(job.probs, job.segs, job.sh, job.plan, st));
  return kOk;
}

// one persistent k_oz_gemm launch on a schedule
static int launch_oz(const OzPlan& plan, const OzProblem* probs, const OzSeg* segs, const OzMaps* maps,
                     double* tbase, double* const* tbases, int* err, cudaStream_t st) {
  if (plan.grid == 0) return kOk;
  k_oz_gemm<<<plan.grid, OZ_THREADS, OZ_SMEM_BYTES, st>>>(probs, segs, maps, plan.d_items.as<OzItem>(),
                                                          plan.d_cta.as<int>(), tbase, tbases, plan.d_ws.as<double>(),
                                                          plan.d_cnt.as<int>(), err); ISCSI_COUNT_LAUNCH();
  ISCSI_CUDA(cudaGetLastError());
  return kOk;
}

static int launch_job(Context& ctx, const OzJob& job, double* tbase, cudaStream_t st) {
  return launch_oz(job.plan, job.d_probs.as<OzProblem>(), job.d_segs.as<OzSeg>(), job.d_maps.as<OzMaps>(), tbase,
                   nullptr, ctx.oz_err.as<int>(), st);
}

// tile numbering of a problem list (bn columns per tile)
static int add_tiles(std::vector<OzProblem>& probs, int bn = OZ_BN) {
  int tiles = 0;
  for (auto& p : probs) {
    p.tiles_n = round_up(p.N, bn) / bn;
    p.tile_begin = tiles;
    tiles += (round_up(p.M, OZ_BM) / OZ_BM) * p.tiles_n;
  }
  return tiles;
}

// ---------------------------------------------------------------------------
// opposite spin

static TcTable ab_table(const Context& ctx, int nvec, long long* bs_elems, long long* exp_elems, int nslice = OZ_S) {
  TcTable tt;
  std::memset(&tt, 0, sizeof(tt));
  tt.nvec = nvec;
  long long bs = 0, ex = 0, flat = 0;
  for (int cl = 0; cl < (int)ctx.cls.size(); ++cl) {
    const ColClass& cc = ctx.cls[cl];
    if (cc.ncol == 0 || cc.mrows == 0) continue;
    TcClass C;
    C.mrows = cc.mrows;
    C.ncols = cc.ncol * nvec;
    C.krows = cc.krows;
    C.kpad = round_up(cc.krows, OZ_BK);
    C.npad = round_up(C.ncols, OZ_BW_ROWS);
    C.hp_start = ctx.hp_class_start[cl];
    C.bs_off = bs;
    C.exp_off = ex;
    C.tot = (long long)C.ncols * C.kpad;
    tt.start[tt.nclass] = flat;
    tt.col_start[tt.nclass + 1] = tt.col_start[tt.nclass] + C.ncols;
    C.wpc = oz_lift_wpc(C.kpad);
    tt.blk_start[tt.nclass + 1] = tt.blk_start[tt.nclass] + (C.ncols + 8 / C.wpc - 1) / (8 / C.wpc);
    tt.c[tt.nclass++] = C;
    flat += C.tot;
    bs += (long long)nslice * C.npad * C.kpad;
    ex += C.ncols;
  }
  tt.start[tt.nclass] = flat;
  *bs_elems = bs;
  *exp_elems = ex;
  return tt;
}

int opposite_tc_operands(Context& ctx, const double* c, double* ttw, int nvec) {
  cudaStream_t st = stream();
  ISCSI_TRY(tc_prepare_g(ctx));
  long long bs_elems = 0, exp_elems = 0;
  TcTable tt = ab_table(ctx, nvec, &bs_elems, &exp_elems);
  if (tt.nclass == 0) return kOk;
  bool rebuild = ctx.oz_ab.nvec != nvec || ctx.oz_ab.tbase != (const void*)ttw;
  if (ctx.oz_bs_elems < bs_elems) {
    ISCSI_TRY(ctx.oz_bs.alloc(sizeof(__nv_bfloat16) * bs_elems));
    ctx.oz_bs_elems = bs_elems;
    rebuild = true;
  }
  if ((long long)(ctx.oz_bexp.bytes / sizeof(int)) < exp_elems) {
    ISCSI_TRY(ctx.oz_bexp.alloc(sizeof(int) * exp_elems));
    rebuild = true;
  }
  if (rebuild) {
    // padding rows of every class stay zero from here on
    ISCSI_CUDA(cudaMemsetAsync(ctx.oz_bs.p, 0, sizeof(__nv_bfloat16) * ctx.oz_bs_elems, st));
    OzJob& job = ctx.oz_ab;
    job.probs.clear();
    job.segs.clear();
    job.maps.clear();
    job.sh.clear();
    long long t_off = 0;
    const TiledOp GA{ctx.oz_gs.as<__nv_bfloat16>(), ctx.oz_kpad / OZ_BK, 0, 0, ctx.oz_glive.as<int>(),
                     ctx.oz_glive_h.data()};
    for (int i = 0; i < tt.nclass; ++i) {
      const TcClass& C = tt.c[i];
      const TiledOp CB{ctx.oz_bs.as<__nv_bfloat16>() + C.bs_off, C.kpad / OZ_BK, 0, 0, nullptr, nullptr};
      OzProblem P;
      std::memset(&P, 0, sizeof(P));
      // T_c sits where the fold expects it: classes in order, mrows x ncols each
      int mrows = C.mrows;
      P.t = (long long)reinterpret_cast<uintptr_t>(ttw + t_off);
      P.t_rel = 0;
      P.ldt = C.ncols;
      P.M = mrows;
      P.N = C.ncols;
      P.seg_begin = (int)job.segs.size();
      P.seg_count = 1;
      P.accumulate = 0;
      t_off += (long long)mrows * C.ncols;
      ISCSI_TRY(add_seg_tiled(job, GA, ctx.oz_gexp.as<int>(), CB, ctx.oz_bexp.as<int>() + C.exp_off, C.kpad,
                              C.ncols));
      job.probs.push_back(P);
    }
    job.tiles = add_tiles(job.probs);
    ISCSI_TRY(upload_job(job, st));
    job.nvec = nvec;
    job.tbase = ttw;
  }
  const SpinSpace& SA = ctx.sp[0];
  const SpinSpace& SB = ctx.sp[1];
  const int nblk = tt.blk_start[tt.nclass];
  if (nblk > 0) {
    int cpb_max = 1;
    for (int i = 0; i < tt.nclass; ++i) cpb_max = std::max(cpb_max, 8 / tt.c[i].wpc);
    k_oz_lift_tiled<<<nblk, kLiftThreads, oz_lift_col_bytes(ctx.n) * cpb_max, st>>>(tt, ctx.n, SA.nhole, SB.nhole, ctx.pair_split.as<int>(), ctx.hp_inv.as<int>(),
                                          SA.lift.as<int>(), SB.lift.as<int>(), SA.level.as<int8_t>(),
                                          ctx.nballow.as<int>(), ctx.off.as<long long>(), c, ctx.ndet,
                                          ctx.oz_bexp.as<int>(), ctx.oz_bs.as<__nv_bfloat16>()); ISCSI_COUNT_LAUNCH();
  }
  ISCSI_CUDA(cudaGetLastError());
  return kOk;
}

int opposite_tc_gemm(Context& ctx) { return launch_job(ctx, ctx.oz_ab, nullptr, stream()); }

// ---------------------------------------------------------------------------
// same spin

// Same-spin level block a goes to the tensor cores when it has more rows and
// allowed beta strings than the context's threshold for this precision (set
// by the autotuner; the default 16 keeps the thinnest blocks on the FMA thin
// kernels of sigma.cu, which stream the wide operand once).
bool samespin_block_on_tc(const Context& ctx, int a, int prec) {
  const SpinSpace& SA = ctx.sp[0];
  int rows = SA.level_start[a + 1] - SA.level_start[a];
  int nba = (int)ctx.nb_allowed_lvl[a];
  const int thr = ctx.route[prec == 32 ? 1 : 0].ss_min;
  return rows > thr && nba > thr;
}

bool ab_on_tc(const Context& ctx, int prec) {
  return (prec == 32 ? options().fp32_tc : options().fp64_tc) && ctx.route[prec == 32 ? 1 : 0].ab_tc;
}

bool samespin_tc_active(const Context& ctx) {
  if (!options().fp64_tc || !options().samespin_tc) return false;
  for (int a = 0; a <= ctx.sp[0].maxlevel; ++a)
    if (samespin_block_on_tc(ctx, a, 64)) return true;
  return false;
}

// cut_only: the matrices changed in place (a per-step one-body term); cut them
// again into the existing buffers, so the work lists keep their pointers
static int tc_prepare_m(Context& ctx, bool cut_only = false) {
  if (ctx.oz_m_ready && !cut_only) return kOk;
  cudaStream_t st = stream();
  ISCSI_TRY(tc_attr());
  ISCSI_TRY(tc_err_buf(ctx));
  const SpinSpace& SA = ctx.sp[0];
  const SpinSpace& SB = ctx.sp[1];
  int nl = SA.maxlevel + 1;
  // M_alpha (the A operand of the alpha part): every level block's rows start
  // at a 128-row tile of their own, columns grouped by level with each group
  // padded to 16, so every segment starts on a block boundary
  if (ctx.na > 0 && ctx.M64[0].p) {
    if (!cut_only) {
      ctx.oz_kbase.assign(nl + 1, 0);
      ctx.oz_mabase.assign(nl + 1, 0);
      for (int a = 0; a < nl; ++a) {
        const int rows = SA.level_start[a + 1] - SA.level_start[a];
        ctx.oz_kbase[a + 1] = ctx.oz_kbase[a] + round_up(rows, OZ_BK);
        ctx.oz_mabase[a + 1] = ctx.oz_mabase[a] + round_up(rows, OZ_BM);
      }
      const int kcols = ctx.oz_kbase[nl], trows = ctx.oz_mabase[nl];
      std::vector<int> colmap(kcols, -1), rowmap(trows, -1);
      for (int a = 0; a < nl; ++a)
        for (int i = SA.level_start[a]; i < SA.level_start[a + 1]; ++i) {
          colmap[ctx.oz_kbase[a] + i - SA.level_start[a]] = i;
          rowmap[ctx.oz_mabase[a] + i - SA.level_start[a]] = i;
        }
      ISCSI_TRY(ctx.oz_macol.alloc(sizeof(int) * kcols));
      ISCSI_TRY(ctx.oz_marow.alloc(sizeof(int) * trows));
      ISCSI_CUDA(cudaMemcpy(ctx.oz_macol.p, colmap.data(), sizeof(int) * kcols, cudaMemcpyHostToDevice));
      ISCSI_CUDA(cudaMemcpy(ctx.oz_marow.p, rowmap.data(), sizeof(int) * trows, cudaMemcpyHostToDevice));
      ctx.oz_ma_rows = trows;
      ctx.oz_ma_ld = kcols;
      ISCSI_TRY(ctx.oz_mas.alloc(sizeof(__nv_bfloat16) * OZ_S * (size_t)trows * kcols));
      ISCSI_TRY(ctx.oz_maexp.alloc(sizeof(int) * (SA.count + OZ_BM)));
      ISCSI_CUDA(cudaMemsetAsync(ctx.oz_maexp.p, 0, sizeof(int) * (SA.count + OZ_BM), st));
      ISCSI_TRY(ctx.oz_malive.alloc(sizeof(int) * (size_t)(trows / OZ_BM) * (kcols / OZ_BK)));
    }
    ISCSI_TRY(slice_tiled(ctx.M64[0].as<double>(), SA.count, SA.count, SA.count, 0, ctx.oz_marow.as<int>(),
                          ctx.oz_macol.as<int>(), OZ_BM, ctx.oz_ma_rows, ctx.oz_ma_ld, ctx.oz_maexp.as<int>(),
                          ctx.oz_mas.as<__nv_bfloat16>(), ctx.oz_malive.as<int>(), st));
    if (!cut_only)
      ISCSI_TRY(live_to_host(ctx.oz_malive, (size_t)(ctx.oz_ma_rows / OZ_BM) * (ctx.oz_ma_ld / OZ_BK),
                             ctx.oz_malive_h));
  }
  if (ctx.nb > 0) {
    // M_beta[B][B'] as the B operand; the stored beta matrix is M_beta^T
    // (or the symmetric alpha matrix when shared)
    const double* Mb = ctx.beta_alias ? ctx.M64[0].as<double>() : ctx.M64[1].as<double>();
    int trans = ctx.beta_alias ? 0 : 1;
    ctx.oz_mb_rows = round_up(SB.count, OZ_BW_ROWS);
    ctx.oz_mb_ld = round_up(SB.count, OZ_BK);
    const size_t nblk = (size_t)(ctx.oz_mb_rows / OZ_BN) * (ctx.oz_mb_ld / OZ_BK);
    if (!cut_only) {
      ISCSI_TRY(ctx.oz_mbs.alloc(sizeof(__nv_bfloat16) * OZ_S * (size_t)ctx.oz_mb_rows * ctx.oz_mb_ld));
      ISCSI_TRY(ctx.oz_mbexp.alloc(sizeof(int) * ctx.oz_mb_rows));
      ISCSI_CUDA(cudaMemsetAsync(ctx.oz_mbexp.p, 0, sizeof(int) * ctx.oz_mb_rows, st));
      ISCSI_TRY(ctx.oz_mblive.alloc(sizeof(int) * nblk));
    }
    ISCSI_TRY(slice_tiled(Mb, SB.count, SB.count, SB.count, trans, nullptr, nullptr, OZ_BN, ctx.oz_mb_rows,
                          ctx.oz_mb_ld, ctx.oz_mbexp.as<int>(), ctx.oz_mbs.as<__nv_bfloat16>(),
                          ctx.oz_mblive.as<int>(), st));
    if (!cut_only) ISCSI_TRY(live_to_host(ctx.oz_mblive, nblk, ctx.oz_mblive_h));
  }
  ctx.oz_m_ready = true;
  return kOk;
}

// workspace layout of the per-call slices of C for (vector v, level block a)
struct SsBlock {
  int a, rows, nba, start;
  long long obase;
  long long bt_off, ca_off;      // slice-0 element offsets in oz_cs
  long long bt_exp, ca_exp;      // offsets in oz_csexp
  int bt_rows, bt_ld, ca_rows, ca_ld;
};

static std::vector<SsBlock> ss_blocks(const Context& ctx, long long* elems, long long* exps, int nslice = OZ_S) {
  std::vector<SsBlock> out;
  const SpinSpace& SA = ctx.sp[0];
  long long e = 0, x = 0;
  for (int a = 0; a <= SA.maxlevel; ++a) {
    SsBlock b;
    b.a = a;
    b.start = SA.level_start[a];
    b.rows = SA.level_start[a + 1] - SA.level_start[a];
    b.nba = (int)ctx.nb_allowed_lvl[a];
    if (b.rows == 0 || b.nba == 0) continue;
    b.obase = ctx.off_h[b.start];
    // C_a^T (alpha part operand): rows = beta strings, K = alpha strings of the block
    b.bt_rows = round_up(b.nba, OZ_BW_ROWS);
    b.bt_ld = round_up(b.rows, OZ_BK);
    b.bt_off = e;
    e += (long long)nslice * b.bt_rows * b.bt_ld;
    b.bt_exp = x;
    x += b.bt_rows;
    // C_a (beta part operand): rows = alpha strings of the block, K = beta strings
    b.ca_rows = round_up(b.rows, OZ_BM);
    b.ca_ld = round_up(b.nba, OZ_BK);
    b.ca_off = e;
    e += (long long)nslice * b.ca_rows * b.ca_ld;
    b.ca_exp = x;
    x += b.ca_rows;
    out.push_back(b);
  }
  *elems = e;
  *exps = x;
  return out;
}

int samespin_tc_operands(Context& ctx, const double* c, double* sigma, int nvec) {
  cudaStream_t st = stream();
  ISCSI_TRY(tc_prepare_m(ctx));
  long long elems1 = 0, exps1 = 0;
  std::vector<SsBlock> blocks = ss_blocks(ctx, &elems1, &exps1);
  long long elems = elems1 * nvec, nexp = exps1 * nvec;
  bool rebuild = ctx.oz_ss.nvec != nvec;
  if (ctx.oz_cs_elems < elems) {
    ISCSI_TRY(ctx.oz_cs.alloc(sizeof(__nv_bfloat16) * elems));
    ctx.oz_cs_elems = elems;
    rebuild = true;
  }
  if ((long long)(ctx.oz_csexp.bytes / sizeof(int)) < nexp) {
    ISCSI_TRY(ctx.oz_csexp.alloc(sizeof(int) * nexp));
    rebuild = true;
  }
  __nv_bfloat16* cs = ctx.oz_cs.as<__nv_bfloat16>();
  int* cx = ctx.oz_csexp.as<int>();
  const SpinSpace& SB = ctx.sp[1];
  if (rebuild) {
    ISCSI_CUDA(cudaMemsetAsync(ctx.oz_cs.p, 0, sizeof(__nv_bfloat16) * ctx.oz_cs_elems, st));
    ISCSI_CUDA(cudaMemsetAsync(ctx.oz_csexp.p, 0, sizeof(int) * nexp, st));
    OzJob& job = ctx.oz_ss;
    job.probs.clear();
    job.segs.clear();
    job.maps.clear();
    job.sh.clear();
    const TiledOp MB{ctx.oz_mbs.as<__nv_bfloat16>(), ctx.oz_mb_ld / OZ_BK, 0, 0, ctx.oz_mblive.as<int>(),
                     ctx.oz_mblive_h.data()};
    for (int v = 0; v < nvec; ++v)
      for (const SsBlock& b : blocks) {
        if (!samespin_block_on_tc(ctx, b.a, 64)) continue;
        OzProblem P;
        std::memset(&P, 0, sizeof(P));
        P.t = (long long)v * ctx.ndet + b.obase;
        P.t_rel = 1;
        P.ldt = b.nba;
        P.M = b.rows;
        P.N = b.nba;
        P.seg_begin = (int)job.segs.size();
        P.accumulate = 1;
        if (ctx.na > 0 && ctx.oz_mas.p)
          for (const SsBlock& b2 : blocks) {
            if (std::abs(b.a - b2.a) > 2) continue;
            const TiledOp MA{ctx.oz_mas.as<__nv_bfloat16>(), ctx.oz_ma_ld / OZ_BK, ctx.oz_mabase[b.a] / OZ_BM,
                             ctx.oz_kbase[b2.a] / OZ_BK, ctx.oz_malive.as<int>(), ctx.oz_malive_h.data()};
            const TiledOp CT{cs + v * elems1 + b2.bt_off, b2.bt_ld / OZ_BK, 0, 0, nullptr, nullptr};
            ISCSI_TRY(add_seg_tiled(job, MA, ctx.oz_maexp.as<int>() + b.start, CT, cx + v * exps1 + b2.bt_exp,
                                    b2.bt_ld, std::min(b.nba, b2.nba)));
            P.seg_count++;
          }
        if (ctx.nb > 0 && ctx.oz_mbs.p) {
          const TiledOp CA{cs + v * elems1 + b.ca_off, b.ca_ld / OZ_BK, 0, 0, nullptr, nullptr};
          ISCSI_TRY(add_seg_tiled(job, CA, cx + v * exps1 + b.ca_exp, MB, ctx.oz_mbexp.as<int>(), b.ca_ld, b.nba));
          P.seg_count++;
        }
        if (P.seg_count > 0) job.probs.push_back(P);
      }
    job.tiles = add_tiles(job.probs);
    ISCSI_TRY(upload_job(job, st));
    job.nvec = nvec;
  }
  // slice this call's C blocks (only the blocks some tensor-core problem reads)
  for (int v = 0; v < nvec; ++v)
    for (const SsBlock& b : blocks) {
      bool used = samespin_block_on_tc(ctx, b.a, 64);
      for (const SsBlock& b2 : blocks)
        if (std::abs(b.a - b2.a) <= 2 && samespin_block_on_tc(ctx, b2.a, 64)) used = true;
      if (!used) continue;
      const double* X = c + (long long)v * ctx.ndet + b.obase;  // [rows][nba]
      if (ctx.na > 0)
        ISCSI_TRY(slice_tiled(X, b.nba, b.rows, b.nba, 1, nullptr, nullptr, OZ_BN, b.bt_rows, b.bt_ld,
                              cx + v * exps1 + b.bt_exp, cs + v * elems1 + b.bt_off, nullptr, st));
      if (ctx.nb > 0 && samespin_block_on_tc(ctx, b.a, 64))
        ISCSI_TRY(slice_tiled(X, b.rows, b.nba, b.nba, 0, nullptr, nullptr, OZ_BM, b.ca_rows, b.ca_ld,
                              cx + v * exps1 + b.ca_exp, cs + v * elems1 + b.ca_off, nullptr, st));
    }
  (void)SB;
  (void)sigma;
  return kOk;
}

int samespin_tc_gemm(Context& ctx, double* sigma) { return launch_job(ctx, ctx.oz_ss, sigma, stream()); }

// ---------------------------------------------------------------------------
// FP32 form: three bf16 terms per element, FP32 accumulation (tc32.cuh)

template <typename V>
static int t3_slice_matrix(const V* X, int rows, int cols, long long ld, int trans, const int* colmap, int ldo,
                           int rows_pad, __nv_bfloat16* out, cudaStream_t st) {
  long long slice = (long long)rows_pad * ldo;
  if (slice > 0) {
    k_t3_slice<V><<<launch_blocks(slice, 256), 256, 0, st>>>(X, rows, cols, ld, trans, colmap, out, slice, ldo,
                                                             rows_pad); ISCSI_COUNT_LAUNCH();
  }
  ISCSI_CUDA(cudaGetLastError());
  return kOk;
}

// k_tc32w_gemm over a problem list
static int launch_t3(int tiles, const OzProblem* probs, int nprobs, const OzSeg* segs, const OzMaps* maps,
                     float* tbase, float* const* tbases, int* err, cudaStream_t st) {
  if (tiles == 0) return kOk;
  k_tc32w_gemm<<<tiles, T3W_THREADS, T3W_SMEM_BYTES, st>>>(probs, nprobs, segs, maps, tbase, tbases, err); ISCSI_COUNT_LAUNCH();
  ISCSI_CUDA(cudaGetLastError());
  return kOk;
}

static int t3_launch(Context& ctx, const OzJob& job, float* tbase, cudaStream_t st) {
  return launch_t3(job.tiles, job.d_probs.as<OzProblem>(), (int)job.probs.size(), job.d_segs.as<OzSeg>(),
                   job.d_maps.as<OzMaps>(), tbase, nullptr, ctx.oz_err.as<int>(), st);
}

static int t3_prepare_g(Context& ctx) {
  if (ctx.t3_gs.p) return kOk;
  ISCSI_TRY(tc_attr());
  ISCSI_TRY(tc_err_buf(ctx));
  int np = ctx.npairs;
  ctx.oz_mpad = round_up(np, OZ_BM);
  ctx.oz_kpad = round_up(np, OZ_BK);
  long long slice = (long long)ctx.oz_mpad * ctx.oz_kpad;
  ISCSI_TRY(ctx.t3_gs.alloc(sizeof(__nv_bfloat16) * slice * T3_S));
  return t3_slice_matrix<double>(ctx.G64.as<double>(), np, np, np, 0, nullptr, ctx.oz_kpad, ctx.oz_mpad,
                                 ctx.t3_gs.as<__nv_bfloat16>(), stream());
}

int opposite_tc32_operands(Context& ctx, const float* c, float* ttw, int nvec) {
  cudaStream_t st = stream();
  ISCSI_TRY(t3_prepare_g(ctx));
  long long bs_elems = 0, exp_elems = 0;
  TcTable tt = ab_table(ctx, nvec, &bs_elems, &exp_elems, T3_S);
  if (tt.nclass == 0) return kOk;
  bool rebuild = ctx.t3_ab.nvec != nvec || ctx.t3_ab.tbase != (const void*)ttw;
  if (ctx.t3_bs_elems < bs_elems) {
    ISCSI_TRY(ctx.t3_bs.alloc(sizeof(__nv_bfloat16) * bs_elems));
    ctx.t3_bs_elems = bs_elems;
    rebuild = true;
  }
  if (rebuild) {
    ISCSI_CUDA(cudaMemsetAsync(ctx.t3_bs.p, 0, sizeof(__nv_bfloat16) * ctx.t3_bs_elems, st));
    OzJob& job = ctx.t3_ab;
    job.probs.clear();
    job.segs.clear();
    job.maps.clear();
    job.sh.clear();
    long long t_off = 0;
    const SliceArray GA{ctx.t3_gs.as<__nv_bfloat16>(), ctx.oz_kpad, ctx.oz_mpad, (long long)ctx.oz_mpad * ctx.oz_kpad};
    for (int i = 0; i < tt.nclass; ++i) {
      const TcClass& C = tt.c[i];
      const SliceArray CB{ctx.t3_bs.as<__nv_bfloat16>() + C.bs_off, C.kpad, C.npad, (long long)C.npad * C.kpad};
      OzProblem P;
      std::memset(&P, 0, sizeof(P));
      P.t = (long long)reinterpret_cast<uintptr_t>(ttw + t_off);
      P.ldt = C.ncols;
      P.M = C.mrows;
      P.N = C.ncols;
      P.seg_begin = (int)job.segs.size();
      P.seg_count = 1;
      t_off += (long long)C.mrows * C.ncols;
      ISCSI_TRY(add_seg(job, GA, 0, 0, nullptr, CB, 0, 0, nullptr, C.kpad, C.ncols, T3_S));
      job.probs.push_back(P);
    }
    job.tiles = add_tiles(job.probs, T3W_BN);
    ISCSI_TRY(upload_job(job, st, false));
    job.nvec = nvec;
    job.tbase = ttw;
  }
  const SpinSpace& SA = ctx.sp[0];
  const SpinSpace& SB = ctx.sp[1];
  if (tt.col_start[tt.nclass] > 0)
  k_t3_lift<<<tt.col_start[tt.nclass], 256, 0, st>>>(tt, ctx.n, SA.nhole, SB.nhole, ctx.pair_split.as<int>(),
                                                       ctx.hp_inv.as<int>(), SA.lift.as<int>(), SB.lift.as<int>(),
                                                       SA.level.as<int8_t>(), ctx.nballow.as<int>(),
                                                       ctx.off.as<long long>(), c, ctx.ndet,
                                                       ctx.t3_bs.as<__nv_bfloat16>()); ISCSI_COUNT_LAUNCH();
  ISCSI_CUDA(cudaGetLastError());
  return kOk;
}

int opposite_tc32_gemm(Context& ctx) { return t3_launch(ctx, ctx.t3_ab, nullptr, stream()); }

bool samespin_tc32_active(const Context& ctx) {
  if (!options().fp32_tc || !options().samespin_tc) return false;
  for (int a = 0; a <= ctx.sp[0].maxlevel; ++a)
    if (samespin_block_on_tc(ctx, a, 32)) return true;
  return false;
}

static int t3_prepare_m(Context& ctx, bool cut_only = false) {
  if (ctx.t3_m_ready && !cut_only) return kOk;
  cudaStream_t st = stream();
  ISCSI_TRY(tc_attr());
  ISCSI_TRY(tc_err_buf(ctx));
  const SpinSpace& SA = ctx.sp[0];
  const SpinSpace& SB = ctx.sp[1];
  int nl = SA.maxlevel + 1;
  // the same level-padded column layout as the FP64 slices
  ctx.oz_kbase.assign(nl + 1, 0);
  for (int a = 0; a < nl; ++a) ctx.oz_kbase[a + 1] = ctx.oz_kbase[a] + round_up(SA.level_start[a + 1] - SA.level_start[a], OZ_BK);
  if (ctx.na > 0 && ctx.M64[0].p) {
    int kcols = ctx.oz_kbase[nl];
    std::vector<int> colmap(kcols, -1);
    for (int a = 0; a < nl; ++a)
      for (int i = SA.level_start[a]; i < SA.level_start[a + 1]; ++i) colmap[ctx.oz_kbase[a] + i - SA.level_start[a]] = i;
    DevBuf dmap;
    ISCSI_TRY(dmap.alloc(sizeof(int) * kcols));
    ISCSI_CUDA(cudaMemcpyAsync(dmap.p, colmap.data(), sizeof(int) * kcols, cudaMemcpyHostToDevice, st));
    ctx.t3_ma_rows = SA.count + OZ_BM;
    ctx.oz_ma_ld = kcols;
    if (!cut_only) ISCSI_TRY(ctx.t3_mas.alloc(sizeof(__nv_bfloat16) * T3_S * (size_t)ctx.t3_ma_rows * kcols));
    ISCSI_TRY(t3_slice_matrix<double>(ctx.M64[0].as<double>(), SA.count, SA.count, SA.count, 0, dmap.as<int>(), kcols,
                                      ctx.t3_ma_rows, ctx.t3_mas.as<__nv_bfloat16>(), st));
    ISCSI_CUDA(cudaStreamSynchronize(st));  // colmap lives until here
  }
  if (ctx.nb > 0) {
    const double* Mb = ctx.beta_alias ? ctx.M64[0].as<double>() : ctx.M64[1].as<double>();
    int trans = ctx.beta_alias ? 0 : 1;
    ctx.oz_mb_rows = round_up(SB.count, OZ_BW_ROWS);
    ctx.oz_mb_ld = round_up(SB.count, OZ_BK);
    if (!cut_only) ISCSI_TRY(ctx.t3_mbs.alloc(sizeof(__nv_bfloat16) * T3_S * (size_t)ctx.oz_mb_rows * ctx.oz_mb_ld));
    ISCSI_TRY(t3_slice_matrix<double>(Mb, SB.count, SB.count, SB.count, trans, nullptr, ctx.oz_mb_ld, ctx.oz_mb_rows,
                                      ctx.t3_mbs.as<__nv_bfloat16>(), st));
  }
  ctx.t3_m_ready = true;
  return kOk;
}

int samespin_tc32_operands(Context& ctx, const float* c, float* sigma, int nvec) {
  cudaStream_t st = stream();
  ISCSI_TRY(t3_prepare_m(ctx));
  long long elems1 = 0, exps1 = 0;
  std::vector<SsBlock> blocks = ss_blocks(ctx, &elems1, &exps1, T3_S);
  long long elems = elems1 * nvec;
  bool rebuild = ctx.t3_ss.nvec != nvec;
  if (ctx.t3_cs_elems < elems) {
    ISCSI_TRY(ctx.t3_cs.alloc(sizeof(__nv_bfloat16) * elems));
    ctx.t3_cs_elems = elems;
    rebuild = true;
  }
  __nv_bfloat16* cs = ctx.t3_cs.as<__nv_bfloat16>();
  if (rebuild) {
    ISCSI_CUDA(cudaMemsetAsync(ctx.t3_cs.p, 0, sizeof(__nv_bfloat16) * ctx.t3_cs_elems, st));
    OzJob& job = ctx.t3_ss;
    job.probs.clear();
    job.segs.clear();
    job.maps.clear();
    job.sh.clear();
    const SliceArray MA{ctx.t3_mas.as<__nv_bfloat16>(), ctx.oz_ma_ld, ctx.t3_ma_rows,
                        (long long)ctx.t3_ma_rows * ctx.oz_ma_ld};
    const SliceArray MB{ctx.t3_mbs.as<__nv_bfloat16>(), ctx.oz_mb_ld, ctx.oz_mb_rows,
                        (long long)ctx.oz_mb_rows * ctx.oz_mb_ld};
    for (int v = 0; v < nvec; ++v)
      for (const SsBlock& b : blocks) {
        if (!samespin_block_on_tc(ctx, b.a, 32)) continue;
        OzProblem P;
        std::memset(&P, 0, sizeof(P));
        P.t = (long long)v * ctx.ndet + b.obase;
        P.t_rel = 1;
        P.ldt = b.nba;
        P.M = b.rows;
        P.N = b.nba;
        P.seg_begin = (int)job.segs.size();
        P.accumulate = 1;
        if (ctx.na > 0 && ctx.t3_mas.p)
          for (const SsBlock& b2 : blocks) {
            if (std::abs(b.a - b2.a) > 2) continue;
            const SliceArray CT{cs + v * elems1 + b2.bt_off, b2.bt_ld, b2.bt_rows, (long long)b2.bt_rows * b2.bt_ld};
            ISCSI_TRY(add_seg(job, MA, b.start, ctx.oz_kbase[b2.a], nullptr, CT, 0, 0, nullptr, b2.bt_ld,
                              std::min(b.nba, b2.nba), T3_S));
            P.seg_count++;
          }
        if (ctx.nb > 0 && ctx.t3_mbs.p) {
          const SliceArray CA{cs + v * elems1 + b.ca_off, b.ca_ld, b.ca_rows, (long long)b.ca_rows * b.ca_ld};
          ISCSI_TRY(add_seg(job, CA, 0, 0, nullptr, MB, 0, 0, nullptr, b.ca_ld, b.nba, T3_S));
          P.seg_count++;
        }
        if (P.seg_count > 0) job.probs.push_back(P);
      }
    job.tiles = add_tiles(job.probs, T3W_BN);
    ISCSI_TRY(upload_job(job, st, false));
    job.nvec = nvec;
  }
  for (int v = 0; v < nvec; ++v)
    for (const SsBlock& b : blocks) {
      bool used = samespin_block_on_tc(ctx, b.a, 32);
      for (const SsBlock& b2 : blocks)
        if (std::abs(b.a - b2.a) <= 2 && samespin_block_on_tc(ctx, b2.a, 32)) used = true;
      if (!used) continue;
      const float* X = c + (long long)v * ctx.ndet + b.obase;  // [rows][nba]
      if (ctx.na > 0)
        ISCSI_TRY(t3_slice_matrix<float>(X, b.nba, b.rows, b.nba, 1, nullptr, b.bt_ld, b.bt_rows,
                                         cs + v * elems1 + b.bt_off, st));
      if (ctx.nb > 0 && samespin_block_on_tc(ctx, b.a, 32))
        ISCSI_TRY(t3_slice_matrix<float>(X, b.rows, b.nba, b.nba, 0, nullptr, b.ca_ld, b.ca_rows,
                                         cs + v * elems1 + b.ca_off, st));
    }
  (void)sigma;
  return kOk;
}

int samespin_tc32_gemm(Context& ctx, float* sigma) { return t3_launch(ctx, ctx.t3_ss, sigma, stream()); }

// The opposite-spin and same-spin problem lists of a context as one list
// (one launch fills the GPU's waves better than two).  Rebuilt when either
// source job changed.
static int build_both(OzJob& both, const OzJob& ab, const OzJob& ss, int bn, cudaStream_t st) {
  if (both.src_ver[0] == ab.version && both.src_ver[1] == ss.version) return kOk;
  both.probs = ab.probs;
  both.segs = ab.segs;
  both.maps = ab.maps;
  const int seg0 = (int)ab.segs.size();
  for (OzProblem P : ss.probs) {
    P.seg_begin += seg0;
    both.probs.push_back(P);
  }
  both.segs.insert(both.segs.end(), ss.segs.begin(), ss.segs.end());
  both.maps.insert(both.maps.end(), ss.maps.begin(), ss.maps.end());
  both.sh = ab.sh;
  both.sh.insert(both.sh.end(), ss.sh.begin(), ss.sh.end());
  both.tiles = add_tiles(both.probs, bn);
  ISCSI_TRY(upload_job(both, st, bn == OZ_BN));
  both.src_ver[0] = ab.version;
  both.src_ver[1] = ss.version;
  return kOk;
}

const OzJob* both_tc_job(Context& ctx, int prec) {
  OzJob& both = prec == 64 ? ctx.oz_both : ctx.t3_both;
  if (build_both(both, prec == 64 ? ctx.oz_ab : ctx.t3_ab, prec == 64 ? ctx.oz_ss : ctx.t3_ss,
                 prec == 64 ? OZ_BN : T3W_BN, stream()) != kOk)
    return nullptr;
  return &both;
}

int both_tc_gemm(Context& ctx, double* sigma) {
  cudaStream_t st = stream();
  ISCSI_TRY(build_both(ctx.oz_both, ctx.oz_ab, ctx.oz_ss, OZ_BN, st));
  return launch_job(ctx, ctx.oz_both, sigma, st);
}

int both_tc32_gemm(Context& ctx, float* sigma) {
  cudaStream_t st = stream();
  ISCSI_TRY(build_both(ctx.t3_both, ctx.t3_ab, ctx.t3_ss, T3W_BN, st));
  return t3_launch(ctx, ctx.t3_both, sigma, st);
}

// one launch of the FP64-accurate (prec 64) or FP32-form (prec 32) contraction
// over a device problem list whose relative outputs use the base table tbases
int launch_tc_problems(const OzProblem* probs, int nprobs, const OzSeg* segs, const OzMaps* maps,
                       void* const* tbases, int tiles, const OzPlan* plan, int prec, int* err, cudaStream_t st) {
  ISCSI_TRY(tc_attr());
  if (prec == 64) {
    if (!plan) return kOk;
    return launch_oz(*plan, probs, segs, maps, nullptr, reinterpret_cast<double* const*>(tbases), err, st);
  }
  if (tiles == 0) return kOk;
  return launch_t3(tiles, probs, nprobs, segs, maps, nullptr, reinterpret_cast<float* const*>(tbases), err, st);
}

// the same-spin string matrices changed in place: cut the slices prepared so far again
int samespin_matrices_changed(Context& ctx) {
  if (ctx.oz_m_ready) ISCSI_TRY(tc_prepare_m(ctx, true));
  if (ctx.t3_m_ready) ISCSI_TRY(t3_prepare_m(ctx, true));
  return kOk;
}

// tensor-core jobs built by other parts of the library (density.cu): segments
// whose K starts at column 0 of both slice arrays
int oz_job_add_seg(OzJob& job, const SliceArray& A, int a_row0, const int* a_exp, const SliceArray& B, int b_row0,
                   const int* b_exp, int K, int nrows_b) {
  return add_seg(job, A, a_row0, 0, a_exp, B, b_row0, 0, b_exp, K, nrows_b);
}

int oz_job_upload(OzJob& job, cudaStream_t st) {
  job.tiles = add_tiles(job.probs);
  return upload_job(job, st);
}

int oz_job_launch(Context& ctx, const OzJob& job, cudaStream_t st) {
  ISCSI_TRY(tc_attr());
  ISCSI_TRY(tc_err_buf(ctx));
  return launch_job(ctx, job, nullptr, st);
}

// the error word of the contraction kernels' bounded waits (device, one int):
// kOk, or kErrWait with a message naming the wait that ran out (its site,
// CTA and position, as oz_wait_code packs them); a raised word is cleared so
// that later launches report only their own waits (synchronises)
int tc_wait_status(int* err, const char* what) {
  if (!err) return kOk;
  int h = 0;
  ISCSI_CUDA(cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost));
  if (!h) return kOk;
  static const char* const kSite[8] = {"an unknown wait",
                                       "a stage's release (producer)",
                                       "the end marker's stage (producer)",
                                       "a stage's data (MMA thread)",
                                       "the accumulators' drain (MMA thread)",
                                       "a chunk's products (epilogue)",
                                       "the split-K meeting (epilogue)",
                                       "a stage's description (MMA thread)"};
  ISCSI_CUDA(cudaMemset(err, 0, sizeof(int)));
  set_error(std::string(what) + ": a bounded device wait ran out in a tensor-core contraction (" + kSite[h & 7] +
            ", CTA " + std::to_string((h >> 19) & 4095) + ", position " + std::to_string((h >> 3) & 0xFFFF) + ")");
  return kErrWait;
}

// The failure path of the contraction kernels' bounded waits, without a fault:
// one CTA waits (oz_wait_bounded, the kernels' own wait) on a barrier that
// nothing arrives on, gives up after `limit` polls and reports through the
// context's error word as the kernels do (site: a stage's data, position 1).
// No tensor memory is involved.
__global__ void k_wait_selftest(int* err, long long limit) {
  __shared__ uint64_t bar;
  __shared__ volatile int abort_s;
  if (threadIdx.x == 0) {
    tc::mbar_init(tc::smem_u32(&bar), 1);
    abort_s = 0;
    tc::fence_mbar_init();
  }
  __syncthreads();
  oz_wait_bounded(&bar, 0, OZ_SITE_FULL, 1, &abort_s, limit);
  __syncthreads();
  if (abort_s && threadIdx.x == 0) atomicCAS(err, 0, abort_s + (int)blockIdx.x * OZ_WAIT_CTA);
}

int tc_wait_selftest(Context& ctx, long long polls) {
  ISCSI_TRY(tc_err_buf(ctx));
  k_wait_selftest<<<1, 64, 0, stream()>>>(ctx.oz_err.as<int>(), polls); ISCSI_COUNT_LAUNCH();
  ISCSI_CUDA(cudaGetLastError());
  return tc_check(ctx);
}

// status of the bounded waits of the context's tensor-core kernels (synchronises)
int tc_check(Context& ctx) {
  const int rc = tc_wait_status(ctx.oz_err.as<int>(), "tensor-core sigma");
  if (rc != kOk) {
    // the aborted launch may have left split-K counters raised: rebuild the
    // context's work lists (and schedules) before the next launch
    ctx.oz_ab.nvec = ctx.oz_ss.nvec = ctx.t3_ab.nvec = ctx.t3_ss.nvec = -1;
    ctx.oz_both.src_ver[0] = ctx.t3_both.src_ver[0] = -1;
  }
  return rc;
}

}  // namespace iscsi
