// sigma_tc.cu -- the opposite-spin contraction of the FP64 sigma step on the
// tensor cores (tcgen05), with FP64 accuracy from exact bf16 slices (ozaki.cuh).
//
// Per sigma call and column level class c:
//   1. k_oz_col_exp   : exponent of the largest |Ct| in each column (X,Y,v)
//   2. k_oz_lift_slice: Ct^T[(X,Y,v)][(q,s)] = s s c[X u q, Y u s] gathered
//                       through the contraction/addition tables and cut into
//                       7 bf16 slices (the B operand, K-major)
//   3. k_oz_gemm      : T_c = G[:M_c, :K_c] Ct_c for all classes in one launch
// G's slices are built once per context (first use).
#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "ozaki.cuh"

namespace iscsi {

struct TcClass {
  int ncols;        // hole pairs x vectors
  int krows;        // K of the class
  int kpad;         // krows rounded up to 16
  int npad;         // ncols rounded up to 64
  int hp_start;     // first hole pair of the class in hp_inv
  long long bs_off; // element offset of the class's slices in the B buffer (slice 0)
  long long exp_off;
  long long tot;    // ncols * kpad (elements gathered)
};

struct TcTable {
  int nclass;
  int nvec;
  TcClass c[2 * kMaxElec];
  long long start[2 * kMaxElec + 1];  // flattened (col, k) element offsets
};

__device__ __forceinline__ double tc_gather(const TcClass& C, int nvec, int col, int k, int n, int nholeA,
                                            int nholeB, const int* __restrict__ pair_of,
                                            const int* __restrict__ hp_inv, const int* __restrict__ liftA,
                                            const int* __restrict__ liftB, const int8_t* __restrict__ alevel,
                                            const int* __restrict__ nballow, const long long* __restrict__ off,
                                            const double* __restrict__ c, long long ndet) {
  if (k >= C.krows) return 0.0;
  int hp = col / nvec, v = col % nvec;
  int xy = hp_inv[C.hp_start + hp];
  int X = xy / nholeB, Y = xy % nholeB;
  int qs = pair_of[k];
  int q = qs / n, s = qs % n;
  int ea = liftA[q * nholeA + X], eb = liftB[s * nholeB + Y];
  if (ea < 0 || eb < 0) return 0.0;
  int Ap = ea >> 1, Bp = eb >> 1;
  if (Bp >= nballow[alevel[Ap]]) return 0.0;
  double x = c[(long long)v * ndet + off[Ap] + Bp];
  return ((ea ^ eb) & 1) ? -x : x;
}

// exponent (frexp) of max |Ct| per column, by atomicMax; exps start at INT_MIN
__global__ void k_oz_col_exp(TcTable tt, int n, int nholeA, int nholeB, const int* __restrict__ pair_of,
                             const int* __restrict__ hp_inv, const int* __restrict__ liftA,
                             const int* __restrict__ liftB, const int8_t* __restrict__ alevel,
                             const int* __restrict__ nballow, const long long* __restrict__ off,
                             const double* __restrict__ c, long long ndet, int* __restrict__ exps) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= tt.start[tt.nclass]) return;
  int cl = 0;
  while (t >= tt.start[cl + 1]) ++cl;
  const TcClass& C = tt.c[cl];
  long long local = t - tt.start[cl];
  int col = (int)(local / C.kpad), k = (int)(local % C.kpad);
  double x = tc_gather(C, tt.nvec, col, k, n, nholeA, nholeB, pair_of, hp_inv, liftA, liftB, alevel, nballow, off,
                       c, ndet);
  int e = INT_MIN;
  if (x != 0.0) frexp(x, &e);
  // one atomic per (warp, column): lanes of the same column reduce together
  int key = (int)(C.exp_off + col);
  unsigned group = __match_any_sync(__activemask(), key);
  int m = __reduce_max_sync(group, e);
  if ((int)(threadIdx.x & 31) == __ffs(group) - 1 && m != INT_MIN) atomicMax(&exps[key], m);
}

__global__ void k_oz_fill_int(int* __restrict__ p, long long count, int value) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < count) p[t] = value;
}

__global__ void k_oz_fix_exp(int* __restrict__ exps, long long count) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < count && exps[t] == INT_MIN) exps[t] = 0;
}

__global__ void k_oz_lift_slice(TcTable tt, int n, int nholeA, int nholeB, const int* __restrict__ pair_of,
                                const int* __restrict__ hp_inv, const int* __restrict__ liftA,
                                const int* __restrict__ liftB, const int8_t* __restrict__ alevel,
                                const int* __restrict__ nballow, const long long* __restrict__ off,
                                const double* __restrict__ c, long long ndet, const int* __restrict__ exps,
                                __nv_bfloat16* __restrict__ bs) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= tt.start[tt.nclass]) return;
  int cl = 0;
  while (t >= tt.start[cl + 1]) ++cl;
  const TcClass& C = tt.c[cl];
  long long local = t - tt.start[cl];
  int col = (int)(local / C.kpad), k = (int)(local % C.kpad);
  double x = tc_gather(C, tt.nvec, col, k, n, nholeA, nholeB, pair_of, hp_inv, liftA, liftB, alevel, nballow, off,
                       c, ndet);
  x = ldexp(x, -exps[C.exp_off + col]);
  long long slice = (long long)C.npad * C.kpad;
  __nv_bfloat16* out = bs + C.bs_off + (long long)col * C.kpad + k;
#pragma unroll
  for (int s = 0; s < OZ_S; ++s) {
    double v = x * 128.0;
    double a = rint(v);
    x = v - a;
    out[s * slice] = __float2bfloat16_rn((float)ldexp(a, -OZ_BITS * s));
  }
}

static int tc_prepare_g(Context& ctx) {
  if (ctx.oz_gs.p) return kOk;
  cudaStream_t st = stream();
  int np = ctx.npairs;
  ctx.oz_mpad = (np + OZ_BM - 1) / OZ_BM * OZ_BM;
  ctx.oz_kpad = (np + OZ_BK - 1) / OZ_BK * OZ_BK;
  long long slice = (long long)ctx.oz_mpad * ctx.oz_kpad;
  ISCSI_TRY(ctx.oz_gs.alloc(sizeof(__nv_bfloat16) * slice * OZ_S));
  ISCSI_TRY(ctx.oz_gexp.alloc(sizeof(int) * np));
  ISCSI_TRY(ctx.oz_err.alloc(sizeof(int)));
  ISCSI_CUDA(cudaMemsetAsync(ctx.oz_err.p, 0, sizeof(int), st));
  k_oz_row_exp<<<np, 256, 0, st>>>(ctx.G64.as<double>(), np, np, np, ctx.oz_gexp.as<int>());
  k_oz_slice<<<launch_blocks(slice, 256), 256, 0, st>>>(ctx.G64.as<double>(), np, np, np, ctx.oz_gexp.as<int>(),
                                                        ctx.oz_gs.as<__nv_bfloat16>(), slice, ctx.oz_kpad,
                                                        ctx.oz_mpad);
  ISCSI_CUDA(cudaGetLastError());
  static bool attr_done = false;
  if (!attr_done) {
    ISCSI_CUDA(cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM_BYTES));
    attr_done = true;
  }
  return kOk;
}

// T_c for all column classes (FP64 out, layout of the fold's workspace)
int opposite_tc(Context& ctx, const double* c, double* ttw, int nvec) {
  cudaStream_t st = stream();
  ISCSI_TRY(tc_prepare_g(ctx));
  TcTable tt;
  std::memset(&tt, 0, sizeof(tt));
  tt.nvec = nvec;
  std::vector<OzProblem> probs;
  long long bs_elems = 0, exp_elems = 0, flat = 0, t_off = 0;
  int tiles = 0;
  for (int cl = 0; cl < (int)ctx.cls.size(); ++cl) {
    const ColClass& cc = ctx.cls[cl];
    if (cc.ncol == 0 || cc.mrows == 0) continue;
    TcClass C;
    C.ncols = cc.ncol * nvec;
    C.krows = cc.krows;
    C.kpad = (cc.krows + OZ_BK - 1) / OZ_BK * OZ_BK;
    C.npad = (C.ncols + OZ_BN - 1) / OZ_BN * OZ_BN;
    C.hp_start = ctx.hp_class_start[cl];
    C.bs_off = bs_elems;
    C.exp_off = exp_elems;
    C.tot = (long long)C.ncols * C.kpad;
    tt.start[tt.nclass] = flat;
    tt.c[tt.nclass++] = C;
    flat += C.tot;
    OzProblem P;
    P.as = nullptr;  // set below (base pointer known after allocation)
    P.a_slice = (long long)ctx.oz_mpad * ctx.oz_kpad;
    P.b_slice = (long long)C.npad * C.kpad;
    P.lda = ctx.oz_kpad;
    P.ldb = C.kpad;
    P.M = cc.mrows;
    P.N = C.ncols;
    P.K = C.kpad;
    P.ldt = C.ncols;
    P.tiles_n = C.npad / OZ_BN;
    P.tile_begin = tiles;
    tiles += ((cc.mrows + OZ_BM - 1) / OZ_BM) * P.tiles_n;
    // T_c sits where the fold expects it: classes in order, mrows x ncols each
    P.t = ttw + t_off;
    t_off += (long long)cc.mrows * C.ncols;
    probs.push_back(P);
    bs_elems += (long long)OZ_S * C.npad * C.kpad;
    exp_elems += C.ncols;
  }
  tt.start[tt.nclass] = flat;
  if (probs.empty()) return kOk;
  if (ctx.oz_bs_elems < bs_elems) {
    ISCSI_TRY(ctx.oz_bs.alloc(sizeof(__nv_bfloat16) * bs_elems));
    // padding rows of every class stay zero from here on
    ISCSI_CUDA(cudaMemsetAsync(ctx.oz_bs.p, 0, sizeof(__nv_bfloat16) * bs_elems, st));
    ctx.oz_bs_elems = bs_elems;
    ctx.oz_layout_nvec = -1;
    ctx.oz_probs_nvec = -1;  // slice base pointers changed
  } else if (ctx.oz_layout_nvec != nvec) {
    ISCSI_CUDA(cudaMemsetAsync(ctx.oz_bs.p, 0, sizeof(__nv_bfloat16) * ctx.oz_bs_elems, st));
  }
  ctx.oz_layout_nvec = nvec;
  if ((long long)(ctx.oz_bexp.bytes / sizeof(int)) < exp_elems) {
    ISCSI_TRY(ctx.oz_bexp.alloc(sizeof(int) * exp_elems));
    ctx.oz_probs_nvec = -1;
  }
  if (ctx.oz_probs_nvec != nvec) {
    // the problem list depends on nvec and the workspaces only: upload once
    ISCSI_TRY(ctx.oz_probs.grow(sizeof(OzProblem) * probs.size()));
    for (size_t i = 0; i < probs.size(); ++i) {
      probs[i].as = ctx.oz_gs.as<__nv_bfloat16>();
      probs[i].a_exp = ctx.oz_gexp.as<int>();
      probs[i].bs = ctx.oz_bs.as<__nv_bfloat16>() + tt.c[i].bs_off;
      probs[i].b_exp = ctx.oz_bexp.as<int>() + tt.c[i].exp_off;
    }
    ISCSI_CUDA(cudaMemcpyAsync(ctx.oz_probs.p, probs.data(), sizeof(OzProblem) * probs.size(),
                               cudaMemcpyHostToDevice, st));
    ISCSI_CUDA(cudaStreamSynchronize(st));  // probs must outlive the copy
    ctx.oz_probs_nvec = nvec;
    ctx.oz_nprobs = (int)probs.size();
    ctx.oz_tiles = tiles;
  }
  k_oz_fill_int<<<launch_blocks(exp_elems, 256), 256, 0, st>>>(ctx.oz_bexp.as<int>(), exp_elems, INT_MIN);
  const SpinSpace& SA = ctx.sp[0];
  const SpinSpace& SB = ctx.sp[1];
  k_oz_col_exp<<<launch_blocks(flat, 256), 256, 0, st>>>(tt, ctx.n, SA.nhole, SB.nhole, ctx.pair_of.as<int>(),
                                                          ctx.hp_inv.as<int>(), SA.lift.as<int>(), SB.lift.as<int>(),
                                                          SA.level.as<int8_t>(), ctx.nballow.as<int>(),
                                                          ctx.off.as<long long>(), c, ctx.ndet, ctx.oz_bexp.as<int>());
  k_oz_fix_exp<<<launch_blocks(exp_elems, 256), 256, 0, st>>>(ctx.oz_bexp.as<int>(), exp_elems);
  k_oz_lift_slice<<<launch_blocks(flat, 256), 256, 0, st>>>(
      tt, ctx.n, SA.nhole, SB.nhole, ctx.pair_of.as<int>(), ctx.hp_inv.as<int>(), SA.lift.as<int>(), SB.lift.as<int>(),
      SA.level.as<int8_t>(), ctx.nballow.as<int>(), ctx.off.as<long long>(), c, ctx.ndet, ctx.oz_bexp.as<int>(),
      ctx.oz_bs.as<__nv_bfloat16>());
  ISCSI_CUDA(cudaGetLastError());
  k_oz_gemm<<<ctx.oz_tiles, OZ_THREADS, OZ_SMEM_BYTES, st>>>(ctx.oz_probs.as<OzProblem>(), ctx.oz_nprobs,
                                                             ctx.oz_err.as<int>());
  ISCSI_CUDA(cudaGetLastError());
  return kOk;
}

// status of the bounded waits of the tensor-core kernels (synchronises)
int tc_check(Context& ctx) {
  if (!ctx.oz_err.p) return kOk;
  int h = 0;
  ISCSI_CUDA(cudaMemcpy(&h, ctx.oz_err.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    set_error("tensor-core sigma: a bounded device wait ran out");
    return kErrWait;
  }
  return kOk;
}

}  // namespace iscsi
