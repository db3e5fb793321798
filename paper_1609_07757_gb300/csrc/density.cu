// density.cu -- one- and two-body density matrices (Sec. "Density matrices",
// Eqs. d1 and d2) on the GPU, spin-resolved:
//   d1[s][p][q]       = <bra| a+_ps a_qs |ket>
//   d2[b][p][q][r][t] = <bra| a+_ps a+_ru a_tu a_qs |ket>,  (s,u) = aa, ab, bb
//
// The paper builds them with the sigma step's class loops, a product of two CI
// coefficients in place of the integral.  Here each two-body block is one
// Gram-type contraction of "lifted" vectors, on the tensor cores with FP64
// accuracy (the exact bf16 slices of ozaki.cuh):
//   ab: L[(q,t)][(X,Y)] = <X,Y| a_tu a_qs |ket> (X, Y: strings with one alpha
//       and one beta electron removed -- the sigma step's hole strings and its
//       lift tables), so d2_ab[p,q,r,t] = sum_XY L_bra[(p,r)] L_ket[(q,t)];
//   aa: L[{u<v}][(Z,B)] = <Z| a_v a_u |A> c[A,B] with A = Z u {u,v} (Z: strings
//       with two alpha electrons removed), so d2_aa[p,q,r,t] =
//       s(p,r) s(q,t) sum_ZB L_bra[{p,r}] L_ket[{q,t}], s(x,y) = +1 if x < y,
//       -1 if x > y; bb likewise with the roles of the spins exchanged.
// Rows of L are orbital pairs sorted by excitation level and columns are
// grouped by their level class c, so class c only reaches the rows with level
// <= k - c: the product is a sum of prefix blocks, cut into row/column regions
// (the block's "staircase"), one tensor-core problem per region pair.  With
// ket = bra the result is symmetric and only the upper regions (and, in a
// diagonal region, the tiles right of each 128-row block's start) are computed.
// An expansion kernel writes the n^4 tensors from the pair-indexed results.
// d1 comes from d2's partial trace when d2 is computed for that spin (sum_r
// d2_ss[p,q,r,r] = (N_s - 1) d1_s[p,q], summed by the expansion kernel), else
// from a direct kernel over the one-hole strings.
#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "ozaki_digits.cuh"

namespace iscsi {

constexpr int kDmMaxBnd = 2 * kMaxElec + 2;

// ---------------------------------------------------------------------------
// host plan

struct DmPart {            // one column level class of a block
  int col_start = 0;       // first column in the block's column list
  int ncol = 0;            // columns (K)
  int rows = 0;            // rows reached (pairs with level <= k - c)
  int ld = 0;              // ncol rounded up to 16
  int rows_pad = 0;        // rows rounded up to 128
  size_t sl_off = 0;       // element offset of its slices in a slice workspace
};

struct DmBlock {
  int kind = 0;            // 0: ab, 1: aa, 2: bb
  int R = 0;               // rows of the pair-indexed result (largest part rows)
  std::vector<DmPart> parts;
  std::vector<int> bnd;    // region boundaries: 0 = bnd[0] < ... < bnd[nreg] = R
  size_t q_off = 0;        // double offset of the R x R result in the result workspace
  size_t exp_off = 0;      // int offset of its row exponents (parts x R128) in an exponent workspace
  int R128 = 0;
};

struct DensityPlan {
  bool built = false;
  DmBlock blk[3];
  // same-spin tables per spin: pair row of {u<v}, two-hole lift, column list (Z, other string)
  DevBuf pp_row[2], lift2[2], cols[2];
  int nz[2] = {0, 0};
  DevBuf q;                      // FP64 results of all blocks
  DevBuf sl_bra, sl_ket;         // bf16 slices of the bra / ket operands
  DevBuf ex_bra, ex_ket;         // row exponents
  size_t sl_elems = 0, q_elems = 0, ex_elems = 0;
  OzJob job_sym, job_gen;        // ket = bra (upper regions only) / general
  bool sym_ready = false, gen_ready = false;
  double bf16_flops[2] = {0, 0}; // bf16 MMA flops of one launch of each job
  double fp64_flops[2] = {0, 0}; // 2 M N K of the computed regions
  cudaEvent_t ev[2] = {nullptr, nullptr};  // around the last contraction launch
  bool timed = false;
  ~DensityPlan() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  }
};

void density_release(Context& ctx) {
  delete ctx.dm;
  ctx.dm = nullptr;
}

static inline int rup(int x, int m) { return (x + m - 1) / m * m; }

// sorted position of an ascending orbital list: colex rank through the context's rank table
static int host_colex(const int* o, int ne) {
  long long r = 0;
  for (int i = 0; i < ne; ++i) r += binom_ll(o[i], i + 1);
  return (int)r;
}

// same-spin tables of spin s: pairs {u<v} sorted by level, strings Z with two
// electrons removed, the two-hole lift <Z| a_v a_u |A>, and the column list
// (Z, string of the other spin) grouped by level class
static int build_samespin(Context& ctx, DensityPlan& P, int s, DmBlock& B) {
  const int n = ctx.n, ne = ctx.sp[s].ne, nocc = ctx.sp[s].nocc, o = 1 - s;
  const SpinSpace& SO = ctx.sp[o];
  std::vector<int> pos(ctx.sp[s].count);
  ISCSI_CUDA(cudaMemcpy(pos.data(), ctx.sp[s].pos.p, sizeof(int) * pos.size(), cudaMemcpyDeviceToHost));
  // pairs u < v by level lu + lv, then (u, v)
  std::vector<std::pair<int, int>> pairs;
  for (int lev = 0; lev <= 2; ++lev)
    for (int u = 0; u < n; ++u)
      for (int v = u + 1; v < n; ++v)
        if ((u >= nocc) + (v >= nocc) == lev) pairs.push_back({u, v});
  const int npp = (int)pairs.size();
  std::vector<int> pp_row(n * n, -1), pair_lev(npp);
  for (int i = 0; i < npp; ++i) {
    pp_row[pairs[i].first * n + pairs[i].second] = i;
    pair_lev[i] = (pairs[i].first >= nocc) + (pairs[i].second >= nocc);
  }
  // strings Z of ne - 2 electrons (lexicographic), with their levels
  std::vector<std::vector<int>> Z;
  {
    int k = ne - 2;
    std::vector<int> c(k);
    for (int i = 0; i < k; ++i) c[i] = i;
    while (true) {
      Z.push_back(c);
      int i = k - 1;
      while (i >= 0 && c[i] == n - k + i) --i;
      if (i < 0) break;
      ++c[i];
      for (int j = i + 1; j < k; ++j) c[j] = c[j - 1] + 1;
    }
  }
  const int nz = (int)Z.size();
  if ((long long)npp * nz >= (1ll << 31)) {
    set_error("iscsi_density: two-hole string table too large");
    return kErrArg;
  }
  std::vector<int> zlev(nz), lift2((size_t)npp * nz, -1);
  for (int z = 0; z < nz; ++z) {
    int l = 0;
    for (int x : Z[z]) l += (x >= nocc);
    zlev[z] = l;
    for (int i = 0; i < npp; ++i) {
      int u = pairs[i].first, v = pairs[i].second;
      if (std::find(Z[z].begin(), Z[z].end(), u) != Z[z].end() ||
          std::find(Z[z].begin(), Z[z].end(), v) != Z[z].end())
        continue;
      std::vector<int> A = Z[z];
      A.push_back(u);
      A.push_back(v);
      std::sort(A.begin(), A.end());
      // a_u acts first on |A>, then a_v on |A \ u>: signs from the occupied orbitals below each
      int below_u = 0, below_v = 0;
      for (int x : A) {
        if (x < u) ++below_u;
        if (x < v && x != u) ++below_v;
      }
      lift2[(size_t)i * nz + z] = (pos[host_colex(A.data(), ne)] << 1) | ((below_u + below_v) & 1);
    }
  }
  // columns (Z, O) by class c = level(Z) + level(O); O over the other spin's level-sorted strings
  int maxc = 0;
  for (int z = 0; z < nz; ++z) maxc = std::max(maxc, zlev[z] + SO.maxlevel);
  std::vector<int> cols;
  B.parts.clear();
  for (int c = 0; c <= maxc; ++c) {
    DmPart pt;
    pt.col_start = (int)(cols.size() / 2);
    for (int z = 0; z < nz; ++z) {
      int lo = c - zlev[z];
      if (lo < 0 || lo > SO.maxlevel) continue;
      for (int O = SO.level_start[lo]; O < SO.level_start[lo + 1]; ++O) {
        cols.push_back(z);
        cols.push_back(O);
      }
    }
    pt.ncol = (int)(cols.size() / 2) - pt.col_start;
    int rows = 0;
    for (int i = 0; i < npp; ++i)
      if (pair_lev[i] <= ctx.kmax - c) rows = i + 1;
    pt.rows = rows;
    if (pt.ncol > 0 && pt.rows > 0) B.parts.push_back(pt);
  }
  P.nz[s] = nz;
  ISCSI_TRY(P.pp_row[s].alloc(sizeof(int) * pp_row.size()));
  ISCSI_CUDA(cudaMemcpy(P.pp_row[s].p, pp_row.data(), sizeof(int) * pp_row.size(), cudaMemcpyHostToDevice));
  ISCSI_TRY(P.lift2[s].alloc(sizeof(int) * std::max<size_t>(1, lift2.size())));
  ISCSI_CUDA(cudaMemcpy(P.lift2[s].p, lift2.data(), sizeof(int) * lift2.size(), cudaMemcpyHostToDevice));
  ISCSI_TRY(P.cols[s].alloc(sizeof(int) * std::max<size_t>(2, cols.size())));
  if (!cols.empty())
    ISCSI_CUDA(cudaMemcpy(P.cols[s].p, cols.data(), sizeof(int) * cols.size(), cudaMemcpyHostToDevice));
  return kOk;
}

static void set_regions(DmBlock& B) {
  std::vector<int> b = {0};
  for (const DmPart& p : B.parts) b.push_back(p.rows);
  std::sort(b.begin(), b.end());
  b.erase(std::unique(b.begin(), b.end()), b.end());
  B.bnd = b;
  B.R = b.back();
  B.R128 = rup(std::max(B.R, 1), OZ_BM);
}

static int plan_build(Context& ctx) {
  if (!ctx.dm) ctx.dm = new DensityPlan();
  DensityPlan& P = *ctx.dm;
  if (P.built) return kOk;
  cudaStream_t st = stream();
  ISCSI_CUDA(cudaStreamSynchronize(st));
  for (int b = 0; b < 3; ++b) {
    P.blk[b] = DmBlock();
    P.blk[b].kind = b;
  }
  // ab: the sigma step's pairs, hole-pair classes and lift tables
  if (ctx.have_ab || (ctx.na > 0 && ctx.nb > 0)) {
    DmBlock& B = P.blk[0];
    for (int c = 0; c < (int)ctx.cls.size(); ++c) {
      const ColClass& cc = ctx.cls[c];
      if (cc.ncol == 0 || cc.mrows == 0) continue;
      DmPart pt;
      pt.col_start = ctx.hp_class_start[c];
      pt.ncol = cc.ncol;
      pt.rows = cc.mrows;
      B.parts.push_back(pt);
    }
  }
  if (ctx.na >= 2) ISCSI_TRY(build_samespin(ctx, P, 0, P.blk[1]));
  if (ctx.nb >= 2) ISCSI_TRY(build_samespin(ctx, P, 1, P.blk[2]));
  // consecutive classes that reach the same rows are one part (their columns
  // are adjacent in the column lists): one longer K instead of several segments
  for (int b = 0; b < 3; ++b) {
    std::vector<DmPart> merged;
    for (const DmPart& pt : P.blk[b].parts) {
      if (!merged.empty() && merged.back().rows == pt.rows &&
          merged.back().col_start + merged.back().ncol == pt.col_start)
        merged.back().ncol += pt.ncol;
      else
        merged.push_back(pt);
    }
    P.blk[b].parts = merged;
  }
  // workspace layout
  size_t sl = 0, q = 0, ex = 0;
  for (int b = 0; b < 3; ++b) {
    DmBlock& B = P.blk[b];
    if (B.parts.empty()) continue;
    if ((int)B.parts.size() > OZ_MAX_SEGS) {
      set_error("iscsi_density: too many column classes for one tensor-core problem");
      return kErrArg;
    }
    set_regions(B);
    for (DmPart& pt : B.parts) {
      pt.ld = rup(pt.ncol, OZ_BK);
      pt.rows_pad = rup(pt.rows, OZ_BM);
      pt.sl_off = sl;
      sl += (size_t)OZ_S * pt.rows_pad * pt.ld;
      sl = (sl + 127) / 128 * 128;  // 256-byte aligned slice arrays (TMA wants 16)
    }
    B.q_off = q;
    q += (size_t)B.R * B.R;
    q = (q + 31) / 32 * 32;
    B.exp_off = ex;
    ex += (size_t)B.parts.size() * B.R128;
  }
  for (cudaEvent_t& e : P.ev) ISCSI_CUDA(cudaEventCreate(&e));
  P.sl_elems = sl;
  P.q_elems = q;
  P.ex_elems = ex;
  if (sl) ISCSI_TRY(P.sl_bra.alloc(sizeof(__nv_bfloat16) * sl));
  if (q) ISCSI_TRY(P.q.alloc(sizeof(double) * q));
  if (ex) {
    ISCSI_TRY(P.ex_bra.alloc(sizeof(int) * ex));
    ISCSI_CUDA(cudaMemset(P.ex_bra.p, 0, sizeof(int) * ex));
  }
  P.built = true;
  return kOk;
}

// ---------------------------------------------------------------------------
// device: operand values, exponents, slices

struct DmGather {
  int kind;                       // 0 ab, 1 aa, 2 bb
  int n, nholeA, nholeB, nz;
  const int* pair_of;             // ab rows -> q * n + t
  const int* hp_inv;              // ab columns -> X * nholeB + Y
  const int* liftA;
  const int* liftB;
  const int* lift2;               // aa / bb: [pair row][Z] -> (string << 1 | neg) or -1
  const int* cols;                // aa / bb: (Z, other string) per column
  const int8_t* alevel;
  const int* nballow;
  const long long* off;
};

__device__ __forceinline__ double dm_value(const DmGather& g, int col, int row, const double* __restrict__ c) {
  int A, B, neg;
  if (g.kind == 0) {
    int xy = g.hp_inv[col];
    int X = xy / g.nholeB, Y = xy - X * g.nholeB;
    int qt = g.pair_of[row];
    int q = qt / g.n, t = qt - q * g.n;
    int ea = g.liftA[q * g.nholeA + X], eb = g.liftB[t * g.nholeB + Y];
    if (ea < 0 || eb < 0) return 0.0;
    A = ea >> 1;
    B = eb >> 1;
    neg = (ea ^ eb) & 1;
  } else {
    int z = g.cols[2 * col], O = g.cols[2 * col + 1];
    int e = g.lift2[(long long)row * g.nz + z];
    if (e < 0) return 0.0;
    A = g.kind == 1 ? (e >> 1) : O;
    B = g.kind == 1 ? O : (e >> 1);
    neg = e & 1;
  }
  if (B >= g.nballow[g.alevel[A]]) return 0.0;
  double x = c[g.off[A] + B];
  return neg ? -x : x;
}

// One block per row of L (rows_pad rows, ld columns): gathers the row once
// (held in registers, kDmRowRegs values per thread, or re-gathered beyond
// that), takes the row exponent e with max |L[row][:]| 2^-e < 1 (0 for an
// all-zero row, and for the padding rows) and writes the row's slices
// out[s][row][k], zero padded.
// With STAGED (the alpha-beta block with at most kDmStage hole strings per
// spin) the row's lift entries -- a+_q |X> and a+_t |Y> for every X and Y,
// with the target alpha string's offset and allowed beta count -- are staged
// in shared memory first, so an element costs the hole-pair table and c.
constexpr int kDmRowRegs = 16;
constexpr int kDmStage = 256;
struct DmStageRow {
  int a[kDmStage], b[kDmStage], lim[kDmStage];
  long long off[kDmStage];
};

template <bool STAGED>
__device__ __forceinline__ double dm_row_value(const DmGather& g, const DmStageRow& S, int col, int row,
                                               const double* __restrict__ c) {
  if (!STAGED) return dm_value(g, col, row, c);
  const int xy = g.hp_inv[col];
  const int X = xy / g.nholeB, Y = xy - (xy / g.nholeB) * g.nholeB;
  const int ea = S.a[X], eb = S.b[Y];
  if (ea < 0 || eb < 0) return 0.0;
  const int B = eb >> 1;
  if (B >= S.lim[X]) return 0.0;
  const double x = c[S.off[X] + B];
  return ((ea ^ eb) & 1) ? -x : x;
}

template <bool STAGED>
__global__ void __launch_bounds__(256) k_dm_lift_slice(DmGather g, int col_start, int ncol, int rows, int ld,
                                                       int rows_pad, const double* __restrict__ c,
                                                       int* __restrict__ e, __nv_bfloat16* __restrict__ out) {
  const int r = blockIdx.x;
  const long long total = (long long)rows_pad * ld;
  __shared__ DmStageRow S;
  if (STAGED && r < rows) {
    const int qt = g.pair_of[r];
    const int q = qt / g.n, t = qt - (qt / g.n) * g.n;
    for (int X = threadIdx.x; X < g.nholeA; X += blockDim.x) {
      const int ea = g.liftA[q * g.nholeA + X];
      S.a[X] = ea;
      if (ea >= 0) {
        const int A = ea >> 1;
        S.off[X] = g.off[A];
        S.lim[X] = g.nballow[g.alevel[A]];
      }
    }
    for (int Y = threadIdx.x; Y < g.nholeB; Y += blockDim.x) S.b[Y] = g.liftB[t * g.nholeB + Y];
  }
  __syncthreads();
  double v[kDmRowRegs];
  int m = 0;
#pragma unroll
  for (int i = 0; i < kDmRowRegs; ++i) {
    const int k = threadIdx.x + i * blockDim.x;
    v[i] = (r < rows && k < ncol) ? dm_row_value<STAGED>(g, S, col_start + k, r, c) : 0.0;
    m = max(m, oz_exp_field(v[i]));
  }
  for (int k = threadIdx.x + kDmRowRegs * blockDim.x; k < ncol; k += blockDim.x)
    if (r < rows) m = max(m, oz_exp_field(dm_row_value<STAGED>(g, S, col_start + k, r, c)));
  m = __reduce_max_sync(0xffffffffu, m);
  __shared__ int sm[8];
  __shared__ int ex_s;
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    int x = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) x = max(x, sm[i]);
    ex_s = x > 0 ? x - 1022 : 0;
    if (r < rows) e[r] = ex_s;
  }
  __syncthreads();
  const int ex = ex_s;
  __nv_bfloat16* row = out + (long long)r * ld;
  int a[OZ_S];
#pragma unroll
  for (int i = 0; i < kDmRowRegs; ++i) {
    const int k = threadIdx.x + i * blockDim.x;
    if (k < ld) {
      oz_digits(v[i], ex, a);
      oz_store_digits(a, row + k, total);
    }
  }
  for (int k = threadIdx.x + kDmRowRegs * blockDim.x; k < ld; k += blockDim.x) {
    const double x = (r < rows && k < ncol) ? dm_row_value<STAGED>(g, S, col_start + k, r, c) : 0.0;
    oz_digits(x, ex, a);
    oz_store_digits(a, row + k, total);
  }
}

// ---------------------------------------------------------------------------
// device: expansion to the n^4 tensors, one-body matrices

struct DmResult {
  const double* q;   // R x R, row-major
  int R, nreg;
  int bnd[kDmMaxBnd];
};

// whether entry (x, y) of a ket = bra result is computed by the contraction:
// regions i < j, or the same region right of the 128-row block's first row
__device__ __forceinline__ bool dm_computed(const DmResult& Q, int x, int y) {
  int i = 0, j = 0;
  while (i + 1 < Q.nreg && x >= Q.bnd[i + 1]) ++i;
  while (j + 1 < Q.nreg && y >= Q.bnd[j + 1]) ++j;
  return i < j || (i == j && y >= Q.bnd[i] + ((x - Q.bnd[i]) / OZ_BM) * OZ_BM);
}

// ket = bra: every entry that was not computed is copied from its transpose,
// 32 x 32 tiles through shared memory (reads and writes coalesced).  Tiles
// wholly above the diagonal are all computed (x < y lies in the computed part).
__global__ void __launch_bounds__(256) k_dm_mirror(DmResult Q, double* __restrict__ q) {
  __shared__ double tile[32][33];
  const int x0 = blockIdx.y * 32, y0 = blockIdx.x * 32;  // destination rows x, columns y
  if (x0 + 31 < y0) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int i = ty; i < 32; i += 8) {  // source rows y0 + i, columns x0 + tx
    const int ys = y0 + i, xs = x0 + tx;
    tile[i][tx] = (ys < Q.R && xs < Q.R) ? q[(long long)ys * Q.R + xs] : 0.0;
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {  // destination row x0 + i, column y0 + tx
    const int x = x0 + i, y = y0 + tx;
    if (x < Q.R && y < Q.R && !dm_computed(Q, x, y)) q[(long long)x * Q.R + y] = tile[tx][i];
  }
}

// Q[x][y] (0 outside the rows any class reaches)
__device__ __forceinline__ double dm_read(const DmResult& Q, int x, int y) {
  if (x >= Q.R || y >= Q.R) return 0.0;
  return Q.q[(long long)x * Q.R + y];
}

struct DmExpand {
  int n, na, nb;
  DmResult blk[3];        // in d2's block order: aa, ab, bb
  const int* pair_index;  // ab: (p, r) -> row
  const int* pp_row[2];   // aa / bb: {u < v} -> row
};

// d2 block b = 0 (aa) or 2 (bb): s(p,r) s(q,t) Q[{p,r}][{q,t}]
__device__ __forceinline__ double dm_samespin(const DmExpand& E, int b, int p, int q, int r, int t) {
  if (p == r || q == t) return 0.0;
  const int* pr = E.pp_row[b == 0 ? 0 : 1];
  int x = pr[min(p, r) * E.n + max(p, r)], y = pr[min(q, t) * E.n + max(q, t)];
  double v = dm_read(E.blk[b], x, y);
  return ((p < r) == (q < t)) ? v : -v;
}

// one block per (p, q) and d2 block b: writes d2[b][p][q][r][t] for all (r, t),
// consecutive threads on consecutive t (coalesced stores; the pair-indexed
// reads are mostly consecutive within a level group)
// A same-spin block's (p, q) block also yields d1_s[p][q] = sum_r d2_ss[p,q,r,r]
// / (N_s - 1) (written when d1 is given and N_s >= 2).
__global__ void __launch_bounds__(256) k_dm_expand(DmExpand E, double* __restrict__ d2, double* __restrict__ d1) {
  const int n = E.n, p = blockIdx.x / n, q = blockIdx.x - (blockIdx.x / n) * n, b = blockIdx.y;
  const long long n2 = (long long)n * n;
  double* __restrict__ out = d2 + (long long)b * n2 * n2 + (long long)blockIdx.x * n2;
  const bool ab = b == 1 && E.na > 0 && E.nb > 0;
  const bool ss = b != 1 && (b == 0 ? E.na : E.nb) >= 2;
  double tr = 0.0;
  for (int rt = threadIdx.x; rt < n * n; rt += blockDim.x) {
    const int r = rt / n, t = rt - (rt / n) * n;
    double v = 0.0;
    if (ab) v = dm_read(E.blk[1], E.pair_index[p * n + r], E.pair_index[q * n + t]);
    else if (ss) v = dm_samespin(E, b, p, q, r, t);
    out[rt] = v;
    if (r == t) tr += v;
  }
  if (!ss || !d1) return;
  __shared__ double red[8];
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tr;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
    const int spin = b == 0 ? 0 : 1;
    d1[(long long)spin * n2 + blockIdx.x] = sum / (double)((spin == 0 ? E.na : E.nb) - 1);
  }
}

// d1_s[p][q] = sum_X s(p,X) s(q,X) sum_O bra[X u p, O] ket[X u q, O] over the
// one-hole strings X of spin s (the lift tables), one block per (p, q)
__global__ void __launch_bounds__(256) k_dm_gamma_direct(int n, int spin, int nhole, const int* __restrict__ lift,
                                                         int na_count, const int8_t* __restrict__ alevel,
                                                         const int* __restrict__ nballow,
                                                         const long long* __restrict__ off,
                                                         const double* __restrict__ bra,
                                                         const double* __restrict__ ket, double* __restrict__ d1) {
  const int p = blockIdx.x / n, q = blockIdx.x % n;
  double acc = 0.0;
  for (int X = 0; X < nhole; ++X) {
    int e1 = lift[p * nhole + X], e2 = lift[q * nhole + X];
    if (e1 < 0 || e2 < 0) continue;
    const double sg = ((e1 ^ e2) & 1) ? -1.0 : 1.0;
    const int s1 = e1 >> 1, s2 = e2 >> 1;
    double part = 0.0;
    if (spin == 0) {
      const int m = min(nballow[alevel[s1]], nballow[alevel[s2]]);
      const double* x = bra + off[s1];
      const double* y = ket + off[s2];
      for (int B = threadIdx.x; B < m; B += blockDim.x) part += x[B] * y[B];
    } else {
      for (int A = threadIdx.x; A < na_count; A += blockDim.x) {
        const int nbA = nballow[alevel[A]];
        if (s1 < nbA && s2 < nbA) part += bra[off[A] + s1] * ket[off[A] + s2];
      }
    }
    acc += sg * part;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double sm[8];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sm[i];
    d1[spin * n * n + blockIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------
// host: operands, work lists, launches

static DmGather gather_of(const Context& ctx, const DensityPlan& P, int b) {
  DmGather g;
  std::memset(&g, 0, sizeof(g));
  g.kind = b;
  g.n = ctx.n;
  g.nholeA = ctx.sp[0].nhole;
  g.nholeB = ctx.sp[1].nhole;
  g.pair_of = ctx.pair_of.as<int>();
  g.hp_inv = ctx.hp_inv.as<int>();
  g.liftA = ctx.sp[0].lift.as<int>();
  g.liftB = ctx.sp[1].lift.as<int>();
  if (b > 0) {
    g.lift2 = P.lift2[b - 1].as<int>();
    g.cols = P.cols[b - 1].as<int>();
    g.nz = P.nz[b - 1];
  }
  g.alevel = ctx.sp[0].level.as<int8_t>();
  g.nballow = ctx.nballow.as<int>();
  g.off = ctx.off.as<long long>();
  return g;
}

// slices and row exponents of every part of every block for one vector
static int cut_operands(Context& ctx, const double* v, __nv_bfloat16* sl, int* ex, cudaStream_t st) {
  DensityPlan& P = *ctx.dm;
  for (int b = 0; b < 3; ++b) {
    const DmBlock& B = P.blk[b];
    if (B.parts.empty()) continue;
    DmGather g = gather_of(ctx, P, b);
    for (size_t i = 0; i < B.parts.size(); ++i) {
      const DmPart& pt = B.parts[i];
      int* e = ex + B.exp_off + i * B.R128;
      if (b == 0 && g.nholeA <= kDmStage && g.nholeB <= kDmStage)
        k_dm_lift_slice<true><<<pt.rows_pad, 256, 0, st>>>(g, pt.col_start, pt.ncol, pt.rows, pt.ld, pt.rows_pad, v,
                                                           e, sl + pt.sl_off);
      else
        k_dm_lift_slice<false><<<pt.rows_pad, 256, 0, st>>>(g, pt.col_start, pt.ncol, pt.rows, pt.ld, pt.rows_pad,
                                                            v, e, sl + pt.sl_off);
      ISCSI_COUNT_LAUNCH();
    }
  }
  ISCSI_CUDA(cudaGetLastError());
  return kOk;
}

// one problem (rows [r0, r1) x columns [c0, c1) of block B's result) with the
// parts that reach both ranges
static int add_problem(DensityPlan& P, OzJob& job, const DmBlock& B, int r0, int r1, int c0, int c1, bool sym,
                       int reg_rows_end, int reg_cols_end, double* flops) {
  OzProblem pr;
  std::memset(&pr, 0, sizeof(pr));
  pr.t = reinterpret_cast<long long>(P.q.as<double>() + B.q_off + (size_t)r0 * B.R + c0);
  pr.t_rel = 0;
  pr.ldt = B.R;
  pr.M = r1 - r0;
  pr.N = c1 - c0;
  pr.seg_begin = (int)job.segs.size();
  pr.accumulate = 0;
  const __nv_bfloat16* abase = P.sl_bra.as<__nv_bfloat16>();
  const __nv_bfloat16* bbase = sym ? abase : P.sl_ket.as<__nv_bfloat16>();
  const int* aex = P.ex_bra.as<int>();
  const int* bex = sym ? aex : P.ex_ket.as<int>();
  for (size_t i = 0; i < B.parts.size(); ++i) {
    const DmPart& pt = B.parts[i];
    if (pt.rows < reg_rows_end || pt.rows < reg_cols_end) continue;
    SliceArray a{abase + pt.sl_off, pt.ld, pt.rows_pad, (long long)pt.rows_pad * pt.ld};
    SliceArray b{bbase + pt.sl_off, pt.ld, pt.rows_pad, (long long)pt.rows_pad * pt.ld};
    ISCSI_TRY(oz_job_add_seg(job, a, r0, aex + B.exp_off + i * B.R128 + r0, b, c0, bex + B.exp_off + i * B.R128 + c0,
                             pt.ld, pr.N));
    flops[0] += 28.0 * 2.0 * pr.M * (double)pr.N * pt.ld;
    flops[1] += 2.0 * pr.M * (double)pr.N * pt.ncol;
  }
  pr.seg_count = (int)job.segs.size() - pr.seg_begin;
  if (pr.seg_count > 0) job.probs.push_back(pr);
  return kOk;
}

static int build_job(Context& ctx, bool sym) {
  DensityPlan& P = *ctx.dm;
  OzJob& job = sym ? P.job_sym : P.job_gen;
  job.probs.clear();
  job.segs.clear();
  job.maps.clear();
  job.sh.clear();
  double f[2] = {0.0, 0.0};
  for (int b = 0; b < 3; ++b) {
    const DmBlock& B = P.blk[b];
    if (B.parts.empty()) continue;
    const int nreg = (int)B.bnd.size() - 1;
    for (int i = 0; i < nreg; ++i)
      for (int j = sym ? i : 0; j < nreg; ++j) {
        const int r0 = B.bnd[i], r1 = B.bnd[i + 1], c0 = B.bnd[j], c1 = B.bnd[j + 1];
        if (sym && i == j) {
          // diagonal region: per 128-row block, the columns from the block's first row on
          for (int rb = r0; rb < r1; rb += OZ_BM)
            ISCSI_TRY(add_problem(P, job, B, rb, std::min(rb + OZ_BM, r1), rb, c1, true, r1, c1, f));
        } else {
          ISCSI_TRY(add_problem(P, job, B, r0, r1, c0, c1, sym, r1, c1, f));
        }
      }
  }
  P.bf16_flops[sym ? 0 : 1] = f[0];
  P.fp64_flops[sym ? 0 : 1] = f[1];
  ISCSI_TRY(oz_job_upload(job, stream()));
  (sym ? P.sym_ready : P.gen_ready) = true;
  return kOk;
}

int density_run(Context& ctx, const double* bra, const double* ket, double* d1, double* d2) {
  cudaStream_t st = stream();
  const bool sym = (ket == nullptr || ket == bra);
  if (!ket) ket = bra;
  const int n = ctx.n;
  DensityPlan* Pp = nullptr;
  DmExpand E;
  std::memset(&E, 0, sizeof(E));
  E.n = n;
  E.na = ctx.na;
  E.nb = ctx.nb;
  E.pair_index = ctx.pair_index.as<int>();
  if (d2) {
    ISCSI_TRY(plan_build(ctx));
    Pp = ctx.dm;
    DensityPlan& P = *Pp;
    if (!sym && !P.sl_ket.p && P.sl_elems) {
      ISCSI_TRY(P.sl_ket.alloc(sizeof(__nv_bfloat16) * P.sl_elems));
      ISCSI_TRY(P.ex_ket.alloc(sizeof(int) * P.ex_elems));
      ISCSI_CUDA(cudaMemsetAsync(P.ex_ket.p, 0, sizeof(int) * P.ex_elems, st));
    }
    if (sym ? !P.sym_ready : !P.gen_ready) ISCSI_TRY(build_job(ctx, sym));
    ISCSI_TRY(cut_operands(ctx, bra, P.sl_bra.as<__nv_bfloat16>(), P.ex_bra.as<int>(), st));
    if (!sym) ISCSI_TRY(cut_operands(ctx, ket, P.sl_ket.as<__nv_bfloat16>(), P.ex_ket.as<int>(), st));
    const OzJob& job = sym ? P.job_sym : P.job_gen;
    if (job.tiles > 0) {
      const bool ev = !ctx.capturing;
      if (ev) ISCSI_CUDA(cudaEventRecord(P.ev[0], st));
      ISCSI_TRY(oz_job_launch(ctx, job, st));
      if (ev) ISCSI_CUDA(cudaEventRecord(P.ev[1], st));
      P.timed = ev;
    }
    // expansion: slot 0 = aa, 1 = ab, 2 = bb (d2's block order)
    const int slot_of_plan[3] = {1, 0, 2};
    for (int b = 0; b < 3; ++b) {
      const DmBlock& B = P.blk[b];
      DmResult& R = E.blk[slot_of_plan[b]];
      R.q = P.q.as<double>() + B.q_off;
      R.R = B.parts.empty() ? 0 : B.R;
      R.nreg = B.parts.empty() ? 0 : (int)B.bnd.size() - 1;
      for (int i = 0; i < (int)B.bnd.size() && i < kDmMaxBnd; ++i) R.bnd[i] = B.bnd[i];
    }
    E.pp_row[0] = P.pp_row[0].as<int>();
    E.pp_row[1] = P.pp_row[1].as<int>();
    if (sym)
      for (int b = 0; b < 3; ++b) {
        const DmResult& R = E.blk[b];
        if (R.R == 0) continue;
        dim3 grid((R.R + 31) / 32, (R.R + 31) / 32);
        k_dm_mirror<<<grid, 256, 0, st>>>(R, const_cast<double*>(R.q)); ISCSI_COUNT_LAUNCH();
      }
    k_dm_expand<<<dim3(n * n, 3), 256, 0, st>>>(E, d2, d1); ISCSI_COUNT_LAUNCH();
    ISCSI_CUDA(cudaGetLastError());
  }
  if (d1) {
    for (int s = 0; s < 2; ++s) {
      const int ne = s == 0 ? ctx.na : ctx.nb;
      if (d2 && ne >= 2) {
        // written by the expansion
      } else if (ne == 0) {
        ISCSI_CUDA(cudaMemsetAsync(d1 + (size_t)s * n * n, 0, sizeof(double) * n * n, st));
      } else {
        k_dm_gamma_direct<<<n * n, 256, 0, st>>>(n, s, ctx.sp[s].nhole, ctx.sp[s].lift.as<int>(), ctx.sp[0].count,
                                                 ctx.sp[0].level.as<int8_t>(), ctx.nballow.as<int>(),
                                                 ctx.off.as<long long>(), bra, ket, d1); ISCSI_COUNT_LAUNCH();
      }
    }
    ISCSI_CUDA(cudaGetLastError());
  }
  return kOk;
}

double density_gemm_ms(Context& ctx) {
  if (!ctx.dm || !ctx.dm->timed) return 0.0;
  if (cudaEventSynchronize(ctx.dm->ev[1]) != cudaSuccess) return 0.0;
  float ms = 0.0f;
  if (cudaEventElapsedTime(&ms, ctx.dm->ev[0], ctx.dm->ev[1]) != cudaSuccess) return 0.0;
  return ms;
}

double density_flops(const Context& ctx, int sym, int which) {
  if (!ctx.dm) return 0.0;
  return which == 0 ? ctx.dm->bf16_flops[sym ? 0 : 1] : ctx.dm->fp64_flops[sym ? 0 : 1];
}

}  // namespace iscsi
