// sigma.cu -- the ISCI sigma step sigma = H_tau c on the GPU.
//
// The 42 generalised matrix-vector products of Eqs. class_to_ex_dx..the_end
// are grouped by what they touch:
//
//   opposite-spin (16 terms of H_{2,0,0}): the separability of Eq. final lets
//     every term factor into an alpha string equation and a beta string
//     equation (Eqs. four-last).  Writing E^a_pq = a+_p a_q through the hole
//     strings X (one electron removed, the intermediate strings of the
//     contraction/addition loops of Sec. "Second part"),
//       sigma[A,B] = sum_{(p,X)->A} sum_{(r,Y)->B} s s T[(p,r),(X,Y)],
//       T[(p,r),(X,Y)] = sum_{q,s} g_pqrs Ct[(q,s),(X,Y)],
//       Ct[(q,s),(X,Y)] = s s c[X u q, Y u s],
//     so the integral-outer loop of the paper becomes a dense contraction
//     over the integral indices (q,s), the intermediate of Eqs. h200ca-h200ab
//     generalised to all terms.  Ct is "lift", T is a grouped GEMM, the gather
//     into sigma is "fold".  Screened units are zeros of G.
//   one-body and same-spin (8 + 18 terms): each spin's surviving units are
//     summed into a dense string Hamiltonian M_sigma at set-up, and the sigma
//     contribution is M_alpha C and C M_beta^T per excitation-level block of the
//     CI vector (the blocks of Fig. cisdt), accumulated into the output tile
//     in registers, so no atomics are needed.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "internal.cuh"

namespace iscsi {

// ---------------------------------------------------------------------------
// grouped, segmented tile GEMM:  C[M x N] (+)= sum_seg A_seg[M x K_seg] B_seg[K_seg x N]

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    k_grouped_gemm(const Problem<T>* __restrict__ probs, int nprobs, const Segment<T>* __restrict__ segs,
                   const T* __restrict__ cbase, T* sbase) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int LA = BM * BK / NT;  // A elements loaded per thread per K step
  constexpr int LB = BK * BN / NT;
  static_assert(BM * BK % NT == 0 && BK * BN % NT == 0, "tile shape");
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN];

  int tile = blockIdx.x;
  int lo = 0, hi = nprobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (probs[mid].tile_begin <= tile) lo = mid;
    else hi = mid - 1;
  }
  const Problem<T> P = probs[lo];
  auto resolve = [&](long long v, int src) -> const T* {
    return src == kSrcC ? cbase + v : src == kSrcSigma ? sbase + v : reinterpret_cast<const T*>(v);
  };
  T* Cp = const_cast<T*>(resolve(P.c, P.csrc));
  int t = tile - P.tile_begin;
  int m0 = (t / P.tiles_n) * BM, n0 = (t % P.tiles_n) * BN;
  int tx = threadIdx.x % (BN / TN), ty = threadIdx.x / (BN / TN);

  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  for (int sg = 0; sg < P.seg_count; ++sg) {
    const Segment<T> S = segs[P.seg_begin + sg];
    const T* Ap = resolve(S.a, S.asrc);
    const T* Bp = resolve(S.b, S.bsrc);
    int bcols = min(S.bcols, P.N);
    T ra[LA], rb[LB];
    auto load = [&](int k0) {
#pragma unroll
      for (int u = 0; u < LA; ++u) {
        int i = threadIdx.x + u * NT;
        int r = i / BK, kk = i % BK;
        int gm = m0 + r, gk = k0 + kk;
        ra[u] = (gm < P.M && gk < S.K) ? Ap[(long long)gm * S.lda + gk] : T(0);
      }
#pragma unroll
      for (int u = 0; u < LB; ++u) {
        int i = threadIdx.x + u * NT;
        int kk = i / BN, cc = i % BN;
        int gk = k0 + kk, gn = n0 + cc;
        rb[u] = (gk < S.K && gn < bcols) ? Bp[(long long)gk * S.ldb + gn] : T(0);
      }
    };
    load(0);
    for (int k0 = 0; k0 < S.K; k0 += BK) {
      __syncthreads();
#pragma unroll
      for (int u = 0; u < LA; ++u) {
        int i = threadIdx.x + u * NT;
        As[i % BK][i / BK] = ra[u];
      }
#pragma unroll
      for (int u = 0; u < LB; ++u) {
        int i = threadIdx.x + u * NT;
        Bs[i / BN][i % BN] = rb[u];
      }
      __syncthreads();
      if (k0 + BK < S.K) load(k0 + BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int gm = m0 + ty * TM + i;
    if (gm >= P.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int gn = n0 + tx * TN + j;
      if (gn >= P.N) continue;
      T* c = Cp + (long long)gm * P.ldc + gn;
      *c = P.accumulate ? *c + acc[i][j] : acc[i][j];
    }
  }
}

// Thin problems (N <= 16 columns, e.g. the single allowed beta string of the
// highest-level CISD block): one warp per output row, lanes split K, the
// per-column partial sums are reduced with shuffles.  The column count is a
// template parameter so no FMA is spent on absent columns.
template <typename T, int NB>
__device__ __forceinline__ void thin_row_seg(T (&acc)[16], const T* __restrict__ Ap, const T* __restrict__ Bp,
                                             int K, long long ldb, int lane) {
  for (int k = lane; k < K; k += 32) {
    T a = Ap[k];
    const T* br = Bp + (long long)k * ldb;
#pragma unroll
    for (int n = 0; n < NB; ++n) acc[n] = fma(a, br[n], acc[n]);
  }
}

template <typename T, int MB>
__device__ __forceinline__ void mthin_col_seg(T (&acc)[16], const T* __restrict__ Ap, long long lda,
                                              const T* __restrict__ Bp, long long ldb, int k0, int k1) {
  for (int k = k0; k < k1; ++k) {
    T b = Bp[(long long)k * ldb];
#pragma unroll
    for (int m = 0; m < MB; ++m) acc[m] = fma(Ap[(long long)m * lda + k], b, acc[m]);
  }
}
template <typename T>
__global__ void __launch_bounds__(256)
    k_grouped_thin(const Problem<T>* __restrict__ probs, int nprobs, const Segment<T>* __restrict__ segs,
                   const T* __restrict__ cbase, T* sbase, int total_rows) {
  int item = blockIdx.x * 8 + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (item >= total_rows) return;
  int lo = 0, hi = nprobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (probs[mid].tile_begin <= item) lo = mid;
    else hi = mid - 1;
  }
  const Problem<T> P = probs[lo];
  int row = item - P.tile_begin;
  auto resolve = [&](long long v, int src) -> const T* {
    return src == kSrcC ? cbase + v : src == kSrcSigma ? sbase + v : reinterpret_cast<const T*>(v);
  };
  T acc[kThinN];
#pragma unroll
  for (int n = 0; n < kThinN; ++n) acc[n] = T(0);
  for (int sg = 0; sg < P.seg_count; ++sg) {
    const Segment<T> S = segs[P.seg_begin + sg];
    const T* Ap = resolve(S.a, S.asrc) + (long long)row * S.lda;
    const T* Bp = resolve(S.b, S.bsrc);
    int bcols = min(S.bcols, P.N);
    switch (bcols) {
#define THIN_CASE(NB) \
  case NB:            \
    thin_row_seg<T, NB>(acc, Ap, Bp, S.K, S.ldb, lane); \
    break;
      THIN_CASE(1) THIN_CASE(2) THIN_CASE(3) THIN_CASE(4) THIN_CASE(5) THIN_CASE(6) THIN_CASE(7) THIN_CASE(8)
      THIN_CASE(9) THIN_CASE(10) THIN_CASE(11) THIN_CASE(12) THIN_CASE(13) THIN_CASE(14) THIN_CASE(15)
      THIN_CASE(16)
#undef THIN_CASE
      default:
        break;
    }
  }
#pragma unroll
  for (int n = 0; n < kThinN; ++n)
    for (int o = 16; o; o >>= 1) acc[n] += __shfl_xor_sync(0xffffffffu, acc[n], o);
  T* Cp = const_cast<T*>(resolve(P.c, P.csrc)) + (long long)row * P.ldc;
#pragma unroll
  for (int n = 0; n < kThinN; ++n)
    if (lane == n && n < P.N) Cp[n] = P.accumulate ? Cp[n] + acc[n] : acc[n];
}

// Problems with at most kThinN rows (e.g. the reference row block): split K
// into chunks of kMthinChunk over the concatenated segments; one thread per
// (output column, K chunk) accumulates up to kThinN rows, partial sums go to
// part[chunk][problem offset + m * N + n] and a second kernel adds them in
// chunk order (deterministic).  tile_begin = first column item of the
// problem, seg K ranges are taken in order.
constexpr int kMthinChunk = 64;

template <typename T>
__global__ void __launch_bounds__(256)
    k_grouped_mthin(const Problem<T>* __restrict__ probs, int nprobs, const Segment<T>* __restrict__ segs,
                    const long long* __restrict__ part_off, const T* __restrict__ cbase, T* sbase, int total_cols,
                    long long part_stride, T* __restrict__ part) {
  int item = blockIdx.x * 256 + threadIdx.x;
  if (item >= total_cols) return;
  int lo = 0, hi = nprobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (probs[mid].tile_begin <= item) lo = mid;
    else hi = mid - 1;
  }
  const Problem<T> P = probs[lo];
  int n = item - P.tile_begin;
  long long k_lo = (long long)blockIdx.y * kMthinChunk, k_hi = k_lo + kMthinChunk;
  auto resolve = [&](long long v, int src) -> const T* {
    return src == kSrcC ? cbase + v : src == kSrcSigma ? sbase + v : reinterpret_cast<const T*>(v);
  };
  T acc[kThinN];
#pragma unroll
  for (int m = 0; m < kThinN; ++m) acc[m] = T(0);
  long long kbase = 0;
  for (int sg = 0; sg < P.seg_count && kbase < k_hi; ++sg) {
    const Segment<T> S = segs[P.seg_begin + sg];
    long long a0 = max(k_lo, kbase), a1 = min(k_hi, kbase + S.K);
    if (a0 < a1 && n < min(S.bcols, P.N)) {
      const T* Ap = resolve(S.a, S.asrc);
      const T* Bp = resolve(S.b, S.bsrc) + n;
      int k0 = (int)(a0 - kbase), k1 = (int)(a1 - kbase);
      switch (P.M) {
#define MTHIN_CASE(MB) \
  case MB:             \
    mthin_col_seg<T, MB>(acc, Ap, S.lda, Bp, S.ldb, k0, k1); \
    break;
        MTHIN_CASE(1) MTHIN_CASE(2) MTHIN_CASE(3) MTHIN_CASE(4) MTHIN_CASE(5) MTHIN_CASE(6) MTHIN_CASE(7)
        MTHIN_CASE(8) MTHIN_CASE(9) MTHIN_CASE(10) MTHIN_CASE(11) MTHIN_CASE(12) MTHIN_CASE(13) MTHIN_CASE(14)
        MTHIN_CASE(15) MTHIN_CASE(16)
#undef MTHIN_CASE
        default:
          break;
      }
    }
    kbase += S.K;
  }
  T* out = part + blockIdx.y * part_stride + part_off[lo];
#pragma unroll
  for (int m = 0; m < kThinN; ++m)
    if (m < P.M) out[(long long)m * P.N + n] = acc[m];
}

template <typename T>
__global__ void k_mthin_reduce(const Problem<T>* __restrict__ probs, int nprobs, const long long* __restrict__ part_off,
                               T* sbase, const T* __restrict__ cbase, int total_cols, int nchunks,
                               long long part_stride, const T* __restrict__ part) {
  int item = blockIdx.x * 256 + threadIdx.x;
  if (item >= total_cols) return;
  int lo = 0, hi = nprobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (probs[mid].tile_begin <= item) lo = mid;
    else hi = mid - 1;
  }
  const Problem<T> P = probs[lo];
  int n = item - P.tile_begin;
  T* Cp = (P.csrc == kSrcC ? const_cast<T*>(cbase) + P.c : P.csrc == kSrcSigma ? sbase + P.c
                                                                              : reinterpret_cast<T*>(P.c)) + n;
  for (int m = 0; m < P.M; ++m) {
    T acc = T(0);
    for (int c = 0; c < nchunks; ++c) acc += part[c * part_stride + part_off[lo] + (long long)m * P.N + n];
    T* dst = Cp + (long long)m * P.ldc;
    *dst = P.accumulate ? *dst + acc : acc;
  }
}

template <typename T>
struct TileCfg;
template <>
struct TileCfg<double> {
  static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
};
template <>
struct TileCfg<float> {
  static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
};

template <typename T>
static int upload_problems(ProblemList<T>& pl, cudaStream_t st) {
  using C = TileCfg<T>;
  // split off the thin problems
  pl.thin.clear();
  pl.mthin.clear();
  std::vector<Problem<T>> wide;
  pl.thin_rows = 0;
  pl.mthin_cols = 0;
  std::vector<long long> part_off;
  long long part_elems = 0;
  int max_k = 0;
  for (auto& p : pl.probs) {
    if (p.M <= kThinN && p.N > kThinN && p.accumulate) {
      Problem<T> q = p;
      q.tile_begin = pl.mthin_cols;
      pl.mthin_cols += q.N;
      pl.mthin.push_back(q);
      part_off.push_back(part_elems);
      part_elems += (long long)q.M * q.N;
      int k = 0;
      for (int sg = 0; sg < q.seg_count; ++sg) k += pl.segs[q.seg_begin + sg].K;
      max_k = std::max(max_k, k);
    } else if (p.N <= kThinN) {
      Problem<T> q = p;
      q.tile_begin = pl.thin_rows;
      pl.thin_rows += q.M;
      pl.thin.push_back(q);
    } else {
      wide.push_back(p);
    }
  }
  pl.probs.swap(wide);
  if (!pl.mthin.empty()) {
    ISCSI_TRY(pl.d_mthin.grow(sizeof(Problem<T>) * pl.mthin.size()));
    ISCSI_CUDA(cudaMemcpyAsync(pl.d_mthin.p, pl.mthin.data(), sizeof(Problem<T>) * pl.mthin.size(),
                               cudaMemcpyHostToDevice, st));
    pl.mthin_chunks = std::max(1, (max_k + kMthinChunk - 1) / kMthinChunk);
    pl.mthin_part_stride = part_elems;
    ISCSI_TRY(pl.d_part_off.grow(sizeof(long long) * part_off.size()));
    ISCSI_CUDA(cudaMemcpyAsync(pl.d_part_off.p, part_off.data(), sizeof(long long) * part_off.size(),
                               cudaMemcpyHostToDevice, st));
    ISCSI_TRY(pl.d_part.grow(sizeof(T) * part_elems * pl.mthin_chunks));
  }
  if (!pl.thin.empty()) {
    ISCSI_TRY(pl.d_thin.grow(sizeof(Problem<T>) * pl.thin.size()));
    ISCSI_CUDA(cudaMemcpyAsync(pl.d_thin.p, pl.thin.data(), sizeof(Problem<T>) * pl.thin.size(),
                               cudaMemcpyHostToDevice, st));
  }
  int tiles = 0;
  for (auto& p : pl.probs) {
    p.tile_begin = tiles;
    p.tiles_n = (p.N + C::BN - 1) / C::BN;
    tiles += ((p.M + C::BM - 1) / C::BM) * p.tiles_n;
  }
  pl.total_tiles = tiles;
  if (pl.probs.empty() && pl.thin.empty() && pl.mthin.empty()) return kOk;
  ISCSI_TRY(pl.d_probs.grow(sizeof(Problem<T>) * std::max<size_t>(1, pl.probs.size())));
  ISCSI_TRY(pl.d_segs.grow(sizeof(Segment<T>) * std::max<size_t>(1, pl.segs.size())));
  if (!pl.probs.empty())
    ISCSI_CUDA(cudaMemcpyAsync(pl.d_probs.p, pl.probs.data(), sizeof(Problem<T>) * pl.probs.size(),
                               cudaMemcpyHostToDevice, st));
  if (!pl.segs.empty())
    ISCSI_CUDA(cudaMemcpyAsync(pl.d_segs.p, pl.segs.data(), sizeof(Segment<T>) * pl.segs.size(),
                               cudaMemcpyHostToDevice, st));
  // the host vectors must outlive the copies
  ISCSI_CUDA(cudaStreamSynchronize(st));
  return kOk;
}

template <typename T>
static int launch_grouped(const ProblemList<T>& pl, const T* cbase, T* sbase, cudaStream_t st) {
  using C = TileCfg<T>;
  if (pl.mthin_cols > 0) {
    dim3 grid((pl.mthin_cols + 255) / 256, pl.mthin_chunks);
    k_grouped_mthin<T><<<grid, 256, 0, st>>>(pl.d_mthin.template as<Problem<T>>(), (int)pl.mthin.size(),
                                             pl.d_segs.template as<Segment<T>>(), pl.d_part_off.template as<long long>(),
                                             cbase, sbase, pl.mthin_cols, pl.mthin_part_stride,
                                             pl.d_part.template as<T>()); ISCSI_COUNT_LAUNCH();
    k_mthin_reduce<T><<<(pl.mthin_cols + 255) / 256, 256, 0, st>>>(
        pl.d_mthin.template as<Problem<T>>(), (int)pl.mthin.size(), pl.d_part_off.template as<long long>(), sbase,
        cbase, pl.mthin_cols, pl.mthin_chunks, pl.mthin_part_stride, pl.d_part.template as<T>()); ISCSI_COUNT_LAUNCH();
    ISCSI_CUDA(cudaGetLastError());
  }
  if (pl.thin_rows > 0) {
    k_grouped_thin<T><<<(pl.thin_rows + 7) / 8, 256, 0, st>>>(pl.d_thin.template as<Problem<T>>(),
                                                              (int)pl.thin.size(), pl.d_segs.template as<Segment<T>>(),
                                                              cbase, sbase, pl.thin_rows); ISCSI_COUNT_LAUNCH();
    ISCSI_CUDA(cudaGetLastError());
  }
  if (pl.total_tiles == 0) return kOk;
  constexpr int NT = (C::BM / C::TM) * (C::BN / C::TN);
  k_grouped_gemm<T, C::BM, C::BN, C::BK, C::TM, C::TN><<<pl.total_tiles, NT, 0, st>>>(
      pl.d_probs.template as<Problem<T>>(), (int)pl.probs.size(), pl.d_segs.template as<Segment<T>>(), cbase,
      sbase); ISCSI_COUNT_LAUNCH();
  ISCSI_CUDA(cudaGetLastError());
  return kOk;
}

// ---------------------------------------------------------------------------
// lift: Ct_c[(q,s)][(X,Y), v] = s_a(q,X) s_b(s,Y) c_v[X u q, Y u s]  (0 outside the space)

constexpr int kMaxClasses = 2 * kMaxElec;

struct ClassTable {
  int nclass;
  long long start[kMaxClasses + 1];  // element offsets (all vectors) of each class block
  int ncol[kMaxClasses];
  int hp_start[kMaxClasses];
};

template <typename T, typename TC>
__global__ void k_lift_ct(ClassTable ct, int nvec, int n, int nholeA, int nholeB, const int* __restrict__ pair_of,
                          const int* __restrict__ hp_inv, const int* __restrict__ liftA,
                          const int* __restrict__ liftB, const int8_t* __restrict__ alevel,
                          const int* __restrict__ nballow, const long long* __restrict__ off,
                          const TC* __restrict__ c, long long ndet, T* __restrict__ out) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= ct.start[ct.nclass]) return;
  int cl = 0;
  while (t >= ct.start[cl + 1]) ++cl;
  long long local = t - ct.start[cl];
  long long width = (long long)ct.ncol[cl] * nvec;
  int k = (int)(local / width);
  int col = (int)(local % width);
  int hp = col / nvec, v = col % nvec;
  int xy = hp_inv[ct.hp_start[cl] + hp];
  int X = xy / nholeB, Y = xy % nholeB;
  int qs = pair_of[k];
  int q = qs / n, s = qs % n;
  int ea = liftA[q * nholeA + X], eb = liftB[s * nholeB + Y];
  T val = T(0);
  if (ea >= 0 && eb >= 0) {
    int Ap = ea >> 1, Bp = eb >> 1;
    if (Bp < nballow[alevel[Ap]]) {
      T x = (T)c[(long long)v * ndet + off[Ap] + Bp];
      val = ((ea ^ eb) & 1) ? -x : x;
    }
  }
  out[t] = val;
}

// fold: sigma_v[A,B] (+)= sum_{(p,X)->A} sum_{(r,Y)->B} s s T_c[pi(p,r)][(X,Y), v]
template <typename T>
__global__ void k_fold(ClassTable ct, int nvec, int n, int na, int nb, int nholeB, const int* __restrict__ decA,
                       const int* __restrict__ decB, const int8_t* __restrict__ hp_class,
                       const int* __restrict__ hp_local, const int* __restrict__ pair_index,
                       const long long* __restrict__ off, const T* __restrict__ tt, long long ndet,
                       T* __restrict__ sigma, int accumulate) {
  int A = blockIdx.x;
  long long o0 = off[A], o1 = off[A + 1];
  long long work = (o1 - o0) * nvec;
  for (long long w = threadIdx.x; w < work; w += blockDim.x) {
    int B = (int)(w / nvec), v = (int)(w % nvec);
    T acc = T(0);
    for (int i = 0; i < na; ++i) {
      int da = decA[A * na + i];
      int X = da >> 9, p = (da >> 1) & 255;
      for (int j = 0; j < nb; ++j) {
        int db = decB[B * nb + j];
        int Y = db >> 9, r = (db >> 1) & 255;
        long long hp = (long long)X * nholeB + Y;
        int cl = hp_class[hp];
        int m = pair_index[p * n + r];
        T x = tt[ct.start[cl] + ((long long)m * ct.ncol[cl] + hp_local[hp]) * nvec + v];
        acc += ((da ^ db) & 1) ? -x : x;
      }
    }
    T* dst = sigma + (long long)v * ndet + o0 + B;
    *dst = accumulate ? *dst + acc : acc;
  }
}

template <typename TA, typename TB>
__global__ void k_convert(const TA* __restrict__ in, TB* __restrict__ out, long long count) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (; t < count; t += stride) out[t] = (TB)in[t];
}

// ---------------------------------------------------------------------------

static ClassTable class_table(const Context& ctx, int nvec) {
  ClassTable ct;
  std::memset(&ct, 0, sizeof(ct));
  ct.nclass = (int)ctx.cls.size();
  long long acc = 0;
  for (int c = 0; c < ct.nclass; ++c) {
    const ColClass& cc = ctx.cls[c];
    ct.start[c] = acc;
    ct.ncol[c] = cc.ncol;
    ct.hp_start[c] = ctx.hp_class_start[c];
    if (cc.ncol > 0 && cc.mrows > 0) acc += (long long)cc.mrows * cc.ncol * nvec;
  }
  ct.start[ct.nclass] = acc;
  return ct;
}

template <typename T>
static const T* mat_ptr(const DevBuf& b) {
  return b.as<T>();
}

// builds the grouped problem lists of one precision for nvec vectors
template <typename T>
static int build_problems(Context& ctx, int nvec, const T* G, const T* Ma, const T* Mb, T* ctw, T* ttw,
                          ProblemList<T>& ab, ProblemList<T>& ss) {
  auto absp = [](const void* p) { return (long long)reinterpret_cast<uintptr_t>(p); };
  cudaStream_t st = stream();
  ab.probs.clear();
  ab.segs.clear();
  ss.probs.clear();
  ss.segs.clear();
  if (ctx.have_ab) {
    ClassTable ct = class_table(ctx, nvec);
    for (int cl = 0; cl < (int)ctx.cls.size(); ++cl) {
      const ColClass& cc = ctx.cls[cl];
      if (cc.ncol == 0 || cc.mrows == 0) continue;
      Segment<T> sgm;
      sgm.a = absp(G);
      sgm.asrc = kSrcAbs;
      sgm.lda = ctx.npairs;
      sgm.b = absp(ctw + ct.start[cl]);
      sgm.bsrc = kSrcAbs;
      sgm.ldb = (long long)cc.ncol * nvec;
      sgm.K = cc.krows;
      sgm.bcols = cc.ncol * nvec;
      Problem<T> p;
      p.c = absp(ttw + ct.start[cl]);
      p.csrc = kSrcAbs;
      p.ldc = (long long)cc.ncol * nvec;
      p.M = cc.mrows;
      p.N = cc.ncol * nvec;
      p.seg_begin = (int)ab.segs.size();
      p.seg_count = 1;
      p.accumulate = 0;
      ab.segs.push_back(sgm);
      ab.probs.push_back(p);
    }
  }
  const SpinSpace& SA = ctx.sp[0];
  const SpinSpace& SB = ctx.sp[1];
  for (int v = 0; v < nvec; ++v) {
    for (int a = 0; a <= SA.maxlevel; ++a) {
      int rows = SA.level_start[a + 1] - SA.level_start[a];
      int nba = (int)ctx.nb_allowed_lvl[a];
      if (rows == 0 || nba == 0) continue;
      const int routed = std::is_same<T, double>::value ? ctx.pl_ss_tc : ctx.pl_ss_tc32;
      if (routed == 1 && samespin_block_on_tc(ctx, a, std::is_same<T, double>::value ? 64 : 32)) continue;
      long long obase = ctx.off_h[SA.level_start[a]];
      Problem<T> p;
      p.c = (long long)v * ctx.ndet + obase;
      p.csrc = kSrcSigma;
      p.ldc = nba;
      p.M = rows;
      p.N = nba;
      p.seg_begin = (int)ss.segs.size();
      p.seg_count = 0;
      p.accumulate = 1;
      if (ctx.na > 0 && Ma) {
        for (int a2 = 0; a2 <= SA.maxlevel; ++a2) {
          int rows2 = SA.level_start[a2 + 1] - SA.level_start[a2];
          int nba2 = (int)ctx.nb_allowed_lvl[a2];
          if (rows2 == 0 || nba2 == 0 || std::abs(a - a2) > 2) continue;
          Segment<T> sgm;
          sgm.a = absp(Ma + (long long)SA.level_start[a] * SA.count + SA.level_start[a2]);
          sgm.asrc = kSrcAbs;
          sgm.lda = SA.count;
          sgm.b = (long long)v * ctx.ndet + ctx.off_h[SA.level_start[a2]];
          sgm.bsrc = kSrcC;
          sgm.ldb = nba2;
          sgm.K = rows2;
          sgm.bcols = std::min(nba, nba2);
          ss.segs.push_back(sgm);
          p.seg_count++;
        }
      }
      if (ctx.nb > 0 && Mb) {
        Segment<T> sgm;
        sgm.a = (long long)v * ctx.ndet + obase;
        sgm.asrc = kSrcC;
        sgm.lda = nba;
        sgm.b = absp(Mb);
        sgm.bsrc = kSrcAbs;
        sgm.ldb = SB.count;
        sgm.K = nba;
        sgm.bcols = nba;
        ss.segs.push_back(sgm);
        p.seg_count++;
      }
      if (p.seg_count > 0) ss.probs.push_back(p);
    }
  }
  ISCSI_TRY(upload_problems(ab, st));
  ISCSI_TRY(upload_problems(ss, st));
  return kOk;
}

double ctx_gemm_flops(const Context& ctx, int which) {
  double f = 0.0;
  if (which == 3) {
    // bf16 MMA flops of the same-spin level blocks on the tensor cores (FP64
    // routing): 28 slice products x 2 M N K, K padded to 16 per segment
    const SpinSpace& SA = ctx.sp[0];
    auto pad = [](double x) { return std::ceil(x / 16.0) * 16.0; };
    for (int a = 0; a <= SA.maxlevel; ++a) {
      if (!samespin_block_on_tc(ctx, a, 64)) continue;
      double rows = SA.level_start[a + 1] - SA.level_start[a], nba = (double)ctx.nb_allowed_lvl[a];
      if (rows == 0 || nba == 0) continue;
      if (ctx.na > 0 && ctx.M64[0].p)
        for (int a2 = 0; a2 <= SA.maxlevel; ++a2) {
          double rows2 = SA.level_start[a2 + 1] - SA.level_start[a2], nba2 = (double)ctx.nb_allowed_lvl[a2];
          if (rows2 == 0 || nba2 == 0 || std::abs(a - a2) > 2) continue;
          f += 28.0 * 2.0 * rows * pad(rows2) * std::min(nba, nba2);
        }
      if (ctx.nb > 0) f += 28.0 * 2.0 * rows * nba * pad(nba);
    }
    return f;
  }
  if (which == 2) {
    // bf16 MMA flops the tensor-core opposite-spin contraction issues: 28 slice
    // products (levels 0..6 of 7 slices) x 2 M N K, K rounded up to 16
    if (!ctx.have_ab) return 0.0;
    for (const ColClass& cc : ctx.cls)
      if (cc.ncol > 0 && cc.mrows > 0)
        f += 28.0 * 2.0 * cc.mrows * (double)((cc.krows + 15) / 16 * 16) * cc.ncol;
    return f;
  }
  if (which == 0) {
    if (!ctx.have_ab) return 0.0;
    for (const ColClass& cc : ctx.cls)
      if (cc.ncol > 0 && cc.mrows > 0) f += 2.0 * cc.mrows * (double)cc.krows * cc.ncol;
    return f;
  }
  const SpinSpace& SA = ctx.sp[0];
  for (int a = 0; a <= SA.maxlevel; ++a) {
    double rows = SA.level_start[a + 1] - SA.level_start[a];
    double nba = (double)ctx.nb_allowed_lvl[a];
    if (rows == 0 || nba == 0) continue;
    if (ctx.na > 0 && ctx.M64[0].p)
      for (int a2 = 0; a2 <= SA.maxlevel; ++a2) {
        double rows2 = SA.level_start[a2 + 1] - SA.level_start[a2];
        double nba2 = (double)ctx.nb_allowed_lvl[a2];
        if (rows2 == 0 || nba2 == 0 || std::abs(a - a2) > 2) continue;
        f += 2.0 * rows * rows2 * std::min(nba, nba2);
      }
    if (ctx.nb > 0) f += 2.0 * rows * nba * nba;
  }
  return f;
}

int sigma_workspace(Context& ctx, int nvec, int precision) {
  // Ct and T are sized in FP64 elements, so both precisions share them
  if (nvec > ctx.nvec_cap) {
    if (ctx.have_ab) {
      ISCSI_TRY(ctx.ct.alloc(sizeof(double) * ctx.ct_elems * nvec));
      ISCSI_TRY(ctx.tt.alloc(sizeof(double) * ctx.ct_elems * nvec));
    }
    ctx.c32.release();
    ctx.s32.release();
    ctx.nvec_cap = nvec;
    ctx.pl_nvec64 = ctx.pl_nvec32 = 0;  // workspace pointers changed: rebuild problem lists
  }
  if (precision == 32 && !ctx.c32.p) {
    ISCSI_TRY(ctx.c32.alloc(sizeof(float) * ctx.ndet * ctx.nvec_cap));
    ISCSI_TRY(ctx.s32.alloc(sizeof(float) * ctx.ndet * ctx.nvec_cap));
    ctx.pl_nvec32 = 0;
  }
  return kOk;
}

// M = M_base + f M_v, elementwise
__global__ void k_shift_m(const double* __restrict__ base, const double* __restrict__ mv, double f,
                          double* __restrict__ out, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    out[i] = base[i] + f * mv[i];
}

// A per-step one-body term (Eq. ham with h(t) = h + f v): the string matrices
// of the one-body and same-spin units become M_base + f M_v, with M_v those of
// the context cpl (h1 = v, no two-electron part, the same space); the FP32
// copies and the tensor-core slices follow.  f = 0 restores M_base exactly.
int onebody_shift(Context& ctx, const Context& cpl, double f) {
  if (f == ctx.m_shift) return kOk;
  cudaStream_t st = stream();
  for (int s = 0; s < 2; ++s) {
    if (!ctx.M64[s].p) continue;
    if (!cpl.M64[s].p) {
      set_error("one-body shift: the coupling context has no matching string matrix");
      return kErrArg;
    }
    const long long m2 = (long long)ctx.sp[s].count * ctx.sp[s].count;
    if (!ctx.M64base[s].p) {
      ISCSI_TRY(ctx.M64base[s].alloc(sizeof(double) * m2));
      ISCSI_CUDA(cudaMemcpyAsync(ctx.M64base[s].p, ctx.M64[s].p, sizeof(double) * m2, cudaMemcpyDeviceToDevice, st));
    }
    k_shift_m<<<launch_blocks(m2, 256), 256, 0, st>>>(ctx.M64base[s].as<double>(), cpl.M64[s].as<double>(), f,
                                                      ctx.M64[s].as<double>(), m2); ISCSI_COUNT_LAUNCH();
    if (ctx.M32[s].p) {
      k_convert<double, float><<<2048, 256, 0, st>>>(ctx.M64[s].as<double>(), ctx.M32[s].as<float>(), m2); ISCSI_COUNT_LAUNCH();
    }
  }
  ISCSI_CUDA(cudaGetLastError());
  ctx.m_shift = f;
  return samespin_matrices_changed(ctx);
}

static int ensure_fp32_matrices(Context& ctx) {
  cudaStream_t st = stream();
  if (ctx.have_ab && !ctx.G32.p) {
    long long g2 = (long long)ctx.npairs * ctx.npairs;
    ISCSI_TRY(ctx.G32.alloc(sizeof(float) * g2));
    k_convert<double, float><<<2048, 256, 0, st>>>(ctx.G64.as<double>(), ctx.G32.as<float>(), g2); ISCSI_COUNT_LAUNCH();
  }
  for (int s = 0; s < 2; ++s) {
    if (!ctx.M64[s].p || ctx.M32[s].p) continue;
    long long m2 = (long long)ctx.sp[s].count * ctx.sp[s].count;
    ISCSI_TRY(ctx.M32[s].alloc(sizeof(float) * m2));
    k_convert<double, float><<<2048, 256, 0, st>>>(ctx.M64[s].as<double>(), ctx.M32[s].as<float>(), m2); ISCSI_COUNT_LAUNCH();
  }
  ISCSI_CUDA(cudaGetLastError());
  return kOk;
}

static int timing_event(Context& ctx, int call, int phase, cudaStream_t st) {
  if (!options().phase_timing || ctx.capturing || call >= Context::kMaxTimed) return kOk;
  size_t idx = (size_t)call * (Context::kPhases + 1) + phase;
  if (ctx.tev.size() <= idx) ctx.tev.resize((size_t)Context::kMaxTimed * (Context::kPhases + 1), nullptr);
  if (!ctx.tev[idx]) ISCSI_CUDA(cudaEventCreate(&ctx.tev[idx]));
  ISCSI_CUDA(cudaEventRecord(ctx.tev[idx], st));
  return kOk;
}

template <typename T, typename TC>
static int sigma_impl(Context& ctx, const TC* c_in, T* s_out, const T* c, T* sigma, int nvec, ProblemList<T>& ab,
                      ProblemList<T>& ss, int& pl_nvec, const T* G, const T* Ma, const T* Mb, int phases) {
  cudaStream_t st = stream();
  T* ctw = ctx.ct.as<T>();
  T* ttw = ctx.tt.as<T>();
  constexpr bool f64 = std::is_same<T, double>::value;
  const int ss_tc = (f64 ? samespin_tc_active(ctx) : samespin_tc32_active(ctx)) ? 1 : 0;
  const bool tc_path = ab_on_tc(ctx, f64 ? 64 : 32);
  // both contractions on the tensor cores: one launch for both problem lists
  // (fewer partly filled waves); sigma starts at zero, the same-spin products
  // add into it, the fold adds last
  const bool comb = ctx.have_ab && tc_path && ss_tc;
  // per-phase events only when the whole step runs in this call
  const bool timed = phases == kPhAll;
  const int call = ctx.ntimed;
  auto ev = [&](int ph) { return timed ? timing_event(ctx, call, ph, st) : kOk; };
  if (phases & kPhPre) {
    // problem lists depend on nvec, the workspaces and the same-spin routing, not on the vectors
    // a new routing (autotuner) rebuilds the FMA lists and the same-spin tensor-core job
    int& routed = f64 ? ctx.pl_ss_tc : ctx.pl_ss_tc32;
    long long& rkey = f64 ? ctx.pl_route_key : ctx.pl_route_key32;
    const Context::Route& R = ctx.route[f64 ? 0 : 1];
    const long long key = ((long long)R.ss_min << 2) | (R.ab_tc << 1) | ss_tc;
    if (routed != ss_tc || rkey != key) {
      routed = ss_tc;
      rkey = key;
      pl_nvec = 0;
      (f64 ? ctx.oz_ss : ctx.t3_ss).nvec = -1;
    }
    if (pl_nvec != nvec) {
      ISCSI_TRY(build_problems<T>(ctx, nvec, G, Ma, Mb, ctw, ttw, ab, ss));
      pl_nvec = nvec;
    }
    ISCSI_TRY(ev(0));
    if (ctx.have_ab && tc_path) {
      // opposite-spin operands for the tensor cores (lift + slice)
      if (f64)
        ISCSI_TRY(opposite_tc_operands(ctx, reinterpret_cast<const double*>(c_in), reinterpret_cast<double*>(ttw),
                                       nvec));
      else
        ISCSI_TRY(opposite_tc32_operands(ctx, reinterpret_cast<const float*>(c_in), reinterpret_cast<float*>(ttw),
                                         nvec));
      if (comb) {
        ISCSI_CUDA(cudaMemsetAsync(sigma, 0, sizeof(T) * ctx.ndet * nvec, st));
        if (f64)
          ISCSI_TRY(samespin_tc_operands(ctx, reinterpret_cast<const double*>(c), reinterpret_cast<double*>(sigma),
                                         nvec));
        else
          ISCSI_TRY(samespin_tc32_operands(ctx, reinterpret_cast<const float*>(c), reinterpret_cast<float*>(sigma),
                                           nvec));
      }
    } else if (ctx.have_ab) {
      ClassTable ct = class_table(ctx, nvec);
      long long tot = ct.start[ct.nclass];
      if (tot > 0) {
        k_lift_ct<T, TC><<<launch_blocks(tot, 256), 256, 0, st>>>(
            ct, nvec, ctx.n, ctx.sp[0].nhole, ctx.sp[1].nhole, ctx.pair_of.as<int>(), ctx.hp_inv.as<int>(),
            ctx.sp[0].lift.as<int>(), ctx.sp[1].lift.as<int>(), ctx.sp[0].level.as<int8_t>(), ctx.nballow.as<int>(),
            ctx.off.as<long long>(), c_in, ctx.ndet, ctw); ISCSI_COUNT_LAUNCH();
        ISCSI_CUDA(cudaGetLastError());
      }
    } else {
      ISCSI_CUDA(cudaMemsetAsync(sigma, 0, sizeof(T) * ctx.ndet * nvec, st));
    }
    ISCSI_TRY(ev(1));
  }
  if (phases & kPhAbGemm) {
    if (comb)
      ISCSI_TRY(f64 ? both_tc_gemm(ctx, reinterpret_cast<double*>(sigma))
                    : both_tc32_gemm(ctx, reinterpret_cast<float*>(sigma)));
    else if (ctx.have_ab && tc_path)
      ISCSI_TRY(f64 ? opposite_tc_gemm(ctx) : opposite_tc32_gemm(ctx));
    else if (ctx.have_ab)
      ISCSI_TRY(launch_grouped<T>(ab, c, sigma, st));
    ISCSI_TRY(ev(2));
  }
  if (phases & kPhMid) {
    if (ctx.have_ab) {
      ClassTable ct = class_table(ctx, nvec);
      k_fold<T><<<ctx.sp[0].count, 256, 0, st>>>(ct, nvec, ctx.n, ctx.na, ctx.nb, ctx.sp[1].nhole,
                                                 ctx.sp[0].dec.as<int>(), ctx.sp[1].dec.as<int>(),
                                                 ctx.hp_class.as<int8_t>(), ctx.hp_local.as<int>(),
                                                 ctx.pair_index.as<int>(), ctx.off.as<long long>(), ttw, ctx.ndet,
                                                 sigma, comb ? 1 : 0); ISCSI_COUNT_LAUNCH();
      ISCSI_CUDA(cudaGetLastError());
    }
    ISCSI_TRY(ev(3));
    ISCSI_TRY(launch_grouped<T>(ss, c, sigma, st));
    if (ss_tc && !comb && f64)
      ISCSI_TRY(samespin_tc_operands(ctx, reinterpret_cast<const double*>(c), reinterpret_cast<double*>(sigma), nvec));
    else if (ss_tc && !comb)
      ISCSI_TRY(samespin_tc32_operands(ctx, reinterpret_cast<const float*>(c), reinterpret_cast<float*>(sigma), nvec));
  }
  if (phases & kPhSsGemm) {
    if (ss_tc && !comb && f64)
      ISCSI_TRY(samespin_tc_gemm(ctx, reinterpret_cast<double*>(sigma)));
    else if (ss_tc && !comb)
      ISCSI_TRY(samespin_tc32_gemm(ctx, reinterpret_cast<float*>(sigma)));
  }
  if (phases & kPhPost) {
    ISCSI_TRY(ev(4));
    if (timed && options().phase_timing && !ctx.capturing && call < Context::kMaxTimed) ctx.ntimed++;
  }
  (void)s_out;
  return kOk;
}

int sigma_run(Context& ctx, const double* c, double* sigma, int nvec, int precision, int phases) {
  cudaStream_t st = stream();
  if (phases == kPhAll) ISCSI_TRY(sigma_autotune(ctx, c, sigma, nvec, precision));
  if (phases & kPhPre) ISCSI_TRY(sigma_workspace(ctx, nvec, precision));
  const double* Ma = ctx.na ? ctx.M64[0].as<double>() : nullptr;
  const double* Mb = ctx.nb ? (ctx.beta_alias ? ctx.M64[0].as<double>() : ctx.M64[1].as<double>()) : nullptr;
  if (precision == 64) {
    ISCSI_TRY(sigma_impl<double, double>(ctx, c, sigma, c, sigma, nvec, ctx.pl_ab64, ctx.pl_ss64, ctx.pl_nvec64,
                                         ctx.G64.as<double>(), Ma, Mb, phases));
    // a GAS restriction: sigma = P H c (zero outside the kept determinants)
    if ((phases & kPhPost) && ctx.gas_nspace) ISCSI_TRY(gas_project(ctx, sigma, sigma, nvec, st));
    return kOk;
  }
  if (phases & kPhPre) ISCSI_TRY(ensure_fp32_matrices(ctx));
  const float* Ma32 = ctx.na ? ctx.M32[0].as<float>() : nullptr;
  const float* Mb32 = ctx.nb ? (ctx.beta_alias ? ctx.M32[0].as<float>() : ctx.M32[1].as<float>()) : nullptr;
  long long cnt = ctx.ndet * nvec;
  if (phases & kPhPre) {
    k_convert<double, float><<<std::min(launch_blocks(cnt, 256), 4096), 256, 0, st>>>(c, ctx.c32.as<float>(), cnt); ISCSI_COUNT_LAUNCH();
  }
  ISCSI_TRY(sigma_impl<float, float>(ctx, ctx.c32.as<float>(), ctx.s32.as<float>(), ctx.c32.as<float>(),
                                     ctx.s32.as<float>(), nvec, ctx.pl_ab32, ctx.pl_ss32, ctx.pl_nvec32,
                                     ctx.G32.as<float>(), Ma32, Mb32, phases));
  if (phases & kPhPost) {
    k_convert<float, double><<<std::min(launch_blocks(cnt, 256), 4096), 256, 0, st>>>(ctx.s32.as<float>(), sigma, cnt); ISCSI_COUNT_LAUNCH();
    if (ctx.gas_nspace) ISCSI_TRY(gas_project(ctx, sigma, sigma, nvec, st));
  }
  ISCSI_CUDA(cudaGetLastError());
  return kOk;
}

// ---------------------------------------------------------------------------
// Autotuner: the kernel routing of a context (which products run on the
// tensor cores, which on the FMA kernels) for one precision and vector count.
// Candidates: the opposite-spin contraction on the tensor cores or not, and
// the same-spin block threshold (16, 64, 256, or none on the tensor cores).
// A model from the flop counts and the kernels' measured rates (tensor-core
// FP64-accurate contraction ~1.1 PFLOP/s of bf16 products, FP32 form ~0.6,
// FP64 FMA ~1.1 TFLOP/s, FP32 FMA ~24 TFLOP/s) keeps the candidates within 3x
// of the best prediction; each of those is timed on the caller's vector (one
// untimed sigma to build its lists, then the best of three timed with CUDA
// events, since close candidates differ by a few percent) and the fastest is
// kept.  Runs once per context, precision and vector count, before
// the first sigma (never during a graph capture).

namespace {

double block_rows(const Context& ctx, int a) {
  return ctx.sp[0].level_start[a + 1] - ctx.sp[0].level_start[a];
}

// predicted ms of one sigma under a routing (contractions only)
double route_model_ms(const Context& ctx, int prec, int ab_tc, int ss_min, int nvec) {
  const bool f64 = prec == 64;
  const double tc_rate = f64 ? 1.1e15 / 28.0 : 0.6e15 / 6.0;  // useful flops/s on the tensor cores
  const double fma_rate = f64 ? 1.1e12 : 2.4e13;
  double t = 0.0;
  const double fab = ctx_gemm_flops(ctx, 0) * nvec;
  t += fab / (ab_tc ? tc_rate : fma_rate);
  const SpinSpace& SA = ctx.sp[0];
  for (int a = 0; a <= SA.maxlevel; ++a) {
    double rows = block_rows(ctx, a), nba = (double)ctx.nb_allowed_lvl[a];
    if (rows == 0 || nba == 0) continue;
    double f = 0.0;
    if (ctx.na > 0 && ctx.M64[0].p)
      for (int a2 = 0; a2 <= SA.maxlevel; ++a2) {
        double rows2 = block_rows(ctx, a2), nba2 = (double)ctx.nb_allowed_lvl[a2];
        if (rows2 == 0 || nba2 == 0 || std::abs(a - a2) > 2) continue;
        f += 2.0 * rows * rows2 * std::min(nba, nba2);
      }
    if (ctx.nb > 0) f += 2.0 * rows * nba * nba;
    const bool on = rows > ss_min && nba > ss_min;
    t += f * nvec / (on ? tc_rate : fma_rate);
  }
  return t * 1e3;
}

}  // namespace

int sigma_autotune(Context& ctx, const double* c, double* sigma, int nvec, int prec) {
  Context::Route& R = ctx.route[prec == 32 ? 1 : 0];
  if (!options().autotune || ctx.capturing || R.tuned_nvec == nvec) return kOk;
  R.tuned_nvec = nvec;  // also stops the trial sigma calls below from tuning again
  const bool tc_ok = prec == 32 ? options().fp32_tc : options().fp64_tc;
  const bool ss_ok = tc_ok && options().samespin_tc;
  struct Cand {
    int ab, ss;
    double pred, ms;
  };
  std::vector<Cand> cands;
  const int thr[4] = {kThinN, 64, 256, 1 << 30};
  for (int ab = tc_ok ? 1 : 0; ab >= 0; --ab)
    for (int i = 0; i < (ss_ok ? 4 : 1); ++i) {
      const int ss = ss_ok ? thr[i] : (1 << 30);
      // thresholds that route the same blocks are the same candidate
      bool dup = false;
      for (const Cand& q : cands) {
        if (q.ab != ab) continue;
        bool same = true;
        for (int a = 0; a <= ctx.sp[0].maxlevel && same; ++a) {
          double rows = block_rows(ctx, a), nba = (double)ctx.nb_allowed_lvl[a];
          same = (rows > q.ss && nba > q.ss) == (rows > ss && nba > ss);
        }
        if (same) dup = true;
      }
      if (!dup) cands.push_back({ab, ss, route_model_ms(ctx, prec, ab, ss, nvec), -1.0});
    }
  double best_pred = 1e300;
  for (const Cand& q : cands) best_pred = std::min(best_pred, q.pred);
  std::vector<Cand> keep;
  for (const Cand& q : cands)
    if (q.pred <= 3.0 * best_pred) keep.push_back(q);
  R.trials.clear();
  if (keep.size() > 1 && best_pred > 0.05) {  // below ~50 us a sigma is launch-bound: nothing to learn
    cudaStream_t st = stream();
    cudaEvent_t e0, e1;
    ISCSI_CUDA(cudaEventCreate(&e0));
    ISCSI_CUDA(cudaEventCreate(&e1));
    for (Cand& q : keep) {
      R.ab_tc = q.ab;
      R.ss_min = q.ss;
      ISCSI_TRY(sigma_run(ctx, c, sigma, nvec, prec));  // builds this routing's lists
      q.ms = 1e300;
      for (int rep = 0; rep < 3; ++rep) {
        ISCSI_CUDA(cudaEventRecord(e0, st));
        ISCSI_TRY(sigma_run(ctx, c, sigma, nvec, prec));
        ISCSI_CUDA(cudaEventRecord(e1, st));
        ISCSI_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        ISCSI_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        q.ms = std::min(q.ms, (double)ms);
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  const Cand* best = &keep[0];
  for (const Cand& q : keep)
    if ((q.ms >= 0 ? q.ms : q.pred) < (best->ms >= 0 ? best->ms : best->pred)) best = &q;
  R.ab_tc = best->ab;
  R.ss_min = best->ss;
  for (const Cand& q : cands) {
    R.trials.push_back(q.ab);
    R.trials.push_back(q.ss >= (1 << 30) ? -1 : q.ss);
    R.trials.push_back(q.pred);
    double ms = -1.0;
    for (const Cand& k2 : keep)
      if (k2.ab == q.ab && k2.ss == q.ss) ms = k2.ms;
    R.trials.push_back(ms);
  }
  return kOk;
}

// ---------------------------------------------------------------------------
// Allocation-free sigma (iscsi_sigma_noalloc).  Some callers cannot call
// cudaMalloc at the time they need sigma: code running under a memory manager
// that owns all device memory, real-time or callback contexts where an
// allocation (which may synchronise the device) is not allowed, or a process
// whose memory is already committed.  For them this variant keeps every
// per-call buffer -- the lifted vector Ct, the product T and the GEMM problem
// lists -- in one file-scope device array of fixed size instead of
// library-allocated workspace.  It computes the FP64 sigma of one vector on the
// FP64 FMA kernels (k_lift_ct, k_grouped_gemm, k_fold: the fp64_tc = 0 route of
// iscsi_sigma), not on the tensor cores, whose per-call operand slices would
// not fit a modest array.  The array belongs to the module: every GPU that
// loads the library holds it until the process exits.  All calls share it, so
// calls whose work overlaps on the GPU (different streams, or several host
// threads) race on it and must be serialised by the caller.  Nothing in it
// has to start at zero: each call overwrites every element it later reads.
// The problem lists stay in the array between calls: a call copies them from
// host memory only when the array last held another context's (or another
// build of this context's) lists.

constexpr size_t kNoAllocScratchBytes = 32u << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// per-device bookkeeping (the array's address, whose lists it holds), guarded
// so that host threads calling at once at least keep it consistent
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {nullptr};
static const Context* g_noalloc_lists_of[64] = {nullptr};  // whose lists the array holds, per device
static long long g_noalloc_lists_gen[64] = {0};

size_t noalloc_scratch_bytes() { return kNoAllocScratchBytes; }

// bytes of scratch one FP64 single-vector sigma of this context needs
size_t noalloc_bytes_needed(const Context& ctx) {
  size_t b = ctx.have_ab ? 2 * sizeof(double) * ctx.ct_elems : 0;
  b = (b + 255) & ~(size_t)255;
  b += 64 * (sizeof(Problem<double>) + sizeof(Segment<double>)) + 256;
  return b;
}

int sigma_noalloc_run(Context& ctx, const double* c, double* sigma) {
  using C = TileCfg<double>;
  cudaStream_t st = stream();
  size_t need = noalloc_bytes_needed(ctx);
  if (need > kNoAllocScratchBytes) {
    set_error("iscsi_sigma_noalloc: this context needs " + std::to_string(need) + " bytes of scratch, above the " +
              std::to_string(kNoAllocScratchBytes) + "-byte static array; use iscsi_sigma");
    return kErrArg;
  }
  // once per device, with that device current: host code only knows the
  // array through its device address
  int dev = 0;
  ISCSI_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("iscsi_sigma_noalloc: device index out of range");
    return kErrArg;
  }
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* ptr = nullptr;
      ISCSI_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
      g_noalloc_ptr[dev] = ptr;
    }
    base = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
  }
  double* ctw = reinterpret_cast<double*>(base);
  double* ttw = ctw + ctx.ct_elems;
  size_t lists_off = ctx.have_ab ? ((2 * sizeof(double) * ctx.ct_elems + 255) & ~(size_t)255) : 0;
  Problem<double>* dprobs = reinterpret_cast<Problem<double>*>(base + lists_off);
  Segment<double>* dsegs = reinterpret_cast<Segment<double>*>(base + lists_off + 64 * sizeof(Problem<double>));

  // problem lists (host vectors, copied into the array below)
  std::vector<Problem<double>> ab, ss;
  std::vector<Segment<double>> segs;
  auto absp = [](const void* p) { return (long long)reinterpret_cast<uintptr_t>(p); };
  const double* G = ctx.G64.as<double>();
  const double* Ma = ctx.na ? ctx.M64[0].as<double>() : nullptr;
  const double* Mb = ctx.nb ? (ctx.beta_alias ? ctx.M64[0].as<double>() : ctx.M64[1].as<double>()) : nullptr;
  ClassTable ct = class_table(ctx, 1);
  if (ctx.have_ab) {
    for (int cl = 0; cl < (int)ctx.cls.size(); ++cl) {
      const ColClass& cc = ctx.cls[cl];
      if (cc.ncol == 0 || cc.mrows == 0) continue;
      Segment<double> g{absp(G), absp(ctw + ct.start[cl]), kSrcAbs, kSrcAbs, ctx.npairs, cc.ncol, cc.krows, cc.ncol};
      Problem<double> p{};
      p.c = absp(ttw + ct.start[cl]);
      p.csrc = kSrcAbs;
      p.ldc = cc.ncol;
      p.M = cc.mrows;
      p.N = cc.ncol;
      p.seg_begin = (int)segs.size();
      p.seg_count = 1;
      p.accumulate = 0;
      segs.push_back(g);
      ab.push_back(p);
    }
  }
  const SpinSpace& SA = ctx.sp[0];
  const SpinSpace& SB = ctx.sp[1];
  for (int a = 0; a <= SA.maxlevel; ++a) {
    int rows = SA.level_start[a + 1] - SA.level_start[a];
    int nba = (int)ctx.nb_allowed_lvl[a];
    if (rows == 0 || nba == 0) continue;
    long long obase = ctx.off_h[SA.level_start[a]];
    Problem<double> p{};
    p.c = obase;
    p.csrc = kSrcSigma;
    p.ldc = nba;
    p.M = rows;
    p.N = nba;
    p.seg_begin = (int)segs.size();
    p.seg_count = 0;
    p.accumulate = 1;
    if (ctx.na > 0 && Ma)
      for (int a2 = 0; a2 <= SA.maxlevel; ++a2) {
        int rows2 = SA.level_start[a2 + 1] - SA.level_start[a2];
        int nba2 = (int)ctx.nb_allowed_lvl[a2];
        if (rows2 == 0 || nba2 == 0 || std::abs(a - a2) > 2) continue;
        segs.push_back({absp(Ma + (long long)SA.level_start[a] * SA.count + SA.level_start[a2]),
                        ctx.off_h[SA.level_start[a2]], kSrcAbs, kSrcC, SA.count, nba2, rows2, std::min(nba, nba2)});
        p.seg_count++;
      }
    if (ctx.nb > 0 && Mb) {
      segs.push_back({obase, absp(Mb), kSrcC, kSrcAbs, nba, SB.count, nba, nba});
      p.seg_count++;
    }
    if (p.seg_count > 0) ss.push_back(p);
  }
  auto tiles_of = [](std::vector<Problem<double>>& v) {
    int tiles = 0;
    for (auto& p : v) {
      p.tile_begin = tiles;
      p.tiles_n = (p.N + C::BN - 1) / C::BN;
      tiles += ((p.M + C::BM - 1) / C::BM) * p.tiles_n;
    }
    return tiles;
  };
  int ab_tiles = tiles_of(ab), ss_tiles = tiles_of(ss);
  std::vector<Problem<double>> all(ab);
  all.insert(all.end(), ss.begin(), ss.end());
  if (all.size() > 64 || segs.size() > 64) {
    set_error("iscsi_sigma_noalloc: too many GEMM problems for the static lists");
    return kErrArg;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_lists_of[dev] != &ctx || g_noalloc_lists_gen[dev] != ctx.noalloc_gen) {
    if (!all.empty())
      ISCSI_CUDA(cudaMemcpyAsync(dprobs, all.data(), sizeof(Problem<double>) * all.size(), cudaMemcpyHostToDevice, st));
    if (!segs.empty())
      ISCSI_CUDA(
          cudaMemcpyAsync(dsegs, segs.data(), sizeof(Segment<double>) * segs.size(), cudaMemcpyHostToDevice, st));
    g_noalloc_lists_of[dev] = &ctx;
    g_noalloc_lists_gen[dev] = ctx.noalloc_gen;
  }
  constexpr int NT = (C::BM / C::TM) * (C::BN / C::TN);
  if (ctx.have_ab) {
    long long tot = ct.start[ct.nclass];
    if (tot > 0) {
      k_lift_ct<double, double><<<launch_blocks(tot, 256), 256, 0, st>>>(
          ct, 1, ctx.n, ctx.sp[0].nhole, ctx.sp[1].nhole, ctx.pair_of.as<int>(), ctx.hp_inv.as<int>(),
          ctx.sp[0].lift.as<int>(), ctx.sp[1].lift.as<int>(), ctx.sp[0].level.as<int8_t>(), ctx.nballow.as<int>(),
          ctx.off.as<long long>(), c, ctx.ndet, ctw);
      ISCSI_COUNT_LAUNCH();
    }
    if (ab_tiles > 0) {
      k_grouped_gemm<double, C::BM, C::BN, C::BK, C::TM, C::TN>
          <<<ab_tiles, NT, 0, st>>>(dprobs, (int)ab.size(), dsegs, c, sigma);
      ISCSI_COUNT_LAUNCH();
    }
    k_fold<double><<<ctx.sp[0].count, 256, 0, st>>>(ct, 1, ctx.n, ctx.na, ctx.nb, ctx.sp[1].nhole,
                                                    ctx.sp[0].dec.as<int>(), ctx.sp[1].dec.as<int>(),
                                                    ctx.hp_class.as<int8_t>(), ctx.hp_local.as<int>(),
                                                    ctx.pair_index.as<int>(), ctx.off.as<long long>(), ttw, ctx.ndet,
                                                    sigma, 0); ISCSI_COUNT_LAUNCH();
  } else {
    ISCSI_CUDA(cudaMemsetAsync(sigma, 0, sizeof(double) * ctx.ndet, st));
  }
  if (ss_tiles > 0) {
    k_grouped_gemm<double, C::BM, C::BN, C::BK, C::TM, C::TN>
        <<<ss_tiles, NT, 0, st>>>(dprobs + ab.size(), (int)ss.size(), dsegs, c, sigma);
    ISCSI_COUNT_LAUNCH();
  }
  ISCSI_CUDA(cudaGetLastError());
  return kOk;
}

}  // namespace iscsi
