// setup.cu -- per-context set-up on the device: string spaces, determinant
// addressing, hole-string (contraction/addition) tables, screened units.
//
// This is the "first part" of the ISCI algorithm (Sec. "First part"): every
// quantity that depends only on the orbital space, the truncation and the
// integrals is built once, so the sigma step ("second part") only multiplies.
// Screening (Eq. sigma_split, with the algorithm's "if |I| > epsilon") is
// applied here, once per integral unit: a dropped unit is a structural zero of
// the matrices below, which is exactly the same as never applying its term.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <numeric>

#include "internal.cuh"

namespace iscsi {

// C(n, k); LLONG_MAX when it does not fit (every partial product r is itself
// the binomial C(n - k + i, i), so the division is exact)
// C(n, k), saturating at LLONG_MAX only when the value itself does not fit:
// after step i, r = C(n - k + i, i), and the product r (n - k + i) is formed in
// 128 bits before the exact division by i
long long binom_ll(int n, int k) {
  if (k < 0 || n < 0 || k > n) return 0;
  if (k > n - k) k = n - k;
  unsigned __int128 r = 1;
  for (int i = 1; i <= k; ++i) {
    r = r * (unsigned __int128)(n - k + i) / (unsigned __int128)i;
    if (r > (unsigned __int128)LLONG_MAX) return LLONG_MAX;
  }
  return (long long)r;
}

int launch_blocks(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > (1ll << 30)) b = 1ll << 30;
  return (int)b;
}

int DevBuf::alloc(size_t nbytes) {
  release();
  if (nbytes == 0) return kOk;
  cudaError_t e = cudaMalloc(&p, nbytes);
  if (e != cudaSuccess) {
    p = nullptr;
    cudaGetLastError();
    set_error(std::string("cudaMalloc of ") + std::to_string(nbytes) + " bytes: " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? kErrNoMem : kErrCuda;
  }
  bytes = nbytes;
  return kOk;
}

int DevBuf::grow(size_t nbytes) {
  if (nbytes <= bytes && p) return kOk;
  return alloc(nbytes);
}

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

Context::~Context() {
  density_release(*this);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
}

// ---------------------------------------------------------------------------
// device helpers: binomials, colex unranking, 256-bit orbital masks

__constant__ long long c_binom[kMaxOrb + 1][kMaxElec + 2];

__device__ __forceinline__ long long dbinom(int n, int k) {
  return (n < 0 || k < 0 || k > n) ? 0 : c_binom[n][k];
}

struct OrbMask {
  unsigned long long w[4];
};

__device__ __forceinline__ void mask_clear(OrbMask& m) { m.w[0] = m.w[1] = m.w[2] = m.w[3] = 0ull; }
__device__ __forceinline__ bool mask_has(const OrbMask& m, int p) { return (m.w[p >> 6] >> (p & 63)) & 1ull; }
__device__ __forceinline__ void mask_flip(OrbMask& m, int p) { m.w[p >> 6] ^= 1ull << (p & 63); }
// number of occupied orbitals below p
__device__ __forceinline__ int mask_below(const OrbMask& m, int p) {
  int w = p >> 6, b = p & 63, c = 0;
  for (int i = 0; i < w; ++i) c += __popcll(m.w[i]);
  if (b) c += __popcll(m.w[w] & ((1ull << b) - 1ull));
  return c;
}
// a_q on |m>: returns sign (+1/-1) or 0
__device__ __forceinline__ int mask_annihilate(OrbMask& m, int q) {
  if (!mask_has(m, q)) return 0;
  int s = (mask_below(m, q) & 1) ? -1 : 1;
  mask_flip(m, q);
  return s;
}
// a+_p on |m>
__device__ __forceinline__ int mask_create(OrbMask& m, int p) {
  if (mask_has(m, p)) return 0;
  int s = (mask_below(m, p) & 1) ? -1 : 1;
  mask_flip(m, p);
  return s;
}

__device__ __forceinline__ long long colex_of(const int* o, int k) {
  long long r = 0;
  for (int i = 0; i < k; ++i) r += dbinom(o[i], i + 1);
  return r;
}

// colex unranking: the k-subset of {0..n-1} with rank r, ascending
__device__ void colex_unrank(long long r, int n, int k, int* o) {
  int hi = n - 1;
  for (int i = k - 1; i >= 0; --i) {
    // largest c <= hi with C(c, i+1) <= r
    int lo = i, h = hi;
    while (lo < h) {
      int mid = (lo + h + 1) >> 1;
      if (dbinom(mid, i + 1) <= r) lo = mid;
      else h = mid - 1;
    }
    o[i] = lo;
    r -= dbinom(lo, i + 1);
    hi = lo - 1;
  }
}

// ---------------------------------------------------------------------------
// string enumeration: unrank every colex rank, then a stable counting sort by
// level (the colex order is kept inside each level)

__global__ void k_unrank(int n, int k, int nocc, long long count, int16_t* orbs, int8_t* level) {
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= count) return;
  int o[kMaxElec];
  colex_unrank(r, n, k, o);
  int l = 0;
  for (int i = 0; i < k; ++i) {
    orbs[r * k + i] = (int16_t)o[i];
    l += (o[i] >= nocc);
  }
  level[r] = (int8_t)l;
}

// per chunk of 256 ranks: how many strings of each level
__global__ void k_level_hist(const int8_t* level, long long count, int nlev, int* chunk_hist) {
  __shared__ int h[kMaxLevels];
  if (threadIdx.x < kMaxLevels) h[threadIdx.x] = 0;
  __syncthreads();
  long long r = blockIdx.x * 256ll + threadIdx.x;
  if (r < count) atomicAdd(&h[level[r]], 1);
  __syncthreads();
  if (threadIdx.x < nlev) chunk_hist[blockIdx.x * nlev + threadIdx.x] = h[threadIdx.x];
}

// exclusive scan of chunk_hist down each level column, plus the level bases;
// one block, one thread per level (the chunk count is small)
__global__ void k_level_scan(int* chunk_hist, int nchunks, int nlev, int* level_count) {
  int l = threadIdx.x;
  if (l >= nlev) return;
  int acc = 0;
  for (int c = 0; c < nchunks; ++c) {
    int v = chunk_hist[c * nlev + l];
    chunk_hist[c * nlev + l] = acc;
    acc += v;
  }
  level_count[l] = acc;
}

// sorted position of each rank = level base + chunk prefix + rank inside the chunk
__global__ void k_scatter_sorted(const int16_t* orbs_r, const int8_t* level_r, long long count, int k, int nlev,
                                 const int* chunk_prefix, const int* level_base, int16_t* orbs_s, int8_t* level_s,
                                 int* pos) {
  __shared__ int warp_cnt[8][kMaxLevels];
  long long r = blockIdx.x * 256ll + threadIdx.x;
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int my = (r < count) ? level_r[r] : -1;
  int rank_in_warp = 0;
  for (int l = 0; l < nlev; ++l) {
    unsigned b = __ballot_sync(0xffffffffu, my == l);
    if (lane == 0) warp_cnt[warp][l] = __popc(b);
    if (my == l) rank_in_warp = __popc(b & ((1u << lane) - 1u));
  }
  __syncthreads();
  if (r >= count) return;
  int before = 0;
  for (int w = 0; w < warp; ++w) before += warp_cnt[w][my];
  int p = level_base[my] + chunk_prefix[blockIdx.x * nlev + my] + before + rank_in_warp;
  pos[r] = p;
  for (int i = 0; i < k; ++i) orbs_s[(long long)p * k + i] = orbs_r[r * k + i];
  level_s[p] = (int8_t)my;
}

// Enumerates the k-subsets of n orbitals sorted by (level, colex), level =
// number of orbitals >= nocc.  Device outputs: orbs [count][k], level [count],
// pos (colex rank -> sorted position).  Host outputs: per-level counts.
static int enumerate_strings(int n, int k, int nocc, DevBuf& orbs, DevBuf& level, DevBuf& pos,
                             std::vector<int>& level_count, cudaStream_t st) {
  long long count = binom_ll(n, k);
  if (count <= 0 || count > (1ll << 30)) {
    set_error("string space too large");
    return kErrArg;
  }
  int nlev = k + 1;
  DevBuf tmp_orbs, tmp_level, hist, lcount, lbase;
  size_t kk = k > 0 ? k : 1;
  ISCSI_TRY(tmp_orbs.alloc(sizeof(int16_t) * count * kk));
  ISCSI_TRY(tmp_level.alloc(count));
  ISCSI_TRY(orbs.alloc(sizeof(int16_t) * count * kk));
  ISCSI_TRY(level.alloc(count));
  ISCSI_TRY(pos.alloc(sizeof(int) * count));
  int nchunks = (int)((count + 255) / 256);
  ISCSI_TRY(hist.alloc(sizeof(int) * nchunks * nlev));
  ISCSI_TRY(lcount.alloc(sizeof(int) * nlev));
  ISCSI_TRY(lbase.alloc(sizeof(int) * nlev));
  k_unrank<<<launch_blocks(count, 256), 256, 0, st>>>(n, k, nocc, count, tmp_orbs.as<int16_t>(),
                                                       tmp_level.as<int8_t>());
  k_level_hist<<<nchunks, 256, 0, st>>>(tmp_level.as<int8_t>(), count, nlev, hist.as<int>());
  k_level_scan<<<1, 32, 0, st>>>(hist.as<int>(), nchunks, nlev, lcount.as<int>());
  level_count.assign(nlev, 0);
  ISCSI_CUDA(cudaMemcpyAsync(level_count.data(), lcount.p, sizeof(int) * nlev, cudaMemcpyDeviceToHost, st));
  ISCSI_CUDA(cudaStreamSynchronize(st));
  std::vector<int> base(nlev, 0);
  for (int l = 1; l < nlev; ++l) base[l] = base[l - 1] + level_count[l - 1];
  ISCSI_CUDA(cudaMemcpyAsync(lbase.p, base.data(), sizeof(int) * nlev, cudaMemcpyHostToDevice, st));
  k_scatter_sorted<<<nchunks, 256, 0, st>>>(tmp_orbs.as<int16_t>(), tmp_level.as<int8_t>(), count, k, nlev,
                                            hist.as<int>(), lbase.as<int>(), orbs.as<int16_t>(),
                                            level.as<int8_t>(), pos.as<int>());
  ISCSI_CUDA(cudaGetLastError());
  ISCSI_CUDA(cudaStreamSynchronize(st));
  return kOk;
}

// ---------------------------------------------------------------------------
// determinant offsets: alpha strings are sorted by level and every alpha
// string of level l carries nballow[l] beta strings, so off[A] is a closed
// form per level (the prefix sum of piecewise-constant row lengths)

__global__ void k_offsets(const int8_t* alevel, int count, const long long* level_off, const int* level_first,
                          const int* nballow, long long* off) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a > count) return;
  if (a == count) {
    int l = alevel[count - 1];
    off[a] = level_off[l] + (long long)(count - level_first[l]) * nballow[l];
    return;
  }
  int l = alevel[a];
  off[a] = level_off[l] + (long long)(a - level_first[l]) * nballow[l];
}

// ---------------------------------------------------------------------------
// hole-string tables (contraction / addition with phases, Eqs. four-last)

// lift[q][X] = pos(X u {q}) << 1 | (sign of a+_q on |X> is negative), or -1 if q in X
__global__ void k_lift(int n, int ne, int nhole, const int16_t* hole_orbs, const int* str_pos, int* lift) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n * nhole) return;
  int q = (int)(t / nhole), X = (int)(t % nhole);
  int o[kMaxElec];
  int below = 0, j = 0;
  bool clash = false;
  for (int i = 0; i < ne - 1; ++i) {
    int x = hole_orbs[(long long)X * (ne - 1) + i];
    if (x == q) clash = true;
    if (x < q) ++below;
  }
  if (clash) {
    lift[t] = -1;
    return;
  }
  for (int i = 0; i < ne - 1; ++i) {
    int x = hole_orbs[(long long)X * (ne - 1) + i];
    if (j == below) o[j++] = q;
    o[j++] = x;
  }
  if (j == below) o[j++] = q;
  int p = str_pos[colex_of(o, ne)];
  lift[t] = (p << 1) | (below & 1);
}

// dec[A][i] = X << 9 | p << 1 | neg for p = A[i], X = A \ {p}, sign (-1)^i of a+_p on |X>
__global__ void k_dec(int ne, int count, const int16_t* orbs, const int* hole_pos, int* dec) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)count * ne) return;
  int A = (int)(t / ne), i = (int)(t % ne);
  int o[kMaxElec];
  int j = 0;
  for (int u = 0; u < ne; ++u)
    if (u != i) o[j++] = orbs[(long long)A * ne + u];
  int X = hole_pos[colex_of(o, ne - 1)];
  int p = orbs[(long long)A * ne + i];
  dec[t] = (X << 9) | (p << 1) | (i & 1);
}

// ---------------------------------------------------------------------------
// integral units and classes

__device__ __forceinline__ long long pidx(int p, int q) {
  return p >= q ? (long long)p * (p + 1) / 2 + q : (long long)q * (q + 1) / 2 + p;
}

__device__ __forceinline__ double eri_g(const double* eri, long long npair, int p, int q, int r, int s) {
  return eri ? eri[pidx(p, q) * npair + pidx(r, s)] : 0.0;
}

// class id of the opposite-spin term with alpha (creator p, annihilator q) and
// beta (creator r, annihilator s); v = index in the virtual space.  The spin
// part kind is 2*[creator in V] + [annihilator in V]: 0 = C^dx A^ex,
// 1 = C^dx A^dx, 2 = C^ex A^ex, 3 = C^ex A^dx.
__constant__ signed char c_ab_class[4][4];

__device__ __forceinline__ int class_ab(bool pv, bool qv, bool rv, bool sv) {
  return 8 + c_ab_class[2 * pv + qv][2 * rv + sv];
}

__device__ __forceinline__ int class_one(int spin, bool pv, bool qv) {
  // H^{P,H}: P = [q in V], H = [p in O]; order H^{1,1}, H^{1,0}, H^{0,1}, H^{0,0}
  int P = qv, H = !pv;
  int idx = (P == 1 && H == 1) ? 0 : (P == 1 && H == 0) ? 1 : (P == 0 && H == 1) ? 2 : 3;
  return 4 * spin + idx;
}

__device__ __forceinline__ int class_ss(int spin, bool pv, bool rv, bool qv, bool sv) {
  int P = (int)qv + (int)sv, H = (int)(!pv) + (int)(!rv);
  // order (2,2),(2,1),(1,2),(2,0),(1,1),(0,2),(1,0),(0,1),(0,0)
  const int tbl[3][3] = {{8, 7, 5}, {6, 4, 2}, {3, 1, 0}};  // [P][H]
  return 24 + 9 * spin + tbl[P][H];
}

__device__ __forceinline__ bool class_on(unsigned long long mask, int cls) { return (mask >> cls) & 1ull; }

__constant__ double c_w_ab[6][6];  // updates per surviving opposite-spin unit, by (alpha kind, beta kind)

__device__ __forceinline__ int pair_kind(int p, int q, int ne) {
  bool pv = p >= ne, qv = q >= ne;
  if (!pv && !qv) return p == q ? 0 : 1;
  if (!pv && qv) return 2;
  if (pv && !qv) return 3;
  return p == q ? 4 : 5;
}

// G[m][k] = g_pqrs for m = pi(p,r), k = pi(q,s) if the unit survives, else 0
// (class labels use the reference's occupied orbitals na, nb; the update
// weights the level split oa, ob)
__global__ void k_build_g(const double* eri, long long npair, int n, int na, int nb, int oa, int ob, int npairs,
                          const int* pair_of, double tau, unsigned long long mask, double* G, double* upd,
                          unsigned long long* nunits) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double my_upd = 0.0;
  unsigned long long my_units = 0;
  if (t < (long long)npairs * npairs) {
    int m = (int)(t / npairs), k = (int)(t % npairs);
    int pr = pair_of[m], qs = pair_of[k];
    int p = pr / n, r = pr % n, q = qs / n, s = qs % n;
    double g = eri_g(eri, npair, p, q, r, s);
    bool keep = fabs(g) > tau && class_on(mask, class_ab(p >= na, q >= na, r >= nb, s >= nb));
    G[t] = keep ? g : 0.0;
    if (keep) {
      my_upd = c_w_ab[pair_kind(p, q, oa)][pair_kind(r, s, ob)];
      my_units = 1;
    }
  }
  // block reduction, one atomic per block
  for (int o = 16; o; o >>= 1) {
    my_upd += __shfl_xor_sync(0xffffffffu, my_upd, o);
    my_units += __shfl_xor_sync(0xffffffffu, my_units, o);
  }
  __shared__ double su[32];
  __shared__ unsigned long long sn[32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    su[w] = my_upd;
    sn[w] = my_units;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0;
    unsigned long long b = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      a += su[i];
      b += sn[i];
    }
    if (b) {
      atomicAdd(upd, a);
      atomicAdd(nunits, b);
    }
  }
}

// Dense string Hamiltonian of one spin from the surviving one-body and
// same-spin units: M[I][J] = sum_units unit * <I|op|J> (stored as M[J][I] when
// transpose is set: the beta part of sigma multiplies the CI block from the
// right, sigma[A,:] += c[A,:] M^T).  Also counts updates:
// each surviving unit that connects J to I is applied once per beta (other
// spin) string allowed beside both I and J.
__global__ void k_build_msame(int n, int ne, int spin, int count, const int16_t* orbs, const int8_t* level,
                              const double* h1, const double* eri, long long npair, double tau,
                              unsigned long long mask, const int* nother_both, int kmax, int transpose, double* M,
                              double* upd, unsigned long long* nunits) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double val = 0.0;
  double u1 = 0.0, u2 = 0.0;
  unsigned long long n1 = 0, n2 = 0;
  if (t < (long long)count * count) {
    int I = (int)(t / count), J = (int)(t % count);
    OrbMask mi, mj;
    mask_clear(mi);
    mask_clear(mj);
    for (int i = 0; i < ne; ++i) {
      mask_flip(mi, orbs[(long long)I * ne + i]);
      mask_flip(mj, orbs[(long long)J * ne + i]);
    }
    int cre[2], ann[2], nc = 0, na_ = 0;
    bool far = false;
    for (int i = 0; i < ne; ++i) {
      int x = orbs[(long long)I * ne + i];
      if (!mask_has(mj, x)) {
        if (nc < 2) cre[nc] = x;
        ++nc;
      }
      int y = orbs[(long long)J * ne + i];
      if (!mask_has(mi, y)) {
        if (na_ < 2) ann[na_] = y;
        ++na_;
      }
    }
    far = nc > 2;
    if (!far) {
      int lI = level[I], lJ = level[J];
      int lmax = lI > lJ ? lI : lJ;
      int rem = kmax - lmax;
      double nboth = rem < 0 ? 0.0 : (double)nother_both[rem > kMaxLevels - 1 ? kMaxLevels - 1 : rem];
      // one-body a+_p a_q
      auto one = [&](int p, int q) {
        double u = h1[p * n + q];
        if (!(fabs(u) > tau) || !class_on(mask, class_one(spin, p >= ne, q >= ne))) return;
        OrbMask m = mj;
        int s = mask_annihilate(m, q);
        s *= mask_create(m, p);
        if (!s) return;
        val += s * u;
        u1 += nboth;
        ++n1;
      };
      // same-spin (g_psrq - g_pqrs) a+_p a+_r a_q a_s, p>r, q>s
      auto two = [&](int c1, int c2, int a1, int a2) {
        int p = c1 > c2 ? c1 : c2, r = c1 > c2 ? c2 : c1;
        int q = a1 > a2 ? a1 : a2, s = a1 > a2 ? a2 : a1;
        if (p == r || q == s) return;
        double u = eri_g(eri, npair, p, s, r, q) - eri_g(eri, npair, p, q, r, s);
        if (!(fabs(u) > tau) || !class_on(mask, class_ss(spin, p >= ne, r >= ne, q >= ne, s >= ne))) return;
        OrbMask m = mj;
        int sg = mask_annihilate(m, s);
        sg *= mask_annihilate(m, q);
        sg *= mask_create(m, r);
        sg *= mask_create(m, p);
        if (!sg) return;
        val += sg * u;
        u2 += nboth;
        ++n2;
      };
      if (nc == 0) {
        for (int i = 0; i < ne; ++i) {
          int p = orbs[(long long)I * ne + i];
          one(p, p);
          for (int j = 0; j < i; ++j) {
            int r = orbs[(long long)I * ne + j];
            two(p, r, p, r);
          }
        }
      } else if (nc == 1) {
        int p = cre[0], q = ann[0];
        one(p, q);
        for (int i = 0; i < ne; ++i) {
          int k = orbs[(long long)J * ne + i];
          if (k != q) two(p, k, q, k);
        }
      } else {
        two(cre[0], cre[1], ann[0], ann[1]);
      }
    }
    M[transpose ? (long long)J * count + I : t] = val;
  }
  // block reductions
  for (int o = 16; o; o >>= 1) {
    u1 += __shfl_xor_sync(0xffffffffu, u1, o);
    u2 += __shfl_xor_sync(0xffffffffu, u2, o);
    n1 += __shfl_xor_sync(0xffffffffu, n1, o);
    n2 += __shfl_xor_sync(0xffffffffu, n2, o);
  }
  __shared__ double s1[32], s2[32];
  __shared__ unsigned long long sn1[32], sn2[32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    s1[w] = u1;
    s2[w] = u2;
    sn1[w] = n1;
    sn2[w] = n2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    unsigned long long c = 0, d = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      a += s1[i];
      b += s2[i];
      c += sn1[i];
      d += sn2[i];
    }
    if (c) {
      atomicAdd(&upd[0], a);
      atomicAdd(&nunits[0], c);
    }
    if (d) {
      atomicAdd(&upd[1], b);
      atomicAdd(&nunits[1], d);
    }
  }
}

// H diagonal: Malpha[A][A] + Mbeta[B][B] + sum_{p in A, r in B} G[pi(p,r)][pi(p,r)]
__global__ void k_diag(int na, int nb, int NA, int NB, const long long* off, const int16_t* aorbs,
                       const int16_t* borbs, const double* Ma, const double* Mb, const double* G, int npairs,
                       const int* pair_index, int n, double* diag) {
  int A = blockIdx.x;
  long long o0 = off[A], o1 = off[A + 1];
  double da = Ma ? Ma[(long long)A * NA + A] : 0.0;
  for (long long I = o0 + threadIdx.x; I < o1; I += blockDim.x) {
    int B = (int)(I - o0);
    double d = da + (Mb ? Mb[(long long)B * NB + B] : 0.0);
    if (G) {
      for (int i = 0; i < na; ++i) {
        int p = aorbs[(long long)A * na + i];
        for (int j = 0; j < nb; ++j) {
          int r = borbs[(long long)B * nb + j];
          int m = pair_index[p * n + r];
          d += G[(long long)m * npairs + m];
        }
      }
    }
    diag[I] = d;
  }
}

// ---------------------------------------------------------------------------

static void host_binom_table() {
  static bool done = false;
  static long long tbl[kMaxOrb + 1][kMaxElec + 2];
  if (done) return;
  for (int n = 0; n <= kMaxOrb; ++n)
    for (int k = 0; k < kMaxElec + 2; ++k) {
      // C(256, 17) overflows; only k <= 17 with n <= 256 is used for strings of
      // at most 16 electrons, and overflowing entries are never reached by the
      // enumerated ranks (they exceed the 2^30 string limit first).
      long double v = 1;
      for (int i = 1; i <= k; ++i) v = v * (n - k + i) / i;
      tbl[n][k] = (k > n) ? 0 : (v > 9.0e18L ? (long long)9e18 : (long long)std::llround((double)v));
    }
  cudaMemcpyToSymbol(c_binom, tbl, sizeof(tbl));
  // the 16 opposite-spin terms of Eqs. class_to_ex_dx..the_end in the paper's
  // order, each as (alpha kind, beta kind); kind = 2*[creator in V] + [annihilator in V]
  signed char t[4][4];
  const int ka[16] = {1, 3, 1, 0, 1, 3, 1, 0, 3, 2, 0, 2, 3, 2, 0, 2};
  const int kb[16] = {1, 1, 3, 1, 0, 3, 2, 3, 0, 1, 0, 3, 2, 0, 2, 2};
  for (int i = 0; i < 16; ++i) t[ka[i]][kb[i]] = (signed char)i;
  cudaMemcpyToSymbol(c_ab_class, t, sizeof(t));
  done = true;
}

// number of (ne-1)-subsets of the orbitals outside {p,q} with the given
// level, for the six (p,q) kinds of pair_kind (inner / outer membership, the
// first nocc orbitals being the inner ones, and p == q)
static double hole_count(int n, int ne, int nocc, int kind, int lvl) {
  // orbitals removed from the inner and the outer orbitals by {p,q}
  static const int rmO[6] = {1, 2, 1, 1, 0, 0};
  static const int rmV[6] = {0, 0, 1, 1, 1, 2};
  int k = ne - 1;
  int o = nocc - rmO[kind], v = (n - nocc) - rmV[kind];
  if (o < 0 || v < 0 || k < 0) return 0.0;
  return (double)binom_ll(o, k - lvl) * (double)binom_ll(v, lvl);
}

int context_build(Context& ctx, int n, int na, int nb, int kmax, const double* h1, const double* eri, double tau,
                  int ninner) {
  cudaStream_t st = stream();
  host_binom_table();
  ISCSI_CUDA(cudaGetLastError());
  static long long builds = 0;
  ctx.noalloc_gen = ++builds;
  // a general one-body operator (a transition operator a+_p a_q, say) has
  // h_pq != h_qp; the string matrices are then not symmetric
  ctx.h1_symmetric = true;
  for (int p = 0; p < n && ctx.h1_symmetric; ++p)
    for (int q = 0; q < p; ++q)
      if (!(h1[(long long)p * n + q] == h1[(long long)q * n + p])) {
        ctx.h1_symmetric = false;
        break;
      }
  ctx.n = n;
  ctx.na = na;
  ctx.nb = nb;
  ctx.kmax = kmax;
  ctx.tau = tau;
  ctx.class_mask = options().class_mask;
  ISCSI_CUDA(cudaEventCreate(&ctx.ev0));
  ISCSI_CUDA(cudaEventCreate(&ctx.ev1));
  ISCSI_CUDA(cudaEventRecord(ctx.ev0, st));

  // --- strings and hole strings per spin
  int nel[2] = {na, nb};
  std::vector<int> lcount[2];
  for (int s = 0; s < 2; ++s) {
    SpinSpace& S = ctx.sp[s];
    S.ne = nel[s];
    S.nocc = ninner < 0 ? S.ne : ninner;
    ISCSI_TRY(enumerate_strings(n, S.ne, S.nocc, S.orbs, S.level, S.pos, lcount[s], st));
    S.count = (int)binom_ll(n, S.ne);
    S.maxlevel = 0;
    for (int l = 0; l < (int)lcount[s].size(); ++l)
      if (lcount[s][l] > 0) S.maxlevel = l;
    S.level_start.assign(S.maxlevel + 2, 0);
    for (int l = 0; l <= S.maxlevel; ++l) S.level_start[l + 1] = S.level_start[l] + lcount[s][l];
  }
  // beta strings with level <= L, alpha strings with level <= L
  auto cnt_le = [&](int s, int L) -> long long {
    if (L < 0) return 0;
    const SpinSpace& S = ctx.sp[s];
    if (L > S.maxlevel) L = S.maxlevel;
    return S.level_start[L + 1];
  };
  // --- determinant addressing
  SpinSpace& SA = ctx.sp[0];
  ctx.nb_allowed_lvl.assign(kMaxLevels, 0);
  for (int l = 0; l < kMaxLevels; ++l) ctx.nb_allowed_lvl[l] = cnt_le(1, kmax - l);
  std::vector<long long> level_off(SA.maxlevel + 1, 0);
  std::vector<int> level_first(SA.maxlevel + 1, 0), nballow_i(kMaxLevels, 0);
  for (int l = 0; l < kMaxLevels; ++l) nballow_i[l] = (int)ctx.nb_allowed_lvl[l];
  long long acc = 0;
  for (int l = 0; l <= SA.maxlevel; ++l) {
    level_off[l] = acc;
    level_first[l] = SA.level_start[l];
    acc += (long long)(SA.level_start[l + 1] - SA.level_start[l]) * ctx.nb_allowed_lvl[l];
  }
  ctx.ndet = acc;
  ctx.gas_ndet = acc;
  if (ctx.ndet <= 0) {
    set_error("empty determinant space");
    return kErrArg;
  }
  {
    DevBuf dlo, dlf;
    ISCSI_TRY(dlo.alloc(sizeof(long long) * level_off.size()));
    ISCSI_TRY(dlf.alloc(sizeof(int) * level_first.size()));
    ISCSI_TRY(ctx.nballow.alloc(sizeof(int) * kMaxLevels));
    ISCSI_TRY(ctx.off.alloc(sizeof(long long) * (SA.count + 1)));
    ISCSI_CUDA(cudaMemcpyAsync(dlo.p, level_off.data(), sizeof(long long) * level_off.size(), cudaMemcpyHostToDevice, st));
    ISCSI_CUDA(cudaMemcpyAsync(dlf.p, level_first.data(), sizeof(int) * level_first.size(), cudaMemcpyHostToDevice, st));
    ISCSI_CUDA(cudaMemcpyAsync(ctx.nballow.p, nballow_i.data(), sizeof(int) * kMaxLevels, cudaMemcpyHostToDevice, st));
    k_offsets<<<launch_blocks(SA.count + 1, 256), 256, 0, st>>>(SA.level.as<int8_t>(), SA.count, dlo.as<long long>(),
                                                                dlf.as<int>(), ctx.nballow.as<int>(),
                                                                ctx.off.as<long long>());
    ISCSI_CUDA(cudaGetLastError());
    ctx.off_h.resize(SA.count + 1);
    ISCSI_CUDA(cudaMemcpyAsync(ctx.off_h.data(), ctx.off.p, sizeof(long long) * (SA.count + 1), cudaMemcpyDeviceToHost, st));
    ISCSI_CUDA(cudaStreamSynchronize(st));
  }

  // --- integrals to the device (temporary)
  long long npair = (long long)n * (n + 1) / 2;
  DevBuf d_h1, d_eri, d_upd, d_units;
  ISCSI_TRY(d_h1.alloc(sizeof(double) * n * n));
  ISCSI_CUDA(cudaMemcpyAsync(d_h1.p, h1, sizeof(double) * n * n, cudaMemcpyHostToDevice, st));
  if (eri) {
    ISCSI_TRY(d_eri.alloc(sizeof(double) * npair * npair));
    ISCSI_CUDA(cudaMemcpyAsync(d_eri.p, eri, sizeof(double) * npair * npair, cudaMemcpyHostToDevice, st));
  }
  ISCSI_TRY(d_upd.alloc(sizeof(double) * 8));
  ISCSI_TRY(d_units.alloc(sizeof(unsigned long long) * 8));
  ISCSI_CUDA(cudaMemsetAsync(d_upd.p, 0, sizeof(double) * 8, st));
  ISCSI_CUDA(cudaMemsetAsync(d_units.p, 0, sizeof(unsigned long long) * 8, st));

  // --- same-spin string Hamiltonians
  unsigned long long cm = ctx.class_mask;
  // with a symmetric one-body part and every one-body and same-spin class
  // kept, M is symmetric (each term's adjoint is present with the same unit)
  // and identical for both spins when na == nb, so one matrix serves alpha and
  // (transposed) beta
  const unsigned long long same_spin_bits = 0xFFull | (0x3FFFFull << 24);
  ctx.beta_alias = (na == nb) && ((cm & same_spin_bits) == same_spin_bits) && ctx.h1_symmetric;
  for (int s = 0; s < 2; ++s) {
    SpinSpace& S = ctx.sp[s];
    if (S.ne == 0) continue;
    if (s == 1 && ctx.beta_alias) {
      // identical matrix; counts are those of alpha with the roles of the spins swapped
      continue;
    }
    long long cnt2 = (long long)S.count * S.count;
    ISCSI_TRY(ctx.M64[s].alloc(sizeof(double) * cnt2));
    std::vector<int> nboth(kMaxLevels, 0);
    for (int L = 0; L < kMaxLevels; ++L) nboth[L] = (int)cnt_le(1 - s, L);
    DevBuf d_nboth;
    ISCSI_TRY(d_nboth.alloc(sizeof(int) * kMaxLevels));
    ISCSI_CUDA(cudaMemcpyAsync(d_nboth.p, nboth.data(), sizeof(int) * kMaxLevels, cudaMemcpyHostToDevice, st));
    k_build_msame<<<launch_blocks(cnt2, 256), 256, 0, st>>>(
        n, S.ne, s, S.count, S.orbs.as<int16_t>(), S.level.as<int8_t>(), d_h1.as<double>(),
        eri ? d_eri.as<double>() : nullptr, npair, tau, cm, d_nboth.as<int>(), kmax, s == 1 ? 1 : 0,
        ctx.M64[s].as<double>(),
        d_upd.as<double>() + 2 * s, d_units.as<unsigned long long>() + 2 * s);
    ISCSI_CUDA(cudaGetLastError());
    ISCSI_CUDA(cudaStreamSynchronize(st));
  }

  // --- hole strings and lift / dec tables of each spin with electrons (the
  // opposite-spin sigma part and the density matrices use them; they do not
  // depend on the integrals)
  ctx.have_ab = (na > 0 && nb > 0 && eri != nullptr);
  std::vector<int> hole_lcount[2];
  {
    DevBuf hole_orbs[2], hole_level[2], hole_pos[2];
    for (int s = 0; s < 2; ++s) {
      SpinSpace& S = ctx.sp[s];
      if (S.ne == 0) continue;
      ISCSI_TRY(enumerate_strings(n, S.ne - 1, S.nocc, hole_orbs[s], hole_level[s], hole_pos[s], hole_lcount[s], st));
      S.nhole = (int)binom_ll(n, S.ne - 1);
      if (S.nhole >= (1 << 22)) {
        set_error("hole-string space too large (>= 2^22)");
        return kErrArg;
      }
      S.hole_level.resize(S.nhole);
      std::vector<int8_t> hl(S.nhole);
      ISCSI_CUDA(cudaMemcpy(hl.data(), hole_level[s].p, S.nhole, cudaMemcpyDeviceToHost));
      S.hole_maxlevel = 0;
      for (int i = 0; i < S.nhole; ++i) {
        S.hole_level[i] = hl[i];
        S.hole_maxlevel = std::max(S.hole_maxlevel, (int)hl[i]);
      }
      ISCSI_TRY(S.lift.alloc(sizeof(int) * (size_t)n * S.nhole));
      ISCSI_TRY(S.dec.alloc(sizeof(int) * (size_t)S.count * S.ne));
      k_lift<<<launch_blocks((long long)n * S.nhole, 256), 256, 0, st>>>(n, S.ne, S.nhole, hole_orbs[s].as<int16_t>(),
                                                                          S.pos.as<int>(), S.lift.as<int>());
      k_dec<<<launch_blocks((long long)S.count * S.ne, 256), 256, 0, st>>>(S.ne, S.count, S.orbs.as<int16_t>(),
                                                                            hole_pos[s].as<int>(), S.dec.as<int>());
      ISCSI_CUDA(cudaGetLastError());
      ISCSI_CUDA(cudaStreamSynchronize(st));
    }
  }
  if (na > 0 && nb > 0) {
    // pair ordering pi(p, r): sorted by level(p) + level(r); within a level
    // sum in 8 x 8 patches of (p, r) (patches by p, then r; inside one, p
    // then r).  A 128-row block of G then covers a 8 x 16 patch of (p, r)
    // and a 16-wide K step a 2 x 8 patch of (q, s), so that a block's units
    // are all small (screened, or with leading zero slices) whenever the
    // integrals decay in either |p - q| or |r - s|, not only in |p - q|.
    ctx.npairs = n * n;
    std::vector<int> pair_of(ctx.npairs), pair_index(ctx.npairs);
    ctx.pair_level_start.assign(4, 0);
    {
      constexpr int kPatch = 8;
      int m = 0;
      for (int lvl = 0; lvl <= 2; ++lvl) {
        ctx.pair_level_start[lvl] = m;
        for (int p0 = 0; p0 < n; p0 += kPatch)
          for (int r0 = 0; r0 < n; r0 += kPatch)
            for (int p = p0; p < std::min(n, p0 + kPatch); ++p)
              for (int r = r0; r < std::min(n, r0 + kPatch); ++r)
                if ((p >= ctx.sp[0].nocc) + (r >= ctx.sp[1].nocc) == lvl) {
                  pair_of[m] = p * n + r;
                  pair_index[p * n + r] = m;
                  ++m;
                }
      }
      ctx.pair_level_start[3] = m;
    }
    ISCSI_TRY(ctx.pair_of.alloc(sizeof(int) * ctx.npairs));
    ISCSI_TRY(ctx.pair_index.alloc(sizeof(int) * ctx.npairs));
    ISCSI_CUDA(cudaMemcpyAsync(ctx.pair_of.p, pair_of.data(), sizeof(int) * ctx.npairs, cudaMemcpyHostToDevice, st));
    ISCSI_CUDA(cudaMemcpyAsync(ctx.pair_index.p, pair_index.data(), sizeof(int) * ctx.npairs, cudaMemcpyHostToDevice, st));
    std::vector<int> pair_split(ctx.npairs);
    for (int m = 0; m < ctx.npairs; ++m) pair_split[m] = ((pair_of[m] / n) << 16) | (pair_of[m] % n);
    ISCSI_TRY(ctx.pair_split.alloc(sizeof(int) * ctx.npairs));
    ISCSI_CUDA(cudaMemcpyAsync(ctx.pair_split.p, pair_split.data(), sizeof(int) * ctx.npairs, cudaMemcpyHostToDevice,
                               st));
    ISCSI_CUDA(cudaStreamSynchronize(st));  // the host vector must outlive the copy

    // hole pairs (X, Y) grouped by column level class c = level(X) + level(Y)
    const SpinSpace& HA = ctx.sp[0];
    const SpinSpace& HB = ctx.sp[1];
    int ncls = HA.hole_maxlevel + HB.hole_maxlevel + 1;
    long long nhp = (long long)HA.nhole * HB.nhole;
    std::vector<int8_t> hpc(nhp);
    std::vector<int> hpl(nhp), hpinv;
    std::vector<int> cls_count(ncls, 0);
    for (int X = 0; X < HA.nhole; ++X)
      for (int Y = 0; Y < HB.nhole; ++Y) {
        int c = HA.hole_level[X] + HB.hole_level[Y];
        hpc[(long long)X * HB.nhole + Y] = (int8_t)c;
        hpl[(long long)X * HB.nhole + Y] = cls_count[c]++;
      }
    ctx.hp_class_start.assign(ncls + 1, 0);
    for (int c = 0; c < ncls; ++c) ctx.hp_class_start[c + 1] = ctx.hp_class_start[c] + cls_count[c];
    hpinv.resize(nhp);
    for (long long t = 0; t < nhp; ++t) hpinv[ctx.hp_class_start[hpc[t]] + hpl[t]] = (int)t;
    ISCSI_TRY(ctx.hp_class.alloc(nhp));
    ISCSI_TRY(ctx.hp_local.alloc(sizeof(int) * nhp));
    ISCSI_TRY(ctx.hp_inv.alloc(sizeof(int) * nhp));
    ISCSI_CUDA(cudaMemcpyAsync(ctx.hp_class.p, hpc.data(), nhp, cudaMemcpyHostToDevice, st));
    ISCSI_CUDA(cudaMemcpyAsync(ctx.hp_local.p, hpl.data(), sizeof(int) * nhp, cudaMemcpyHostToDevice, st));
    ISCSI_CUDA(cudaMemcpyAsync(ctx.hp_inv.p, hpinv.data(), sizeof(int) * nhp, cudaMemcpyHostToDevice, st));
    // per column class: rows of T_c and of Ct_c (pairs whose level leaves room)
    ctx.cls.clear();
    ctx.ct_elems = 0;
    for (int c = 0; c < ncls; ++c) {
      ColClass cc;
      cc.level = c;
      cc.ncol = cls_count[c];
      int room = kmax - c;
      int rows = room < 0 ? 0 : ctx.pair_level_start[std::min(room, 2) + 1];
      cc.mrows = rows;
      cc.krows = rows;
      cc.ct_off = ctx.ct_elems;
      if (cc.ncol > 0 && rows > 0) ctx.ct_elems += (size_t)rows * cc.ncol;
      ctx.cls.push_back(cc);
    }
  }
  if (ctx.have_ab) {
    // opposite-spin updates per surviving unit, by (alpha pair kind, beta pair kind)
    double w[6][6];
    const int qv_of[6] = {0, 0, 1, 0, 1, 1}, pv_of[6] = {0, 0, 0, 1, 1, 1};
    for (int ka = 0; ka < 6; ++ka)
      for (int kb = 0; kb < 6; ++kb) {
        double tot = 0.0;
        for (int lx = 0; lx <= na - 1; ++lx)
          for (int ly = 0; ly <= nb - 1; ++ly) {
            int src = lx + qv_of[ka] + ly + qv_of[kb];
            int dst = lx + pv_of[ka] + ly + pv_of[kb];
            if (src <= kmax && dst <= kmax)
              tot += hole_count(n, na, ctx.sp[0].nocc, ka, lx) * hole_count(n, nb, ctx.sp[1].nocc, kb, ly);
          }
        w[ka][kb] = tot;
      }
    ISCSI_CUDA(cudaMemcpyToSymbol(c_w_ab, w, sizeof(w)));

    long long g2 = (long long)ctx.npairs * ctx.npairs;
    ISCSI_TRY(ctx.G64.alloc(sizeof(double) * g2));
    k_build_g<<<launch_blocks(g2, 256), 256, 0, st>>>(d_eri.as<double>(), npair, n, na, nb, ctx.sp[0].nocc,
                                                      ctx.sp[1].nocc, ctx.npairs,
                                                      ctx.pair_of.as<int>(), tau, cm, ctx.G64.as<double>(),
                                                      d_upd.as<double>() + 4, d_units.as<unsigned long long>() + 4);
    ISCSI_CUDA(cudaGetLastError());
  }

  // --- statistics
  double upd[8];
  unsigned long long units[8];
  ISCSI_CUDA(cudaMemcpyAsync(upd, d_upd.p, sizeof(upd), cudaMemcpyDeviceToHost, st));
  ISCSI_CUDA(cudaMemcpyAsync(units, d_units.p, sizeof(units), cudaMemcpyDeviceToHost, st));
  ISCSI_CUDA(cudaStreamSynchronize(st));
  if (ctx.beta_alias) {
    // the beta counts follow from the alpha matrix with the spins' roles swapped;
    // with na == nb the strings and level tables of both spins coincide
    upd[2] = upd[0];
    upd[3] = upd[1];
    units[2] = units[0];
    units[3] = units[1];
  }
  ctx.updates_onebody = (na ? upd[0] : 0) + (nb ? upd[2] : 0);
  ctx.updates_samespin = (na ? upd[1] : 0) + (nb ? upd[3] : 0);
  ctx.updates_opposite = ctx.have_ab ? upd[4] : 0.0;
  ctx.units_onebody = (long long)((na ? units[0] : 0) + (nb ? units[2] : 0));
  ctx.units_samespin = (long long)((na ? units[1] : 0) + (nb ? units[3] : 0));
  ctx.units_opposite = ctx.have_ab ? (long long)units[4] : 0;
  // the one-body and same-spin counters count (unit, string pair) hits in M;
  // unit totals below count distinct integral terms
  ctx.units_onebody_total = (long long)(na ? n * n : 0) + (nb ? n * n : 0);
  long long pairs = (long long)n * (n - 1) / 2;
  ctx.units_samespin_total = (eri ? ((na >= 2 ? pairs * pairs : 0) + (nb >= 2 ? pairs * pairs : 0)) : 0);
  ctx.units_opposite_total = ctx.have_ab ? (long long)n * n * n * n : 0;

  // --- diagonal
  ISCSI_TRY(ctx.diag.alloc(sizeof(double) * ctx.ndet));
  {
    const double* Ma = na ? ctx.M64[0].as<double>() : nullptr;
    const double* Mb = nb ? (ctx.beta_alias ? ctx.M64[0].as<double>() : ctx.M64[1].as<double>()) : nullptr;
    k_diag<<<SA.count, 128, 0, st>>>(na, nb, SA.count, ctx.sp[1].count, ctx.off.as<long long>(),
                                     SA.orbs.as<int16_t>(), ctx.sp[1].orbs.as<int16_t>(), Ma, Mb,
                                     ctx.have_ab ? ctx.G64.as<double>() : nullptr, ctx.npairs,
                                     ctx.have_ab ? ctx.pair_index.as<int>() : nullptr, n, ctx.diag.as<double>());
    ISCSI_CUDA(cudaGetLastError());
  }
  ISCSI_CUDA(cudaEventRecord(ctx.ev1, st));
  ISCSI_CUDA(cudaStreamSynchronize(st));
  float ms = 0;
  cudaEventElapsedTime(&ms, ctx.ev0, ctx.ev1);
  ctx.init_ms = ms;
  return kOk;
}

}  // namespace iscsi
