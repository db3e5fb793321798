// davidson.cu -- lowest eigenpairs of H_tau (Eq. hcec) by a device-resident
// Davidson iteration around the sigma step (Eq. sigma).  The paper names
// Davidson as the usual optimisation step that follows sigma; its own runs
// used imaginary-time propagation instead (Sec. "Basis and calculation set up").
//
// Everything lives on the device: the basis V, its images W = H V, the Ritz
// vectors X and residuals R, the subspace matrix S = V^T W, its eigen-
// decomposition and a small control block (DavCtl) holding the basis size,
// Ritz values, residual norms and flags.  Every kernel reads the basis size
// from the control block, so one iteration is a fixed launch sequence:
//
//   restart      thick restart to the lowest nkeep Ritz pairs when the next
//                expansion would overflow the basis (flag set by check)
//   precondition t_j = (r_j - eps_j x_j) / (theta_j - diag) (Olsen's correction,
//                option), zero for converged roots
//   orthogonalise block Gram-Schmidt against V (a second pass only where the
//                first removed more than 30% of a column), then two passes of
//                Cholesky QR within the block; directions that keep no more
//                than 1e-8 of their norm are dropped
//   sigma        W_new = H T (the FP64 or FP32 sigma path)
//   append       T, W_new join V, W; the new rows and columns of S
//   eig          one-CTA parallel Jacobi on S (Brent-Luk round-robin order)
//   ritz         X = V Y, R = W Y - X diag(theta), |R_j|
//   check        convergence (all |R_j| <= tol and |d theta| <= etol),
//                restart decision
//
// which is captured once as a CUDA graph and replayed each iteration; the host
// reads the control block back (one small copy) to decide whether to stop.
// Projections, Rayleigh-Ritz, residual norms and the orthonormalisation are
// FP64.  With the mixed-precision option the sigma steps run in FP32 until
// every residual norm is below switch_tol (or stops improving near the FP32
// floor); then the basis is collapsed to the lowest 2k Ritz vectors, their
// images are recomputed with the FP64 sigma, and the iteration finishes in
// FP64, so the returned energies are Rayleigh quotients of the FP64 operator.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "internal.cuh"

namespace iscsi {

constexpr int kMaxRoots = 32;
constexpr int kVecThreads = 256;
constexpr int kVecBlocks = 4 * 152;  // streaming kernels: 4 blocks per SM
constexpr int kDotT = 8;             // tall-skinny dot products: 8 x 8 vectors per block

struct DavCtl {
  int m;        // basis size
  int k;        // block: roots iterated
  int kw;       // roots wanted (the first kw of the block decide convergence)
  int maxsub;   // basis capacity
  int iter;     // completed checks
  int restart;  // 1: thick restart at the start of the next expansion
  int nkeep;    // Ritz pairs kept by that restart
  int added;    // vectors appended by the last expansion
  int status;   // kStatus* bits
  double tol, etol, rmax, dmax;
  int reorth;    // 1: the block needs a second Gram-Schmidt pass
  int olsen;    // 1: Olsen's correction in the preconditioner
  double theta[kMaxRoots], theta_prev[kMaxRoots], rnorm[kMaxRoots], nrm0[kMaxRoots], eps[kMaxRoots];
  int active[kMaxRoots];
};
enum { kStatusConverged = 1, kStatusNonFinite = 2, kStatusNoDirection = 4 };

__device__ __forceinline__ double dav_den(double th, double d) {
  double den = th - d;
  if (fabs(den) < 1e-8) den = den < 0 ? -1e-8 : 1e-8;
  return den;
}

__device__ __forceinline__ double block_sum(double x, double* red) {
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = x;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;  // valid in thread 0
}

// ---------------------------------------------------------------------------
// FP64-accurate products on the FP32 units.  GB300 issues FP64 at about 1/64
// of its FP32 rate, so the tall-skinny products of the iteration (projections,
// Ritz vectors, restarts) are formed in double-float arithmetic: each double
// is split exactly into a float pair (hi = its leading 24 significant bits,
// lo = the rest rounded, 2^-48 relative), a product is the exact product of the
// high parts (fmaf gives its rounding error) plus the cross terms in FP32, and
// a sum is a float pair renormalised after every term by Knuth's error-free
// two-sum (about 3e-14 of sum |x y| over a thread's few hundred terms, which
// FP64 sums of the same length match).  Magnitudes below 2^-126 (the float
// range) are flushed to zero, far below the iteration's tolerances for the
// unit-norm basis and its images.  Reductions across threads stay FP64.
struct Df {
  float s, c;
};

__device__ __forceinline__ void df_split(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  const unsigned int sgn = (unsigned int)(b >> 63) << 31;
  const int eh = E - 1023 + 127;
  if (eh < 1 || eh > 254) {
    hi = 0.0f;
    lo = 0.0f;
    return;
  }
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  hi = __uint_as_float(sgn | ((unsigned int)eh << 23) | (unsigned int)(m >> 29));
  const int el = E - 1075 + 127;  // the low 29 bits L are worth L 2^(E - 1075)
  const float l = el >= 1 ? __fmul_rn(__int2float_rn((int)(m & 0x1FFFFFFFull)), __uint_as_float((unsigned int)el << 23))
                          : 0.0f;
  lo = sgn ? -l : l;
}

__device__ __forceinline__ void df_fma(Df& a, float xh, float xl, float yh, float yl) {
  const float p = __fmul_rn(xh, yh);
  const float e = __fmaf_rn(xh, yh, -p);                 // xh yh - p, exact
  const float cr = __fmaf_rn(xh, yl, __fmul_rn(xl, yh));  // cross terms
  const float s = __fadd_rn(a.s, p);                     // two-sum of a.s and p
  const float bb = __fsub_rn(s, a.s);
  const float t = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  const float c = __fadd_rn(a.c, __fadd_rn(t, __fadd_rn(e, cr)));
  const float s2 = __fadd_rn(s, c);                      // renormalise
  a.c = __fsub_rn(c, __fsub_rn(s2, s));
  a.s = s2;
}

__device__ __forceinline__ double df_value(const Df& a) { return (double)a.s + (double)a.c; }

// partial[b][i][j] = sum over block b's elements of A_i[e] B_j[e], for
// i < na = (na_dev ? *na_dev : 0) + na_add and j < nb; rows_cap bounds na.
// Each block takes kDotT rows of A and NB columns of B (NB = nb when nb <= 8,
// so no FMA is spent on absent columns: GB300's FP64 rate, not HBM, bounds
// these products).
template <int NB>
__global__ void __launch_bounds__(kVecThreads) k_tsdots(const double* __restrict__ A, const int* __restrict__ na_dev,
                                                        int na_add, const double* __restrict__ B, int nb, long long N,
                                                        double* __restrict__ partial, int rows_cap,
                                                        const int* __restrict__ gate) {
  if (gate && !*gate) return;
  const int na = (na_dev ? *na_dev : 0) + na_add;
  const int tiles_b = (nb + NB - 1) / NB;
  const int i0 = (blockIdx.y / tiles_b) * kDotT, j0 = (blockIdx.y % tiles_b) * NB;
  if (i0 >= na) return;
  const int ra = min(kDotT, na - i0);
  Df acc[kDotT][NB];
#pragma unroll
  for (int a = 0; a < kDotT; ++a)
#pragma unroll
    for (int b = 0; b < NB; ++b) acc[a][b] = Df{0.0f, 0.0f};
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride) {
    float bh[NB], bl[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) df_split((j0 + b < nb) ? B[(long long)(j0 + b) * N + e] : 0.0, bh[b], bl[b]);
#pragma unroll
    for (int a = 0; a < kDotT; ++a)
      if (a < ra) {
        float ah, al;
        df_split(A[(long long)(i0 + a) * N + e], ah, al);
#pragma unroll
        for (int b = 0; b < NB; ++b) df_fma(acc[a][b], ah, al, bh[b], bl[b]);
      }
  }
  __shared__ double red[kVecThreads / 32][kDotT * NB];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < kDotT; ++a)
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      double x = df_value(acc[a][b]);
      for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) red[warp][a * NB + b] = x;
    }
  __syncthreads();
  if (threadIdx.x < kDotT * NB) {
    double x = 0.0;
    for (int w = 0; w < kVecThreads / 32; ++w) x += red[w][threadIdx.x];
    const int a = threadIdx.x / NB, b = threadIdx.x % NB;
    if (a < ra && j0 + b < nb) partial[((long long)blockIdx.x * rows_cap + i0 + a) * nb + j0 + b] = x;
  }
}

// x[0] + x[stride] + ... + x[(parts - 1) stride] by one warp in a fixed order
// (lane l sums l, l + 32, ...; then a butterfly whose two operands are the same
// on both lanes of every exchange, so every lane returns the same value, and
// every run the same)
__device__ __forceinline__ double warp_sum_strided(const double* __restrict__ x, long long stride, int parts,
                                                   int lane) {
  double s = 0.0;
  for (int p = lane; p < parts; p += 32) s += x[(long long)p * stride];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// C[i][j] = sum over blocks of partial[b][i][j], one warp per element
// (nothing when gate points at 0)
__global__ void k_tsreduce(const double* __restrict__ partial, int parts, const int* __restrict__ na_dev, int na_add,
                           int nb, int rows_cap, double* __restrict__ C, const int* __restrict__ gate) {
  if (gate && !*gate) return;
  const int na = (na_dev ? *na_dev : 0) + na_add;
  const int t = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (t >= na * nb) return;  // whole warps
  const double x = warp_sum_strided(partial + t, (long long)rows_cap * nb, parts, lane);
  if (lane == 0) C[t] = x;
}

// X_j = sum_i V_i Y[i][j], R_j = sum_i W_i Y[i][j] - theta_j X_j for j in
// [j0, j0 + KC) (j < k); partial[b][j] = block b's part of |R_j|^2
template <int KC>
__global__ void __launch_bounds__(kVecThreads) k_dav_ritz(const double* __restrict__ V, const double* __restrict__ W,
                                                          const DavCtl* __restrict__ ctl, const double* __restrict__ Y,
                                                          int ldy, int j0, long long N, double* __restrict__ X,
                                                          double* __restrict__ R, double* __restrict__ partial) {
  extern __shared__ float sYf[];  // [2][m][KC]: Y split into float pairs
  __shared__ double red[kVecThreads / 32];
  const int m = ctl->m, k = ctl->k;
  const int cnt = min(KC, k - j0);
  if (cnt <= 0) return;
  float* sYh = sYf;
  float* sYl = sYf + m * KC;
  for (int t = threadIdx.x; t < m * KC; t += blockDim.x)
    df_split((t % KC < cnt) ? Y[(t / KC) * ldy + j0 + t % KC] : 0.0, sYh[t], sYl[t]);
  double th[KC];
#pragma unroll
  for (int j = 0; j < KC; ++j) th[j] = j < cnt ? ctl->theta[j0 + j] : 0.0;
  __syncthreads();
  double rr[KC];
#pragma unroll
  for (int j = 0; j < KC; ++j) rr[j] = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride) {
    Df x[KC], r[KC];
#pragma unroll
    for (int j = 0; j < KC; ++j) x[j] = r[j] = Df{0.0f, 0.0f};
    for (int i = 0; i < m; ++i) {
      float vh, vl, wh, wl;
      df_split(V[(long long)i * N + e], vh, vl);
      df_split(W[(long long)i * N + e], wh, wl);
#pragma unroll
      for (int j = 0; j < KC; ++j) {
        df_fma(x[j], vh, vl, sYh[i * KC + j], sYl[i * KC + j]);
        df_fma(r[j], wh, wl, sYh[i * KC + j], sYl[i * KC + j]);
      }
    }
#pragma unroll
    for (int j = 0; j < KC; ++j)
      if (j < cnt) {
        const double xv = df_value(x[j]);
        const double rv = df_value(r[j]) - th[j] * xv;
        X[(long long)(j0 + j) * N + e] = xv;
        R[(long long)(j0 + j) * N + e] = rv;
        rr[j] = fma(rv, rv, rr[j]);
      }
  }
#pragma unroll
  for (int j = 0; j < KC; ++j) {
    const double t = block_sum(rr[j], red);
    if (threadIdx.x == 0 && j < cnt) partial[(long long)blockIdx.x * k + j0 + j] = t;
  }
}

// out_j = sum_{i<m} V_i Y[i][j0 + j] for j < min(KC, nkeep - j0); only when a
// restart is pending
template <int KC>
__global__ void __launch_bounds__(kVecThreads) k_dav_restart_lincomb(const double* __restrict__ V,
                                                                     const DavCtl* __restrict__ ctl,
                                                                     const double* __restrict__ Y, int ldy, int j0,
                                                                     long long N, double* __restrict__ out) {
  extern __shared__ float sYcf[];  // [2][m][KC]
  if (!ctl->restart) return;
  const int m = ctl->m;
  const int cnt = min(KC, ctl->nkeep - j0);
  if (cnt <= 0) return;
  float* sYh = sYcf;
  float* sYl = sYcf + m * KC;
  for (int t = threadIdx.x; t < m * KC; t += blockDim.x)
    df_split((t % KC < cnt) ? Y[(t / KC) * ldy + j0 + t % KC] : 0.0, sYh[t], sYl[t]);
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride) {
    Df acc[KC];
#pragma unroll
    for (int j = 0; j < KC; ++j) acc[j] = Df{0.0f, 0.0f};
    for (int i = 0; i < m; ++i) {
      float vh, vl;
      df_split(V[(long long)i * N + e], vh, vl);
#pragma unroll
      for (int j = 0; j < KC; ++j) df_fma(acc[j], vh, vl, sYh[i * KC + j], sYl[i * KC + j]);
    }
#pragma unroll
    for (int j = 0; j < KC; ++j)
      if (j < cnt) out[(long long)(j0 + j) * N + e] = df_value(acc[j]);
  }
}

// dst[0 : nkeep N] = src[...] when a restart is pending
__global__ void k_dav_restart_copy(double* __restrict__ dst, const double* __restrict__ src,
                                   const DavCtl* __restrict__ ctl, long long N) {
  if (!ctl->restart) return;
  const long long total = (long long)ctl->nkeep * N;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += stride) dst[t] = src[t];
}

// after a restart the basis is the Ritz basis: S = diag(theta_0 .. theta_{nkeep-1})
__global__ void k_dav_restart_S(DavCtl* __restrict__ ctl, double* __restrict__ S, int lds,
                                const double* __restrict__ theta_all) {
  if (!ctl->restart) return;
  const int m = ctl->m, nk = ctl->nkeep;
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    const int i = t / m, j = t % m;
    S[(long long)i * lds + j] = (i == j && i < nk) ? theta_all[i] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl->m = nk;
    ctl->restart = 0;
  }
}

// t_j = (r_j - eps_j x_j) / (theta_j - d) with the denominator kept away from
// zero (eps_j = 0 without Olsen's correction); zero for roots already
// converged (no new direction)
__global__ void __launch_bounds__(kVecThreads) k_dav_precond(const double* __restrict__ R,
                                                             const double* __restrict__ X,
                                                             const double* __restrict__ diag,
                                                             const DavCtl* __restrict__ ctl, long long N,
                                                             double* __restrict__ T) {
  __shared__ double th[kMaxRoots], ep[kMaxRoots];
  __shared__ int on[kMaxRoots];
  const int k = ctl->k;
  if (threadIdx.x < k) {
    th[threadIdx.x] = ctl->theta[threadIdx.x];
    ep[threadIdx.x] = ctl->olsen ? ctl->eps[threadIdx.x] : 0.0;
    on[threadIdx.x] = ctl->rnorm[threadIdx.x] > 0.1 * ctl->tol;
  }
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride) {
    const double d = diag[e];
    for (int j = 0; j < k; ++j) {
      const double r = R[(long long)j * N + e] - (ep[j] != 0.0 ? ep[j] * X[(long long)j * N + e] : 0.0);
      T[(long long)j * N + e] = on[j] ? r / dav_den(th[j], d) : 0.0;
    }
  }
}

// norms of the corrections before projection (G = T^T T) and the directions
// that take part in this expansion
__global__ void k_dav_set_nrm0(DavCtl* __restrict__ ctl, const double* __restrict__ G) {
  const int k = ctl->k, j = threadIdx.x;
  if (j < k) {
    const double g = G[j * k + j];
    ctl->nrm0[j] = sqrt(fmax(g, 0.0));
    ctl->active[j] = g > 0.0 && isfinite(g);
  }
}

// T_j -= sum_{i<m} V_i C[i][j] for all j < k (k <= KC); nothing when gate points at 0
template <int KC>
__global__ void __launch_bounds__(kVecThreads) k_dav_project(const double* __restrict__ V,
                                                             const DavCtl* __restrict__ ctl,
                                                             const double* __restrict__ C, long long N,
                                                             double* __restrict__ T, const int* __restrict__ gate) {
  extern __shared__ float sCf[];  // [2][m][KC]
  if (gate && !*gate) return;
  const int m = ctl->m, k = ctl->k;
  float* sCh = sCf;
  float* sCl = sCf + m * KC;
  for (int t = threadIdx.x; t < m * KC; t += blockDim.x)
    df_split((t % KC < k) ? C[(t / KC) * k + t % KC] : 0.0, sCh[t], sCl[t]);
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride) {
    Df acc[KC];
#pragma unroll
    for (int j = 0; j < KC; ++j) acc[j] = Df{0.0f, 0.0f};
    for (int i = 0; i < m; ++i) {
      float vh, vl;
      df_split(V[(long long)i * N + e], vh, vl);
#pragma unroll
      for (int j = 0; j < KC; ++j) df_fma(acc[j], vh, vl, sCh[i * KC + j], sCl[i * KC + j]);
    }
#pragma unroll
    for (int j = 0; j < KC; ++j)
      if (j < k) T[(long long)j * N + e] -= df_value(acc[j]);
  }
}

// Second Gram-Schmidt pass only where the first removed more than 30% of a
// column's norm (the criterion of Daniel, Gragg, Kaufman and Stewart, Math.
// Comp. 30 (1976) 772); otherwise one pass already leaves the block orthogonal
// to the basis to working precision.
__global__ void k_dav_reorth(DavCtl* __restrict__ ctl, const double* __restrict__ G) {
  if (threadIdx.x != 0) return;
  const int k = ctl->k;
  int re = 0;
  for (int j = 0; j < k; ++j)
    if (ctl->active[j] && sqrt(fmax(G[j * k + j], 0.0)) < 0.7 * ctl->nrm0[j]) re = 1;
  ctl->reorth = re;
}

// Olsen's correction (Olsen, Jorgensen and Simons, Chem. Phys. Lett. 169
// (1990) 463): t_j = M_j^-1 (r_j - eps_j x_j) with M_j = diag(theta_j - H_ii)
// and eps_j = (x_j . M_j^-1 r_j) / (x_j . M_j^-1 x_j), so that t_j is
// orthogonal to x_j in the M_j metric.  partial[b][2j], [2j+1]: block b's
// parts of the two products.
__global__ void __launch_bounds__(kVecThreads) k_dav_olsen_dots(const double* __restrict__ R,
                                                                const double* __restrict__ X,
                                                                const double* __restrict__ diag,
                                                                const DavCtl* __restrict__ ctl, long long N,
                                                                double* __restrict__ partial) {
  __shared__ double red[kVecThreads / 32];
  if (!ctl->olsen) return;
  const int k = ctl->k;
  for (int j = 0; j < k; ++j) {
    const double th = ctl->theta[j];
    double a = 0.0, b = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride) {
      const double x = X[(long long)j * N + e], inv = 1.0 / dav_den(th, diag[e]);
      a = fma(x * inv, R[(long long)j * N + e], a);
      b = fma(x * inv, x, b);
    }
    a = block_sum(a, red);
    b = block_sum(b, red);
    if (threadIdx.x == 0) {
      partial[(long long)blockIdx.x * 2 * k + 2 * j] = a;
      partial[(long long)blockIdx.x * 2 * k + 2 * j + 1] = b;
    }
  }
}

// one warp per root (kMaxRoots warps)
__global__ void k_dav_olsen_eps(DavCtl* __restrict__ ctl, const double* __restrict__ partial, int parts) {
  const int k = ctl->k, j = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (j >= k) return;
  if (!ctl->olsen) {
    if (lane == 0) ctl->eps[j] = 0.0;
    return;
  }
  const double a = warp_sum_strided(partial + 2 * j, 2ll * k, parts, lane);
  const double b = warp_sum_strided(partial + 2 * j + 1, 2ll * k, parts, lane);
  if (lane == 0) ctl->eps[j] = (b != 0.0 && isfinite(a / b)) ? a / b : 0.0;
}

// Cholesky QR of the correction block from G = T^T T: upper R with R^T R = G
// over the active columns, Rinv = R^-1 (zero rows/columns for dropped ones).
// A column is dropped when its remaining norm is at most 1e-8 times its norm
// before projection (first pass) or times its current norm (second pass).
__global__ void k_dav_cholqr(DavCtl* __restrict__ ctl, const double* __restrict__ G, double* __restrict__ Rinv,
                             int first_pass) {
  __shared__ double Rm[kMaxRoots][kMaxRoots], Ri[kMaxRoots][kMaxRoots];
  if (threadIdx.x != 0) return;
  const int k = ctl->k;
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) Rm[i][j] = Ri[i][j] = 0.0;
  for (int j = 0; j < k; ++j) {
    if (!ctl->active[j]) continue;
    double d = G[j * k + j];
    for (int i = 0; i < j; ++i) d -= Rm[i][j] * Rm[i][j];
    const double ref = first_pass ? ctl->nrm0[j] : sqrt(fmax(G[j * k + j], 0.0));
    if (!(d > 0.0) || sqrt(d) <= 1e-8 * ref) {
      ctl->active[j] = 0;
      continue;
    }
    Rm[j][j] = sqrt(d);
    for (int l = j + 1; l < k; ++l) {
      if (!ctl->active[l]) continue;
      double x = G[j * k + l];
      for (int i = 0; i < j; ++i) x -= Rm[i][j] * Rm[i][l];
      Rm[j][l] = x / Rm[j][j];
    }
  }
  // inverse of the upper-triangular R on the active columns
  for (int j = 0; j < k; ++j) {
    if (!ctl->active[j]) continue;
    Ri[j][j] = 1.0 / Rm[j][j];
    for (int i = j - 1; i >= 0; --i) {
      if (!ctl->active[i]) continue;
      double x = 0.0;
      for (int l = i + 1; l <= j; ++l) x += Rm[i][l] * Ri[l][j];
      Ri[i][j] = -x / Rm[i][i];
    }
  }
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) Rinv[i * k + j] = Ri[i][j];
}

// T <- T Rinv (in place, all k <= KC columns per element)
template <int KC>
__global__ void __launch_bounds__(kVecThreads) k_dav_transform(double* __restrict__ T,
                                                               const double* __restrict__ Rinv,
                                                               const DavCtl* __restrict__ ctl, long long N) {
  __shared__ double sR[KC * KC];
  const int k = ctl->k;
  for (int t = threadIdx.x; t < KC * KC; t += blockDim.x) {
    const int i = t / KC, j = t % KC;
    sR[t] = (i < k && j < k) ? Rinv[i * k + j] : 0.0;
  }
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride) {
    double t[KC];
#pragma unroll
    for (int j = 0; j < KC; ++j) t[j] = j < k ? T[(long long)j * N + e] : 0.0;
#pragma unroll
    for (int j = 0; j < KC; ++j)
      if (j < k) {
        double x = 0.0;
#pragma unroll
        for (int i = 0; i <= j; ++i) x = fma(t[i], sR[i * KC + j], x);
        T[(long long)j * N + e] = x;
      }
  }
}

// the active columns of T and W_new join the basis at positions m, m+1, ...
__global__ void __launch_bounds__(kVecThreads) k_dav_append_vec(double* __restrict__ V, double* __restrict__ W,
                                                                const double* __restrict__ T,
                                                                const double* __restrict__ Wn,
                                                                const DavCtl* __restrict__ ctl, long long N) {
  __shared__ int slot[kMaxRoots];
  const int k = ctl->k, m = ctl->m;
  if (threadIdx.x == 0) {
    int s = 0;
    for (int j = 0; j < k; ++j) slot[j] = ctl->active[j] ? s++ : -1;
  }
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride)
    for (int j = 0; j < k; ++j)
      if (slot[j] >= 0) {
        V[(long long)(m + slot[j]) * N + e] = T[(long long)j * N + e];
        W[(long long)(m + slot[j]) * N + e] = Wn[(long long)j * N + e];
      }
}

// new rows/columns of S from C1 = V[0:m]^T W_new and C2 = T^T W_new; m grows
__global__ void k_dav_append_S(DavCtl* __restrict__ ctl, double* __restrict__ S, int lds,
                               const double* __restrict__ C1, const double* __restrict__ C2) {
  __shared__ int slot[kMaxRoots];
  __shared__ int added;
  const int k = ctl->k, m = ctl->m;
  if (threadIdx.x == 0) {
    int s = 0;
    for (int j = 0; j < k; ++j) slot[j] = ctl->active[j] ? s++ : -1;
    added = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < m * k; t += blockDim.x) {
    const int i = t / k, j = t % k;
    if (slot[j] < 0) continue;
    const int p = m + slot[j];
    S[(long long)i * lds + p] = S[(long long)p * lds + i] = C1[i * k + j];
  }
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    const int j = t / k, l = t % k;
    if (slot[j] < 0 || slot[l] < 0) continue;
    S[(long long)(m + slot[j]) * lds + (m + slot[l])] = 0.5 * (C2[j * k + l] + C2[l * k + j]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl->m = m + added;
    ctl->added = added;
    if (added == 0) ctl->status |= kStatusNoDirection;
  }
}

// S[0:cnt][0:cnt] from C = V[0:cnt]^T W[0:cnt] (symmetrised); the basis is
// those cnt vectors
__global__ void k_dav_init_S(DavCtl* __restrict__ ctl, double* __restrict__ S, int lds, const double* __restrict__ C,
                             int cnt) {
  for (int t = threadIdx.x; t < cnt * cnt; t += blockDim.x) {
    const int i = t / cnt, j = t % cnt;
    S[(long long)i * lds + j] = 0.5 * (C[i * cnt + j] + C[j * cnt + i]);
  }
  if (threadIdx.x == 0) {
    ctl->m = cnt;
    ctl->restart = 0;
  }
}

// request a restart to the lowest nkeep Ritz pairs (used when the precision changes)
__global__ void k_dav_request_restart(DavCtl* __restrict__ ctl, int nkeep) {
  if (threadIdx.x == 0) {
    ctl->restart = 1;
    ctl->nkeep = nkeep;
    ctl->status = 0;
  }
}

// Symmetric eigen-decomposition of S[0:m][0:m] by cyclic Jacobi rotations
// (Golub & Van Loan, "Matrix Computations", Sec. 8.5) in the parallel
// round-robin order of Brent and Luk: each round rotates m/2 disjoint (p, q)
// pairs at once.  A, Q are m x m work arrays (shared or global memory).
// Eigenvalues ascending into theta_all, eigenvector j into column j of Y;
// ctl->theta gets the lowest k.
__global__ void __launch_bounds__(256) k_dav_eigh(DavCtl* __restrict__ ctl, const double* __restrict__ S, int lds,
                                                  double* gA, double* gQ, double* __restrict__ Y, int ldy,
                                                  double* __restrict__ theta_all, int use_smem) {
  extern __shared__ double dyn[];
  __shared__ double cs[192], sn[192];
  __shared__ int pp[192], qq[192];
  __shared__ double red[8];
  __shared__ int stop;
  const int m = ctl->m;
  double* A = use_smem ? dyn : gA;
  double* Q = use_smem ? dyn + m * m : gQ;
  const int me = m + (m & 1);
  const int npair = me / 2;
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    const int i = t / m, j = t % m;
    A[t] = S[(long long)i * lds + j];
    Q[t] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 60 && m > 1; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const double x = A[t] * A[t];
      tot += x;
      if (t / m != t % m) off += x;
    }
    off = block_sum(off, red);
    tot = block_sum(tot, red);
    if (threadIdx.x == 0) stop = !(off > 1e-30 * tot) || off == 0.0;
    __syncthreads();
    if (stop) break;
    for (int r = 0; r < me - 1; ++r) {
      for (int i = threadIdx.x; i < npair; i += blockDim.x) {
        const int a = i == 0 ? 0 : ((i - 1 + r) % (me - 1)) + 1;
        const int b = ((me - 2 - i + r) % (me - 1)) + 1;
        const int p = min(a, b), q = max(a, b);
        double c = 1.0, s = 0.0;
        if (q < m) {
          const double apq = A[p * m + q];
          if (fabs(apq) >= 1e-300) {
            const double tau = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
            const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        pp[i] = p;
        qq[i] = q;
        cs[i] = c;
        sn[i] = s;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < npair * m; t += blockDim.x) {  // rows p, q
        const int i = t / m, col = t % m;
        const int p = pp[i], q = qq[i];
        if (q >= m || sn[i] == 0.0) continue;
        const double c = cs[i], s = sn[i];
        const double apk = A[p * m + col], aqk = A[q * m + col];
        A[p * m + col] = c * apk - s * aqk;
        A[q * m + col] = s * apk + c * aqk;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < npair * m; t += blockDim.x) {  // columns p, q and Q
        const int i = t / m, row = t % m;
        const int p = pp[i], q = qq[i];
        if (q >= m || sn[i] == 0.0) continue;
        const double c = cs[i], s = sn[i];
        const double akp = A[row * m + p], akq = A[row * m + q];
        A[row * m + p] = c * akp - s * akq;
        A[row * m + q] = s * akp + c * akq;
        const double ykp = Q[row * m + p], ykq = Q[row * m + q];
        Q[row * m + p] = c * ykp - s * ykq;
        Q[row * m + q] = s * ykp + c * ykq;
      }
      __syncthreads();
    }
  }
  // ascending order: rank of each eigenvalue (ties by index)
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double li = A[i * m + i];
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      const double lj = A[j * m + j];
      rank += (lj < li) || (lj == li && j < i);
    }
    theta_all[rank] = li;
    for (int row = 0; row < m; ++row) Y[(long long)row * ldy + rank] = Q[row * m + i];
  }
  __syncthreads();
  for (int j = threadIdx.x; j < ctl->k && j < m; j += blockDim.x) ctl->theta[j] = theta_all[j];
}

// residual norms, convergence and the restart decision
// (one warp per root for the residual norms: kMaxRoots warps)
__global__ void k_dav_check(DavCtl* __restrict__ ctl, const double* __restrict__ partial, int parts) {
  const int k = ctl->k, j = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (j < k) {
    const double x = warp_sum_strided(partial + j, k, parts, lane);
    if (lane == 0) ctl->rnorm[j] = sqrt(fmax(x, 0.0));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double rmax = 0.0, dmax = 0.0;
    bool finite = true;
    for (int i = 0; i < k; ++i) {
      if (i < ctl->kw) {
        rmax = fmax(rmax, ctl->rnorm[i]);
        dmax = fmax(dmax, fabs(ctl->theta[i] - ctl->theta_prev[i]));
      }
      if (!isfinite(ctl->theta[i]) || !isfinite(ctl->rnorm[i])) finite = false;
      ctl->theta_prev[i] = ctl->theta[i];
    }
    ctl->rmax = rmax;
    ctl->dmax = dmax;
    ctl->iter += 1;
    if (!finite) ctl->status |= kStatusNonFinite;
    if (finite && ctl->iter > 1 && rmax <= ctl->tol && dmax <= ctl->etol) ctl->status |= kStatusConverged;
    const int m = ctl->m;
    if (m + k > ctl->maxsub) {
      ctl->restart = 1;
      ctl->nkeep = max(k, min(m - k, ctl->maxsub / 2));
    }
  }
}

__global__ void k_unit_vectors(double* __restrict__ V, const long long* __restrict__ idx, int k, long long N) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride)
    for (int j = 0; j < k; ++j) V[(long long)j * N + e] = (e == idx[j]) ? 1.0 : 0.0;
}

// ---------------------------------------------------------------------------
// host side

namespace {

// column block of the lincomb kernels: k itself up to 8 (no work on absent
// columns), else 16 or 32
int kc_for(int k) { return k <= 8 ? std::max(k, 1) : k <= 16 ? 16 : 32; }

struct Dav {
  Context& ctx;
  long long N;
  int k, maxsub, kc, parts, rows_cap, eig_smem;
  cudaStream_t st;
  DevBuf ctl_d, S, Y, thetas, eigA, eigQ, partial, C1, C2, G, Rinv, rr_part;
  DevBuf rq;  // x_j . r_j and x_j . x_j of the returned vectors
  double *V = nullptr, *W = nullptr, *X = nullptr, *R = nullptr, *T = nullptr, *Wn = nullptr, *tmp = nullptr;
  DavCtl* ctl = nullptr;

  Dav(Context& c, int k_, int maxsub_) : ctx(c), N(c.ndet), k(k_), maxsub(maxsub_), st(stream()) {
    kc = kc_for(k);
    // blocks of the streaming kernels: 1 to 4 per SM, about 8 or more elements
    // per thread (fewer block partials to reduce on small spaces)
    const long long per_wave = 152ll * kVecThreads * 8;
    parts = 152 * (int)std::min<long long>(kVecBlocks / 152, std::max<long long>(1, (N + per_wave - 1) / per_wave));
    rows_cap = maxsub + k;
    const int eb = 2 * maxsub * maxsub * (int)sizeof(double);
    eig_smem = eb <= 160 * 1024 ? eb : 0;
  }

  int setup() {
    ISCSI_TRY(ctx.dv_V.grow(sizeof(double) * (size_t)maxsub * N));
    ISCSI_TRY(ctx.dv_W.grow(sizeof(double) * (size_t)maxsub * N));
    // X, R, T, W_new and the restart buffer
    const size_t nk = std::max(k, maxsub / 2);
    ISCSI_TRY(ctx.dv_tmp.grow(sizeof(double) * ((size_t)4 * k + nk) * N));
    V = ctx.dv_V.as<double>();
    W = ctx.dv_W.as<double>();
    X = ctx.dv_tmp.as<double>();
    R = X + (size_t)k * N;
    T = R + (size_t)k * N;
    Wn = T + (size_t)k * N;
    tmp = Wn + (size_t)k * N;
    ISCSI_TRY(ctl_d.alloc(sizeof(DavCtl)));
    ctl = ctl_d.as<DavCtl>();
    ISCSI_TRY(S.alloc(sizeof(double) * (size_t)maxsub * maxsub));
    ISCSI_TRY(Y.alloc(sizeof(double) * (size_t)maxsub * maxsub));
    ISCSI_TRY(thetas.alloc(sizeof(double) * maxsub));
    ISCSI_TRY(eigA.alloc(sizeof(double) * (size_t)maxsub * maxsub));
    ISCSI_TRY(eigQ.alloc(sizeof(double) * (size_t)maxsub * maxsub));
    ISCSI_TRY(partial.alloc(sizeof(double) * (size_t)parts * rows_cap * 2 * k));
    ISCSI_TRY(C1.alloc(sizeof(double) * (size_t)rows_cap * 2 * k));
    ISCSI_TRY(C2.alloc(sizeof(double) * (size_t)k * k));
    ISCSI_TRY(G.alloc(sizeof(double) * (size_t)k * k));
    ISCSI_TRY(Rinv.alloc(sizeof(double) * (size_t)k * k));
    ISCSI_TRY(rr_part.alloc(sizeof(double) * (size_t)parts * 2 * k));
    ISCSI_CUDA(cudaMemsetAsync(S.p, 0, sizeof(double) * (size_t)maxsub * maxsub, st));
    return attributes();
  }

  int attributes() {
    const int lim = 200 * 1024;
    if ((long long)sizeof(double) * maxsub * kc > lim) {
      set_error("iscsi_davidson: subspace too large for the shared-memory staging");
      return kErrArg;
    }
#define ISCSI_DAV_ATTR(KC)                                                                                 \
  ISCSI_CUDA(cudaFuncSetAttribute(k_dav_ritz<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));    \
  ISCSI_CUDA(cudaFuncSetAttribute(k_dav_project<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)); \
  ISCSI_CUDA(cudaFuncSetAttribute(k_dav_restart_lincomb<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    ISCSI_DAV_ATTR(4)
    ISCSI_DAV_ATTR(8)
    ISCSI_DAV_ATTR(16)
    ISCSI_DAV_ATTR(32)
#undef ISCSI_DAV_ATTR
    if (eig_smem) ISCSI_CUDA(cudaFuncSetAttribute(k_dav_eigh, cudaFuncAttributeMaxDynamicSharedMemorySize, eig_smem));
    return kOk;
  }

  template <int NB>
  void dots_t(const double* A, const int* na_dev, int na_add, const double* B, int nb, const int* gate) {
    const int tiles = ((rows_cap + kDotT - 1) / kDotT) * ((nb + NB - 1) / NB);
    k_tsdots<NB><<<dim3(parts, tiles), kVecThreads, 0, st>>>(A, na_dev, na_add, B, nb, N, partial.as<double>(),
                                                             rows_cap, gate); ISCSI_COUNT_LAUNCH();
  }
  // C[i][j] = A_i . B_j for i < (na_dev ? *na_dev : 0) + na_add, j < nb; when
  // gate is given, only if *gate != 0 at run time
  void dots(const double* A, const int* na_dev, int na_add, const double* B, int nb, double* C,
            const int* gate = nullptr) {
    switch (nb) {
      case 1: dots_t<1>(A, na_dev, na_add, B, nb, gate); break;
      case 2: dots_t<2>(A, na_dev, na_add, B, nb, gate); break;
      case 3: dots_t<3>(A, na_dev, na_add, B, nb, gate); break;
      case 4: dots_t<4>(A, na_dev, na_add, B, nb, gate); break;
      case 5: dots_t<5>(A, na_dev, na_add, B, nb, gate); break;
      case 6: dots_t<6>(A, na_dev, na_add, B, nb, gate); break;
      case 7: dots_t<7>(A, na_dev, na_add, B, nb, gate); break;
      default: dots_t<8>(A, na_dev, na_add, B, nb, gate); break;
    }
    k_tsreduce<<<(rows_cap * nb + 7) / 8, 256, 0, st>>>(partial.as<double>(), parts, na_dev, na_add, nb, rows_cap,
                                                            C, gate); ISCSI_COUNT_LAUNCH();
  }

  template <int KC>
  void ritz_t() {
    const size_t sm = sizeof(double) * (size_t)maxsub * KC;
    for (int j0 = 0; j0 < k; j0 += KC) {
      k_dav_ritz<KC><<<parts, kVecThreads, sm, st>>>(V, W, ctl, Y.as<double>(), maxsub, j0, N, X, R,
                                                     rr_part.as<double>()); ISCSI_COUNT_LAUNCH();
    }
  }
  template <int KC>
  void project_t(const double* C, const int* gate) {
    k_dav_project<KC><<<parts, kVecThreads, sizeof(double) * (size_t)maxsub * KC, st>>>(V, ctl, C, N, T, gate); ISCSI_COUNT_LAUNCH();
  }
  template <int KC>
  void transform_t() {
    k_dav_transform<KC><<<parts, kVecThreads, 0, st>>>(T, Rinv.as<double>(), ctl, N); ISCSI_COUNT_LAUNCH();
  }
  template <int KC>
  void restart_t() {
    const size_t sm = sizeof(double) * (size_t)maxsub * KC;
    const int nk = std::max(k, maxsub / 2);
    for (int pass = 0; pass < 2; ++pass) {
      double* src = pass == 0 ? V : W;
      for (int j0 = 0; j0 < nk; j0 += KC) {
        k_dav_restart_lincomb<KC><<<parts, kVecThreads, sm, st>>>(src, ctl, Y.as<double>(), maxsub, j0, N, tmp); ISCSI_COUNT_LAUNCH();
      }
      k_dav_restart_copy<<<parts, kVecThreads, 0, st>>>(src, tmp, ctl, N); ISCSI_COUNT_LAUNCH();
    }
    k_dav_restart_S<<<1, 256, 0, st>>>(ctl, S.as<double>(), maxsub, thetas.as<double>()); ISCSI_COUNT_LAUNCH();
  }
  void ritz() {
    switch (kc) {
      case 1: ritz_t<1>(); break;
      case 2: ritz_t<2>(); break;
      case 3: ritz_t<3>(); break;
      case 4: ritz_t<4>(); break;
      case 5: ritz_t<5>(); break;
      case 6: ritz_t<6>(); break;
      case 7: ritz_t<7>(); break;
      case 8: ritz_t<8>(); break;
      case 16: ritz_t<16>(); break;
      default: ritz_t<32>(); break;
    }
  }
  void transform() {
    switch (kc) {
      case 1: transform_t<1>(); break;
      case 2: transform_t<2>(); break;
      case 3: transform_t<3>(); break;
      case 4: transform_t<4>(); break;
      case 5: transform_t<5>(); break;
      case 6: transform_t<6>(); break;
      case 7: transform_t<7>(); break;
      case 8: transform_t<8>(); break;
      case 16: transform_t<16>(); break;
      default: transform_t<32>(); break;
    }
  }
  void restart() {
    switch (kc) {
      case 1: restart_t<1>(); break;
      case 2: restart_t<2>(); break;
      case 3: restart_t<3>(); break;
      case 4: restart_t<4>(); break;
      case 5: restart_t<5>(); break;
      case 6: restart_t<6>(); break;
      case 7: restart_t<7>(); break;
      case 8: restart_t<8>(); break;
      case 16: restart_t<16>(); break;
      default: restart_t<32>(); break;
    }
  }
  void project(const double* C, const int* gate = nullptr) {
    switch (kc) {
      case 1: project_t<1>(C, gate); break;
      case 2: project_t<2>(C, gate); break;
      case 3: project_t<3>(C, gate); break;
      case 4: project_t<4>(C, gate); break;
      case 5: project_t<5>(C, gate); break;
      case 6: project_t<6>(C, gate); break;
      case 7: project_t<7>(C, gate); break;
      case 8: project_t<8>(C, gate); break;
      case 16: project_t<16>(C, gate); break;
      default: project_t<32>(C, gate); break;
    }
  }

  // eigen-decomposition of S, Ritz vectors and residuals, convergence check
  int evaluate() {
    k_dav_eigh<<<1, 256, eig_smem, st>>>(ctl, S.as<double>(), maxsub, eigA.as<double>(), eigQ.as<double>(),
                                         Y.as<double>(), maxsub, thetas.as<double>(), eig_smem ? 1 : 0); ISCSI_COUNT_LAUNCH();
    ritz();
    k_dav_check<<<1, 32 * kMaxRoots, 0, st>>>(ctl, rr_part.as<double>(), parts); ISCSI_COUNT_LAUNCH();
    ISCSI_CUDA(cudaGetLastError());
    return kOk;
  }

  // orthonormalise the k columns of T against V[0:m] and among themselves
  int orthonormalise_block(bool set_norms) {
    if (set_norms) {
      dots(T, nullptr, k, T, k, G.as<double>());
      k_dav_set_nrm0<<<1, 32, 0, st>>>(ctl, G.as<double>()); ISCSI_COUNT_LAUNCH();
    }
    // Gram-Schmidt against the basis; the second pass runs only when needed
    dots(V, &ctl->m, 0, T, k, C1.as<double>());
    project(C1.as<double>());
    dots(T, nullptr, k, T, k, G.as<double>());
    k_dav_reorth<<<1, 32, 0, st>>>(ctl, G.as<double>()); ISCSI_COUNT_LAUNCH();
    dots(V, &ctl->m, 0, T, k, C1.as<double>(), &ctl->reorth);
    project(C1.as<double>(), &ctl->reorth);
    dots(T, nullptr, k, T, k, G.as<double>(), &ctl->reorth);
    // Cholesky QR within the block, twice
    for (int pass = 0; pass < 2; ++pass) {
      if (pass) dots(T, nullptr, k, T, k, G.as<double>());
      k_dav_cholqr<<<1, 32, 0, st>>>(ctl, G.as<double>(), Rinv.as<double>(), pass == 0 ? 1 : 0); ISCSI_COUNT_LAUNCH();
      transform();
    }
    ISCSI_CUDA(cudaGetLastError());
    return kOk;
  }

  // one iteration after an evaluation, in two halves around the sigma of the
  // new directions T -> W_new: expand the basis, evaluate again
  int pre_sigma() {
    // Olsen's epsilon from the Ritz vectors of the last evaluation (a restart
    // below replaces V, not X)
    k_dav_olsen_dots<<<parts, kVecThreads, 0, st>>>(R, X, ctx.diag.as<double>(), ctl, N, rr_part.as<double>()); ISCSI_COUNT_LAUNCH();
    k_dav_olsen_eps<<<1, 32 * kMaxRoots, 0, st>>>(ctl, rr_part.as<double>(), parts); ISCSI_COUNT_LAUNCH();
    restart();
    k_dav_precond<<<parts, kVecThreads, 0, st>>>(R, X, ctx.diag.as<double>(), ctl, N, T); ISCSI_COUNT_LAUNCH();
    return orthonormalise_block(true);
  }
  int post_sigma() {
    dots(V, &ctl->m, 0, Wn, k, C1.as<double>());
    dots(T, nullptr, k, Wn, k, C2.as<double>());
    k_dav_append_vec<<<parts, kVecThreads, 0, st>>>(V, W, T, Wn, ctl, N); ISCSI_COUNT_LAUNCH();
    k_dav_append_S<<<1, 256, 0, st>>>(ctl, S.as<double>(), maxsub, C1.as<double>(), C2.as<double>()); ISCSI_COUNT_LAUNCH();
    return evaluate();
  }

  // basis = the cnt orthonormal columns at V (cnt a multiple of k); W = H V in
  // sigma calls of k vectors each (the call shape the captured iteration
  // uses); S; evaluate
  int start_from_basis(int prec, int cnt) {
    for (int j0 = 0; j0 < cnt; j0 += k)
      ISCSI_TRY(sigma_run(ctx, V + (size_t)j0 * N, W + (size_t)j0 * N, k, prec));
    dots(V, nullptr, cnt, W, cnt, C1.as<double>());
    k_dav_init_S<<<1, 256, 0, st>>>(ctl, S.as<double>(), maxsub, C1.as<double>(), cnt); ISCSI_COUNT_LAUNCH();
    return evaluate();
  }

  // keep the lowest cnt Ritz vectors of the current basis and rebuild their
  // images with the given precision (the switch from FP32 to FP64 sigma)
  int collapse(int prec, int cnt) {
    k_dav_request_restart<<<1, 32, 0, st>>>(ctl, cnt); ISCSI_COUNT_LAUNCH();
    switch (kc) {
      case 1: restart_v<1>(); break;
      case 2: restart_v<2>(); break;
      case 3: restart_v<3>(); break;
      case 4: restart_v<4>(); break;
      case 5: restart_v<5>(); break;
      case 6: restart_v<6>(); break;
      case 7: restart_v<7>(); break;
      case 8: restart_v<8>(); break;
      case 16: restart_v<16>(); break;
      default: restart_v<32>(); break;
    }
    return start_from_basis(prec, cnt);
  }
  template <int KC>
  void restart_v() {
    const size_t sm = sizeof(double) * (size_t)maxsub * KC;
    for (int j0 = 0; j0 < 2 * k; j0 += KC) {
      k_dav_restart_lincomb<KC><<<parts, kVecThreads, sm, st>>>(V, ctl, Y.as<double>(), maxsub, j0, N, tmp); ISCSI_COUNT_LAUNCH();
    }
    k_dav_restart_copy<<<parts, kVecThreads, 0, st>>>(V, tmp, ctl, N); ISCSI_COUNT_LAUNCH();
  }

  int read_ctl(DavCtl& h) {
    ISCSI_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(DavCtl), cudaMemcpyDeviceToHost, st));
    ISCSI_CUDA(cudaStreamSynchronize(st));
    return kOk;
  }
};

// kernel nodes of a captured graph (counted per replay in the launch statistics)
long long graph_kernels(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return 0;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
  long long c = 0;
  for (size_t i = 0; i < n; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++c;
  }
  return c;
}

struct IterGraph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t x = nullptr;
  long long kernels = 0;
  IterGraph() = default;
  IterGraph(const IterGraph&) = delete;
  IterGraph& operator=(const IterGraph&) = delete;
  ~IterGraph() { reset(); }
  void reset() {
    if (x) cudaGraphExecDestroy(x);
    if (g) cudaGraphDestroy(g);
    x = nullptr;
    g = nullptr;
    kernels = 0;
  }
};

// basis capacity: max_subspace vectors per root when set, else 12 per root up
// to 96 (at least 4 per root): with many roots the FP64 subspace work (its
// eigen-decomposition grows as m^3, the vector products as m k) costs more
// than the extra iterations a smaller basis needs (16 roots: 96 vectors
// converge in 53 iterations against 43 with 192, 1.4x faster overall)
int subspace_size(long long N, int k) {
  const int per_root = options().max_subspace;
  const long long want = per_root > 0 ? (long long)std::max(2, per_root) * k
                                      : std::min<long long>(12ll * k, std::max<long long>(4ll * k, 96));
  int maxsub = (int)std::min<long long>(N, want);
  maxsub = std::min(maxsub, 384);
  if (maxsub < 2 * k && N > k) maxsub = (int)std::min<long long>(N, 2 * k);
  if (maxsub < k) maxsub = k;
  return maxsub;
}

// start vectors of one instance: the caller's (orthonormalised) or unit
// vectors on the k lowest diagonal entries
int start_vectors(Dav& d, DavCtl& h, const double* vecs) {
  Context& ctx = d.ctx;
  const long long N = d.N;
  const int k = d.k;
  cudaStream_t st = d.st;
  if (vecs && options().guess_from_vecs) {
    ISCSI_CUDA(cudaMemcpyAsync(d.T, vecs, sizeof(double) * k * N, cudaMemcpyDeviceToDevice, st));
    if (ctx.gas_nspace) ISCSI_TRY(gas_project(ctx, d.T, d.T, k, st));  // onto the GAS space
    ISCSI_TRY(d.orthonormalise_block(true));  // the basis is still empty (m = 0)
    ISCSI_TRY(d.read_ctl(h));
    for (int j = 0; j < k; ++j)
      if (!h.active[j]) {
        set_error("iscsi_davidson: start vectors are linearly dependent");
        return kErrArg;
      }
    ISCSI_CUDA(cudaMemcpyAsync(d.V, d.T, sizeof(double) * k * N, cudaMemcpyDeviceToDevice, st));
    return kOk;
  }
  std::vector<double> dg(N);
  ISCSI_CUDA(cudaMemcpyAsync(dg.data(), ctx.diag.p, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
  ISCSI_CUDA(cudaStreamSynchronize(st));
  // the candidates: every determinant, or the kept ones under a GAS restriction
  std::vector<long long> idx;
  idx.reserve(ctx.gas_ndet);
  for (long long i = 0; i < N; ++i)
    if (!ctx.gas_nspace || ctx.gas_mask_h[i]) idx.push_back(i);
  if ((long long)idx.size() < k) {
    set_error("iscsi_davidson: fewer determinants in the space than vectors in the block");
    return kErrArg;
  }
  std::partial_sort(idx.begin(), idx.begin() + k, idx.end(),
                    [&](long long a, long long b) { return dg[a] < dg[b] || (dg[a] == dg[b] && a < b); });
  idx.resize(k);
  DevBuf didx;
  ISCSI_TRY(didx.alloc(sizeof(long long) * k));
  ISCSI_CUDA(cudaMemcpyAsync(didx.p, idx.data(), sizeof(long long) * k, cudaMemcpyHostToDevice, st));
  k_unit_vectors<<<kVecBlocks, kVecThreads, 0, st>>>(d.V, didx.as<long long>(), k, N); ISCSI_COUNT_LAUNCH();
  ISCSI_CUDA(cudaGetLastError());
  ISCSI_CUDA(cudaStreamSynchronize(st));
  return kOk;
}

// the bounded waits of the merged contractions of a batch (synchronises)
int batch_wait_status(const std::unique_ptr<SigmaBatch> (&sb)[2]) {
  for (int g = 0; g < 2; ++g) {
    if (!sb[g] || !sb[g]->err.p) continue;
    ISCSI_TRY(tc_wait_status(sb[g]->err.as<int>(), "iscsi_davidson"));
  }
  return kOk;
}

}  // namespace

// Davidson for several independent contexts at once.  Every active instance
// keeps its own device-resident state; one iteration is: the pre-sigma half of
// every instance, one batched sigma per precision group (the contractions of
// all members merged, batch.cu), the post-sigma half of every instance.  That
// sequence is captured into one CUDA graph per set of active instances and
// replayed; instances leave the set when they converge (or fail), switch
// precision, or reach maxiter, and the graph is captured again.
static int davidson_batch_body(const std::vector<Context*>& ctxs, int kw, double tol, double* energies,
                               double* const* vecs, int* statuses) {
  const Options& opt = options();
  const int n = (int)ctxs.size();
  if (kw > kMaxRoots) {
    set_error("iscsi_davidson: at most 32 roots");
    return kErrArg;
  }
  // the block: the wanted roots and block_extra more (they widen the
  // expansion; convergence is judged on the wanted roots only)
  long long ndet_min = ctxs[0]->gas_ndet;
  for (const Context* c : ctxs) ndet_min = std::min(ndet_min, c->gas_ndet);
  // (the caller's start vectors fill a block of the wanted roots only)
  const int extra = vecs && opt.guess_from_vecs ? 0 : std::max(0, opt.block_extra);
  const int k = (int)std::min<long long>(std::min(kMaxRoots, kw + extra), ndet_min);
  cudaStream_t st = stream();
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  const bool mixed = (opt.precision == 32);
  std::vector<std::unique_ptr<Dav>> D(n);
  std::vector<DavCtl> H(n);
  std::vector<int> prec(n, mixed ? 32 : 64), status(n, kErrNoConv), active(n, 1), iters(n, 0), best_it(n, 0),
      fp32_iters(n, 0);
  std::vector<double> best_r(n, 1e300);
  std::vector<std::vector<double>> rhist(n);
  for (int i = 0; i < n; ++i) {
    D[i].reset(new Dav(*ctxs[i], k, subspace_size(ctxs[i]->gas_ndet, k)));  // basis <= dimension of the space
    ISCSI_TRY(D[i]->setup());
    DavCtl& h = H[i];
    std::memset(&h, 0, sizeof(h));
    h.k = k;
    h.kw = kw;
    h.maxsub = D[i]->maxsub;
    h.tol = tol;
    h.etol = opt.etol;
    h.olsen = opt.olsen ? 1 : 0;
    ISCSI_CUDA(cudaMemcpyAsync(D[i]->ctl, &h, sizeof(DavCtl), cudaMemcpyHostToDevice, st));
    ISCSI_TRY(start_vectors(*D[i], h, vecs ? vecs[i] : nullptr));
    ISCSI_TRY(D[i]->start_from_basis(prec[i], k));
  }

  IterGraph graph;
  std::unique_ptr<SigmaBatch> sb[2];  // [0]: FP64 members, [1]: FP32 members
  std::vector<int> members;
  bool changed = true, warm = false, graph_failed = false;
  // the halves of every instance run on concurrent pool streams
  StreamPool dpool;
  ISCSI_TRY(dpool.init(std::min(n, 16)));
  auto halves = [&](bool pre) -> int {
    ISCSI_TRY(dpool.fork(st));
    int rc2 = kOk;
    for (size_t j = 0; j < members.size() && rc2 == kOk; ++j) {
      Dav& d = *D[members[j]];
      d.st = dpool.at((int)j);
      rc2 = pre ? d.pre_sigma() : d.post_sigma();
      d.st = st;
    }
    ISCSI_TRY(rc2);
    return dpool.join(st);
  };
  auto sequence = [&]() -> int {
    ISCSI_TRY(halves(true));
    for (int g = 0; g < 2; ++g)
      if (sb[g] && !sb[g]->ctxs.empty()) ISCSI_TRY(sigma_batch_sequence(*sb[g]));
    return halves(false);
  };
  int rc = kOk;
  for (int it = 1; it <= opt.maxiter; ++it) {
    // the state of every active instance (one small copy each, one synchronisation)
    for (int i = 0; i < n; ++i)
      if (active[i]) ISCSI_CUDA(cudaMemcpyAsync(&H[i], D[i]->ctl, sizeof(DavCtl), cudaMemcpyDeviceToHost, st));
    ISCSI_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < n; ++i) {
      if (!active[i]) continue;
      const DavCtl& h = H[i];
      rhist[i].push_back(h.rmax);
      const bool fp32_phase = mixed && prec[i] == 32;
      if (h.status & kStatusNonFinite) {
        status[i] = kErrNan;
        active[i] = 0;
      } else if (!fp32_phase && (h.status & kStatusConverged)) {
        status[i] = kOk;
        active[i] = 0;
      } else if (!fp32_phase && (h.status & kStatusNoDirection)) {
        status[i] = h.rmax <= tol ? kOk : kErrNoConv;  // the subspace cannot grow
        active[i] = 0;
      } else if (fp32_phase) {
        // the FP32 phase ends at switch_tol, or when its residual stops
        // improving near the FP32 rounding floor (best residual within 1e3 of
        // switch_tol and not improved by 10% in 8 iterations; early plateaus
        // of the iteration itself do not count)
        if (h.rmax < 0.9 * best_r[i]) {
          best_r[i] = h.rmax;
          best_it[i] = iters[i];
        }
        const bool stalled = iters[i] - best_it[i] >= 8 && best_r[i] <= 1e3 * opt.switch_tol;
        if (h.rmax <= opt.switch_tol || stalled || (h.status & kStatusNoDirection)) {
          // keep the lowest Ritz vectors (2k when the basis holds them) and
          // recompute their images with the FP64 sigma
          prec[i] = 64;
          fp32_iters[i] = iters[i] + 1;
          ISCSI_TRY(D[i]->collapse(64, h.m >= 2 * k ? 2 * k : k));
          changed = true;
        }
      }
      if (!active[i]) changed = true;
    }
    // instances of the next iteration
    std::vector<int> next;
    for (int i = 0; i < n; ++i)
      if (active[i]) next.push_back(i);
    if (next.empty()) break;
    if (changed || next != members) {
      members = next;
      graph.reset();
      ISCSI_TRY(batch_wait_status(sb));
      for (int g = 0; g < 2; ++g) sb[g].reset(new SigmaBatch());
      for (int i : members) {
        SigmaBatch& b = *sb[prec[i] == 32 ? 1 : 0];
        b.ctxs.push_back(ctxs[i]);
        b.cs.push_back(D[i]->T);
        b.ss.push_back(D[i]->Wn);
        b.nvec = k;
        b.prec = prec[i];
      }
      changed = false;
      warm = false;  // the first pass of a new set runs directly (it builds the merged lists)
    }
    if (graph.x) {
      ISCSI_CUDA(cudaGraphLaunch(graph.x, st));
      g_launch_count += graph.kernels;
      for (int i : members) ctxs[i]->last_davidson_graph = 1;
    } else if (!warm || !opt.use_graph || graph_failed) {
      ISCSI_TRY(sequence());
      warm = true;
    } else {
      long long before = g_launch_count;
      for (int i : members) ctxs[i]->capturing = true;
      cudaError_t ce = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
      int crc = ce == cudaSuccess ? sequence() : kErrCuda;
      cudaGraph_t g = nullptr;
      cudaError_t ee = ce == cudaSuccess ? cudaStreamEndCapture(st, &g) : ce;
      for (int i : members) ctxs[i]->capturing = false;
      g_launch_count = before;
      if (ce == cudaSuccess && crc == kOk && ee == cudaSuccess && g &&
          cudaGraphInstantiate(&graph.x, g, 0) == cudaSuccess) {
        graph.g = g;
        graph.kernels = graph_kernels(g);
        ISCSI_CUDA(cudaGraphLaunch(graph.x, st));
        g_launch_count += graph.kernels;
        for (int i : members) ctxs[i]->last_davidson_graph = 1;
      } else {
        if (g) cudaGraphDestroy(g);
        graph_failed = true;
        cudaGetLastError();
        ISCSI_TRY(sequence());
      }
    }
    for (int i : members) ++iters[i];
  }
  ISCSI_TRY(batch_wait_status(sb));
  // results: the last evaluation of every instance.  The energies returned are
  // the Rayleigh quotients of the vectors returned, rho_j = theta_j + x_j.r_j /
  // x_j.x_j with r_j = W y_j - theta_j x_j the last residual: the Ritz values
  // of the projected matrix also carry the basis' small departure from
  // orthonormality (~2e-12 Eh at full CI n = 60)
  std::vector<std::vector<double>> rqh(n, std::vector<double>(2 * (size_t)kw * kw, 0.0));
  for (int i = 0; i < n; ++i) {
    Dav& d = *D[i];
    ISCSI_CUDA(cudaMemcpyAsync(&H[i], d.ctl, sizeof(DavCtl), cudaMemcpyDeviceToHost, st));
    ISCSI_TRY(d.rq.grow(sizeof(double) * 2 * (size_t)kw * kw));
    d.st = st;
    d.dots(d.X, nullptr, kw, d.R, kw, d.rq.as<double>());
    d.dots(d.X, nullptr, kw, d.X, kw, d.rq.as<double>() + (size_t)kw * kw);
    ISCSI_CUDA(cudaMemcpyAsync(rqh[i].data(), d.rq.p, sizeof(double) * 2 * (size_t)kw * kw, cudaMemcpyDeviceToHost,
                               st));
  }
  ISCSI_CUDA(cudaStreamSynchronize(st));
  for (int i = 0; i < n; ++i) {
    if (status[i] == kErrNoConv && prec[i] == 64 && (H[i].status & kStatusConverged)) status[i] = kOk;
    for (int j = 0; j < kw; ++j) {
      const double xr = rqh[i][(size_t)j * kw + j], xx = rqh[i][(size_t)kw * kw + (size_t)j * kw + j];
      const double rho = H[i].theta[j] + (xx > 0.0 ? xr / xx : 0.0);
      energies[(size_t)i * kw + j] = std::isfinite(rho) ? rho : H[i].theta[j];
    }
    if (vecs && vecs[i])
      ISCSI_CUDA(cudaMemcpyAsync(vecs[i], D[i]->X, sizeof(double) * kw * D[i]->N, cudaMemcpyDeviceToDevice, st));
    if (statuses) statuses[i] = status[i];
  }
  cudaEventRecord(e1, st);
  ISCSI_CUDA(cudaStreamSynchronize(st));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int i = 0; i < n; ++i) {
    Context& c = *ctxs[i];
    c.last_davidson_ms = ms;
    c.last_davidson_iters = H[i].iter;
    c.last_davidson_fp32_iters = mixed ? (prec[i] == 64 ? fp32_iters[i] : iters[i]) : 0;
    c.last_davidson_rhist = rhist[i];
  }
  for (int i = 0; i < n; ++i)
    if (status[i] != kOk) {
      rc = status[i];
      if (status[i] == kErrNoConv) set_error("iscsi_davidson: no convergence within maxiter");
      if (status[i] == kErrNan) set_error("iscsi_davidson: NaN or Inf in the subspace");
      break;
    }
  return rc;
}

// The iteration runs on a stream of its own (the legacy default stream, which
// callers often use, cannot be captured into a graph), ordered after the
// caller's stream on entry and before it on exit.
int davidson_batch_run(const std::vector<Context*>& ctxs, int nroots, double tol, double* energies,
                       double* const* vecs, int* statuses) {
  cudaStream_t user = stream();
  cudaStream_t ds = nullptr;
  cudaEvent_t ev = nullptr;
  ISCSI_CUDA(cudaStreamCreateWithFlags(&ds, cudaStreamNonBlocking));
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaStreamDestroy(ds);
    set_error("iscsi_davidson: cudaEventCreate failed");
    return kErrCuda;
  }
  for (Context* c : ctxs) c->last_davidson_graph = 0;
  cudaEventRecord(ev, user);
  cudaStreamWaitEvent(ds, ev, 0);
  set_stream(ds);
  int rc = davidson_batch_body(ctxs, nroots, tol, energies, vecs, statuses);
  cudaEventRecord(ev, ds);
  cudaStreamWaitEvent(user, ev, 0);
  set_stream(user);
  cudaStreamSynchronize(ds);
  cudaStreamDestroy(ds);
  cudaEventDestroy(ev);
  return rc;
}

int davidson_run(Context& ctx, int nroots, double tol, double* energies, double* vecs) {
  std::vector<Context*> one(1, &ctx);
  double* v[1] = {vecs};
  return davidson_batch_run(one, nroots, tol, energies, v, nullptr);
}

}  // namespace iscsi
