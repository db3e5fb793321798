// davidson.cu -- lowest eigenpairs of H_tau (Eq. hcec) by a Davidson iteration
// around the sigma step (Eq. sigma).  The paper names Davidson as the usual
// optimisation step that follows sigma; its own runs used imaginary-time
// propagation instead (Sec. "Basis and calculation set up").
//
// Vectors (subspace basis V, images W = H V, Ritz vectors, residuals) live on
// the device in FP64.  Projections, Rayleigh-Ritz, residual norms and the
// Gram-Schmidt orthonormalisation are FP64.  With the mixed-precision option
// the sigma steps run in FP32 until every residual norm is below switch_tol;
// then the basis is collapsed to the current Ritz vectors, their images are
// recomputed with the FP64 sigma, and the iteration finishes in FP64, so the
// returned energies are Rayleigh quotients of the FP64 operator.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace iscsi {

constexpr int kDotTile = 8;
constexpr int kDotThreads = 256;

// partial[b][i*nw + j] = sum over this block's slice of V_i[e] * W_j[e]
__global__ void k_dots(const double* __restrict__ V, int nv, const double* __restrict__ W, int nw, long long N,
                       double* __restrict__ partial, int npair_tiles_j) {
  int ti = blockIdx.y / npair_tiles_j, tj = blockIdx.y % npair_tiles_j;
  int i0 = ti * kDotTile, j0 = tj * kDotTile;
  double acc[kDotTile][kDotTile];
#pragma unroll
  for (int a = 0; a < kDotTile; ++a)
#pragma unroll
    for (int b = 0; b < kDotTile; ++b) acc[a][b] = 0.0;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride) {
    double v[kDotTile], w[kDotTile];
#pragma unroll
    for (int a = 0; a < kDotTile; ++a) v[a] = (i0 + a < nv) ? V[(long long)(i0 + a) * N + e] : 0.0;
#pragma unroll
    for (int b = 0; b < kDotTile; ++b) w[b] = (j0 + b < nw) ? W[(long long)(j0 + b) * N + e] : 0.0;
#pragma unroll
    for (int a = 0; a < kDotTile; ++a)
#pragma unroll
      for (int b = 0; b < kDotTile; ++b) acc[a][b] = fma(v[a], w[b], acc[a][b]);
  }
  __shared__ double red[kDotThreads / 32][kDotTile * kDotTile];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < kDotTile; ++a)
#pragma unroll
    for (int b = 0; b < kDotTile; ++b) {
      double x = acc[a][b];
      for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) red[warp][a * kDotTile + b] = x;
    }
  __syncthreads();
  if (threadIdx.x < kDotTile * kDotTile) {
    double x = 0.0;
    for (int w_ = 0; w_ < kDotThreads / 32; ++w_) x += red[w_][threadIdx.x];
    int a = threadIdx.x / kDotTile, b = threadIdx.x % kDotTile;
    if (i0 + a < nv && j0 + b < nw) partial[(long long)blockIdx.x * nv * nw + (i0 + a) * nw + (j0 + b)] = x;
  }
}

__global__ void k_reduce_partials(const double* __restrict__ partial, int nparts, int count, double* __restrict__ out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  double x = 0.0;
  for (int p = 0; p < nparts; ++p) x += partial[(long long)p * count + t];
  out[t] = x;
}

// X_j = sum_i V_i Y[i][j] (j < k); if W != nullptr: R_j = sum_i W_i Y[i][j] - theta_j X_j
// Y is m x k row-major (ld = k).  k <= 32.
__global__ void k_ritz(const double* __restrict__ V, const double* __restrict__ W, int m, const double* __restrict__ Y,
                       int k, const double* __restrict__ theta, long long N, double* __restrict__ X,
                       double* __restrict__ R) {
  extern __shared__ double sY[];
  for (int t = threadIdx.x; t < m * k; t += blockDim.x) sY[t] = Y[t];
  __syncthreads();
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride) {
    double x[32], r[32];
    for (int j = 0; j < k; ++j) x[j] = r[j] = 0.0;
    for (int i = 0; i < m; ++i) {
      double v = V[(long long)i * N + e];
      double w = W ? W[(long long)i * N + e] : 0.0;
      for (int j = 0; j < k; ++j) {
        x[j] = fma(v, sY[i * k + j], x[j]);
        if (W) r[j] = fma(w, sY[i * k + j], r[j]);
      }
    }
    for (int j = 0; j < k; ++j) {
      X[(long long)j * N + e] = x[j];
      if (W) R[(long long)j * N + e] = r[j] - theta[j] * x[j];
    }
  }
}

// out_j = sum_i V_i Y[i][j0 + j] for j < cnt <= 32 (Y is m x ldy row-major)
__global__ void k_lincomb(const double* __restrict__ V, int m, const double* __restrict__ Y, int ldy, int j0, int cnt,
                          long long N, double* __restrict__ out) {
  extern __shared__ double sYc[];
  for (int t = threadIdx.x; t < m * cnt; t += blockDim.x) sYc[t] = Y[(t / cnt) * ldy + j0 + (t % cnt)];
  __syncthreads();
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride) {
    double acc[32];
    for (int j = 0; j < cnt; ++j) acc[j] = 0.0;
    for (int i = 0; i < m; ++i) {
      double v = V[(long long)i * N + e];
      for (int j = 0; j < cnt; ++j) acc[j] = fma(v, sYc[i * cnt + j], acc[j]);
    }
    for (int j = 0; j < cnt; ++j) out[(long long)j * N + e] = acc[j];
  }
}

// T_j -= sum_i V_i C[i][j] for j < k (C is m x k row-major), then nothing else
__global__ void k_project_out(const double* __restrict__ V, int m, const double* __restrict__ C, int k, long long N,
                              double* __restrict__ T) {
  extern __shared__ double sC[];
  for (int t = threadIdx.x; t < m * k; t += blockDim.x) sC[t] = C[t];
  __syncthreads();
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride) {
    double acc[32];
    for (int j = 0; j < k; ++j) acc[j] = 0.0;
    for (int i = 0; i < m; ++i) {
      double v = V[(long long)i * N + e];
      for (int j = 0; j < k; ++j) acc[j] = fma(v, sC[i * k + j], acc[j]);
    }
    for (int j = 0; j < k; ++j) T[(long long)j * N + e] -= acc[j];
  }
}

// t_j[e] = r_j[e] / (theta_j - d[e]), with the denominator kept away from zero
__global__ void k_precondition(const double* __restrict__ R, const double* __restrict__ diag,
                               const double* __restrict__ theta, int k, long long N, double* __restrict__ T) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride) {
    double d = diag[e];
    for (int j = 0; j < k; ++j) {
      double den = theta[j] - d;
      if (fabs(den) < 1e-8) den = den < 0 ? -1e-8 : 1e-8;
      T[(long long)j * N + e] = R[(long long)j * N + e] / den;
    }
  }
}

__global__ void k_scale_vecs(double* __restrict__ T, const double* __restrict__ f, int k, long long N) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride)
    for (int j = 0; j < k; ++j) T[(long long)j * N + e] *= f[j];
}

__global__ void k_unit_vectors(double* __restrict__ V, const long long* __restrict__ idx, int k, long long N) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride)
    for (int j = 0; j < k; ++j) V[(long long)j * N + e] = (e == idx[j]) ? 1.0 : 0.0;
}

// ---------------------------------------------------------------------------
// host side

// Symmetric eigen-decomposition by cyclic Jacobi rotations (Golub & Van Loan,
// "Matrix Computations", Sec. 8.5).  A (n x n, row-major) is overwritten; the
// eigenvalues come back ascending with eigenvector columns in Y (row-major).
static void jacobi_eigh(std::vector<double> A, int n, std::vector<double>& w, std::vector<double>& Y) {
  Y.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Y[(size_t)i * n + i] = 1.0;
  auto at = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double x = at(i, j) * at(i, j);
        tot += x;
        if (i != j) off += x;
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = at(p, q);
        if (std::fabs(apq) < 1e-300) continue;
        double app = at(p, p), aqq = at(q, q);
        double tau = (aqq - app) / (2.0 * apq);
        double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- J^T A J
          double akp = at(k, p), akq = at(k, q);
          at(k, p) = c * akp - s * akq;
          at(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = at(p, k), aqk = at(q, k);
          at(p, k) = c * apk - s * aqk;
          at(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double ykp = Y[(size_t)k * n + p], ykq = Y[(size_t)k * n + q];
          Y[(size_t)k * n + p] = c * ykp - s * ykq;
          Y[(size_t)k * n + q] = s * ykp + c * ykq;
        }
      }
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return at(a, a) < at(b, b); });
  w.resize(n);
  std::vector<double> Ys((size_t)n * n);
  for (int jj = 0; jj < n; ++jj) {
    w[jj] = at(order[jj], order[jj]);
    for (int i = 0; i < n; ++i) Ys[(size_t)i * n + jj] = Y[(size_t)i * n + order[jj]];
  }
  Y.swap(Ys);
}

struct DavWork {
  Context& ctx;
  long long N;
  cudaStream_t st;
  DevBuf partial, small_d, small_d2;
  int blocks;
  explicit DavWork(Context& c) : ctx(c), N(c.ndet), st(stream()) {
    blocks = (int)std::min<long long>(4 * 152, (N + kDotThreads - 1) / kDotThreads);
    if (blocks < 1) blocks = 1;
  }
  // host out[i*nw + j] = V_i . W_j
  int dots(const double* V, int nv, const double* W, int nw, std::vector<double>& out) {
    int tj = (nw + kDotTile - 1) / kDotTile, ti = (nv + kDotTile - 1) / kDotTile;
    int parts = std::min(blocks, 152);
    ISCSI_TRY(partial.grow(sizeof(double) * (size_t)parts * nv * nw));
    ISCSI_TRY(small_d.grow(sizeof(double) * (size_t)nv * nw));
    dim3 grid(parts, ti * tj);
    k_dots<<<grid, kDotThreads, 0, st>>>(V, nv, W, nw, N, partial.as<double>(), tj);
    k_reduce_partials<<<launch_blocks((long long)nv * nw, 128), 128, 0, st>>>(partial.as<double>(), parts, nv * nw,
                                                                             small_d.as<double>());
    ISCSI_CUDA(cudaGetLastError());
    out.resize((size_t)nv * nw);
    ISCSI_CUDA(cudaMemcpyAsync(out.data(), small_d.p, sizeof(double) * nv * nw, cudaMemcpyDeviceToHost, st));
    ISCSI_CUDA(cudaStreamSynchronize(st));
    return kOk;
  }
  int upload(const std::vector<double>& h, DevBuf& d) {
    ISCSI_TRY(d.grow(sizeof(double) * std::max<size_t>(1, h.size())));
    ISCSI_CUDA(cudaMemcpyAsync(d.p, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, st));
    return kOk;
  }
  // T_j -= V (V^T T_j), applied twice; T has k vectors
  int orthogonalise(const double* V, int m, double* T, int k) {
    if (m == 0) return kOk;
    for (int pass = 0; pass < 2; ++pass) {
      std::vector<double> C;
      ISCSI_TRY(dots(V, m, T, k, C));  // C[i*k + j] = V_i . T_j
      ISCSI_TRY(upload(C, small_d2));
      k_project_out<<<blocks, 256, sizeof(double) * m * k, st>>>(V, m, small_d2.as<double>(), k, N, T);
      ISCSI_CUDA(cudaGetLastError());
      ISCSI_CUDA(cudaStreamSynchronize(st));  // C must stay alive until the copy is consumed
    }
    return kOk;
  }
};

int davidson_run(Context& ctx, int nroots, double tol, double* energies, double* vecs) {
  const Options& opt = options();
  long long N = ctx.ndet;
  int k = nroots;
  int maxsub = (int)std::min<long long>(N, (long long)std::max(2, opt.max_subspace) * k);
  // the Ritz kernels stage the m x k coefficient block in 48 KB of shared memory
  maxsub = std::min(maxsub, 6144 / k);
  if (maxsub < 2 * k && N > k) maxsub = std::min<long long>(N, 2 * k);
  if (maxsub < k) maxsub = k;
  if (k > 32) {
    set_error("iscsi_davidson: at most 32 roots");
    return kErrArg;
  }
  DavWork dw(ctx);
  cudaStream_t st = dw.st;
  ISCSI_TRY(ctx.dv_V.grow(sizeof(double) * (size_t)maxsub * N));
  ISCSI_TRY(ctx.dv_W.grow(sizeof(double) * (size_t)maxsub * N));
  ISCSI_TRY(ctx.dv_tmp.grow(sizeof(double) * (size_t)2 * k * N));  // X and R
  DevBuf dT, dth, dY, dscale, dYall, restart;
  ISCSI_TRY(dT.alloc(sizeof(double) * (size_t)k * N));
  ISCSI_TRY(restart.alloc(sizeof(double) * (size_t)std::max(k, maxsub / 2) * N));
  double* V = ctx.dv_V.as<double>();
  double* W = ctx.dv_W.as<double>();
  double* X = ctx.dv_tmp.as<double>();
  double* R = X + (size_t)k * N;
  double* T = dT.as<double>();
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);

  // --- initial guesses
  if (vecs && opt.guess_from_vecs) {
    ISCSI_CUDA(cudaMemcpyAsync(V, vecs, sizeof(double) * k * N, cudaMemcpyDeviceToDevice, st));
  } else {
    std::vector<double> d(N);
    ISCSI_CUDA(cudaMemcpyAsync(d.data(), ctx.diag.p, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    ISCSI_CUDA(cudaStreamSynchronize(st));
    std::vector<long long> idx(N);
    for (long long i = 0; i < N; ++i) idx[i] = i;
    std::partial_sort(idx.begin(), idx.begin() + k, idx.end(),
                      [&](long long a, long long b) { return d[a] < d[b] || (d[a] == d[b] && a < b); });
    idx.resize(k);
    DevBuf didx;
    ISCSI_TRY(didx.alloc(sizeof(long long) * k));
    ISCSI_CUDA(cudaMemcpyAsync(didx.p, idx.data(), sizeof(long long) * k, cudaMemcpyHostToDevice, st));
    k_unit_vectors<<<dw.blocks, 256, 0, st>>>(V, didx.as<long long>(), k, N);
    ISCSI_CUDA(cudaGetLastError());
    ISCSI_CUDA(cudaStreamSynchronize(st));
  }
  // orthonormalise the start block (Gram-Schmidt, one vector at a time)
  auto normalise = [&](double* vv, int cnt, std::vector<double>& norms) -> int {
    std::vector<double> g;
    ISCSI_TRY(dw.dots(vv, cnt, vv, cnt, g));
    norms.resize(cnt);
    std::vector<double> f(cnt);
    for (int j = 0; j < cnt; ++j) {
      norms[j] = std::sqrt(std::max(0.0, g[(size_t)j * cnt + j]));
      f[j] = norms[j] > 0 ? 1.0 / norms[j] : 0.0;
    }
    ISCSI_TRY(dw.upload(f, dscale));
    k_scale_vecs<<<dw.blocks, 256, 0, st>>>(vv, dscale.as<double>(), cnt, N);
    ISCSI_CUDA(cudaGetLastError());
    ISCSI_CUDA(cudaStreamSynchronize(st));
    return kOk;
  };
  {
    std::vector<double> nrm;
    for (int j = 0; j < k; ++j) {
      ISCSI_TRY(dw.orthogonalise(V, j, V + (size_t)j * N, 1));
      ISCSI_TRY(normalise(V + (size_t)j * N, 1, nrm));
      if (nrm[0] < 1e-12) {
        set_error("iscsi_davidson: start vectors are linearly dependent");
        return kErrArg;
      }
    }
  }

  bool mixed = (opt.precision == 32);
  ctx.last_davidson_fp32_iters = 0;
  int prec = mixed ? 32 : 64;
  int m = k;
  ISCSI_TRY(sigma_run(ctx, V, W, k, prec));
  std::vector<double> S((size_t)maxsub * maxsub, 0.0);
  auto update_S = [&](int from, int to) -> int {
    // blk[i][j - from] = V_i . W_j for i < to, from <= j < to
    std::vector<double> blk;
    ISCSI_TRY(dw.dots(V, to, W + (size_t)from * N, to - from, blk));
    int w_ = to - from;
    for (int i = 0; i < from; ++i)
      for (int j = from; j < to; ++j) S[(size_t)i * maxsub + j] = S[(size_t)j * maxsub + i] = blk[(size_t)i * w_ + (j - from)];
    // inside the new block the two products V_i.W_j and V_j.W_i are averaged
    for (int i = from; i < to; ++i)
      for (int j = i; j < to; ++j) {
        double x = 0.5 * (blk[(size_t)i * w_ + (j - from)] + blk[(size_t)j * w_ + (i - from)]);
        S[(size_t)i * maxsub + j] = S[(size_t)j * maxsub + i] = x;
      }
    return kOk;
  };
  ISCSI_TRY(update_S(0, m));

  std::vector<double> theta_prev(k, 0.0), theta(k, 0.0), rnorm(k, 0.0);
  double best_r = 1e300;
  int best_it = 0;
  int status = kErrNoConv;
  int iter = 0;
  for (iter = 1; iter <= opt.maxiter; ++iter) {
    // Rayleigh-Ritz in the subspace
    std::vector<double> Sm((size_t)m * m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) Sm[(size_t)i * m + j] = S[(size_t)i * maxsub + j];
    std::vector<double> w, Y;
    jacobi_eigh(Sm, m, w, Y);
    std::vector<double> Yk((size_t)m * k);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < k; ++j) Yk[(size_t)i * k + j] = Y[(size_t)i * m + j];
    for (int j = 0; j < k; ++j) theta[j] = w[j];
    ISCSI_TRY(dw.upload(Yk, dY));
    ISCSI_TRY(dw.upload(theta, dth));
    k_ritz<<<dw.blocks, 256, sizeof(double) * m * k, st>>>(V, W, m, dY.as<double>(), k, dth.as<double>(), N, X, R);
    ISCSI_CUDA(cudaGetLastError());
    std::vector<double> rr;
    ISCSI_TRY(dw.dots(R, k, R, k, rr));
    double rmax = 0.0, dmax = 0.0;
    bool finite = true;
    for (int j = 0; j < k; ++j) {
      rnorm[j] = std::sqrt(std::max(0.0, rr[(size_t)j * k + j]));
      rmax = std::max(rmax, rnorm[j]);
      dmax = std::max(dmax, std::fabs(theta[j] - theta_prev[j]));
      if (!std::isfinite(theta[j]) || !std::isfinite(rnorm[j])) finite = false;
    }
    if (!finite) {
      set_error("iscsi_davidson: NaN or Inf in the subspace");
      status = kErrNan;
      break;
    }
    bool fp32_phase = mixed && prec == 32;
    // the FP32 phase ends at switch_tol or when its residual stops improving
    // (the FP32 rounding floor): best residual not improved by 10% in 8 iterations
    if (fp32_phase) {
      if (rmax < 0.9 * best_r) {
        best_r = rmax;
        best_it = iter;
      }
    }
    if (fp32_phase && (rmax <= opt.switch_tol || iter - best_it >= 8)) {
      // collapse to the Ritz vectors and recompute their images in FP64
      ISCSI_CUDA(cudaMemcpyAsync(V, X, sizeof(double) * k * N, cudaMemcpyDeviceToDevice, st));
      std::vector<double> nrm;
      for (int j = 0; j < k; ++j) {
        ISCSI_TRY(dw.orthogonalise(V, j, V + (size_t)j * N, 1));
        ISCSI_TRY(normalise(V + (size_t)j * N, 1, nrm));
      }
      prec = 64;
      ctx.last_davidson_fp32_iters = iter;
      m = k;
      ISCSI_TRY(sigma_run(ctx, V, W, k, prec));
      ISCSI_TRY(update_S(0, m));
      theta_prev = theta;
      continue;
    }
    if (!fp32_phase && iter > 1 && rmax <= tol && dmax <= opt.etol) {
      status = kOk;
      break;
    }
    theta_prev = theta;
    // thick restart when the basis is full: keep the lowest nkeep Ritz pairs
    if (m + k > maxsub) {
      int nkeep = std::max(k, std::min(m - k, maxsub / 2));
      std::vector<double> Yall((size_t)m * nkeep);
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < nkeep; ++j) Yall[(size_t)i * nkeep + j] = Y[(size_t)i * m + j];
      ISCSI_TRY(dw.upload(Yall, dYall));
      for (int pass = 0; pass < 2; ++pass) {
        double* src = pass == 0 ? V : W;
        for (int j0 = 0; j0 < nkeep; j0 += 32) {
          int cnt = std::min(32, nkeep - j0);
          k_lincomb<<<dw.blocks, 256, sizeof(double) * m * cnt, st>>>(src, m, dYall.as<double>(), nkeep, j0, cnt, N,
                                                                     restart.as<double>() + (size_t)j0 * N);
        }
        ISCSI_CUDA(cudaGetLastError());
        ISCSI_CUDA(cudaMemcpyAsync(src, restart.p, sizeof(double) * nkeep * N, cudaMemcpyDeviceToDevice, st));
      }
      std::fill(S.begin(), S.end(), 0.0);
      for (int j = 0; j < nkeep; ++j) S[(size_t)j * maxsub + j] = w[j];
      m = nkeep;
      ISCSI_CUDA(cudaStreamSynchronize(st));
    }
    // corrections from the unconverged residuals
    k_precondition<<<dw.blocks, 256, 0, st>>>(R, ctx.diag.as<double>(), dth.as<double>(), k, N, T);
    ISCSI_CUDA(cudaGetLastError());
    int added = 0;
    std::vector<double> nrm0, nrm;
    for (int j = 0; j < k; ++j) {
      if (rnorm[j] <= tol * 0.1) continue;  // converged root: no new direction
      double* tj = T + (size_t)j * N;
      double* dst = V + (size_t)(m + added) * N;
      ISCSI_CUDA(cudaMemcpyAsync(dst, tj, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
      ISCSI_TRY(normalise(dst, 1, nrm0));
      if (nrm0[0] == 0.0) continue;
      ISCSI_TRY(dw.orthogonalise(V, m + added, dst, 1));
      ISCSI_TRY(normalise(dst, 1, nrm));
      if (nrm[0] < 1e-8) continue;  // no new direction
      ++added;
    }
    if (added == 0) {
      // the subspace cannot grow: report what we have
      status = (rmax <= tol) ? kOk : kErrNoConv;
      break;
    }
    ISCSI_TRY(sigma_run(ctx, V + (size_t)m * N, W + (size_t)m * N, added, prec));
    ISCSI_TRY(update_S(m, m + added));
    m += added;
  }
  for (int j = 0; j < k; ++j) energies[j] = theta[j];
  if (vecs) ISCSI_CUDA(cudaMemcpyAsync(vecs, X, sizeof(double) * k * N, cudaMemcpyDeviceToDevice, st));
  cudaEventRecord(e1, st);
  ISCSI_CUDA(cudaStreamSynchronize(st));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx.last_davidson_ms = ms;
  ctx.last_davidson_iters = iter;
  if (status == kErrNoConv) set_error("iscsi_davidson: no convergence within maxiter");
  return status;
}

}  // namespace iscsi
