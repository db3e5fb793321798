// propagate.cu -- time propagation of a CI vector under H(t) = H_tau + f(t) V
// (Eq. ham with a time-dependent one-body part h(t) = h + f(t) v, the
// two-body part constant), by the short-iterative Lanczos propagator (the
// paper's SIAL, Sec. "Application"): for a step of length dt with the field
// held at its sample f_k,
//   q_0 = c / |c|,  Lanczos on H_k = H_tau + f_k V: m basis vectors q_j, the
//   tridiagonal T (alpha_j = <q_j|H_k q_j>, beta_j = |residual_j|),
//   c <- |c| Q exp(-i T dt) e_1        (real time; c complex)
//   c <- Q exp(-T dt) e_1 / |...|       (imaginary time; c real, normalised).
// Every sigma is the library's: the one-body term f_k V enters the context's
// string matrices for the step (M <- M_base + f_k M_v, with M_v those of a
// second context built with h1 = v and no two-electron integrals on the same
// space; restored at the end), so a Krylov vector costs one sigma of H_k; a
// complex vector is stored as [re; im] and its sigma is one call with nvec = 2.  The basis is kept orthogonal by two classical Gram-Schmidt passes
// against all earlier vectors (inner products by two-pass deterministic
// reductions).  The m x m eigenproblem of T runs on the host (Jacobi) after
// one synchronisation per step.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace iscsi {

constexpr int kPrThreads = 256;
constexpr int kPrBlocks = 152 * 4;  // partial sums per inner product, added in a fixed order

// partial inner products <q_k | w> (k < nk) of nc-component vectors (nc = 2:
// complex [re; im], the conjugate on q; nc = 1: real): part[(block * nk + k) * 2 + {re, im}]
__global__ void __launch_bounds__(kPrThreads) k_pr_dots(const double* __restrict__ Q, long long qstride, int nk,
                                                        const double* __restrict__ w, int nc, long long ndet,
                                                        double* __restrict__ part) {
  __shared__ double sre[kPrThreads / 32], sim[kPrThreads / 32];
  const long long per = (ndet + gridDim.x - 1) / gridDim.x;
  const long long i0 = blockIdx.x * per, i1 = min(ndet, i0 + per);
  for (int k = 0; k < nk; ++k) {
    const double* q = Q + k * qstride;
    double re = 0.0, im = 0.0;
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const double qr = q[i], wr = w[i];
      if (nc == 2) {
        const double qi = q[ndet + i], wi = w[ndet + i];
        re += qr * wr + qi * wi;
        im += qr * wi - qi * wr;
      } else {
        re += qr * wr;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if ((threadIdx.x & 31) == 0) {
      sre[threadIdx.x >> 5] = re;
      sim[threadIdx.x >> 5] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int j = 0; j < (int)(blockDim.x >> 5); ++j) {
        a += sre[j];
        b += sim[j];
      }
      part[((long long)blockIdx.x * nk + k) * 2] = a;
      part[((long long)blockIdx.x * nk + k) * 2 + 1] = b;
    }
    __syncthreads();
  }
}

// Control block of one propagation step (device memory).
struct PrCtl {
  double h[kPrMaxKrylov][2];   // coefficients of the current Gram-Schmidt pass
  double alpha[kPrMaxKrylov];  // diagonal of T
  double beta[kPrMaxKrylov];   // beta[j] = |residual after q_j|
  double beta0;                // |c|
  double y[kPrMaxKrylov][2];   // combination coefficients of the step's result
};

// sums the partial products, one warp per (k, re/im) with a fixed reduction
// order (lane l takes blocks l, l + 32, ..., then a shuffle tree);
// mode 0: h[k] = sum (a Gram-Schmidt pass; alpha[j] += Re h[j] with j = nk - 1);
// mode 1: beta[j] = sqrt(sum_re); mode 2: beta0 = sqrt(sum_re)
__global__ void k_pr_sum(const double* __restrict__ part, int parts, int nk, int mode, int j, PrCtl* __restrict__ ctl) {
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (t >= 2 * nk) return;
  const int k = t >> 1, c = t & 1;
  double s = 0.0;
  for (int b = lane; b < parts; b += 32) s += part[((long long)b * nk + k) * 2 + c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane != 0) return;
  if (mode == 0) {
    ctl->h[k][c] = s;
    if (k == nk - 1 && c == 0) ctl->alpha[j] += s;
  } else if (c == 0) {
    const double r = sqrt(fmax(s, 0.0));
    if (mode == 1) ctl->beta[j] = r;
    else ctl->beta0 = r;
  }
}

// w -= sum_k h[k] q_k  (complex coefficients for nc = 2)
__global__ void __launch_bounds__(kPrThreads) k_pr_update(const double* __restrict__ Q, long long qstride, int nk,
                                                          double* __restrict__ w, int nc, long long ndet,
                                                          const PrCtl* __restrict__ ctl) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ndet;
       i += (long long)gridDim.x * blockDim.x) {
    double wr = w[i], wi = nc == 2 ? w[ndet + i] : 0.0;
    for (int k = 0; k < nk; ++k) {
      const double hr = ctl->h[k][0], hi = ctl->h[k][1];
      const double qr = Q[k * qstride + i];
      if (nc == 2) {
        const double qi = Q[k * qstride + ndet + i];
        wr -= hr * qr - hi * qi;
        wi -= hr * qi + hi * qr;
      } else {
        wr -= hr * qr;
      }
    }
    w[i] = wr;
    if (nc == 2) w[ndet + i] = wi;
  }
}

// dst = src / s with s = beta0 (which = -1) or beta[which]; a vanishing s
// (an invariant subspace) gives dst = 0
__global__ void __launch_bounds__(kPrThreads) k_pr_scale(const double* __restrict__ src, double* __restrict__ dst,
                                                         long long count, const PrCtl* __restrict__ ctl, int which) {
  const double s = which < 0 ? ctl->beta0 : ctl->beta[which];
  const double ref = ctl->beta0 > 0.0 ? 1.0 : 0.0;
  const double inv = (s > 1e-300 && ref > 0.0) ? 1.0 / s : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i] * inv;
}

// c = sum_j y_j q_j  (complex y for nc = 2)
__global__ void __launch_bounds__(kPrThreads) k_pr_combine(const double* __restrict__ Q, long long qstride, int m,
                                                           double* __restrict__ c, int nc, long long ndet,
                                                           const PrCtl* __restrict__ ctl) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ndet;
       i += (long long)gridDim.x * blockDim.x) {
    double cr = 0.0, ci = 0.0;
    for (int j = 0; j < m; ++j) {
      const double yr = ctl->y[j][0], yi = ctl->y[j][1];
      const double qr = Q[j * qstride + i];
      if (nc == 2) {
        const double qi = Q[j * qstride + ndet + i];
        cr += yr * qr - yi * qi;
        ci += yr * qi + yi * qr;
      } else {
        cr += yr * qr;
      }
    }
    c[i] = cr;
    if (nc == 2) c[ndet + i] = ci;
  }
}

// Eigenpairs of a real symmetric m x m matrix (row-major, overwritten) by the
// cyclic Jacobi method: each rotation zeroes one off-diagonal pair, with
// tan(phi) = sgn(theta) / (|theta| + sqrt(theta^2 + 1)), theta = (a_qq - a_pp) / (2 a_pq);
// sweeps until the off-diagonal mass is negligible.  S holds the eigenvectors as columns.
static void jacobi_eigh(std::vector<double>& A, int m, std::vector<double>& w, std::vector<double>& S) {
  S.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) S[(size_t)i * m + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int p = 0; p < m; ++p)
      for (int q = 0; q < m; ++q) {
        tot += A[(size_t)p * m + q] * A[(size_t)p * m + q];
        if (p != q) off += A[(size_t)p * m + q] * A[(size_t)p * m + q];
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = A[(size_t)p * m + q];
        if (apq == 0.0) continue;
        const double theta = (A[(size_t)q * m + q] - A[(size_t)p * m + p]) / (2.0 * apq);
        const double t = std::fabs(theta) > 1e150 ? 0.5 / theta
                                                  : (theta >= 0 ? 1.0 : -1.0) /
                                                        (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < m; ++k) {  // columns p, q
          const double akp = A[(size_t)k * m + p], akq = A[(size_t)k * m + q];
          A[(size_t)k * m + p] = cs * akp - sn * akq;
          A[(size_t)k * m + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < m; ++k) {  // rows p, q
          const double apk = A[(size_t)p * m + k], aqk = A[(size_t)q * m + k];
          A[(size_t)p * m + k] = cs * apk - sn * aqk;
          A[(size_t)q * m + k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < m; ++k) {
          const double skp = S[(size_t)k * m + p], skq = S[(size_t)k * m + q];
          S[(size_t)k * m + p] = cs * skp - sn * skq;
          S[(size_t)k * m + q] = sn * skp + cs * skq;
        }
      }
  }
  w.resize(m);
  for (int i = 0; i < m; ++i) w[i] = A[(size_t)i * m + i];
}

static int pr_blocks(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 8)); }

static int propagate_steps(Context& ctx, Context* cpl, double* c, int nsteps, double dt, const double* field, int m,
                           int imaginary, double* diag) {
  cudaStream_t st = stream();
  const int nc = imaginary ? 1 : 2;
  const long long N = ctx.ndet, qs = (long long)nc * N;
  const int prec = options().precision;
  // workspace: basis [m + 1][nc][N], sigma [nc][N], partial sums, control
  const size_t need = sizeof(double) * ((size_t)(m + 1) * qs + (size_t)qs);
  if (ctx.pr_ws.bytes < need) ISCSI_TRY(ctx.pr_ws.grow(need));
  if (ctx.pr_part.bytes < sizeof(double) * 2 * kPrBlocks * (m + 1))
    ISCSI_TRY(ctx.pr_part.grow(sizeof(double) * 2 * kPrBlocks * (m + 1)));
  if (!ctx.pr_ctl.p) ISCSI_TRY(ctx.pr_ctl.alloc(sizeof(PrCtl)));
  double* Q = ctx.pr_ws.as<double>();
  double* W = Q + (size_t)(m + 1) * qs;
  double* part = ctx.pr_part.as<double>();
  PrCtl* ctl = ctx.pr_ctl.as<PrCtl>();
  const int gb = pr_blocks(N);
  PrCtl h;
  std::vector<double> T, w, S;
  for (int step = 0; step < nsteps; ++step) {
    const double f = field ? field[step] : 0.0;
    if (cpl) ISCSI_TRY(onebody_shift(ctx, *cpl, f));
    ISCSI_CUDA(cudaMemsetAsync(ctl, 0, sizeof(PrCtl), st));
    // q_0 = c / |c|
    k_pr_dots<<<kPrBlocks, kPrThreads, 0, st>>>(c, 0, 1, c, nc, N, part); ISCSI_COUNT_LAUNCH();
    k_pr_sum<<<1, 64, 0, st>>>(part, kPrBlocks, 1, 2, 0, ctl); ISCSI_COUNT_LAUNCH();
    k_pr_scale<<<pr_blocks(qs), kPrThreads, 0, st>>>(c, Q, qs, ctl, -1); ISCSI_COUNT_LAUNCH();
    for (int j = 0; j < m; ++j) {
      double* qj = Q + (size_t)j * qs;
      ISCSI_TRY(sigma_run(ctx, qj, W, nc, prec));
      for (int pass = 0; pass < 2; ++pass) {
        k_pr_dots<<<kPrBlocks, kPrThreads, 0, st>>>(Q, qs, j + 1, W, nc, N, part); ISCSI_COUNT_LAUNCH();
        k_pr_sum<<<(2 * (j + 1) + 7) / 8, 256, 0, st>>>(part, kPrBlocks, j + 1, 0, j, ctl); ISCSI_COUNT_LAUNCH();
        k_pr_update<<<gb, kPrThreads, 0, st>>>(Q, qs, j + 1, W, nc, N, ctl); ISCSI_COUNT_LAUNCH();
      }
      k_pr_dots<<<kPrBlocks, kPrThreads, 0, st>>>(W, 0, 1, W, nc, N, part); ISCSI_COUNT_LAUNCH();
      k_pr_sum<<<1, 64, 0, st>>>(part, kPrBlocks, 1, 1, j, ctl); ISCSI_COUNT_LAUNCH();
      if (j + 1 < m) {
        k_pr_scale<<<pr_blocks(qs), kPrThreads, 0, st>>>(W, Q + (size_t)(j + 1) * qs, qs, ctl, j); ISCSI_COUNT_LAUNCH();
      }
    }
    ISCSI_CUDA(cudaGetLastError());
    ISCSI_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(PrCtl), cudaMemcpyDeviceToHost, st));
    ISCSI_CUDA(cudaStreamSynchronize(st));
    if (!std::isfinite(h.beta0)) {
      set_error("iscsi_propagate: NaN or Inf in the vector");
      return kErrNan;
    }
    // the m x m problem: T = S diag(w) S^T; z = exp(-i T dt) e_1 or exp(-T dt) e_1
    // (an invariant subspace found early leaves zero rows and columns in T)
    int mm = m;
    for (int j = 0; j + 1 < m; ++j)
      if (!(h.beta[j] > 1e-300)) {
        mm = j + 1;
        break;
      }
    T.assign((size_t)mm * mm, 0.0);
    for (int j = 0; j < mm; ++j) {
      T[(size_t)j * mm + j] = h.alpha[j];
      if (j + 1 < mm) T[(size_t)j * mm + j + 1] = T[(size_t)(j + 1) * mm + j] = h.beta[j];
    }
    jacobi_eigh(T, mm, w, S);
    const double wmin = *std::min_element(w.begin(), w.end());
    std::vector<std::complex<double>> z(mm, 0.0);
    for (int l = 0; l < mm; ++l) {
      const std::complex<double> e = imaginary ? std::complex<double>(std::exp(-(w[l] - wmin) * dt), 0.0)
                                               : std::exp(std::complex<double>(0.0, -w[l] * dt));
      const double s0 = S[l];  // e_1^T column l
      for (int j = 0; j < mm; ++j) z[j] += S[(size_t)j * mm + l] * e * s0;
    }
    double scale = h.beta0;
    if (imaginary) {
      double nz = 0.0;
      for (int j = 0; j < mm; ++j) nz += std::norm(z[j]);
      scale = nz > 0.0 ? 1.0 / std::sqrt(nz) : 0.0;
    }
    PrCtl up = h;
    for (int j = 0; j < kPrMaxKrylov; ++j) up.y[j][0] = up.y[j][1] = 0.0;
    for (int j = 0; j < mm; ++j) {
      up.y[j][0] = scale * z[j].real();
      up.y[j][1] = scale * z[j].imag();
    }
    if (diag) {
      // error indicator of the step: |c| beta_m |e_m^T exp(.) e_1| (the
      // residual of the Krylov approximation), and <c|H_k|c> / <c|c>
      diag[2 * step] = mm == m ? h.beta0 * h.beta[m - 1] * std::abs(z[m - 1]) * (imaginary ? scale / h.beta0 : 1.0)
                               : 0.0;
      diag[2 * step + 1] = h.alpha[0];
    }
    ISCSI_CUDA(cudaMemcpyAsync(ctl, &up, sizeof(PrCtl), cudaMemcpyHostToDevice, st));
    k_pr_combine<<<gb, kPrThreads, 0, st>>>(Q, qs, mm, c, nc, N, ctl); ISCSI_COUNT_LAUNCH();
    ISCSI_CUDA(cudaGetLastError());
    ISCSI_CUDA(cudaStreamSynchronize(st));  // 'up' is read by the copy
  }
  return tc_check(ctx);
}

int propagate_run(Context& ctx, Context* cpl, double* c, int nsteps, double dt, const double* field, int m,
                  int imaginary, double* diag) {
  int s = propagate_steps(ctx, cpl, c, nsteps, dt, field, m, imaginary, diag);
  // the context's string matrices lose the step's one-body term, also after an error
  int r = cpl ? onebody_shift(ctx, *cpl, 0.0) : kOk;
  return s != kOk ? s : r;
}

}  // namespace iscsi
