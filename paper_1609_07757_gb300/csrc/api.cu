// api.cu -- the C ABI (include/iscsi.h): argument checks, contexts, options.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>

#include "../../include/iscsi.h"
#include "internal.cuh"

namespace iscsi {

static std::string g_error = "no error";
long long g_launch_count = 0;
static cudaStream_t g_stream = nullptr;
static Options g_options;
static std::map<int, std::unique_ptr<Context>> g_ctx;
static int g_current = 0;
static int g_next_handle = 1;

void set_error(const std::string& msg) { g_error = msg; }
const char* last_error() { return g_error.c_str(); }
Options& options() { return g_options; }
cudaStream_t stream() { return g_stream; }
void set_stream(cudaStream_t s) { g_stream = s; }

static Context* current() {
  auto it = g_ctx.find(g_current);
  return it == g_ctx.end() ? nullptr : it->second.get();
}

}  // namespace iscsi

using namespace iscsi;

#define NEED_CTX(ctxvar)                        \
  Context* ctxvar = current();                  \
  if (!ctxvar) {                                \
    set_error("no current context (iscsi_init)"); \
    return ISCSI_E_NOINIT;                      \
  }

extern "C" {

}  // extern "C"

// a new current context; ninner < 0: excitation levels, else levels count the
// electrons outside the first ninner orbitals.  gas: a GAS spec applied before
// the context is registered (nullptr: none)
struct GasSpec {
  int nspace;
  const int *sizes, *cmin, *cmax;
};

static iscsi_status init_context(int norb, int nalpha, int nbeta, int max_excitation, const double* h1,
                                 const double* eri, double tau, int ninner, const GasSpec* gas) {
  if (norb < 1 || norb > kMaxOrb || nalpha < 0 || nbeta < 0 || nalpha > norb || nbeta > norb ||
      nalpha > kMaxElec || nbeta > kMaxElec || max_excitation < 0 || !h1 || !(tau >= 0.0) || std::isinf(tau)) {
    set_error("iscsi_init: invalid argument (limits: 1<=norb<=256, 0<=n_sigma<=min(norb,16), "
              "max_excitation>=0, tau>=0 finite, h1 != NULL)");
    return ISCSI_E_ARG;
  }
  // the dense same-spin string Hamiltonians and the opposite-spin unit matrix must fit
  long long na_str = binom_ll(norb, nalpha), nb_str = binom_ll(norb, nbeta);
  if (na_str > (1ll << 26) || nb_str > (1ll << 26)) {
    set_error("iscsi_init: string space too large for the dense same-spin string Hamiltonian");
    return ISCSI_E_ARG;
  }
  auto ctx = std::make_unique<Context>();
  int s = context_build(*ctx, norb, nalpha, nbeta, max_excitation, h1, eri, tau, ninner);
  if (s == kOk && gas) {
    s = gas_set(*ctx, gas->nspace, gas->sizes, gas->cmin, gas->cmax);
    // the level truncation alone gives the GAS space: no projection needed
    if (s == kOk && ctx->gas_ndet == ctx->ndet) s = gas_set(*ctx, 0, nullptr, nullptr, nullptr);
  }
  if (s != kOk) {
    cudaGetLastError();
    return s;
  }
  int h = g_next_handle++;
  g_ctx[h] = std::move(ctx);
  g_current = h;
  return ISCSI_OK;
}

// determinants with at most kmax electrons (alpha + beta) outside the first e orbitals
static double split_dim(int n, int na, int nb, int e, int kmax) {
  auto cnt = [&](int ne, int l) { return (double)binom_ll(e, ne - l) * (double)binom_ll(n - e, l); };
  double tot = 0.0;
  for (int la = 0; la <= na; ++la)
    for (int lb = 0; lb <= nb && la + lb <= kmax; ++lb) tot += cnt(na, la) * cnt(nb, lb);
  return tot;
}

extern "C" {

iscsi_status iscsi_init(int norb, int nalpha, int nbeta, int max_excitation, const double* h1, const double* eri,
                        double tau) {
  return init_context(norb, nalpha, nbeta, max_excitation, h1, eri, tau, -1, nullptr);
}

iscsi_status iscsi_init_gas(int norb, int nalpha, int nbeta, int nspace, const int* sizes, const int* cmin,
                            const int* cmax, const double* h1, const double* eri, double tau) {
  const int N = nalpha + nbeta;
  if (norb < 1 || norb > kMaxOrb || nalpha < 0 || nbeta < 0 || nspace < 1 || nspace > kGasMaxSpaces || !sizes ||
      !cmin || !cmax) {
    set_error("iscsi_init_gas: invalid argument (1 to 8 subspaces with sizes and limits)");
    return ISCSI_E_ARG;
  }
  int edge = 0;
  for (int j = 0; j < nspace; ++j) {
    if (sizes[j] < 1 || cmin[j] < 0 || cmax[j] < cmin[j] || cmax[j] > N) {
      set_error("iscsi_init_gas: subspace sizes >= 1 and limits 0 <= cmin <= cmax <= electrons");
      return ISCSI_E_ARG;
    }
    edge += sizes[j];
  }
  if (edge != norb) {
    set_error("iscsi_init_gas: subspace sizes must add up to the orbital count");
    return ISCSI_E_ARG;
  }
  // the enclosing space: full CI, or the level truncation of one accumulated
  // lower limit (at least cmin[j] electrons in the first e_j orbitals), the
  // smallest of them
  int best_inner = -1, best_k = N;
  double best = split_dim(norb, nalpha, nbeta, 0, N);  // every string at level ne: full CI
  edge = 0;
  for (int j = 0; j + 1 < nspace; ++j) {
    edge += sizes[j];
    const int k = N - cmin[j];
    const double d = split_dim(norb, nalpha, nbeta, edge, k);
    if (d < best) {
      best = d;
      best_inner = edge;
      best_k = k;
    }
  }
  const GasSpec spec{nspace, sizes, cmin, cmax};
  return init_context(norb, nalpha, nbeta, best_k, h1, eri, tau, best_inner, &spec);
}

iscsi_status iscsi_sigma(const void* c, void* sigma, int nvec) {
  NEED_CTX(ctx);
  if (!c || !sigma || nvec < 1) {
    set_error("iscsi_sigma: NULL pointer or nvec < 1");
    return ISCSI_E_ARG;
  }
  const double* cin = static_cast<const double*>(c);
  if (ctx->gas_nspace) {  // sigma = P H P c: the projected input in a context buffer
    ISCSI_TRY(ctx->gas_in.grow(sizeof(double) * (size_t)ctx->ndet * nvec));
    ISCSI_TRY(gas_project(*ctx, cin, ctx->gas_in.as<double>(), nvec, stream()));
    cin = ctx->gas_in.as<double>();
  }
  return sigma_run(*ctx, cin, static_cast<double*>(sigma), nvec, options().precision);
}

iscsi_status iscsi_sigma_noalloc(const void* c, void* sigma) {
  NEED_CTX(ctx);
  if (!c || !sigma) {
    set_error("iscsi_sigma_noalloc: NULL pointer");
    return ISCSI_E_ARG;
  }
  if (ctx->gas_nspace) {
    set_error("iscsi_sigma_noalloc: not with a GAS restriction; use iscsi_sigma");
    return ISCSI_E_ARG;
  }
  return sigma_noalloc_run(*ctx, static_cast<const double*>(c), static_cast<double*>(sigma));
}

iscsi_status iscsi_sigma_host(const double* c, double* sigma, int nvec) {
  NEED_CTX(ctx);
  if (!c || !sigma || nvec < 1) {
    set_error("iscsi_sigma_host: NULL pointer or nvec < 1");
    return ISCSI_E_ARG;
  }
  cudaStream_t st = stream();
  size_t bytes = sizeof(double) * (size_t)ctx->ndet * nvec;
  // staging buffers kept by the context (no allocation on repeated calls)
  DevBuf& dc = ctx->host_io[0];
  DevBuf& ds = ctx->host_io[1];
  ISCSI_TRY(dc.grow(bytes));
  ISCSI_TRY(ds.grow(bytes));
  ISCSI_CUDA(cudaMemcpyAsync(dc.p, c, bytes, cudaMemcpyHostToDevice, st));
  if (ctx->gas_nspace) ISCSI_TRY(gas_project(*ctx, dc.as<double>(), dc.as<double>(), nvec, st));
  ISCSI_TRY(sigma_run(*ctx, dc.as<double>(), ds.as<double>(), nvec, options().precision));
  ISCSI_CUDA(cudaMemcpyAsync(sigma, ds.p, bytes, cudaMemcpyDeviceToHost, st));
  ISCSI_CUDA(cudaStreamSynchronize(st));
  return tc_check(*ctx);
}

iscsi_status iscsi_density(const void* bra, const void* ket, void* d1, void* d2) {
  NEED_CTX(ctx);
  if (!bra || (!d1 && !d2)) {
    set_error("iscsi_density: bra is NULL or both outputs are NULL");
    return ISCSI_E_ARG;
  }
  return density_run(*ctx, static_cast<const double*>(bra), static_cast<const double*>(ket),
                     static_cast<double*>(d1), static_cast<double*>(d2));
}

iscsi_status iscsi_density_host(const double* bra, const double* ket, double* d1, double* d2) {
  NEED_CTX(ctx);
  if (!bra || (!d1 && !d2)) {
    set_error("iscsi_density_host: bra is NULL or both outputs are NULL");
    return ISCSI_E_ARG;
  }
  cudaStream_t st = stream();
  const size_t vb = sizeof(double) * (size_t)ctx->ndet;
  const size_t n2 = (size_t)ctx->n * ctx->n, b1 = sizeof(double) * 2 * n2, b2 = sizeof(double) * 3 * n2 * n2;
  // staging buffers kept by the context (no allocation on repeated calls)
  DevBuf& db = ctx->host_io[0];
  DevBuf& dk = ctx->host_io[1];
  DevBuf& o1 = ctx->host_io[2];
  DevBuf& o2 = ctx->host_io[3];
  const bool has_ket = ket && ket != bra;
  ISCSI_TRY(db.grow(vb));
  ISCSI_CUDA(cudaMemcpyAsync(db.p, bra, vb, cudaMemcpyHostToDevice, st));
  if (has_ket) {
    ISCSI_TRY(dk.grow(vb));
    ISCSI_CUDA(cudaMemcpyAsync(dk.p, ket, vb, cudaMemcpyHostToDevice, st));
  }
  if (d1) ISCSI_TRY(o1.grow(b1));
  if (d2) ISCSI_TRY(o2.grow(b2));
  ISCSI_TRY(density_run(*ctx, db.as<double>(), has_ket ? dk.as<double>() : nullptr, d1 ? o1.as<double>() : nullptr,
                        d2 ? o2.as<double>() : nullptr));
  if (d1) ISCSI_CUDA(cudaMemcpyAsync(d1, o1.p, b1, cudaMemcpyDeviceToHost, st));
  if (d2) ISCSI_CUDA(cudaMemcpyAsync(d2, o2.p, b2, cudaMemcpyDeviceToHost, st));
  ISCSI_CUDA(cudaStreamSynchronize(st));
  return tc_check(*ctx);
}

iscsi_status iscsi_propagate(void* c, int nsteps, double dt, const double* field, int coupling, int krylov,
                             int imaginary, double* diag) {
  NEED_CTX(ctx);
  if (!c || nsteps < 1 || !std::isfinite(dt) || dt == 0.0 || krylov < 2 || krylov > kPrMaxKrylov ||
      (imaginary != 0 && imaginary != 1) || (imaginary && dt < 0.0)) {
    set_error("iscsi_propagate: invalid argument (c != NULL, nsteps >= 1, finite dt != 0 (> 0 in imaginary "
              "time), 2 <= krylov <= 64, imaginary 0 or 1)");
    return ISCSI_E_ARG;
  }
  Context* cpl = nullptr;
  if (coupling) {
    auto it = g_ctx.find(coupling);
    if (it == g_ctx.end() || it->second.get() == ctx) {
      set_error("iscsi_propagate: unknown coupling handle, or the current context itself");
      return ISCSI_E_ARG;
    }
    cpl = it->second.get();
    if (cpl->n != ctx->n || cpl->na != ctx->na || cpl->nb != ctx->nb || cpl->kmax != ctx->kmax ||
        cpl->ndet != ctx->ndet || cpl->sp[0].nocc != ctx->sp[0].nocc || cpl->sp[1].nocc != ctx->sp[1].nocc) {
      set_error("iscsi_propagate: the coupling context is on a different determinant space");
      return ISCSI_E_ARG;
    }
  }
  if (field && !cpl) {
    set_error("iscsi_propagate: a field needs a coupling context");
    return ISCSI_E_ARG;
  }
  if (!ctx->h1_symmetric || (cpl && !cpl->h1_symmetric)) {
    set_error("iscsi_propagate: a one-body part that is not symmetric (the propagator needs Hermitian operators)");
    return ISCSI_E_ARG;
  }
  if (field)
    for (int k = 0; k < nsteps; ++k)
      if (!std::isfinite(field[k])) {
        set_error("iscsi_propagate: non-finite field sample");
        return ISCSI_E_ARG;
      }
  // a GAS restriction: the start vector is projected onto the kept determinants
  if (ctx->gas_nspace)
    ISCSI_TRY(gas_project(*ctx, static_cast<double*>(c), static_cast<double*>(c), imaginary ? 1 : 2, stream()));
  return propagate_run(*ctx, cpl, static_cast<double*>(c), nsteps, dt, field, krylov, imaginary, diag);
}

iscsi_status iscsi_set_gas(int nspace, const int* sizes, const int* cmin, const int* cmax, long long* ndet_gas) {
  NEED_CTX(ctx);
  ISCSI_TRY(gas_set(*ctx, nspace, sizes, cmin, cmax));
  if (ndet_gas) *ndet_gas = ctx->gas_ndet;
  return ISCSI_OK;
}

iscsi_status iscsi_gas_mask(void* mask) {
  NEED_CTX(ctx);
  if (!mask) {
    set_error("iscsi_gas_mask: NULL pointer");
    return ISCSI_E_ARG;
  }
  cudaStream_t st = stream();
  if (ctx->gas_nspace)
    ISCSI_CUDA(cudaMemcpyAsync(mask, ctx->gas_mask.p, ctx->ndet, cudaMemcpyDeviceToDevice, st));
  else
    ISCSI_CUDA(cudaMemsetAsync(mask, 1, ctx->ndet, st));
  return ISCSI_OK;
}

iscsi_status iscsi_check_bounded_wait(long long polls) {
  NEED_CTX(ctx);
  if (polls < 1024 || polls > (1ll << 24)) {
    set_error("iscsi_check_bounded_wait: polls must lie in [1024, 2^24]");
    return ISCSI_E_ARG;
  }
  return tc_wait_selftest(*ctx, polls);
}

iscsi_status iscsi_check_schedule(int nprob, const int* M, const int* N, const int* nseg, const int* K,
                                  const int* nrows_b, int nsm, double* balance, int* counts) {
  if (nprob < 1 || nprob > 4096 || !M || !N || !nseg || !K || !nrows_b || nsm < 1 || nsm > 1024 || !balance ||
      !counts) {
    set_error("iscsi_check_schedule: invalid argument (1 <= nprob <= 4096, 1 <= nsm <= 1024, non-NULL arrays)");
    return ISCSI_E_ARG;
  }
  static const unsigned char tiled_marker = 0;  // marks segments as tiled (bulk-copy costs); never read
  const auto* tiled = reinterpret_cast<const __nv_bfloat16*>(&tiled_marker);
  std::vector<OzProblem> probs(nprob);
  std::vector<OzSeg> segs;
  long long tiles = 0;
  for (int p = 0; p < nprob; ++p) {
    if (M[p] < 1 || N[p] < 1 || nseg[p] < 1 || nseg[p] > 64 || M[p] > (1 << 24) || N[p] > (1 << 24)) {
      set_error("iscsi_check_schedule: problem sizes out of range (M, N in [1, 2^24], 1 <= nseg <= 64)");
      return ISCSI_E_ARG;
    }
    OzProblem& P = probs[p];
    std::memset(&P, 0, sizeof(P));
    P.M = M[p];
    P.N = N[p];
    P.ldt = N[p];
    P.seg_begin = (int)segs.size();
    P.seg_count = nseg[p];
    for (int g = 0; g < nseg[p]; ++g) {
      const int i = P.seg_begin + g;
      if (K[i] < 0 || K[i] % OZ_BK || K[i] > (1 << 24) || nrows_b[i] < 1 || nrows_b[i] > N[p]) {
        set_error("iscsi_check_schedule: segment out of range (K a multiple of 16 in [0, 2^24], 1 <= nrows_b <= N)");
        return ISCSI_E_ARG;
      }
      OzSeg S;
      std::memset(&S, 0, sizeof(S));
      S.K = K[i];
      S.nrows_b = nrows_b[i];
      S.a_tiled = tiled;
      S.b_tiled = tiled;
      segs.push_back(S);
    }
    tiles += (long long)((M[p] + OZ_BM - 1) / OZ_BM) * ((N[p] + OZ_BN - 1) / OZ_BN);
    if (tiles > (1 << 20)) {
      set_error("iscsi_check_schedule: more than 2^20 output tiles");
      return ISCSI_E_ARG;
    }
  }
  std::vector<OzSegHost> sh(segs.size());
  OzPlan plan;
  int errors = 0;
  const int s = oz_plan_check(probs, segs, sh, nsm, plan, errors);
  if (s != kOk) return s;
  *balance = plan.model_balance;
  counts[0] = plan.grid;
  counts[1] = (int)plan.items.size();
  counts[2] = (int)tiles;
  counts[3] = plan.counters;
  counts[4] = errors;
  return ISCSI_OK;
}

iscsi_status iscsi_davidson(int nroots, double tol, double* energies, void* vecs) {
  NEED_CTX(ctx);
  if (nroots < 1 || nroots > ctx->gas_ndet || !(tol > 0) || !energies) {
    set_error("iscsi_davidson: invalid argument (1 <= nroots <= determinants of the space, tol > 0, energies)");
    return ISCSI_E_ARG;
  }
  if (!ctx->h1_symmetric) {
    set_error("iscsi_davidson: the context's one-body part is not symmetric (not a Hamiltonian)");
    return ISCSI_E_ARG;
  }
  int s = davidson_run(*ctx, nroots, tol, energies, static_cast<double*>(vecs));
  int w = tc_check(*ctx);
  return s != ISCSI_OK ? s : w;
}

long long iscsi_ndet(void) {
  Context* ctx = current();
  return ctx ? ctx->ndet : -1;
}

long long iscsi_nstrings(int spin) {
  Context* ctx = current();
  if (!ctx || spin < 0 || spin > 1) return -1;
  return ctx->sp[spin].count;
}

iscsi_status iscsi_get_strings(int spin, int* orbitals, int* levels) {
  NEED_CTX(ctx);
  if (spin < 0 || spin > 1) {
    set_error("iscsi_get_strings: spin must be 0 or 1");
    return ISCSI_E_ARG;
  }
  const SpinSpace& S = ctx->sp[spin];
  cudaStream_t st = stream();
  if (orbitals && S.ne > 0) {
    std::vector<int16_t> o((size_t)S.count * S.ne);
    ISCSI_CUDA(cudaMemcpyAsync(o.data(), S.orbs.p, sizeof(int16_t) * o.size(), cudaMemcpyDeviceToHost, st));
    ISCSI_CUDA(cudaStreamSynchronize(st));
    for (size_t i = 0; i < o.size(); ++i) orbitals[i] = o[i];
  }
  if (levels) {
    std::vector<int8_t> l(S.count);
    ISCSI_CUDA(cudaMemcpyAsync(l.data(), S.level.p, S.count, cudaMemcpyDeviceToHost, st));
    ISCSI_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < S.count; ++i) levels[i] = l[i];
  }
  return ISCSI_OK;
}

long long iscsi_det_index(const int* alpha_orbitals, const int* beta_orbitals) {
  Context* ctx = current();
  if (!ctx) return ISCSI_E_NOINIT;
  // colex rank of each list, then the sorted position from the device map
  const int* lists[2] = {alpha_orbitals, beta_orbitals};
  int pos[2] = {0, 0}, lvl[2] = {0, 0};
  for (int s = 0; s < 2; ++s) {
    const SpinSpace& S = ctx->sp[s];
    long long rank = 0;
    for (int i = 0; i < S.ne; ++i) {
      int o = lists[s] ? lists[s][i] : -1;
      if (o < 0 || o >= ctx->n || (i > 0 && o <= lists[s][i - 1])) return -1;
      rank += binom_ll(o, i + 1);
      lvl[s] += (o >= S.nocc);
    }
    int p = 0;
    if (cudaMemcpy(&p, S.pos.as<int>() + rank, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    pos[s] = p;
  }
  if (lvl[0] + lvl[1] > ctx->kmax) return -1;
  return ctx->off_h[pos[0]] + pos[1];
}

iscsi_status iscsi_diagonal(void* diag) {
  NEED_CTX(ctx);
  if (!diag) {
    set_error("iscsi_diagonal: NULL pointer");
    return ISCSI_E_ARG;
  }
  ISCSI_CUDA(cudaMemcpyAsync(diag, ctx->diag.p, sizeof(double) * ctx->ndet, cudaMemcpyDeviceToDevice, stream()));
  return ISCSI_OK;
}

iscsi_status iscsi_set_stream(void* s) {
  set_stream(static_cast<cudaStream_t>(s));
  return ISCSI_OK;
}

iscsi_status iscsi_set_option(const char* key, double value) {
  if (!key || std::isnan(value)) {
    set_error("iscsi_set_option: NULL key or NaN value");
    return ISCSI_E_ARG;
  }
  Options& o = options();
  std::string k(key);
  auto bad = [&]() {
    set_error("iscsi_set_option: value out of range for " + k);
    return ISCSI_E_ARG;
  };
  if (k == "precision") {
    if (value != 32 && value != 64) return bad();
    o.precision = (int)value;
  } else if (k == "class_mask_lo") {
    if (value < 0 || value > 4294967295.0) return bad();
    o.class_mask = (o.class_mask & ~0xFFFFFFFFull) | (unsigned long long)value;
  } else if (k == "class_mask_hi") {
    if (value < 0 || value > 1023) return bad();
    o.class_mask = (o.class_mask & 0xFFFFFFFFull) | ((unsigned long long)value << 32);
  } else if (k == "maxiter") {
    if (value < 1 || value > 100000) return bad();
    o.maxiter = (int)value;
  } else if (k == "max_subspace") {
    if (value != 0 && (value < 2 || value > 64)) return bad();
    o.max_subspace = (int)value;
  } else if (k == "etol") {
    if (value <= 0) return bad();
    o.etol = value;
  } else if (k == "switch_tol") {
    if (value <= 0) return bad();
    o.switch_tol = value;
  } else if (k == "guess_from_vecs") {
    o.guess_from_vecs = value != 0;
  } else if (k == "use_graph") {
    o.use_graph = value != 0;
  } else if (k == "olsen") {
    o.olsen = value != 0;
  } else if (k == "block_extra") {
    if (value < 0 || value > 31) return bad();
    o.block_extra = (int)value;
  } else if (k == "fp64_tc") {
    o.fp64_tc = value != 0;
  } else if (k == "samespin_tc") {
    o.samespin_tc = value != 0;
  } else if (k == "fp32_tc") {
    o.fp32_tc = value != 0;
  } else if (k == "autotune") {
    o.autotune = value != 0;
  } else if (k == "phase_timing") {
    o.phase_timing = value != 0;
    Context* ctx = current();
    if (ctx) ctx->ntimed = 0;  // restart the per-call record
    g_launch_count = 0;
  } else {
    set_error("iscsi_set_option: unknown key " + k);
    return ISCSI_E_ARG;
  }
  return ISCSI_OK;
}

iscsi_status iscsi_stats(char* json, int len) {
  NEED_CTX(ctx);
  if (!json || len < 2) {
    set_error("iscsi_stats: buffer too small");
    return ISCSI_E_ARG;
  }
  // per-phase sigma times of the recorded calls
  double phase_ms[Context::kPhases] = {0, 0, 0, 0};
  int ncalls = ctx->ntimed;
  if (ncalls > 0) {
    ISCSI_CUDA(cudaStreamSynchronize(stream()));
    for (int c = 0; c < ncalls; ++c)
      for (int p = 0; p < Context::kPhases; ++p) {
        float ms = 0;
        cudaEvent_t a = ctx->tev[(size_t)c * (Context::kPhases + 1) + p];
        cudaEvent_t b = ctx->tev[(size_t)c * (Context::kPhases + 1) + p + 1];
        if (cudaEventElapsedTime(&ms, a, b) == cudaSuccess) phase_ms[p] += ms;
      }
  }
  double upd = ctx->updates_onebody + ctx->updates_samespin + ctx->updates_opposite;
  char buf[4096];
  std::snprintf(
      buf, sizeof(buf),
      "{\"norb\": %d, \"nalpha\": %d, \"nbeta\": %d, \"max_excitation\": %d, \"tau\": %.17g, \"ndet\": %lld, "
      "\"nstrings\": [%d, %d], \"units_total\": {\"onebody\": %lld, \"samespin\": %lld, \"opposite\": %lld}, "
      "\"units_kept_opposite\": %lld, \"unit_hits_onebody\": %lld, \"unit_hits_samespin\": %lld, "
      "\"updates\": {\"onebody\": %.17g, \"samespin\": %.17g, \"opposite\": %.17g, \"total\": %.17g}, "
      "\"init_ms\": %.6f, \"timed_calls\": %d, \"phase_ms\": {\"lift\": %.6f, \"opposite_gemm\": %.6f, "
      "\"fold\": %.6f, \"samespin_gemm\": %.6f}, \"davidson_iters\": %d, \"davidson_ms\": %.6f, "
      "\"opposite_gemm_flops\": %.17g, \"samespin_gemm_flops\": %.17g, \"opposite_tc_bf16_flops\": %.17g, "
      "\"fp64_tc\": %d, \"samespin_tc\": %d, \"fp32_tc\": %d, \"davidson_fp32_iters\": %d, "
      "\"davidson_graph\": %d, \"kernel_launches\": %lld}",
      ctx->n, ctx->na, ctx->nb, ctx->kmax, ctx->tau, ctx->ndet, ctx->sp[0].count, ctx->sp[1].count,
      ctx->units_onebody_total, ctx->units_samespin_total, ctx->units_opposite_total, ctx->units_opposite,
      ctx->units_onebody, ctx->units_samespin, ctx->updates_onebody, ctx->updates_samespin,
      ctx->updates_opposite, upd, ctx->init_ms, ncalls, phase_ms[0], phase_ms[1], phase_ms[2], phase_ms[3],
      ctx->last_davidson_iters, ctx->last_davidson_ms, ctx_gemm_flops(*ctx, 0), ctx_gemm_flops(*ctx, 1),
      ctx_gemm_flops(*ctx, 2), options().fp64_tc, options().samespin_tc, options().fp32_tc,
      ctx->last_davidson_fp32_iters, ctx->last_davidson_graph, g_launch_count);
  // largest residual norm per Davidson iteration of the last run (up to 400)
  std::string out(buf);
  out.pop_back();  // closing brace
  out += ", \"davidson_rmax\": [";
  const size_t nh = std::min<size_t>(ctx->last_davidson_rhist.size(), 400);
  for (size_t i = 0; i < nh; ++i) {
    char v[32];
    std::snprintf(v, sizeof(v), i ? ", %.3e" : "%.3e", ctx->last_davidson_rhist[i]);
    out += v;
  }
  out += "]";
  // whether the opposite- and same-spin tensor-core products run as one launch
  {
    char v[512];
    auto both = [&](int prec) {
      return ctx->have_ab && ab_on_tc(*ctx, prec) && (prec == 64 ? samespin_tc_active(*ctx) : samespin_tc32_active(*ctx));
    };
    std::snprintf(v, sizeof(v), ", \"samespin_tc_bf16_flops\": %.17g, \"both_tc_fp64\": %d, \"both_tc_fp32\": %d",
                  ctx_gemm_flops(*ctx, 3), both(64) ? 1 : 0, both(32) ? 1 : 0);
    out += v;
    // the schedule of the FP64 tensor-core launch sigma makes (the combined
    // list when both contractions run there): bf16 MMA flops it issues (live
    // slices of non-screened blocks only), its CTAs, work items, split tiles
    // and the cost model's balance
    {
      const OzJob& J = both(64) ? ctx->oz_both : ctx->oz_ab;
      const OzPlan& pl = J.plan;
      std::snprintf(v, sizeof(v),
                    ", \"tc_schedule_fp64\": {\"issued_bf16_flops\": %.17g, \"grid\": %d, \"items\": %d, "
                    "\"split_tiles\": %d, \"tiles\": %d, \"model_balance\": %.4f}",
                    pl.issued_products, pl.grid, (int)pl.items.size(), pl.counters, J.tiles, pl.model_balance);
      out += v;
    }
    // GAS restriction: subspaces (0: none) and kept determinants
    std::snprintf(v, sizeof(v), ", \"gas_subspaces\": %d, \"gas_ndet\": %lld, \"level_split\": [%d, %d]",
                  ctx->gas_nspace, ctx->gas_ndet, ctx->sp[0].nocc, ctx->sp[1].nocc);
    out += v;
    // the density matrices' contraction (after the first iscsi_density call with d2):
    // bf16 MMA flops and 2 M N K of one launch, ket = bra and general
    std::snprintf(v, sizeof(v),
                  ", \"density_bf16_flops\": [%.17g, %.17g], \"density_fp64_flops\": [%.17g, %.17g], "
                  "\"density_gemm_ms\": %.6g",
                  density_flops(*ctx, 1, 0), density_flops(*ctx, 0, 0), density_flops(*ctx, 1, 1),
                  density_flops(*ctx, 0, 1), density_gemm_ms(*ctx));
    out += v;
  }
  // the autotuner's routing per precision and its trials (ab_tc, ss_min or -1 =
  // none on the tensor cores, predicted ms, measured ms or -1 = pruned)
  for (int p = 0; p < 2; ++p) {
    const Context::Route& R = ctx->route[p];
    char v[192];
    std::snprintf(v, sizeof(v),
                  ", \"route_fp%d\": {\"ab_tc\": %d, \"ss_min\": %d, \"tuned_nvec\": %d, \"trials\": [",
                  p == 0 ? 64 : 32, R.ab_tc, R.ss_min >= (1 << 30) ? -1 : R.ss_min, R.tuned_nvec);
    out += v;
    for (size_t i = 0; i + 3 < R.trials.size(); i += 4) {
      std::snprintf(v, sizeof(v), "%s[%d, %d, %.4g, %.4g]", i ? ", " : "", (int)R.trials[i],
                    (int)R.trials[i + 1], R.trials[i + 2], R.trials[i + 3]);
      out += v;
    }
    out += "]}";
  }
  out += "}";
  std::strncpy(json, out.c_str(), len - 1);
  json[len - 1] = 0;
  if (out.size() >= (size_t)len) {
    set_error("iscsi_stats: buffer too small");
    return ISCSI_E_ARG;
  }
  return ISCSI_OK;
}

double iscsi_updates_per_sigma(void) {
  Context* ctx = current();
  if (!ctx) return -1;
  return ctx->updates_onebody + ctx->updates_samespin + ctx->updates_opposite;
}

const char* iscsi_last_error(void) { return last_error(); }

void iscsi_finalize(void) {
  batch_reset();
  g_ctx.clear();
  g_current = 0;
}

iscsi_status iscsi_batch_sigma(const int* handles, const void* const* cs, void* const* sigmas, int count, int nvec) {
  if (count < 1 || nvec < 1 || !handles || !cs || !sigmas) {
    set_error("iscsi_batch_sigma: invalid argument");
    return ISCSI_E_ARG;
  }
  std::vector<Context*> ctxs(count);
  std::vector<const double*> c(count);
  std::vector<double*> s(count);
  for (int i = 0; i < count; ++i) {
    auto it = g_ctx.find(handles[i]);
    if (it == g_ctx.end() || !cs[i] || !sigmas[i]) {
      set_error("iscsi_batch_sigma: unknown handle or NULL vector at position " + std::to_string(i));
      return ISCSI_E_ARG;
    }
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) {
        set_error("iscsi_batch_sigma: a context appears twice");
        return ISCSI_E_ARG;
      }
    if (it->second->gas_nspace) {
      set_error("iscsi_batch_sigma: the context at position " + std::to_string(i) +
                " has a GAS restriction; use iscsi_sigma");
      return ISCSI_E_ARG;
    }
    ctxs[i] = it->second.get();
    c[i] = static_cast<const double*>(cs[i]);
    s[i] = static_cast<double*>(sigmas[i]);
  }
  return batch_sigma(ctxs, c, s, nvec, options().precision == 32 ? 32 : 64);
}

iscsi_status iscsi_batch_check(void) { return batch_check(); }

iscsi_status iscsi_batch_davidson(const int* handles, int count, int nroots, double tol, double* energies,
                                  void* const* vecs, int* statuses) {
  if (count < 1 || !handles || nroots < 1 || !(tol > 0) || !energies) {
    set_error("iscsi_batch_davidson: invalid argument");
    return ISCSI_E_ARG;
  }
  std::vector<Context*> ctxs(count);
  for (int i = 0; i < count; ++i) {
    auto it = g_ctx.find(handles[i]);
    if (it == g_ctx.end() || nroots > it->second->gas_ndet) {
      set_error("iscsi_batch_davidson: unknown handle, or more roots than determinants, at position " +
                std::to_string(i));
      return ISCSI_E_ARG;
    }
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) {
        set_error("iscsi_batch_davidson: a context appears twice");
        return ISCSI_E_ARG;
      }
    if (!it->second->h1_symmetric) {
      set_error("iscsi_batch_davidson: the one-body part of the context at position " + std::to_string(i) +
                " is not symmetric (not a Hamiltonian)");
      return ISCSI_E_ARG;
    }
    ctxs[i] = it->second.get();
  }
  int s = davidson_batch_run(ctxs, nroots, tol, energies, reinterpret_cast<double* const*>(vecs), statuses);
  for (Context* c : ctxs) {
    int w = tc_check(*c);
    if (w != ISCSI_OK && s == ISCSI_OK) s = w;
  }
  return s;
}

int iscsi_ctx_current(void) { return current() ? g_current : 0; }

iscsi_status iscsi_ctx_use(int handle) {
  if (g_ctx.find(handle) == g_ctx.end()) {
    set_error("iscsi_ctx_use: unknown handle");
    return ISCSI_E_ARG;
  }
  g_current = handle;
  return ISCSI_OK;
}

iscsi_status iscsi_ctx_destroy(int handle) {
  auto it = g_ctx.find(handle);
  if (it == g_ctx.end()) {
    set_error("iscsi_ctx_destroy: unknown handle");
    return ISCSI_E_ARG;
  }
  batch_reset();  // a cached batch may refer to this context
  g_ctx.erase(it);
  if (g_current == handle) g_current = 0;
  return ISCSI_OK;
}

}  // extern "C"
