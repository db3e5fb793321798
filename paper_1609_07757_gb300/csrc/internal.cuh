// internal.cuh -- shared declarations of the ISCI sigma library (GB300, sm_103a).
//
// Data layout in HBM (one context):
//   strings      per spin: orbitals [count][ne] (int16), level [count] (int8),
//                colex rank -> sorted position [count] (int32)
//   addressing   off[A] (int64, [NA+1]), beta strings allowed per alpha level
//   hole strings per spin: the (ne-1)-electron strings X; lift[q][X] gives the
//                string X u {q} and the sign of a+_q on |X> (Eqs. four-last:
//                contraction and addition with their phases)
//   G            opposite-spin units g_pqrs, screened (zeros where |g| <= tau
//                or the class is masked), [M x K] with rows m = pi(p, r) and
//                columns k = pi(q, s), pairs sorted by excitation level
//   Msame        per spin, the dense string Hamiltonian of the surviving
//                one-body and same-spin units, [N_sigma x N_sigma]
//   Ct, T        per column level class c: lifted vector Ct_c [K_c x Ncol_c]
//                and product T_c = G[:M_c, :K_c] Ct_c
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "ozaki_types.cuh"

namespace iscsi {

constexpr int kMaxOrb = 256;
constexpr int kMaxElec = 16;
constexpr int kNumClasses = 42;
constexpr int kMaxLevels = kMaxElec + 1;

// status codes (mirror include/iscsi.h)
constexpr int kOk = 0, kErrArg = -1, kErrNoMem = -2, kErrCuda = -3, kErrNoConv = -4, kErrNoInit = -5,
              kErrNan = -6, kErrWait = -7;

void set_error(const std::string& msg);

// kernel launches of the sigma path since the last reset (iscsi_stats)
extern long long g_launch_count;
#define ISCSI_COUNT_LAUNCH() (++::iscsi::g_launch_count)
const char* last_error();

#define ISCSI_CUDA(...)                                                                         \
  do {                                                                                          \
    cudaError_t e_ = (__VA_ARGS__);                                                             \
    if (e_ != cudaSuccess) {                                                                    \
      ::iscsi::set_error(std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_));            \
      return e_ == cudaErrorMemoryAllocation ? ::iscsi::kErrNoMem : ::iscsi::kErrCuda;          \
    }                                                                                           \
  } while (0)

#define ISCSI_TRY(...)       \
  do {                       \
    int s_ = (__VA_ARGS__);  \
    if (s_ != 0) return s_;  \
  } while (0)

// A device buffer owned by a context.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  int alloc(size_t nbytes);
  int grow(size_t nbytes);  // keeps nothing
  void release();
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

struct SpinSpace {
  int ne = 0;
  int nocc = 0;        // a string's level counts its electrons at orbitals >= nocc (nocc = ne: the
                       // excitation level of Eq. ci_hierarchy; else a two-subspace GAS split)
  int count = 0;       // C(n, ne)
  int maxlevel = 0;
  std::vector<int> level_start;   // first sorted index of each level, size maxlevel+2
  DevBuf orbs, level, pos;        // int16 [count][ne], int8 [count], int32 [count]
  // hole strings
  int nhole = 0;                  // C(n, ne-1), 0 when ne == 0
  int hole_maxlevel = 0;
  std::vector<int> hole_level;    // host, [nhole]
  DevBuf lift;                    // int32 [n][nhole]: (pos << 1 | neg) or -1
  DevBuf dec;                     // int32 [count][ne]: (X << 9 | p << 1 | neg)
};

// Operand addresses of the grouped GEMM are either absolute (src 0: the value
// is a device pointer) or element offsets into the vectors of the call
// (src 1: into c, src 2: into sigma), so problem lists survive new vectors.
enum { kSrcAbs = 0, kSrcC = 1, kSrcSigma = 2 };

// One GEMM segment: C[M x N] (+)= A[M x K] * B[K x N]; B columns >= bcols read as 0.
template <typename T>
struct Segment {
  long long a, b;
  int asrc, bsrc;
  long long lda, ldb;
  int K, bcols;
};

template <typename T>
struct Problem {
  long long c;
  int csrc;
  long long ldc;
  int M, N;
  int seg_begin, seg_count;
  int tile_begin;   // first global tile of this problem
  int tiles_n;      // tiles along N
  int accumulate;   // 1: C += ..., 0: C = ...
};

template <typename T>
struct ProblemList {
  std::vector<Problem<T>> probs;
  std::vector<Segment<T>> segs;
  int total_tiles = 0;
  DevBuf d_probs, d_segs;
  // problems with at most kThinN columns run one warp per output row
  std::vector<Problem<T>> thin;
  DevBuf d_thin;
  int thin_rows = 0;
  // problems with at most kThinN rows run one thread per output column
  std::vector<Problem<T>> mthin;
  DevBuf d_mthin, d_part_off, d_part;
  int mthin_cols = 0;
  int mthin_chunks = 1;
  long long mthin_part_stride = 0;
};
constexpr int kThinN = 16;

// one bf16 slice array [OZ_S][rows][ld] as TMA sees it
struct SliceArray {
  const __nv_bfloat16* base;
  int ld;
  long long rows, slice;
};

// host copies of a segment's live-slice maps (OzSeg::a_live / b_live), read
// by the scheduler's cost model (null: every slice live)
struct OzSegHost {
  const int* a_live = nullptr;
  const int* b_live = nullptr;
};

// schedule of one persistent k_oz_gemm launch (oz_schedule.cu): work items in
// execution order, CTA b running [cta_start[b], cta_start[b + 1]); split-K
// workspace (slots blocks of 128 x 64 doubles) and its counters
struct OzPlan {
  std::vector<OzItem> items;
  std::vector<int> cta_start;
  int grid = 0;
  int slots = 0, counters = 0;
  double issued_products = 0;  // bf16 MMA flops the launch issues (live slices only)
  double model_cycles = 0;     // predicted cycles of the busiest CTA
  double model_balance = 1;    // average over busiest predicted CTA load
  DevBuf d_items, d_cta, d_ws, d_cnt;
};
// host only: plan for nsm SMs and count the plan's faults (tiles whose K steps
// are not covered exactly once in part order, misnumbered parts, workspace
// slots or counters used other than once, CTAs without work)
int oz_plan_check(const std::vector<OzProblem>& probs, const std::vector<OzSeg>& segs,
                  const std::vector<OzSegHost>& sh, int nsm, OzPlan& plan, int& errors);
int oz_plan_build(const std::vector<OzProblem>& probs, const std::vector<OzSeg>& segs,
                  const std::vector<OzSegHost>& sh, OzPlan& plan, cudaStream_t st);

// a tensor-core work list (problems + segments) kept on the device
struct OzJob {
  std::vector<OzProblem> probs;
  std::vector<OzSeg> segs;
  std::vector<OzMaps> maps;  // one per segment
  std::vector<OzSegHost> sh; // one per segment (FP64-accurate jobs)
  OzPlan plan;               // FP64-accurate jobs: the persistent launch's schedule
  DevBuf d_probs, d_segs, d_maps;
  int tiles = 0;
  int nvec = -1;
  const void* tbase = nullptr;
  long long version = 0;  // bumped at every rebuild (launches over several contexts re-merge)
  long long src_ver[2] = {-1, -1};  // a combined job: versions of the jobs it was built from
};

struct DensityPlan;     // density.cu

struct ColClass {       // column level class c = level(X) + level(Y)
  int level = 0;
  int ncol = 0;         // hole pairs in the class
  int mrows = 0;        // pairs pi with level <= kmax - c (rows of T_c)
  int krows = 0;        // same count for the K dimension
  size_t ct_off = 0;    // element offset of Ct_c / T_c in the workspace (per vector set)
};

struct Context {
  int n = 0, na = 0, nb = 0, kmax = 0;
  double tau = 0;
  unsigned long long class_mask = 0;
  SpinSpace sp[2];
  long long ndet = 0;
  std::vector<long long> off_h;           // host copy of off
  std::vector<long long> nb_allowed_lvl;  // beta strings allowed per alpha level
  DevBuf off, nballow;                    // int64 [NA+1], int32 [kMaxLevels]
  // opposite-spin part
  int npairs = 0;                         // n*n
  std::vector<int> pair_level_start;      // first pair of each level sum (0..2), size 4
  DevBuf pair_of, pair_index;             // int32 [npairs] -> p*n+r ; int32 [n*n] -> m
  DevBuf pair_split;                      // int32 [npairs] -> (p << 16) | r (no division in the lifts)
  std::vector<ColClass> cls;
  DevBuf hp_class, hp_local;              // int8 / int32 [nholeA * nholeB]
  DevBuf hp_inv;                          // int32 [total hole pairs] -> X * nholeB + Y, grouped by class
  std::vector<int> hp_class_start;        // start of each class in hp_inv
  DevBuf G64, G32;                        // [npairs x npairs]
  bool have_ab = false;
  // same-spin parts
  DevBuf M64[2], M32[2];                  // [count x count] per spin (beta aliases alpha when equal)
  DevBuf M64base[2];                      // M64 without a per-step one-body term (propagation)
  double m_shift = 0.0;                   // the factor f of that term now in M64
  bool beta_alias = false;
  bool h1_symmetric = true;  // h_pq == h_qp exactly (a Hermitian one-body part)
  DevBuf diag;                            // FP64 [ndet]
  // workspaces
  size_t ct_elems = 0;                    // elements of all Ct_c (= of all T_c) for one vector
  DevBuf ct, tt;                          // Ct and T for nvec_cap vectors (in the active precision)
  DevBuf c32, s32;                        // FP32 copies for the FP32 path
  int nvec_cap = 0;
  int ws_prec = 0;
  ProblemList<double> pl_ab64, pl_ss64;
  ProblemList<float> pl_ab32, pl_ss32;
  int pl_nvec64 = 0, pl_nvec32 = 0;
  // tensor-core FP64 contractions (sigma_tc.cu); the slice arrays are tiled
  // (ozaki_types.cuh) with live-slice maps per block (device and host)
  DevBuf oz_gs, oz_gexp, oz_bs, oz_bexp, oz_err;
  DevBuf oz_glive, oz_malive, oz_mblive;
  std::vector<int> oz_glive_h, oz_malive_h, oz_mblive_h;
  std::vector<int> oz_mabase;  // first tiled row of each alpha level block in M_alpha's slices
  int oz_mpad = 0, oz_kpad = 0;
  long long oz_bs_elems = 0;
  OzJob oz_ab, oz_ss, oz_both;  // oz_both: oz_ab and oz_ss as one problem list
  DevBuf oz_mas, oz_maexp, oz_mbs, oz_mbexp, oz_cs, oz_csexp;
  std::vector<int> oz_kbase;
  int oz_ma_rows = 0, oz_ma_ld = 0, oz_mb_rows = 0, oz_mb_ld = 0;
  int t3_ma_rows = 0;                 // rows of the FP32 form's M_alpha slices (TMA layout)
  DevBuf oz_marow, oz_macol;          // tiled row -> alpha string, column -> alpha string of M_alpha's slices
  long long oz_cs_elems = 0;
  bool oz_m_ready = false;
  // kernel routing per precision ([0] FP64, [1] FP32), chosen by the autotuner
  struct Route {
    int ab_tc = 1;           // opposite-spin contraction on the tensor cores (else FMA kernels)
    int ss_min = kThinN;     // same-spin level blocks with more rows and allowed beta strings
                             // than this run on the tensor cores (else FMA kernels)
    int tuned_nvec = 0;      // vector count the autotuner ran for (0: not yet)
    std::vector<double> trials;  // (ab_tc, ss_min, predicted ms, measured ms) per candidate
  } route[2];
  long long pl_route_key = -1, pl_route_key32 = -1;  // routing the grouped-GEMM lists were built for
  int pl_ss_tc = -1;  // same-spin routing the FP64 grouped-GEMM list was built for
  // FP32 form of the tensor-core contractions (three bf16 terms per element)
  OzJob t3_ab, t3_ss, t3_both;
  DevBuf t3_gs, t3_bs, t3_mas, t3_mbs, t3_cs;
  long long t3_bs_elems = 0, t3_cs_elems = 0;
  bool t3_m_ready = false;
  int pl_ss_tc32 = -1;  // same-spin routing the FP32 grouped-GEMM list was built for
  // statistics
  double updates_onebody = 0, updates_samespin = 0, updates_opposite = 0;
  long long units_onebody = 0, units_samespin = 0, units_opposite = 0;
  long long units_onebody_total = 0, units_samespin_total = 0, units_opposite_total = 0;
  double last_sigma_ms = 0, init_ms = 0;
  // per-phase timing of sigma calls (option "phase_timing"): events recorded on
  // the library stream around lift, opposite-spin GEMM, fold, same-spin GEMM
  static constexpr int kPhases = 4;
  static constexpr int kMaxTimed = 512;
  std::vector<cudaEvent_t> tev;  // [kMaxTimed][kPhases + 1]
  int ntimed = 0;
  int last_davidson_iters = 0;
  int last_davidson_fp32_iters = 0;  // iterations of the FP32 phase (mixed precision)
  std::vector<double> last_davidson_rhist;  // largest residual norm per iteration
  double last_davidson_ms = 0;
  // Davidson buffers
  DevBuf dv_V, dv_W, dv_tmp, dv_small;
  bool capturing = false;  // a CUDA graph capture of a Davidson iteration is in progress
  int last_davidson_graph = 0;  // 1: the last Davidson run replayed captured iterations
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // density matrices (density.cu): string tables, workspaces and work lists, built at first use
  DensityPlan* dm = nullptr;
  // time propagation (propagate.cu): Krylov basis and sigma buffers, partial sums, control block
  DevBuf pr_ws, pr_part, pr_ctl;
  // device staging of the host-buffer entry points (iscsi_sigma_host, iscsi_density_host)
  DevBuf host_io[4];
  // GAS restriction (gas.cu): 0 subspaces = none; which determinants are kept
  int gas_nspace = 0;
  long long gas_ndet = 0;
  DevBuf gas_mask;                  // uint8 [ndet], 1 = kept
  std::vector<uint8_t> gas_mask_h;  // host copy (start vectors of the Davidson method)
  DevBuf gas_in;                    // projected copy of a caller's vectors
  long long noalloc_gen = 0;        // distinct per build (iscsi_sigma_noalloc keeps its lists in its array)
  ~Context();
};

struct Options {
  int precision = 64;
  unsigned long long class_mask = (1ull << kNumClasses) - 1;
  int maxiter = 300;
  int max_subspace = 0;  // Davidson basis vectors per root; 0: automatic
  double etol = 1e-10;
  double switch_tol = 1e-6;  // mixed precision: FP32 sigma until every residual is below this
  int guess_from_vecs = 0;
  int use_graph = 1;
  int olsen = 1;        // Olsen's correction in the Davidson preconditioner
  int block_extra = 0;  // Davidson block: the wanted roots and this many more
  int phase_timing = 0;
  int fp64_tc = 1;      // FP64 opposite-spin contraction on the tensor cores (exact bf16 slices)
  int samespin_tc = 1;  // same for the same-spin blocks large enough for a 128 x 64 tile
  int fp32_tc = 1;      // FP32 form: contractions on the tensor cores (three bf16 terms, FP32 accumulation)
  int autotune = 1;     // time the routing candidates at the first sigma of each vector count
};

// gas.cu: GAS restriction (P H P, P the projector onto the kept determinants)
constexpr int kGasMaxSpaces = 8;
int gas_set(Context& ctx, int nspace, const int* sizes, const int* cmin, const int* cmax);
// dst = P src for nvec vectors (a copy when there is no restriction; src == dst allowed)
int gas_project(const Context& ctx, const double* src, double* dst, int nvec, cudaStream_t st);

Options& options();
cudaStream_t stream();
void set_stream(cudaStream_t s);

// setup.cu
// ninner < 0: levels are excitation levels (nocc = ne per spin); else every spin's level counts
// its electrons outside the first ninner orbitals
int context_build(Context& ctx, int n, int na, int nb, int kmax, const double* h1, const double* eri, double tau,
                  int ninner = -1);

// sigma.cu
// phases of one sigma step (a batch over several contexts runs each phase for
// all contexts, with the two contractions merged into one launch each)
enum { kPhPre = 1, kPhAbGemm = 2, kPhMid = 4, kPhSsGemm = 8, kPhPost = 16, kPhAll = 31 };
int sigma_run(Context& ctx, const double* c, double* sigma, int nvec, int precision, int phases = kPhAll);
int sigma_workspace(Context& ctx, int nvec, int precision);
// algorithmic flops per sigma per vector of the opposite-spin GEMM (which = 0)
// or of the same-spin GEMMs (which = 1): 2 x M x K x N summed over problems;
// which = 2: bf16 MMA flops of the tensor-core opposite-spin contraction
double ctx_gemm_flops(const Context& ctx, int which);

// sigma_tc.cu: tensor-core FP64 contractions
int opposite_tc_operands(Context& ctx, const double* c, double* ttw, int nvec);  // slices of Ct
int opposite_tc_gemm(Context& ctx);                                                // T = G Ct
bool samespin_block_on_tc(const Context& ctx, int a, int prec);
bool samespin_tc_active(const Context& ctx);
bool ab_on_tc(const Context& ctx, int prec);
int sigma_autotune(Context& ctx, const double* c, double* sigma, int nvec, int prec);
int samespin_tc_operands(Context& ctx, const double* c, double* sigma, int nvec);  // slices of C, job
int samespin_tc_gemm(Context& ctx, double* sigma);                                 // sigma += same-spin
int opposite_tc32_operands(Context& ctx, const float* c, float* ttw, int nvec);   // FP32 form
int opposite_tc32_gemm(Context& ctx);
bool samespin_tc32_active(const Context& ctx);
int samespin_tc32_operands(Context& ctx, const float* c, float* sigma, int nvec);
int samespin_tc32_gemm(Context& ctx, float* sigma);
int both_tc_gemm(Context& ctx, double* sigma);  // opposite- and same-spin contractions, one launch
int both_tc32_gemm(Context& ctx, float* sigma);
const OzJob* both_tc_job(Context& ctx, int prec);  // that combined job (built when needed), or nullptr
// one launch over a device problem list whose relative outputs use the base
// table tbases: the FP64-accurate kernel on plan's schedule (prec 64), else
// the FP32-form kernel over `tiles` tiles
int launch_tc_problems(const OzProblem* probs, int nprobs, const OzSeg* segs, const OzMaps* maps,
                       void* const* tbases, int tiles, const OzPlan* plan, int prec, int* err, cudaStream_t st);
int tc_check(Context& ctx);
int tc_wait_selftest(Context& ctx, long long polls);
int tc_wait_status(int* err, const char* what);
int samespin_matrices_changed(Context& ctx);  // re-cut the same-spin operand slices in place
// M <- M_base + f M_v (cpl: the context of v); f = 0 restores (sigma.cu)
int onebody_shift(Context& ctx, const Context& cpl, double f);
// jobs assembled elsewhere: append a segment (K from column 0 of both arrays),
// number the tiles and upload, launch k_oz_gemm
int oz_job_add_seg(OzJob& job, const SliceArray& A, int a_row0, const int* a_exp, const SliceArray& B, int b_row0,
                   const int* b_exp, int K, int nrows_b);
int oz_job_upload(OzJob& job, cudaStream_t st);
int oz_job_launch(Context& ctx, const OzJob& job, cudaStream_t st);

// density.cu: one- and two-body density matrices (Eqs. d1, d2)
int density_run(Context& ctx, const double* bra, const double* ket, double* d1, double* d2);
void density_release(Context& ctx);
// flops of one launch of the density contraction (sym: ket = bra); which 0:
// bf16 MMA flops, 1: 2 M N K of the computed regions; 0 before the first call
double density_flops(const Context& ctx, int sym, int which);
double density_gemm_ms(Context& ctx);  // duration of the last contraction launch (synchronises), 0 if none

// allocation-free single-vector FP64 sigma on a static device array (sigma.cu)
int sigma_noalloc_run(Context& ctx, const double* c, double* sigma);
size_t noalloc_bytes_needed(const Context& ctx);
size_t noalloc_scratch_bytes();

// propagate.cu: steps of the short-iterative Lanczos propagator of H_tau + f_k V
// (cpl: the context of V, or nullptr); c device [2][ndet] (real time) or
// [ndet] (imaginary time); diag: host [2 * nsteps] or nullptr
constexpr int kPrMaxKrylov = 64;
int propagate_run(Context& ctx, Context* cpl, double* c, int nsteps, double dt, const double* field, int m,
                  int imaginary, double* diag);

// davidson.cu
int davidson_run(Context& ctx, int nroots, double tol, double* energies, double* vecs);
int davidson_batch_run(const std::vector<Context*>& ctxs, int nroots, double tol, double* energies,
                       double* const* vecs, int* statuses);

// batch.cu
// Streams for the independent per-context work of a batch: fork() makes every
// pool stream wait for the main stream, join() makes the main stream wait for
// all of them.  Captured into a graph, the per-context chains become parallel
// branches that the GPU runs concurrently.
struct StreamPool {
  std::vector<cudaStream_t> s;
  std::vector<cudaEvent_t> done;
  cudaEvent_t start = nullptr;
  StreamPool() = default;
  StreamPool(const StreamPool&) = delete;
  StreamPool& operator=(const StreamPool&) = delete;
  ~StreamPool();
  int init(int n);
  int fork(cudaStream_t main);
  int join(cudaStream_t main);
  cudaStream_t at(int i) const { return s[i % s.size()]; }
};

// one problem list over the tensor-core jobs of several contexts
struct MergedJob {
  std::vector<OzProblem> probs;
  std::vector<OzSeg> segs;
  std::vector<OzMaps> maps;
  std::vector<OzSegHost> sh;
  OzPlan plan;  // FP64-accurate batches
  DevBuf d_probs, d_segs, d_maps, d_tbases;
  std::vector<const OzJob*> src;
  std::vector<long long> ver;
  std::vector<void*> tbases;
  int tiles = 0;
};
// sigma_i = H(ctxs[i]) cs[i] for several contexts, contractions merged
struct SigmaBatch {
  std::vector<Context*> ctxs;
  std::vector<const double*> cs;
  std::vector<double*> ss;
  int nvec = 0, prec = 0;
  MergedJob ab, sst;  // the opposite-spin (or combined) jobs; the same-spin-only jobs
  DevBuf err;
  StreamPool pool;
};
int sigma_batch_sequence(SigmaBatch& B);  // launches on stream(); capturable once warmed up
int batch_sigma(const std::vector<Context*>& ctxs, const std::vector<const double*>& cs,
                const std::vector<double*>& ss, int nvec, int prec);
int batch_check();
void batch_reset();
bool batch_graph_active();

// small helpers shared by the .cu files
long long binom_ll(int n, int k);
int launch_blocks(long long work, int threads);

}  // namespace iscsi
