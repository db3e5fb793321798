// batch.cu -- the sigma step for many independent contexts at once (the
// batching form: many instances of uneven orbital counts in one pass).
//
// Each phase of the sigma step runs for every context in turn, except the two
// tensor-core contractions: the opposite-spin products of all contexts form
// one problem list and run as one k_oz_gemm (or k_tc32w_gemm) launch, and so do
// the same-spin level-block products.  Problems keep their per-context
// output addressing through a table of output bases (OzProblem::tb).  From the
// second call with the same contexts, vectors, vector count and precision,
// the whole sequence is replayed from one captured CUDA graph, so a batch of
// any size costs one launch on the host.
#include <algorithm>
#include <cstring>
#include <memory>
#include <vector>

#include "internal.cuh"

namespace iscsi {

namespace {

// one problem list over the given jobs; rebuilt only when a job changed
int merge_jobs(MergedJob& mj, const std::vector<const OzJob*>& jobs, const std::vector<void*>& tbases, int prec,
               cudaStream_t st) {
  bool same = mj.src == jobs && mj.tbases == tbases;
  for (size_t i = 0; same && i < jobs.size(); ++i) same = mj.ver[i] == jobs[i]->version;
  if (same) return kOk;
  mj.probs.clear();
  mj.segs.clear();
  mj.maps.clear();
  mj.sh.clear();
  mj.tiles = 0;
  for (size_t i = 0; i < jobs.size(); ++i) {
    const OzJob& J = *jobs[i];
    const int seg0 = (int)mj.segs.size();
    for (OzProblem P : J.probs) {
      P.seg_begin += seg0;
      P.tile_begin += mj.tiles;
      P.tb = (int)i;
      mj.probs.push_back(P);
    }
    mj.segs.insert(mj.segs.end(), J.segs.begin(), J.segs.end());
    mj.maps.insert(mj.maps.end(), J.maps.begin(), J.maps.end());
    mj.sh.insert(mj.sh.end(), J.sh.begin(), J.sh.end());
    mj.tiles += J.tiles;
  }
  ISCSI_TRY(mj.d_probs.grow(sizeof(OzProblem) * std::max<size_t>(1, mj.probs.size())));
  ISCSI_TRY(mj.d_segs.grow(sizeof(OzSeg) * std::max<size_t>(1, mj.segs.size())));
  ISCSI_TRY(mj.d_maps.grow(sizeof(OzMaps) * std::max<size_t>(1, mj.maps.size())));
  ISCSI_TRY(mj.d_tbases.grow(sizeof(void*) * std::max<size_t>(1, tbases.size())));
  if (!mj.probs.empty())
    ISCSI_CUDA(cudaMemcpyAsync(mj.d_probs.p, mj.probs.data(), sizeof(OzProblem) * mj.probs.size(),
                               cudaMemcpyHostToDevice, st));
  if (!mj.segs.empty())
    ISCSI_CUDA(cudaMemcpyAsync(mj.d_segs.p, mj.segs.data(), sizeof(OzSeg) * mj.segs.size(), cudaMemcpyHostToDevice,
                               st));
  if (!mj.maps.empty())
    ISCSI_CUDA(cudaMemcpyAsync(mj.d_maps.p, mj.maps.data(), sizeof(OzMaps) * mj.maps.size(), cudaMemcpyHostToDevice,
                               st));
  if (!tbases.empty())
    ISCSI_CUDA(cudaMemcpyAsync(mj.d_tbases.p, tbases.data(), sizeof(void*) * tbases.size(), cudaMemcpyHostToDevice,
                               st));
  ISCSI_CUDA(cudaStreamSynchronize(st));  // the host vectors may change after this call
  // the FP64-accurate kernel is persistent: all contexts' tiles share one schedule
  if (prec == 64) ISCSI_TRY(oz_plan_build(mj.probs, mj.segs, mj.sh, mj.plan, st));
  mj.src = jobs;
  mj.tbases = tbases;
  mj.ver.resize(jobs.size());
  for (size_t i = 0; i < jobs.size(); ++i) mj.ver[i] = jobs[i]->version;
  return kOk;
}

int launch_merged(const MergedJob& mj, int prec, int* err, cudaStream_t st) {
  if (mj.tiles == 0) return kOk;
  return launch_tc_problems(mj.d_probs.as<OzProblem>(), (int)mj.probs.size(), mj.d_segs.as<OzSeg>(),
                            mj.d_maps.as<OzMaps>(), mj.d_tbases.as<void*>(), mj.tiles, &mj.plan, prec, err, st);
}

struct BatchState {
  SigmaBatch sb;
  cudaStream_t bs = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t x = nullptr;
  long long kernels = 0;
  bool failed = false;
  int calls = 0;
  BatchState() = default;
  BatchState(const BatchState&) = delete;
  BatchState& operator=(const BatchState&) = delete;
  ~BatchState() {
    if (bs) cudaStreamSynchronize(bs);
    if (x) cudaGraphExecDestroy(x);
    if (g) cudaGraphDestroy(g);
    if (ev) cudaEventDestroy(ev);
    if (bs) cudaStreamDestroy(bs);
  }
};

std::unique_ptr<BatchState> g_batch;

}  // namespace

StreamPool::~StreamPool() {
  for (cudaEvent_t e : done) cudaEventDestroy(e);
  if (start) cudaEventDestroy(start);
  for (cudaStream_t x : s) {
    cudaStreamSynchronize(x);
    cudaStreamDestroy(x);
  }
}

int StreamPool::init(int n) {
  if ((int)s.size() >= n) return kOk;
  if (!start) ISCSI_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  while ((int)s.size() < n) {
    cudaStream_t x;
    cudaEvent_t e;
    ISCSI_CUDA(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
    ISCSI_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    s.push_back(x);
    done.push_back(e);
  }
  return kOk;
}

int StreamPool::fork(cudaStream_t main) {
  ISCSI_CUDA(cudaEventRecord(start, main));
  for (cudaStream_t x : s) ISCSI_CUDA(cudaStreamWaitEvent(x, start, 0));
  return kOk;
}

int StreamPool::join(cudaStream_t main) {
  for (size_t i = 0; i < s.size(); ++i) {
    ISCSI_CUDA(cudaEventRecord(done[i], s[i]));
    ISCSI_CUDA(cudaStreamWaitEvent(main, done[i], 0));
  }
  return kOk;
}

namespace {

// both contractions of the context on the tensor cores (one combined list)
bool both_tc(const Context& c, int prec) {
  return c.have_ab && ab_on_tc(c, prec) && (prec == 64 ? samespin_tc_active(c) : samespin_tc32_active(c));
}

// one phase of every context, each on a pool stream (concurrent chains);
// skip_tc: only the contexts whose opposite-spin contraction is not on the
// tensor cores (those run in the merged launch)
int phase_all(SigmaBatch& B, int phase, bool skip_tc = false) {
  cudaStream_t main = stream();
  ISCSI_TRY(B.pool.fork(main));
  int rc = kOk;
  for (size_t i = 0; i < B.ctxs.size() && rc == kOk; ++i) {
    if (skip_tc && ab_on_tc(*B.ctxs[i], B.prec)) continue;
    set_stream(B.pool.at((int)i));
    rc = sigma_run(*B.ctxs[i], B.cs[i], B.ss[i], B.nvec, B.prec, phase);
  }
  set_stream(main);
  ISCSI_TRY(rc);
  return B.pool.join(main);
}

}  // namespace

// the whole batch, launch by launch on stream() (also what a capture records):
// the per-context phases run on concurrent pool streams, the merged
// contractions on the main stream between them
int sigma_batch_sequence(SigmaBatch& B) {
  cudaStream_t st = stream();
  const int n = (int)B.ctxs.size();
  if (!B.err.p) {
    ISCSI_TRY(B.err.alloc(sizeof(int)));
    ISCSI_CUDA(cudaMemsetAsync(B.err.p, 0, sizeof(int), st));
  }
  ISCSI_TRY(B.pool.init(std::min(n, 16)));
  // each context's routing is tuned by plain sigma calls before it joins a batch
  for (int i = 0; i < n; ++i)
    if (!B.ctxs[i]->capturing) ISCSI_TRY(sigma_autotune(*B.ctxs[i], B.cs[i], B.ss[i], B.nvec, B.prec));
  ISCSI_TRY(phase_all(B, kPhPre));
  {
    // opposite spin: the tensor-core contexts in one launch, the others on
    // their own
    {
      std::vector<const OzJob*> jobs;
      std::vector<void*> tb;
      for (int i = 0; i < n; ++i) {
        Context& c = *B.ctxs[i];
        if (!c.have_ab || !ab_on_tc(c, B.prec)) continue;
        const OzJob* J = B.prec == 64 ? &c.oz_ab : &c.t3_ab;
        void* base = nullptr;  // the opposite-spin outputs are absolute (the context's T workspace)
        if (both_tc(c, B.prec)) {
          // the context's combined list: its same-spin outputs are relative to its sigma
          J = both_tc_job(c, B.prec);
          if (!J) return kErrCuda;
          base = B.prec == 64 ? static_cast<void*>(B.ss[i]) : static_cast<void*>(c.s32.as<float>());
        }
        jobs.push_back(J);
        tb.push_back(base);
      }
      ISCSI_TRY(merge_jobs(B.ab, jobs, tb, B.prec, st));
      ISCSI_TRY(launch_merged(B.ab, B.prec, B.err.as<int>(), st));
    }
    ISCSI_TRY(phase_all(B, kPhAbGemm, /*skip_tc=*/true));
  }
  ISCSI_TRY(phase_all(B, kPhMid));
  {
    std::vector<const OzJob*> jobs;
    std::vector<void*> tb;
    for (int i = 0; i < n; ++i) {
      Context& c = *B.ctxs[i];
      const bool on = B.prec == 64 ? samespin_tc_active(c) : samespin_tc32_active(c);
      if (!on || both_tc(c, B.prec)) continue;  // combined contexts ran above
      jobs.push_back(B.prec == 64 ? &c.oz_ss : &c.t3_ss);
      tb.push_back(B.prec == 64 ? static_cast<void*>(B.ss[i]) : static_cast<void*>(c.s32.as<float>()));
    }
    ISCSI_TRY(merge_jobs(B.sst, jobs, tb, B.prec, st));
    ISCSI_TRY(launch_merged(B.sst, B.prec, B.err.as<int>(), st));
  }
  ISCSI_TRY(phase_all(B, kPhPost));
  return kOk;
}

namespace {

long long graph_kernel_nodes(cudaGraph_t g) {
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

int batch_run(BatchState& B) {
  if (B.x) {
    ISCSI_CUDA(cudaGraphLaunch(B.x, B.bs));
    g_launch_count += B.kernels;
    return kOk;
  }
  if (B.calls == 0 || !options().use_graph || B.failed) return sigma_batch_sequence(B.sb);
  // second call with this batch: capture it, then replay
  long long before = g_launch_count;
  for (Context* c : B.sb.ctxs) c->capturing = true;
  cudaError_t ce = cudaStreamBeginCapture(B.bs, cudaStreamCaptureModeThreadLocal);
  int rc = ce == cudaSuccess ? sigma_batch_sequence(B.sb) : kErrCuda;
  cudaGraph_t g = nullptr;
  cudaError_t ee = ce == cudaSuccess ? cudaStreamEndCapture(B.bs, &g) : ce;
  for (Context* c : B.sb.ctxs) c->capturing = false;
  g_launch_count = before;
  if (ce == cudaSuccess && rc == kOk && ee == cudaSuccess && g && cudaGraphInstantiate(&B.x, g, 0) == cudaSuccess) {
    B.g = g;
    B.kernels = graph_kernel_nodes(g);
    ISCSI_CUDA(cudaGraphLaunch(B.x, B.bs));
    g_launch_count += B.kernels;
    return kOk;
  }
  if (g) cudaGraphDestroy(g);
  B.x = nullptr;
  B.failed = true;
  cudaGetLastError();
  return sigma_batch_sequence(B.sb);
}

}  // namespace

void batch_reset() { g_batch.reset(); }

int batch_sigma(const std::vector<Context*>& ctxs, const std::vector<const double*>& cs,
                const std::vector<double*>& ss, int nvec, int prec) {
  if (!g_batch || g_batch->sb.ctxs != ctxs || g_batch->sb.cs != cs || g_batch->sb.ss != ss ||
      g_batch->sb.nvec != nvec || g_batch->sb.prec != prec) {
    g_batch.reset(new BatchState());
    BatchState& B = *g_batch;
    B.sb.ctxs = ctxs;
    B.sb.cs = cs;
    B.sb.ss = ss;
    B.sb.nvec = nvec;
    B.sb.prec = prec;
    ISCSI_TRY(B.sb.err.alloc(sizeof(int)));
    ISCSI_CUDA(cudaMemset(B.sb.err.p, 0, sizeof(int)));
    ISCSI_CUDA(cudaStreamCreateWithFlags(&B.bs, cudaStreamNonBlocking));
    ISCSI_CUDA(cudaEventCreateWithFlags(&B.ev, cudaEventDisableTiming));
  }
  BatchState& B = *g_batch;
  // run on the batch's own (capturable) stream, ordered after and before the caller's
  cudaStream_t user = stream();
  ISCSI_CUDA(cudaEventRecord(B.ev, user));
  ISCSI_CUDA(cudaStreamWaitEvent(B.bs, B.ev, 0));
  set_stream(B.bs);
  int rc = batch_run(B);
  set_stream(user);
  ++B.calls;
  ISCSI_CUDA(cudaEventRecord(B.ev, B.bs));
  ISCSI_CUDA(cudaStreamWaitEvent(user, B.ev, 0));
  return rc;
}

// status of the bounded waits of the merged launches (synchronises)
int batch_check() {
  if (!g_batch || !g_batch->sb.err.p) return kOk;
  const int rc = tc_wait_status(g_batch->sb.err.as<int>(), "batched sigma");
  // the aborted launch may have left split-K counters raised: the next call
  // builds the batch (lists, schedules, graph) anew
  if (rc == kErrWait) g_batch.reset();
  return rc;
}

bool batch_graph_active() { return g_batch && g_batch->x; }

}  // namespace iscsi
