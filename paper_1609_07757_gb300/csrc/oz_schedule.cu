// oz_schedule.cu -- the host-built schedule of the persistent FP64-accurate
// contraction (k_oz_gemm): which CTA computes which output tile, or which
// split-K part of it, and in what order.
//
// One CTA runs on each SM for the whole launch.  The schedule
//   1. lists the output tiles of every problem in bands of 8 row tiles, the
//      tiles of a band column by column, so that the tiles that run at the
//      same time on different SMs share A row tiles and B column tiles in L2;
//   2. deals the tiles out in that order, each to the CTA with the least work
//      so far (list scheduling), with a cost model of the kernel: per issued K
//      step the larger of the MMA time (products of live slices) and the
//      load time, plus a per-item overhead;
//   3. takes back the tiles that would end after the balanced finish time
//      and cuts them along K into parts that fill the CTAs up to a common
//      level (water filling), so the last wave ends together; the parts of a
//      tile are added in part order by whichever finishes last (ozaki.cuh).
// Steps whose blocks are all zero (screened) cost nothing and are never
// issued, so the schedule follows the screen.
#include <algorithm>
#include <cstring>
#include <functional>
#include <queue>
#include <vector>

#include "internal.cuh"

namespace iscsi {

namespace {

// cost model (SM clock cycles), measured on GB300: the ten MMAs of a full
// step take ~968 cycles (28 slice products); one contiguous bulk copy streams
// ~66 bytes per cycle into an SM, TMA boxes of 32-byte rows ~32
constexpr double kCycPerProduct = 968.0 / 28.0;
constexpr double kBulkBytesPerCyc = 60.0;
constexpr double kTmaBytesPerCyc = 30.0;
constexpr double kStepOverhead = 20.0;
constexpr double kItemOverhead = 2500.0;
constexpr double kPartOverhead = 2000.0;  // partial block written, then read by the combining part

struct Tile {
  int prob, mt, nt;
  int nsteps;   // K steps of the problem (all segments)
  double cost;  // whole tile
};

class Planner {
 public:
  Planner(const std::vector<OzProblem>& probs, const std::vector<OzSeg>& segs, const std::vector<OzSegHost>& sh)
      : probs_(probs), segs_(segs), sh_(sh) {}

  // cost of each K step of a tile (0: not issued)
  void step_costs(const Tile& T, std::vector<double>& c) const {
    c.assign(T.nsteps, 0.0);
    const OzProblem& P = probs_[T.prob];
    int cstep = 0;
    for (int g = 0; g < P.seg_count; ++g) {
      const OzSeg& S = segs_[P.seg_begin + g];
      const OzSegHost& H = sh_[P.seg_begin + g];
      const int nst = S.K / OZ_BK;
      if (T.nt * OZ_BN < S.nrows_b) {
        const bool tiled = S.a_tiled != nullptr;
        for (int ks = 0; ks < nst; ++ks) {
          const int la = H.a_live ? H.a_live[(long long)(S.a_rt0 + T.mt) * S.a_kst + S.a_ks0 + ks] : OZ_S;
          const int lb = H.b_live ? H.b_live[(long long)(S.b_rt0 + T.nt) * S.b_kst + S.b_ks0 + ks] : OZ_S;
          const int m = la + lb - OZ_S;  // live levels: products m (m + 1) / 2
          if (m <= 0) continue;
          const double mma = kCycPerProduct * m * (m + 1) / 2.0;
          const double bytes = tiled ? (double)m * (OZ_A_SLICE_BYTES + OZ_B_SLICE_BYTES) : (double)OZ_STAGE_BYTES;
          const double load = bytes / (tiled ? kBulkBytesPerCyc : kTmaBytesPerCyc);
          c[cstep + ks] = std::max(mma, load) + kStepOverhead;
        }
      }
      cstep += nst;
    }
  }

  int build(int nsm, OzPlan& plan) {
    // 1. tiles in banded order
    std::vector<Tile> tiles;
    plan.issued_products = 0.0;
    for (int p = 0; p < (int)probs_.size(); ++p) {
      const OzProblem& P = probs_[p];
      const int tm = (P.M + OZ_BM - 1) / OZ_BM, tn = (P.N + OZ_BN - 1) / OZ_BN;
      int nsteps = 0;
      for (int g = 0; g < P.seg_count; ++g) nsteps += segs_[P.seg_begin + g].K / OZ_BK;
      for (int b0 = 0; b0 < tm; b0 += 8)
        for (int nt = 0; nt < tn; ++nt)
          for (int mt = b0; mt < std::min(tm, b0 + 8); ++mt) tiles.push_back({p, mt, nt, nsteps, 0.0});
    }
    std::vector<double> sc;
    double total = 0.0;
    for (Tile& T : tiles) {
      step_costs(T, sc);
      double c = kItemOverhead;
      for (double x : sc) c += x;
      T.cost = c;
      total += c;
      plan.issued_products += products_of(T);
    }
    const int ncta = std::max(1, nsm);  // split-K parts spread small problems over every SM
    // 2. list scheduling
    struct Slot {
      std::vector<OzItem> items;
      double load = 0.0;
    };
    std::vector<Slot> cta(ncta);
    std::vector<std::vector<int>> tile_of(ncta);  // tile index of each whole item
    using Q = std::pair<double, int>;
    std::priority_queue<Q, std::vector<Q>, std::greater<Q>> heap;
    for (int b = 0; b < ncta; ++b) heap.push({0.0, b});
    for (int i = 0; i < (int)tiles.size(); ++i) {
      Q q = heap.top();
      heap.pop();
      const Tile& T = tiles[i];
      cta[q.second].items.push_back({T.prob, T.mt, T.nt, 0, T.nsteps, 0, 1, -1, -1});
      tile_of[q.second].push_back(i);
      cta[q.second].load += T.cost;
      heap.push({cta[q.second].load, q.second});
    }
    // 3. take back the tiles ending late, cut them into parts (water filling)
    const double target = total / ncta;
    std::vector<int> pool;
    for (int b = 0; b < ncta; ++b) {
      while (!cta[b].items.empty() && cta[b].load > target * 1.02) {
        const int i = tile_of[b].back();
        pool.push_back(i);
        cta[b].load -= tiles[i].cost;
        cta[b].items.pop_back();
        tile_of[b].pop_back();
      }
    }
    std::sort(pool.begin(), pool.end());  // banded order again
    plan.slots = 0;
    plan.counters = 0;
    if (!pool.empty()) {
      std::vector<int> order(ncta);
      for (int b = 0; b < ncta; ++b) order[b] = b;
      std::sort(order.begin(), order.end(), [&](int x, int y) { return cta[x].load < cta[y].load; });
      // Fill the CTAs in order of increasing load up to a common level, each
      // CTA taking consecutive pieces of the pool (parts of at least min_part:
      // smaller ones cost more in overhead than they balance); the level is
      // the lowest at which the pool fits (binary search on a dry run).
      const double min_part = 4.0 * (kItemOverhead + kPartOverhead);
      std::vector<std::vector<double>> psc(pool.size());
      for (size_t q = 0; q < pool.size(); ++q) step_costs(tiles[pool[q]], psc[q]);
      struct Part {
        int tile, s0, s1, cta;
      };
      std::vector<Part> parts;
      auto fill = [&](double lev, bool commit) -> bool {
        std::vector<double> load(ncta);
        for (int b = 0; b < ncta; ++b) load[b] = cta[b].load;
        auto room = [&](int b) { return lev - load[b] - kItemOverhead - kPartOverhead; };
        size_t oi = 0;
        if (commit) parts.clear();
        for (size_t q = 0; q < pool.size(); ++q) {
          const Tile& T = tiles[pool[q]];
          const std::vector<double>& sc = psc[q];
          double left = T.cost - kItemOverhead;
          int s = 0;
          do {
            while (oi < order.size() && room(order[oi]) < min_part) ++oi;
            if (oi == order.size()) return false;
            const int b = order[oi];
            const double cap = room(b);
            int e = s;
            double got = 0.0;
            if (left - cap < min_part) {
              e = T.nsteps;  // the rest of the tile
              got = left;
            } else {
              while (e < T.nsteps && got + sc[e] <= cap) got += sc[e++];
              if (e == s) got += sc[e++];  // at least one step
            }
            if (commit) parts.push_back({pool[q], s, e, b});
            load[b] += got + kItemOverhead + kPartOverhead;
            left -= got;
            s = e;
          } while (s < T.nsteps);
        }
        if (commit)
          for (int b = 0; b < ncta; ++b) cta[b].load = load[b];
        return true;
      };
      double lo = target, hi = target;
      for (int rep = 0; rep < 60 && !fill(hi, false); ++rep) hi = hi * 1.25 + min_part;
      for (int rep = 0; rep < 40; ++rep) {
        const double mid = 0.5 * (lo + hi);
        (fill(mid, false) ? hi : lo) = mid;
      }
      fill(hi, true);
      // number the parts of split tiles and hand them to their CTAs
      for (size_t i = 0; i < parts.size();) {
        size_t j = i;
        while (j < parts.size() && parts[j].tile == parts[i].tile) ++j;
        const int np = (int)(j - i);
        const Tile& T = tiles[parts[i].tile];
        for (size_t q = i; q < j; ++q) {
          OzItem it{T.prob, T.mt, T.nt, parts[q].s0, parts[q].s1, 0, 1, -1, -1};
          if (np > 1) {
            it.part = (int)(q - i);
            it.nparts = np;
            it.slot = plan.slots;
            it.cnt = plan.counters;
          }
          cta[parts[q].cta].items.push_back(it);
        }
        if (np > 1) {
          plan.slots += np;
          ++plan.counters;
        }
        i = j;
      }
    }
    // flatten (CTAs without items are left out)
    plan.items.clear();
    plan.cta_start.assign(1, 0);
    double mx = 0.0;
    for (int b = 0; b < ncta; ++b) {
      if (cta[b].items.empty()) continue;
      plan.items.insert(plan.items.end(), cta[b].items.begin(), cta[b].items.end());
      plan.cta_start.push_back((int)plan.items.size());
      mx = std::max(mx, cta[b].load);
    }
    plan.grid = (int)plan.cta_start.size() - 1;
    plan.model_cycles = mx;
    plan.model_balance = mx > 0 ? total / (plan.grid * mx) : 1.0;
    return kOk;
  }

 private:
  // bf16 slice products of a whole tile (x 2 M N K per step)
  double products_of(const Tile& T) const {
    const OzProblem& P = probs_[T.prob];
    double prod = 0.0;
    for (int g = 0; g < P.seg_count; ++g) {
      const OzSeg& S = segs_[P.seg_begin + g];
      const OzSegHost& H = sh_[P.seg_begin + g];
      if (T.nt * OZ_BN >= S.nrows_b) continue;
      for (int ks = 0; ks < S.K / OZ_BK; ++ks) {
        const int la = H.a_live ? H.a_live[(long long)(S.a_rt0 + T.mt) * S.a_kst + S.a_ks0 + ks] : OZ_S;
        const int lb = H.b_live ? H.b_live[(long long)(S.b_rt0 + T.nt) * S.b_kst + S.b_ks0 + ks] : OZ_S;
        const int m = la + lb - OZ_S;
        if (m > 0) prod += m * (m + 1) / 2;
      }
    }
    return prod * 2.0 * OZ_BM * OZ_BN * OZ_BK;
  }

  const std::vector<OzProblem>& probs_;
  const std::vector<OzSeg>& segs_;
  const std::vector<OzSegHost>& sh_;
};

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        n <= 0)
      n = 148;
  }
  return n;
}

}  // namespace

int oz_plan_build(const std::vector<OzProblem>& probs, const std::vector<OzSeg>& segs,
                  const std::vector<OzSegHost>& sh, OzPlan& plan, cudaStream_t st) {
  if (sh.size() != segs.size()) {
    set_error("tensor-core schedule: segment host records missing");
    return kErrArg;
  }
  Planner pl(probs, segs, sh);
  ISCSI_TRY(pl.build(sm_count(), plan));
  ISCSI_TRY(plan.d_items.grow(sizeof(OzItem) * std::max<size_t>(1, plan.items.size())));
  ISCSI_TRY(plan.d_cta.grow(sizeof(int) * plan.cta_start.size()));
  if (!plan.items.empty())
    ISCSI_CUDA(cudaMemcpyAsync(plan.d_items.p, plan.items.data(), sizeof(OzItem) * plan.items.size(),
                               cudaMemcpyHostToDevice, st));
  ISCSI_CUDA(cudaMemcpyAsync(plan.d_cta.p, plan.cta_start.data(), sizeof(int) * plan.cta_start.size(),
                             cudaMemcpyHostToDevice, st));
  const size_t wsb = sizeof(double) * (size_t)std::max(1, plan.slots) * OZ_BM * OZ_BN;
  if (plan.d_ws.bytes < wsb) ISCSI_TRY(plan.d_ws.grow(wsb));
  const size_t cb = sizeof(int) * (size_t)std::max(1, plan.counters);
  if (plan.d_cnt.bytes < cb) ISCSI_TRY(plan.d_cnt.grow(cb));
  ISCSI_CUDA(cudaMemsetAsync(plan.d_cnt.p, 0, plan.d_cnt.bytes, st));
  ISCSI_CUDA(cudaStreamSynchronize(st));  // the host vectors may change after this call
  return kOk;
}

}  // namespace iscsi
