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
//      tile are added in part order by whichever finishes last (ozaki.cuh);
//   4. repeats 2-3 with a few take-back thresholds and smallest part sizes
//      and keeps the plan whose busiest CTA is predicted to end first: when
//      single tiles come close to the balanced load (short launches), the
//      CTAs that hold them keep gaps too small for a part unless those tiles
//      are cut as well.
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
    // Tiles close to the balanced load leave gaps too small for a part, and
    // a part's fixed cost is large against a short launch: try a few take-back
    // thresholds and part sizes, keep the plan whose busiest CTA ends first
    // (the first, least split, unless another ends at least 1 % sooner).  No
    // plan ends before the balanced load (parts only add overhead), so a first
    // plan within 1 % of it cannot be replaced and the others are not tried
    // (large launches, whose plans are also rebuilt most often: batches of
    // many contexts).
    const double ovh = kItemOverhead + kPartOverhead;
    const double variants[][2] = {{1.02, 4.0}, {0.97, 2.0}, {0.9, 2.0}, {0.75, 1.0}, {0.0, 1.0}};
    std::vector<Slot> best, cur;
    int best_slots = 0, best_counters = 0;
    double best_max = 0.0;
    for (const auto& v : variants) {
      int slots = 0, counters = 0;
      const double mx = attempt(tiles, total / ncta, ncta, v[0], v[1] * ovh, cur, slots, counters);
      if (best.empty() || mx < 0.99 * best_max) {
        best.swap(cur);
        best_max = mx;
        best_slots = slots;
        best_counters = counters;
      }
      if (best_max * 0.99 <= total / ncta) break;
    }
    plan.slots = best_slots;
    plan.counters = best_counters;
    std::vector<Slot>& cta = best;
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
  struct Slot {
    std::vector<OzItem> items;
    double load = 0.0;
  };

  // One schedule: list scheduling of whole tiles, then the tiles of CTAs
  // loaded above thr x target taken back and water-filled in parts of at
  // least min_part.  Returns the busiest CTA's predicted load.
  double attempt(const std::vector<Tile>& tiles, double target, int ncta, double thr, double min_part,
                 std::vector<Slot>& cta, int& slots, int& counters) const {
    cta.assign(ncta, Slot());
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
    std::vector<int> pool;
    for (int b = 0; b < ncta; ++b) {
      while (!cta[b].items.empty() && cta[b].load > target * thr) {
        const int i = tile_of[b].back();
        pool.push_back(i);
        cta[b].load -= tiles[i].cost;
        cta[b].items.pop_back();
        tile_of[b].pop_back();
      }
    }
    std::sort(pool.begin(), pool.end());  // banded order again
    slots = 0;
    counters = 0;
    if (!pool.empty()) {
      std::vector<int> order(ncta);
      for (int b = 0; b < ncta; ++b) order[b] = b;
      std::sort(order.begin(), order.end(),
                [&](int x, int y) { return cta[x].load < cta[y].load || (cta[x].load == cta[y].load && x < y); });
      // Fill the CTAs in order of increasing load up to a common level, each
      // CTA taking consecutive pieces of the pool; the level is the lowest at
      // which the pool fits (binary search on a dry run).  Step costs are
      // taken only for the tiles that get cut.
      std::vector<std::vector<double>> psc(pool.size());
      struct Part {
        int tile, s0, s1, cta;
      };
      std::vector<Part> parts;
      std::vector<double> load(ncta);
      auto fill = [&](double lev, bool commit) -> bool {
        for (int b = 0; b < ncta; ++b) load[b] = cta[b].load;
        auto room = [&](int b) { return lev - load[b] - kItemOverhead - kPartOverhead; };
        size_t oi = 0;
        if (commit) parts.clear();
        for (size_t q = 0; q < pool.size(); ++q) {
          const Tile& T = tiles[pool[q]];
          std::vector<double>& sc = psc[q];
          double left = T.cost - kItemOverhead;
          int s = 0;
          do {
            while (oi < order.size() && room(order[oi]) < min_part) ++oi;
            if (oi == order.size()) return false;
            const int b = order[oi];
            const double cap = room(b);
            int e = s;
            double got = 0.0;
            // what is left of the tile fits; or would leave less than a part
            // behind (the rest of a small tile goes whole; of a larger one, a
            // part of min_part stays for the next CTA); or is cut at the level
            const double want = left <= cap ? left : left - cap >= min_part ? cap : left >= 2.0 * min_part ? left - min_part : left;
            if (want >= left) {
              e = T.nsteps;
              got = left;
            } else {
              if (sc.empty()) step_costs(T, sc);
              while (e < T.nsteps && got + sc[e] <= want) got += sc[e++];
              if (e == s) got += sc[e++];  // at least one step
            }
            if (commit) parts.push_back({pool[q], s, e, b});
            load[b] += got + kItemOverhead + kPartOverhead;
            left -= got;
            s = e;
          } while (s < T.nsteps);
        }
        return true;
      };
      double lo = target, hi = target;
      for (int rep = 0; rep < 60 && !fill(hi, false); ++rep) hi = hi * 1.25 + min_part;
      for (int rep = 0; rep < 40; ++rep) {
        const double mid = 0.5 * (lo + hi);
        (fill(mid, false) ? hi : lo) = mid;
      }
      fill(hi, true);
      for (int b = 0; b < ncta; ++b) cta[b].load = load[b];
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
            it.slot = slots;
            it.cnt = counters;
          } else {
            load[parts[q].cta] -= kPartOverhead;  // a whole tile has no partial block
          }
          cta[parts[q].cta].items.push_back(it);
        }
        if (np > 1) {
          slots += np;
          ++counters;
        }
        i = j;
      }
      for (int b = 0; b < ncta; ++b) cta[b].load = load[b];
    }
    double mx = 0.0;
    for (int b = 0; b < ncta; ++b) mx = std::max(mx, cta[b].load);
    return mx;
  }

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

int oz_plan_check(const std::vector<OzProblem>& probs, const std::vector<OzSeg>& segs,
                  const std::vector<OzSegHost>& sh, int nsm, OzPlan& plan, int& errors) {
  if (sh.size() != segs.size() || nsm < 1) {
    set_error("tensor-core schedule check: segment host records missing or no SMs");
    return kErrArg;
  }
  Planner pl(probs, segs, sh);
  ISCSI_TRY(pl.build(nsm, plan));
  errors = 0;
  const int nitems = (int)plan.items.size();
  if (plan.grid < 1 || plan.grid > nsm || (int)plan.cta_start.size() != plan.grid + 1 || plan.cta_start[0] != 0 ||
      plan.cta_start[plan.grid] != nitems)
    ++errors;
  for (int b = 0; b < plan.grid && !errors; ++b)
    if (plan.cta_start[b + 1] <= plan.cta_start[b]) ++errors;  // no CTA runs without work
  // every tile's K steps exactly once; a split tile's parts numbered in K
  // order, sharing one counter and one run of workspace slots
  std::vector<std::vector<const OzItem*>> of_tile;
  std::vector<long long> first_tile(probs.size() + 1, 0);
  for (size_t p = 0; p < probs.size(); ++p) {
    const long long tm = (probs[p].M + OZ_BM - 1) / OZ_BM, tn = (probs[p].N + OZ_BN - 1) / OZ_BN;
    first_tile[p + 1] = first_tile[p] + tm * tn;
  }
  of_tile.resize(first_tile.back());
  for (const OzItem& it : plan.items) {
    if (it.prob < 0 || it.prob >= (int)probs.size()) {
      ++errors;
      continue;
    }
    const OzProblem& P = probs[it.prob];
    const int tn = (P.N + OZ_BN - 1) / OZ_BN, tm = (P.M + OZ_BM - 1) / OZ_BM;
    if (it.mt < 0 || it.mt >= tm || it.nt < 0 || it.nt >= tn) {
      ++errors;
      continue;
    }
    of_tile[first_tile[it.prob] + (long long)it.mt * tn + it.nt].push_back(&it);
  }
  std::vector<int> slot_used(std::max(0, plan.slots), 0), cnt_used(std::max(0, plan.counters), 0);
  for (size_t p = 0; p < probs.size(); ++p) {
    int nsteps = 0;
    for (int g = 0; g < probs[p].seg_count; ++g) nsteps += segs[probs[p].seg_begin + g].K / OZ_BK;
    for (long long t = first_tile[p]; t < first_tile[p + 1]; ++t) {
      std::vector<const OzItem*>& v = of_tile[t];
      std::sort(v.begin(), v.end(), [](const OzItem* x, const OzItem* y) { return x->s0 < y->s0; });
      const int np = (int)v.size();
      int s = 0;
      bool ok = np > 0;
      for (int q = 0; q < np && ok; ++q) {
        const OzItem& it = *v[q];
        ok = it.s0 == s && (it.s1 > it.s0 || nsteps == 0) && it.s1 <= nsteps;
        s = it.s1;
        if (np == 1) {
          ok = ok && it.nparts == 1;
        } else {
          ok = ok && it.nparts == np && it.part == q && it.slot == v[0]->slot && it.cnt == v[0]->cnt &&
               it.slot >= 0 && it.slot + np <= plan.slots && it.cnt >= 0 && it.cnt < plan.counters;
          if (ok) ++slot_used[it.slot + q];
        }
      }
      ok = ok && s == nsteps;
      if (ok && np > 1) ++cnt_used[v[0]->cnt];
      if (!ok) ++errors;
    }
  }
  for (int x : slot_used) errors += x != 1;
  for (int x : cnt_used) errors += x != 1;
  return kOk;
}

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
