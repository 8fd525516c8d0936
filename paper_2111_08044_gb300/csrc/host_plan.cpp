// Fusion planner (host, FP64): groups the period's two-qubit gates into
// passes over the state, each applying one fused 2^n x 2^n unitary on a
// window of n consecutive sites.  This is the single-device form of the
// paper's fused >= 7-qubit operators (Sec. II: contractions on index
// groups of 2^7 to fit the matrix unit).
//
// Search: beam search over (gates done, current window), its levels
// expanded on the host's cores and its result cached per gate structure.  A pass may take
// every pending gate inside its window whose predecessors are done.  Moving
// the window by more than 7 sites costs extra relabel-only passes (the
// state layout changes through a 7-bit row index), as does returning to the
// period's first window at the end of the period, because every period
// starts from the same layout.  That first window sits at site 0 (the
// natural layout), or, for a cyclic plan, at the start s <= 7 that needs
// the fewest passes: the state then stays in the layout of window s from
// one period to the next, and a single relabel pass at the start of an
// evolution (and the last period's last pass writing the natural layout)
// take it there and back.
#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_set>

#include "sv_internal.h"

namespace fsv {

namespace {

constexpr int kMaxShift = 7;

struct Dag {
  std::vector<int> bond;
  std::vector<std::vector<int>> pred;
  std::vector<std::vector<int>> by_bond;  // gate indices per bond, in order
};

Dag make_dag(const std::vector<Gate2>& gates, int L) {
  Dag d;
  d.by_bond.resize(L);
  std::vector<int> last(L, -1);
  for (size_t k = 0; k < gates.size(); ++k) {
    const int b = gates[k].bond;
    d.bond.push_back(b);
    std::vector<int> p;
    if (last[b] >= 0) p.push_back(last[b]);
    if (last[b + 1] >= 0 && last[b + 1] != last[b]) p.push_back(last[b + 1]);
    d.pred.push_back(p);
    d.by_bond[b].push_back((int)k);
    last[b] = last[b + 1] = (int)k;
  }
  return d;
}

struct State {
  std::vector<uint64_t> done;
  int count = 0;
  int lo = -1;
  // the pass that led here: its gates, the relabel-only passes before it,
  // and the state it came from (level, index among that level's kept states)
  std::vector<int> ab;
  int relabels = 0;
  int plevel = -1, pindex = -1;
};

inline bool test(const std::vector<uint64_t>& s, int k) { return (s[k >> 6] >> (k & 63)) & 1; }
inline void set(std::vector<uint64_t>& s, int k) { s[k >> 6] |= 1ull << (k & 63); }

std::vector<int> absorb(const Dag& d, std::vector<uint64_t>& done, int lo, int n) {
  // the pending gates on the window's bonds, in the period's order (a gate
  // taken here can ready a later one in the same window)
  std::vector<int> cand;
  for (int b = lo; b + 1 < lo + n && b < (int)d.by_bond.size(); ++b)
    for (int k : d.by_bond[b])
      if (!test(done, k)) cand.push_back(k);
  std::sort(cand.begin(), cand.end());
  std::vector<int> ab;
  for (int k : cand) {
    bool ready = true;
    for (int p : d.pred[k])
      if (!test(done, p)) {
        ready = false;
        break;
      }
    if (ready) {
      set(done, (int)k);
      ab.push_back((int)k);
    }
  }
  return ab;
}

int shift_cost(int from, int to) {
  const int delta = std::abs(to - from);
  return delta <= kMaxShift ? 0 : (delta + kMaxShift - 1) / kMaxShift - 1;
}

size_t key_hash(const State& s) {
  size_t h = (size_t)s.lo * 0x9E3779B97F4A7C15ull;
  for (uint64_t w : s.done) h ^= w + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
  return h;
}

}  // namespace

namespace {

using Hist = std::vector<std::pair<int, std::vector<int>>>;  // (lo or -1, gates) per pass

// The beam search: the best sequence of windows for the gate DAG.  The kept
// states of a level are expanded on the host's cores; their candidates are
// merged in the order a single thread would produce them, so the plan does
// not depend on the thread count.  States link to their parents; the
// sequence of passes is read back once at the end.
Hist plan_search(const Dag& dag, int L, int n, int ng, int start) {
  const int words = (ng + 63) / 64;
  const size_t beam = ng <= 200 ? 256 : 32;
  // levels[k]: states after k passes (relabel-only passes included)
  std::vector<std::vector<State>> levels(1);
  std::vector<std::vector<State>> archive;  // kept states per level (parents)
  State s0;
  s0.done.assign(words, 0);
  levels[0].push_back(s0);
  int best_total = 1 << 30;
  State best;
  int best_tail = 0;  // relabel-only passes back to the start after the last window
  struct Cand {
    State t;
    int kk;
  };
  const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  for (int k = 0; k < (int)levels.size() && k < best_total; ++k) {
    std::vector<State> lv = std::move(levels[k]);
    levels[k].clear();
    std::sort(lv.begin(), lv.end(), [](const State& a, const State& b) {
      if (a.count != b.count) return a.count > b.count;
      return a.lo < b.lo;
    });
    std::unordered_set<size_t> seen;
    if ((int)archive.size() <= k) archive.resize(k + 1);
    std::vector<State>& kept = archive[k];
    for (auto& s : lv) {
      if (kept.size() >= beam) break;
      if (seen.insert(key_hash(s)).second) kept.push_back(std::move(s));
    }
    std::vector<std::vector<Cand>> per(kept.size());
    auto expand = [&](size_t i0, size_t i1) {
      for (size_t i = i0; i < i1; ++i) {
        const State& s = kept[i];
        // the first window is the period's start
        const int lo_min = s.lo < 0 ? start : 0, lo_max = s.lo < 0 ? start : L - n;
        for (int lo = lo_min; lo <= lo_max; ++lo) {
          State t;
          t.done = s.done;
          t.ab = absorb(dag, t.done, lo, n);
          if (t.ab.empty()) continue;
          t.count = s.count + (int)t.ab.size();
          t.lo = lo;
          const int cost = 1 + (s.lo < 0 ? 0 : shift_cost(s.lo, lo));
          t.relabels = cost - 1;
          t.plevel = k;
          t.pindex = (int)i;
          per[i].push_back({std::move(t), k + cost});
        }
      }
    };
    const size_t nt = std::min<size_t>(hw, kept.size() / 4);
    if (nt <= 1) {
      expand(0, kept.size());
    } else {
      std::vector<std::thread> th;
      const size_t chunk = (kept.size() + nt - 1) / nt;
      for (size_t t = 0; t < nt; ++t)
        th.emplace_back(expand, t * chunk, std::min(kept.size(), (t + 1) * chunk));
      for (auto& x : th) x.join();
    }
    for (auto& cs : per)
      for (Cand& c : cs) {
        if (c.t.count == ng) {
          const int total = c.kk + shift_cost(c.t.lo, start);
          if (total < best_total) {
            best_total = total;
            best = c.t;
            best_tail = shift_cost(c.t.lo, start);
          }
          continue;
        }
        if ((int)levels.size() <= c.kk) levels.resize(c.kk + 1);
        levels[c.kk].push_back(std::move(c.t));
      }
  }
  // read the passes back along the parent links
  Hist rev;
  for (int e = 0; e < best_tail; ++e) rev.push_back({-1, {}});
  const State* st = &best;
  while (st && st->plevel >= 0) {
    rev.push_back({st->lo, st->ab});
    for (int e = 0; e < st->relabels; ++e) rev.push_back({-1, {}});
    st = &archive[st->plevel][st->pindex];
  }
  return Hist(rev.rbegin(), rev.rend());
}

// The plan from the best start: site 0 only, or (cyclic) every start
// s <= 7 (a single relabel pass then reaches it from the natural layout),
// the fewest passes winning and the smaller start breaking ties.
Hist best_plan(const Dag& dag, int L, int n, int ng, bool cyclic) {
  Hist best = plan_search(dag, L, n, ng, 0);
  const int smax = cyclic ? std::min(kMaxShift, L - n) : 0;
  for (int s = 1; s <= smax; ++s) {
    Hist h = plan_search(dag, L, n, ng, s);
    if (h.size() < best.size()) best.swap(h);
  }
  return best;
}

// Plans depend only on the gate structure (bond sequence, L, n), not on the
// gate values: a rebuild with new parameters reuses the search.
Hist cached_plan(const Dag& dag, int L, int n, int ng, bool cyclic) {
  static std::mutex mu;
  static std::map<std::vector<int>, Hist> cache;
  std::vector<int> key{L, n, cyclic ? 1 : 0};
  key.insert(key.end(), dag.bond.begin(), dag.bond.end());
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  Hist h = best_plan(dag, L, n, ng, cyclic);
  std::lock_guard<std::mutex> lk(mu);
  if (cache.size() >= 64) cache.clear();
  cache.emplace(std::move(key), h);
  return h;
}

}  // namespace

std::vector<MultiPass> multigate_plan(int L, const std::vector<Gate2>& gates, int w) {
  // Greedy: each pass takes the window of w sites that absorbs the most
  // pending gates (the lowest such window on ties).  The state keeps the
  // natural layout, so a window may move anywhere between passes.
  const Dag dag = make_dag(gates, L);
  const int ng = (int)gates.size();
  std::vector<uint64_t> done((ng + 63) / 64, 0);
  int count = 0;
  std::vector<MultiPass> out;
  std::vector<int> last_gate(L, -1);
  for (int k = 0; k < ng; ++k) {
    last_gate[gates[k].bond] = k;
    last_gate[gates[k].bond + 1] = k;
  }
  while (count < ng) {
    int best_lo = -1;
    std::vector<int> best;
    for (int lo = 0; lo + w <= L; ++lo) {
      std::vector<uint64_t> d = done;
      std::vector<int> ab = absorb(dag, d, lo, w);
      if (ab.size() > best.size()) {
        best.swap(ab);
        best_lo = lo;
      }
    }
    if (best.empty()) break;  // cannot happen for a gate DAG of bonds inside the chain
    for (int g : best) set(done, g);
    count += (int)best.size();
    MultiPass p;
    p.lo = best_lo;
    p.gates = best;
    for (int g : best)
      for (int site : {gates[g].bond, gates[g].bond + 1})
        if (last_gate[site] == g) p.x_sites.push_back(site);
    std::sort(p.x_sites.begin(), p.x_sites.end());
    out.push_back(std::move(p));
  }
  if (!out.empty()) out.back().diag = true;
  return out;
}

std::vector<BlockPass> fusion_plan(int L, const std::vector<Gate2>& gates, int n, bool cyclic) {
  const Dag dag = make_dag(gates, L);
  const int ng = (int)gates.size();
  const Hist hist = cached_plan(dag, L, n, ng, cyclic);
  int start = 0;
  for (const auto& h : hist)
    if (h.first >= 0) {
      start = h.first;
      break;
    }
  // Materialise passes: fused unitaries, energy flags.  A relabel-only pass
  // keeps an identity unitary on a window that steps toward the next one.
  std::vector<BlockPass> out;
  const size_t dim = (size_t)1 << n;
  std::vector<int> last_gate(L, -1);
  for (int k = 0; k < ng; ++k) {
    last_gate[gates[k].bond] = k;
    last_gate[gates[k].bond + 1] = k;
  }
  int prev_lo = start;
  for (size_t h = 0; h < hist.size(); ++h) {
    BlockPass p;
    p.n = n;
    if (hist[h].first >= 0) {
      p.lo = hist[h].first;
      p.gates = hist[h].second;
    } else {
      // find the next real window (or the start at the end) and step toward it
      int target = start;
      for (size_t q = h + 1; q < hist.size(); ++q)
        if (hist[q].first >= 0) {
          target = hist[q].first;
          break;
        }
      const int step = std::max(-kMaxShift, std::min(kMaxShift, target - prev_lo));
      p.lo = prev_lo + step;
    }
    p.U.assign(dim * dim, cd(0.0, 0.0));
    for (size_t e = 0; e < dim; ++e) p.U[e * dim + e] = 1.0;
    for (int g : p.gates) {
      // U <- G_embedded U, G on local bits (j, j+1) with r = 2 b_j + b_{j+1}
      const int j = gates[g].bond - p.lo;
      std::vector<cd> nu(dim * dim, cd(0.0, 0.0));
      for (size_t row = 0; row < dim; ++row) {
        const int rr = 2 * (int)((row >> j) & 1) + (int)((row >> (j + 1)) & 1);
        const size_t rbase = row & ~(((size_t)3) << j);
        for (int cc = 0; cc < 4; ++cc) {
          const cd gv = gates[g].m[4 * rr + cc];
          if (gv == cd(0.0, 0.0)) continue;
          const size_t src = rbase | ((size_t)(cc >> 1) << j) | ((size_t)(cc & 1) << (j + 1));
          for (size_t col = 0; col < dim; ++col) nu[row * dim + col] += gv * p.U[src * dim + col];
        }
      }
      p.U.swap(nu);
      for (int site : {gates[g].bond, gates[g].bond + 1})
        if (last_gate[site] == g) p.x_sites.push_back(site);
    }
    std::sort(p.x_sites.begin(), p.x_sites.end());
    prev_lo = p.lo;
    out.push_back(std::move(p));
  }
  if (!out.empty()) out.back().diag = true;
  return out;
}

}  // namespace fsv
