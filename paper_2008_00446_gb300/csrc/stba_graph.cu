// Camera graph of a problem (host code).  Two cameras are joined when they observe a common point; the
// edge lists, once, every such pair of observations.  The graph does not depend on the cluster assignment:
// under any assignment the off-diagonal blocks of the clustered reduced camera systems (Eq. 10, 13) are
// sums over exactly the edge pairs whose two cameras share a cluster, and its edge weights (the number of
// co-visible points) are those of the camera graph that stochastic graph clustering samples from (Sec. 4.4).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "stba_internal.cuh"

namespace stba {

namespace {

template <typename F>
void parallel_ranges(int count, F&& f) {
  int nt = (int)std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()), 16u);
  nt = std::max(1, std::min(nt, count / 64));
  if (nt <= 1) {
    f(0, count);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) {
    const int b = (int)((int64_t)count * t / nt), e = (int)((int64_t)count * (t + 1) / nt);
    th.emplace_back([&f, b, e] { f(b, e); });
  }
  for (auto& x : th) x.join();
}

}  // namespace

// base_cam[bo]: camera of base position bo (observations sorted by (point, camera)); pt_off: point runs.
// Without with_pairs only the edges and their weights are formed.
void build_camera_graph(int m, int n, const std::vector<int>& pt_off, const std::vector<int>& base_cam,
                        CameraGraph& g, bool with_pairs) {
  const int q = (int)base_cam.size();
  std::vector<int> base_pt(q);
  for (int i = 0; i < n; ++i)
    for (int o = pt_off[i]; o < pt_off[i + 1]; ++o) base_pt[o] = i;
  // base positions of every camera, ascending
  std::vector<int> cam_off(m + 1, 0), cam_pos(q);
  for (int o = 0; o < q; ++o) cam_off[base_cam[o] + 1]++;
  for (int j = 0; j < m; ++j) cam_off[j + 1] += cam_off[j];
  {
    std::vector<int> f(cam_off.begin(), cam_off.end() - 1);
    for (int o = 0; o < q; ++o) cam_pos[f[base_cam[o]]++] = o;
  }
  // pass 1: for every camera x, its partners y < x (ascending) and the number of common points
  std::vector<std::vector<int2>> part(m);   // (y, count)
  parallel_ranges(m, [&](int xb, int xe) {
    std::vector<int> cnt(m, 0), touched;
    for (int x = xb; x < xe; ++x) {
      touched.clear();
      for (int e = cam_off[x]; e < cam_off[x + 1]; ++e) {
        const int a = cam_pos[e], b = pt_off[base_pt[a]];
        for (int o = b; o < a; ++o) {   // the point's observations by cameras y < x precede a
          const int y = base_cam[o];
          if (cnt[y]++ == 0) touched.push_back(y);
        }
      }
      std::sort(touched.begin(), touched.end());
      part[x].resize(touched.size());
      for (size_t t = 0; t < touched.size(); ++t) {
        part[x][t] = make_int2(touched[t], cnt[touched[t]]);
        cnt[touched[t]] = 0;
      }
    }
  });
  g.edge_off.assign(m + 1, 0);
  for (int x = 0; x < m; ++x) g.edge_off[x + 1] = g.edge_off[x] + (int)part[x].size();
  const int E = g.edge_off[m];
  g.edge_y.resize(E);
  g.edge_w.resize(E);
  g.pair_off.assign(E + 1, 0);
  for (int x = 0; x < m; ++x)
    for (size_t t = 0; t < part[x].size(); ++t) {
      const int e = g.edge_off[x] + (int)t;
      g.edge_y[e] = part[x][t].x;
      g.edge_w[e] = part[x][t].y;
      g.pair_off[e + 1] = part[x][t].y;
    }
  for (int e = 0; e < E; ++e) g.pair_off[e + 1] += g.pair_off[e];
  if (!with_pairs) return;
  g.pairs.resize(g.pair_off[E]);
  // pass 2: the observation pairs of every edge, ordered by point
  parallel_ranges(m, [&](int xb, int xe) {
    std::vector<int64_t> cur(m, 0);
    for (int x = xb; x < xe; ++x) {
      for (int t = g.edge_off[x]; t < g.edge_off[x + 1]; ++t) cur[g.edge_y[t]] = g.pair_off[t];
      for (int e = cam_off[x]; e < cam_off[x + 1]; ++e) {
        const int a = cam_pos[e], b = pt_off[base_pt[a]];
        for (int o = b; o < a; ++o) g.pairs[cur[base_cam[o]]++] = make_int2(a, o);
      }
    }
  });
}

// ------------------------------------------------------------------------------------------------------
// Stochastic graph clustering (Sec. 4.4).  Clusters start as single cameras and are joined one pair at a
// time; a join of neighbouring clusters X, Y (at least one camera edge between them, |X| + |Y| <= Gamma)
// is drawn with probability proportional to exp(beta dQ(X, Y)) (Eq. 16), dQ being the increase of the
// modularity Q = 1/(2s) sum over edges of delta(nu_i, nu_j) (w_ij - k_i k_j / (2s)), i.e.
// dQ(X, Y) = (W_XY - P_XY / (2s)) / (2s) with W_XY the weight and P_XY the sum of k_i k_j over the camera
// edges between X and Y.  The process ends when no join is allowed.
//
// Sampling: every neighbouring cluster pair has one record (W, P and its two clusters, which are always
// the current roots); the records of allowed pairs are in a list.  An entry drawn uniformly is accepted
// with probability exp(beta (dQ - B)), B >= every dQ of the list, which makes the accepted pair follow
// Eq. 16 exactly (rejection sampling).  Entries whose record died (merged into another pair) or whose pair
// stopped being allowed (a side grew; sizes only grow) are removed when drawn.  B is the largest dQ seen
// so far; after a run of rejections it is recomputed from the list.
//
// A join moves the records of the cluster with the shorter record list to the other cluster: a record
// (small, z) merges into the existing record (big, z), or becomes (big, z).  The existing record is found
// without a global table for the pairs that never moved: a pair of current roots (big, z) is either the
// untouched camera edge big-z (every camera edge keeps its record until one of its two cameras stops
// being a root) or a record that moved, and moved records are kept in a small table keyed by their two
// roots.  The camera edges of camera `big` are marked in a per-camera array during the join, so that
// lookup touches no memory outside the walked records but the small table.  The initial records and the
// camera-edge lists are the same for every draw and are built once per graph.
namespace {

struct SplitMix64 {   // Steele, Lea and Flood, "Fast splittable pseudorandom number generators" (2014)
  uint64_t x;
  uint64_t next() {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }   // [0, 1)
  size_t below(size_t n) { return (size_t)(uniform() * (double)n); }
};

// (cluster, cluster) -> record of a moved pair; linear probing, key and value in one 16-byte slot.  Keys
// are never erased: a key whose cluster stopped being a root is never asked for again (cluster ids are
// camera ids and a joined cluster never comes back), and the rehash drops such keys.
struct MovedTable {
  static constexpr uint64_t EMPTY = ~0ull;
  struct Slot {
    uint64_t key;
    int64_t val;
  };
  std::vector<Slot> slot;
  size_t mask = 0, used = 0;
  static uint64_t key_of(int a, int b) {
    return a < b ? ((uint64_t)(uint32_t)a << 32) | (uint32_t)b : ((uint64_t)(uint32_t)b << 32) | (uint32_t)a;
  }
  static size_t hash(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    return (size_t)x;
  }
  void init(size_t n) {   // room for n keys at a load of at most 1/2
    size_t cap = 16;
    while (cap < 2 * n) cap <<= 1;
    slot.assign(cap, Slot{EMPTY, -1});
    mask = cap - 1;
    used = 0;
  }
  int find(int a, int b) const {
    const uint64_t x = key_of(a, b);
    for (size_t i = hash(x) & mask;; i = (i + 1) & mask) {
      if (slot[i].key == x) return (int)slot[i].val;
      if (slot[i].key == EMPTY) return -1;
    }
  }
  void insert(int a, int b, int v) {   // the key must be absent
    const uint64_t x = key_of(a, b);
    size_t i = hash(x) & mask;
    while (slot[i].key != EMPTY) i = (i + 1) & mask;
    ++used;
    slot[i] = Slot{x, v};
  }
};

struct alignas(32) PairRec {   // a neighbouring cluster pair: its clusters (a = -1 once dead) and W, P
  int a, b;
  double W, P;
};

std::mutex g_sgc_base_mutex;

}  // namespace

// The state every draw on one graph starts from (read-only, shared by the draws of a batch).
struct SgcBase {
  int m = 0, E = 0;
  double two_s = 0.0, B0 = -INFINITY;   // 2 s, and the largest dQ over the camera edges
  std::vector<PairRec> rec;              // one record per camera edge
  std::vector<int> inc_off;              // camera -> its camera edges (CSR)
  std::vector<int2> inc;                 // (camera edge, partner camera)
};

static std::shared_ptr<const SgcBase> sgc_base(const CameraGraph& g, int m) {
  std::lock_guard<std::mutex> lock(g_sgc_base_mutex);
  if (g.sgc_base) return g.sgc_base;
  auto S = std::make_shared<SgcBase>();
  const int E = (int)g.edge_y.size();
  S->m = m;
  S->E = E;
  std::vector<double> k(m, 0.0);
  S->inc_off.assign(m + 1, 0);
  double s = 0.0;
  for (int x = 0; x < m; ++x)
    for (int e = g.edge_off[x]; e < g.edge_off[x + 1]; ++e) {
      const int y = g.edge_y[e];
      k[x] += g.edge_w[e];
      k[y] += g.edge_w[e];
      S->inc_off[x + 1]++;
      S->inc_off[y + 1]++;
      s += g.edge_w[e];
    }
  for (int x = 0; x < m; ++x) S->inc_off[x + 1] += S->inc_off[x];
  S->inc.resize(2 * (size_t)E);
  std::vector<int> fill(S->inc_off.begin(), S->inc_off.end() - 1);
  S->rec.resize(E);
  S->two_s = 2.0 * s;
  for (int x = 0; x < m; ++x)
    for (int e = g.edge_off[x]; e < g.edge_off[x + 1]; ++e) {
      const int y = g.edge_y[e];
      S->rec[e] = PairRec{x, y, (double)g.edge_w[e], k[x] * k[y]};
      S->inc[fill[x]++] = make_int2(e, y);
      S->inc[fill[y]++] = make_int2(e, x);
      S->B0 = std::max(S->B0, (S->rec[e].W - S->rec[e].P / S->two_s) / S->two_s);
    }
  g.sgc_base = S;
  return S;
}

static void sgc_draw(const SgcBase& S, int gamma, double beta, uint64_t seed, int* labels, int* nclusters) {
  const int m = S.m, E = S.E;
  const double two_s = S.two_s;
  auto dq = [&](const PairRec& e) { return (e.W - e.P / two_s) / two_s; };
  std::vector<PairRec> rec(S.rec);
  std::vector<int> parent(m), size(m, 1), mark(m, -1);
  for (int i = 0; i < m; ++i) parent[i] = i;
  std::vector<std::vector<int>> extra(m);   // records moved to a cluster (besides its camera's edges)
  MovedTable moved;
  moved.init(1024);
  std::vector<int> list;   // entries: allowed pairs (and, until drawn, dead or no longer allowed ones)
  if (gamma >= 2) {
    list.resize(E);
    for (int e = 0; e < E; ++e) list[e] = e;
  }
  double B = S.B0;
  auto rehash = [&]() {   // keep the keys whose two clusters still exist
    MovedTable nt;
    nt.init(std::max<size_t>(1024, 2 * moved.used));
    for (const auto& sl : moved.slot)
      if (sl.key != MovedTable::EMPTY) {
        const int x = (int)(sl.key >> 32), y = (int)(sl.key & 0xffffffffu);
        if (parent[x] == x && parent[y] == y) nt.insert(x, y, (int)sl.val);
      }
    moved = std::move(nt);
  };
  SplitMix64 rng{seed};
  int rejections = 0;
  std::vector<int> walk;
  // The positions of the next AHEAD draws are drawn early, so that their list entries and then their
  // records are fetched while earlier draws are processed (each a random access into arrays of many MB).
  // A position is drawn uniformly over the list as it is at that moment and used when its turn comes if
  // the list still reaches it, else a fresh position is drawn: the list changes in between only through
  // the entries processed meanwhile, which do not depend on the pending positions, so every draw stays
  // uniform over the current list.
  constexpr int AHEAD = 16;
  size_t ahead[AHEAD] = {};
  int head = 0;
  if (!list.empty())
    for (int k = 0; k < AHEAD; ++k) {
      ahead[k] = rng.below(list.size());
      __builtin_prefetch(&list[ahead[k]]);
    }
  while (!list.empty()) {
    size_t r = ahead[head] < list.size() ? ahead[head] : rng.below(list.size());
    ahead[head] = rng.below(list.size());
    __builtin_prefetch(&list[ahead[head]]);
    head = head + 1 == AHEAD ? 0 : head + 1;
    {   // the entry fetched half a window ago: fetch its record now
      const size_t mid = ahead[(head + AHEAD / 2) % AHEAD];
      if (mid < list.size()) __builtin_prefetch(&rec[list[mid]]);
    }
    const int ei = list[r];
    PairRec& e = rec[ei];
    if (e.a < 0 || size[e.a] + size[e.b] > gamma) {   // merged into another pair, or no longer allowed
      list[r] = list.back();
      list.pop_back();
      continue;
    }
    if (!(rng.uniform() < std::exp(beta * (dq(e) - B)))) {
      if (++rejections >= 64) {   // tighten the bound to the largest dQ still in the list
        double nb = -INFINITY;
        for (size_t t = 0; t < list.size();) {
          const PairRec& f = rec[list[t]];
          if (f.a < 0 || size[f.a] + size[f.b] > gamma) {
            list[t] = list.back();
            list.pop_back();
            continue;
          }
          nb = std::max(nb, dq(f));
          ++t;
        }
        B = nb;
        rejections = 0;
      }
      continue;
    }
    rejections = 0;
    list[r] = list.back();
    list.pop_back();
    // join: the records of the cluster with the shorter list move to the other one
    int big = e.a, small = e.b;
    auto len = [&](int x) { return (size_t)(S.inc_off[x + 1] - S.inc_off[x]) + extra[x].size(); };
    if (len(big) < len(small)) std::swap(big, small);
    e.a = -1;
    walk.clear();
    for (int u = S.inc_off[small]; u < S.inc_off[small + 1]; ++u) walk.push_back(S.inc[u].x);
    walk.insert(walk.end(), extra[small].begin(), extra[small].end());
    std::vector<int>().swap(extra[small]);
    for (int u = S.inc_off[big]; u < S.inc_off[big + 1]; ++u) mark[S.inc[u].y] = S.inc[u].x;
    const int nw = (int)walk.size();
    constexpr int D = 8;   // records are fetched D entries ahead of their use
    for (int i = 0; i < std::min(nw, D); ++i) __builtin_prefetch(&rec[walk[i]]);
    for (int i = 0; i < nw; ++i) {
      if (i + D < nw) __builtin_prefetch(&rec[walk[i + D]]);
      PairRec& f = rec[walk[i]];
      if (f.a < 0) continue;
      const int z = f.a == small ? f.b : f.a;
      int t = mark[z];   // the camera edge big-z, untouched while both are roots
      if (t < 0) t = moved.find(big, z);
      if (t >= 0) {   // both sides touch z: the two cluster pairs become one
        rec[t].W += f.W;
        rec[t].P += f.P;
        f.a = -1;
        B = std::max(B, dq(rec[t]));
      } else {
        if (f.a == small) f.a = big; else f.b = big;
        moved.insert(big, z, walk[i]);
        extra[big].push_back(walk[i]);
      }
    }
    for (int u = S.inc_off[big]; u < S.inc_off[big + 1]; ++u) mark[S.inc[u].y] = -1;
    parent[small] = big;
    size[big] += size[small];
    if (2 * moved.used > moved.mask) rehash();
  }
  // clusters numbered by their smallest camera
  auto root = [&](int i) {
    while (parent[i] != i) i = parent[i] = parent[parent[i]];
    return i;
  };
  std::vector<int> id(m, -1);
  int l = 0;
  for (int i = 0; i < m; ++i) {
    const int r = root(i);
    if (id[r] < 0) id[r] = l++;
    labels[i] = id[r];
  }
  *nclusters = l;
}

void sgc_sample(const CameraGraph& g, int m, int gamma, double beta, uint64_t seed, int* labels, int* nclusters) {
  const auto S = sgc_base(g, m);
  sgc_draw(*S, gamma, beta, seed, labels, nclusters);
}

void sgc_sample_batch(const CameraGraph& g, int m, int gamma, double beta, uint64_t seed, int count, int* labels,
                      int* nclusters) {
  const auto S = sgc_base(g, m);
  parallel_ranges(count * 64, [&](int b, int e) {
    for (int t = (b + 63) / 64; t < (e + 63) / 64 && t < count; ++t)
      sgc_draw(*S, gamma, beta, seed + (uint64_t)t, labels + (size_t)t * m, nclusters + t);
  });
}

}  // namespace stba
