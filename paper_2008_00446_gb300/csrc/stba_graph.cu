// Camera graph of a problem (host code).  Two cameras are joined when they observe a common point; the
// edge lists, once, every such pair of observations.  The graph does not depend on the cluster assignment:
// under any assignment the off-diagonal blocks of the clustered reduced camera systems (Eq. 10, 13) are
// sums over exactly the edge pairs whose two cameras share a cluster, and its edge weights (the number of
// co-visible points) are those of the camera graph that stochastic graph clustering samples from (Sec. 4.4).
#include <algorithm>
#include <cmath>
#include <cstdint>
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
// Sampling: the allowed cluster pairs are kept in a list, one entry each; an entry drawn uniformly is
// accepted with probability exp(beta (dQ - B)), B >= every dQ of the list, which makes the accepted pair
// follow Eq. 16 exactly (rejection sampling).  Pairs that stopped being allowed (a side grew) are dropped
// from the list when drawn, since sizes only grow.  B is the largest dQ seen so far; after a run of
// rejections it is recomputed from the list.  Cluster pairs are found through one open-addressing table
// keyed by the two cluster ids; every cluster keeps the list of its incident pair records, and a join
// walks the shorter list of the two.
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

struct JoinEdge {
  int a, b;       // clusters (root cameras)
  double W, P;    // sum of w_ij and of k_i k_j over the camera edges between them
  int pos;        // index in the list of allowed pairs, -1 once it is dropped
  bool alive;
};

// (cluster, cluster) -> pair record; linear probing with tombstones, rebuilt when half full
struct PairTable {
  static constexpr uint64_t EMPTY = ~0ull, TOMB = ~0ull - 1;
  std::vector<uint64_t> key;
  std::vector<int> val;
  size_t mask = 0, used = 0;
  static uint64_t k(int a, int b) {
    return a < b ? ((uint64_t)(uint32_t)a << 32) | (uint32_t)b : ((uint64_t)(uint32_t)b << 32) | (uint32_t)a;
  }
  static size_t h(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    return (size_t)x;
  }
  void init(size_t n) {
    size_t cap = 16;
    while (cap < 4 * n) cap <<= 1;
    key.assign(cap, EMPTY);
    val.assign(cap, -1);
    mask = cap - 1;
    used = 0;
  }
  int find(int a, int b) const {
    const uint64_t x = k(a, b);
    for (size_t i = h(x) & mask;; i = (i + 1) & mask) {
      if (key[i] == x) return val[i];
      if (key[i] == EMPTY) return -1;
    }
  }
  void insert(int a, int b, int v) {   // the key must be absent
    const uint64_t x = k(a, b);
    size_t i = h(x) & mask;
    while (key[i] != EMPTY && key[i] != TOMB) i = (i + 1) & mask;
    if (key[i] == EMPTY) ++used;
    key[i] = x;
    val[i] = v;
  }
  void erase(int a, int b) {
    const uint64_t x = k(a, b);
    for (size_t i = h(x) & mask;; i = (i + 1) & mask) {
      if (key[i] == x) {
        key[i] = TOMB;
        return;
      }
      if (key[i] == EMPTY) return;
    }
  }
};

}  // namespace

void sgc_sample(const CameraGraph& g, int m, int gamma, double beta, uint64_t seed, int* labels, int* nclusters) {
  const int E = (int)g.edge_y.size();
  std::vector<double> k(m, 0.0);
  std::vector<int> deg(m, 0);
  double s = 0.0;
  for (int x = 0; x < m; ++x)
    for (int e = g.edge_off[x]; e < g.edge_off[x + 1]; ++e) {
      const int y = g.edge_y[e];
      k[x] += g.edge_w[e];
      k[y] += g.edge_w[e];
      deg[x]++;
      deg[y]++;
      s += g.edge_w[e];
    }
  std::vector<int> parent(m), size(m, 1);
  for (int i = 0; i < m; ++i) parent[i] = i;
  std::vector<JoinEdge> edges(E);
  std::vector<std::vector<int>> inc(m);
  for (int i = 0; i < m; ++i) inc[i].reserve(deg[i]);
  PairTable table;
  table.init(E);
  std::vector<int> list;
  list.reserve(E);
  const double two_s = 2.0 * s;
  auto dq = [&](const JoinEdge& e) { return (e.W - e.P / two_s) / two_s; };
  double B = -INFINITY;
  for (int x = 0; x < m; ++x)
    for (int e = g.edge_off[x]; e < g.edge_off[x + 1]; ++e) {
      const int y = g.edge_y[e];
      edges[e] = JoinEdge{x, y, (double)g.edge_w[e], k[x] * k[y], -1, true};
      inc[x].push_back(e);
      inc[y].push_back(e);
      table.insert(x, y, e);
      if (gamma >= 2) {
        edges[e].pos = (int)list.size();
        list.push_back(e);
        B = std::max(B, dq(edges[e]));
      }
    }
  auto drop = [&](int e) {   // O(1) removal from the list of allowed pairs
    const int p = edges[e].pos;
    if (p < 0) return;
    const int last = list.back();
    list[p] = last;
    edges[last].pos = p;
    list.pop_back();
    edges[e].pos = -1;
  };
  auto rebuild = [&]() {
    table.init(E);
    for (int e = 0; e < E; ++e)
      if (edges[e].alive) table.insert(edges[e].a, edges[e].b, e);
  };
  SplitMix64 rng{seed};
  int rejections = 0;
  while (!list.empty()) {
    const size_t r = rng.below(list.size());
    const int ei = list[r];
    JoinEdge& e = edges[ei];
    if (size[e.a] + size[e.b] > gamma) {   // a side grew past the cap: no longer an allowed join
      drop(ei);
      continue;
    }
    const double d = dq(e);
    if (!(rng.uniform() < std::exp(beta * (d - B)))) {
      if (++rejections >= 64) {   // tighten the bound to the largest dQ still in the list
        double nb = -INFINITY;
        for (size_t t = 0; t < list.size();) {
          const JoinEdge& f = edges[list[t]];
          if (size[f.a] + size[f.b] > gamma) {
            drop(list[t]);
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
    // join: the records of the cluster with the shorter list move to the other one
    int big = e.a, small = e.b;
    if (inc[big].size() < inc[small].size()) std::swap(big, small);
    e.alive = false;
    drop(ei);
    table.erase(big, small);
    for (const int ez : inc[small]) {
      JoinEdge& f = edges[ez];
      if (!f.alive) continue;
      const int z = f.a == small ? f.b : f.a;
      table.erase(small, z);
      const int t = table.find(big, z);
      if (t >= 0) {   // both sides touch z: the two cluster pairs become one
        edges[t].W += f.W;
        edges[t].P += f.P;
        f.alive = false;
        drop(ez);
        B = std::max(B, dq(edges[t]));
      } else {
        if (f.a == small) f.a = big; else f.b = big;
        table.insert(big, z, ez);
        inc[big].push_back(ez);
      }
    }
    std::vector<int>().swap(inc[small]);
    parent[small] = big;
    size[big] += size[small];
    if (2 * table.used > table.mask) rebuild();
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

void sgc_sample_batch(const CameraGraph& g, int m, int gamma, double beta, uint64_t seed, int count, int* labels,
                      int* nclusters) {
  parallel_ranges(count * 64, [&](int b, int e) {
    for (int t = (b + 63) / 64; t < (e + 63) / 64 && t < count; ++t)
      sgc_sample(g, m, gamma, beta, seed + (uint64_t)t, labels + (size_t)t * m, nclusters + t);
  });
}

}  // namespace stba
