// Camera graph of a problem (host code).  Two cameras are joined when they observe a common point; the
// edge lists, once, every such pair of observations.  The graph does not depend on the cluster assignment:
// under any assignment the off-diagonal blocks of the clustered reduced camera systems (Eq. 10, 13) are
// sums over exactly the edge pairs whose two cameras share a cluster, and its edge weights (the number of
// co-visible points) are those of the camera graph that stochastic graph clustering samples from (Sec. 4.4).
#include <algorithm>
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
void build_camera_graph(int m, int n, const std::vector<int>& pt_off, const std::vector<int>& base_cam,
                        CameraGraph& g) {
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

}  // namespace stba
