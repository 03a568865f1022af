// C ABI of libstba.so (include/stba.h): context management, host-side preprocessing of the visibility
// graph for a cluster assignment, and the enqueue of one LM iteration (Algorithm 1) on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "stba_internal.cuh"

using namespace stba;

namespace {

thread_local std::string g_create_error;   // message of the last failed stba_create on this thread

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct GrowBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct stba_ctx {
  stba_options opt{};
  Settings set{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  // re-ordering graphs of the two buffer states (argument bytes -> executable graph)
  std::vector<unsigned char> reorder_key[2];
  cudaGraphExec_t reorder_exec[2] = {nullptr, nullptr};
  int reorder_next = 0;
  cudaStream_t side_stream = nullptr;           // trailing updates of the factorisation
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_rfork = nullptr, ev_rjoin = nullptr;   // the re-ordering's side branch (chunk listing)
  cudaEvent_t ev_sfork = nullptr, ev_sjoin = nullptr;   // the S' build's side branch (pair pass)
  cudaEvent_t ev_copy = nullptr;                        // the factorisation's scaled copy beside panel 0
  std::vector<cudaEvent_t> ev_panel, ev_update;  // one per tile step (grown, never shrunk)
  std::string err;
  int64_t m = 0, n = 0, q = 0;
  int l = 0, nv = 0;
  bool mixed = false;
  bool f32f = false;                   // the cluster factor is FP32 (mixed precision without factor_fp64)
  size_t bytes_base = 0;
  std::vector<void*> allocs;            // problem-lifetime device buffers

  // host copies of the input observations (original order) and the (point, camera) order
  std::vector<int> in_cam, in_pt;
  std::vector<double> in_uv;
  std::vector<int> base_order;          // observation indices sorted by (point, camera)
  std::vector<int> h_pt_off;            // [n+1]

  // host structures of the current cluster assignment
  std::vector<int> h_clusters, h_cluster_cams, h_cluster_cam_off, h_np, h_nk;
  std::vector<int64_t> h_S_off, h_v_off;
  std::vector<int> h_panel_off, h_update_off;
  int64_t S_total = 0, v_total = 0;
  int max_np = 0;
  int build_items = 0;

  // device arrays
  double *cams = nullptr, *pts = nullptr, *obs_uv = nullptr;
  float* obs_uvf = nullptr;
  int *obs_cam = nullptr, *obs_vp = nullptr, *obs_pt = nullptr, *obs_perm = nullptr, *obs_base = nullptr;
  int *vp_off = nullptr, *vp_point = nullptr, *pt_vp_off = nullptr, *pt_off = nullptr;
  int *cam_local = nullptr, *cam_cluster = nullptr, *cluster_cams = nullptr, *cluster_cam_off = nullptr;
  int *cluster_np = nullptr, *cluster_n = nullptr;
  int64_t *S_off = nullptr, *v_off = nullptr;
  CamLists clist{};
  CamSlots cslots{};
  PairChunks pchunks{};
  CameraGraph cgraph;                   // camera graph with its observation pairs (host copy)
  void* Gbuf = nullptr;
  // re-ordering for new assignments: fixed arguments, the two inverse maps (previous / current), scratch
  ReorderArgs reorder{};
  int* inv[2] = {nullptr, nullptr};
  int inv_cur = 0;
  bool have_order = false;               // an assignment is in place (its residual order is defined)
  int *key = nullptr, *tile_sum = nullptr;
  long long* counts = nullptr;
  // buffers sized by the cluster layout, kept while the next layout fits
  GrowBuf g_panel, g_update, g_res, g_diag, g_S, g_b, g_L, g_Dinv, g_Ldiag, g_scale, g_x, g_r, g_blob;
  // pinned staging of the per-assignment arrays (two, used in turn; an event marks each one's copy)
  void* stage_h[2] = {nullptr, nullptr};
  size_t stage_bytes[2] = {0, 0};
  cudaEvent_t stage_ev[2] = {nullptr, nullptr};
  int stage_cur = 0;
  bool counts_known = true;             // c->nv and c->n_pairs read back since the last assignment
  int64_t n_pairs = 0;
  CholPlan cplan{};
  FactorBuffers fbuf{};
  bool use_pcg = false;                 // STBA_SOLVER_PCG_FULL: no cluster systems, CG on the full system
  bool use_spcg = false;                // STBA_SOLVER_PCG_CLUSTERS: the cluster systems by CG, matrix-free
  PcgBuffers pcg{};
  int* fail_flags = nullptr;

  // scratch (real = float in mixed mode, double in FP64 mode)
  void *vp_acc = nullptr, *vp_info = nullptr, *pt_info = nullptr, *pt_acc = nullptr, *S = nullptr, *b = nullptr, *vgrad = nullptr,
       *t_acc = nullptr;
  double *dc = nullptr, *dp = nullptr, *partial = nullptr, *cam_rt = nullptr;
  float *cam_df = nullptr, *pt_df = nullptr;   // double-float tables of the mixed-mode cost
  float *cams_f = nullptr, *pts_f = nullptr, *dcf = nullptr;   // FP32 copies (mixed precision)
  float4* obs_uvdf = nullptr;
  void *res_cur = nullptr, *res_cand = nullptr;   // residuals at x and at x + dx (working precision)
  DevState* st = nullptr;

  // tape of recorded iterations for stba_adjoint: x_t before every iteration, its record after it, and
  // the cluster assignment it used
  int tape_cap = 0, tape_len = 0;
  bool tape_broken = false;             // parameters or damping were replaced between recorded iterations
  double* tape_x = nullptr;             // [tape_cap][9m + 3n]
  stba_iter_info* tape_info = nullptr;  // [tape_cap]
  std::vector<int> tape_cluster_id;     // per recorded iteration, index into tape_clusters
  std::vector<std::vector<int>> tape_clusters;
  std::vector<void*> tape_allocs;
  AdjointBuffers adj{};                 // reverse-pass buffers, allocated with the tape
  double* adj_save_x = nullptr;         // [9m + 3n] the final parameters, kept across the reverse pass

  // graph / timing
  cudaGraphExec_t graph = nullptr;      // the current iteration graph, one of graph_cache
  // executable iteration graphs by launch structure (the number of tile steps and which launches each step
  // has vary between clusterings): a new clustering's capture updates the one of its structure in place
  std::vector<std::pair<uint64_t, cudaGraphExec_t>> graph_cache;
  bool graph_stale = false;             // the cluster layout changed since the graph was captured
  int tile = 32;                        // factorisation tile (stba_autotune may change the FP32 one)
  int update_tc = 0;                    // trailing updates on the tensor cores (FP32 factor, tile 64)
  int split_panel = 0;                  // split panel: diagonal-tile factor + inverse, then the tiles below
  int persistent = 0;                   // one persistent launch of 8-CTA clusters factors every cluster
  int solve_cs = 8;                     // CTAs per thread-block cluster of the cluster solves
  int panel_choice = STBA_FACTOR_PANEL_DEFAULT;   // option, or the autotuner's choice; DEFAULT decides per
                                                  // assignment (set_clusters_host)
  // sharded iteration (stba_set_shard): this process's rank among `shard_world`, the transport, the clusters
  // it owns under the current assignment (host and device), and the exchange buffers
  int shard_rank = 0, shard_world = 1, shard_host_staging = 1;
  stba_allreduce_fn shard_fn = nullptr;
  void* shard_user = nullptr;
  std::vector<int> h_owned;             // [l]
  std::vector<int> h_cam_nobs;          // [m] observations of every camera (the cost model of the ownership)
  int* cl_owned = nullptr;              // [m] device (l <= m); all 1 unless sharded
  double* xch = nullptr;                // [9 n + 1] device: point sums, then the failure count
  void* xch_host = nullptr;             // pinned staging of an exchange
  size_t xch_host_bytes = 0;
  std::vector<int> h_diag_count;        // split panel: diagonal items of every step
  bool capturing = false;
  bool timing = false;
  int launches_per_iter = 0;
  double factor_flops = 0;
  cudaEvent_t ev[NSTAGES + 1] = {};
  float stage_ms[NSTAGES] = {};
  bool have_stage_times = false;
};

namespace {

stba_status fail(stba_ctx* c, stba_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(c, STBA_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
stba_status dalloc(stba_ctx* c, T** p, size_t count) {
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(c, STBA_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  c->allocs.push_back((void*)*p);
  c->bytes_base += bytes;
  return STBA_OK;
}

template <typename T>
stba_status dalloc_into(stba_ctx* c, T** p, size_t count, std::vector<void*>& list) {
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(c, STBA_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  list.push_back((void*)*p);
  return STBA_OK;
}

template <typename T>
stba_status upload(stba_ctx* c, T** p, const std::vector<T>& h) {
  stba_status s = dalloc(c, p, h.size());
  if (s != STBA_OK) return s;
  if (!h.empty()) CK(cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
  return STBA_OK;
}

stba_status copy_in(stba_ctx* c, void* host_dst, const void* src, size_t bytes) {
  if (bytes == 0) return STBA_OK;
  if (is_device_ptr(src)) {
    CK(cudaMemcpy(host_dst, src, bytes, cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(host_dst, src, bytes);
  }
  return STBA_OK;
}

stba_status copy_out(stba_ctx* c, void* dst, const void* dev_src, size_t bytes) {
  if (bytes == 0 || !dst) return STBA_OK;
  CK(cudaMemcpyAsync(dst, dev_src, bytes, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return STBA_OK;
}

void free_list(stba_ctx* c, std::vector<void*>& v) {
  for (void* p : v) cudaFree(p);
  v.clear();
}

DevProblem dev_problem(const stba_ctx* c) {
  DevProblem P;
  P.m = (int)c->m;
  P.n = (int)c->n;
  P.q = (int)c->q;
  P.l = c->l;
  P.nv = c->nv;
  P.cams = c->cams;
  P.pts = c->pts;
  P.obs_cam = c->obs_cam;
  P.obs_vp = c->obs_vp;
  P.obs_pt = c->obs_pt;
  P.obs_base = c->obs_base;
  P.obs_uv = c->obs_uv;
  P.obs_uvf = c->obs_uvf;
  P.obs_uvdf = c->obs_uvdf;
  P.cams_f = c->cams_f;
  P.pts_f = c->pts_f;
  P.vp_off = c->vp_off;
  P.vp_point = c->vp_point;
  P.pt_vp_off = c->pt_vp_off;
  P.pt_off = c->pt_off;
  P.cam_local = c->cam_local;
  P.cam_cluster = c->cam_cluster;
  P.cluster_cams = c->cluster_cams;
  P.cluster_cam_off = c->cluster_cam_off;
  P.cluster_np = c->cluster_np;
  P.cluster_n = c->cluster_n;
  P.S_off = c->S_off;
  P.v_off = c->v_off;
  P.huber_a = c->opt.huber_a;
  P.res_f = c->mixed ? (const float*)c->res_cur : nullptr;
  P.res_d = c->mixed ? nullptr : (const double*)c->res_cur;
  P.base_pos = c->inv[c->inv_cur];
  P.pair_recompute = c->opt.pair_blocks == STBA_PAIR_BLOCKS_STORED ? 0 : 1;   // recomputed by default
  P.sharded = c->shard_world > 1 ? 1 : 0;
  P.cluster_owned = c->cl_owned;
  return P;
}

template <typename real>
Scratch<real> scratch(const stba_ctx* c) {
  Scratch<real> W;
  W.vp_acc = (real*)c->vp_acc;
  W.vp_info = (real*)c->vp_info;
  W.pt_info = (real*)c->pt_info;
  W.pt_acc = (real*)c->pt_acc;
  W.S = (double*)c->S;
  W.b = (double*)c->b;
  W.vgrad = (real*)c->vgrad;
  W.t_acc = (real*)c->t_acc;
  W.dc = c->dc;
  W.dcf = c->dcf;
  W.dp = c->dp;
  W.partial = c->partial;
  return W;
}


// ------------------------------------------------------------------------------------------------------
// Device buffer that keeps its allocation while a new size fits (grown by a quarter when it does not).
template <typename T>
stba_status ensure(stba_ctx* c, GrowBuf& g, T** p, size_t count) {
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  if (bytes > g.bytes) {
    if (g.ptr) cudaFree(g.ptr);
    g.ptr = nullptr;
    g.bytes = 0;
    const size_t want = bytes + bytes / 4;
    if (cudaMalloc(&g.ptr, want) != cudaSuccess) {
      cudaGetLastError();
      g.ptr = nullptr;
      return fail(c, STBA_ERR_OOM, "cudaMalloc of %zu bytes failed", want);
    }
    g.bytes = want;
  }
  *p = reinterpret_cast<T*>(g.ptr);
  return STBA_OK;
}

template <typename T>
stba_status put(stba_ctx* c, T* dst, const std::vector<T>& h) {
  if (!h.empty()) CK(cudaMemcpyAsync(dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
  return STBA_OK;
}

// The number of virtual points and of camera-pair instances of the current assignment (device counters
// written by the re-ordering); synchronises the stream the first time after a new assignment.
stba_status refresh_counts(stba_ctx* c) {
  if (c->counts_known) return STBA_OK;
  long long h[2];
  CK(cudaMemcpyAsync(h, c->counts, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->nv = (int)h[0];
  c->n_pairs = h[1];
  c->counts_known = true;
  return STBA_OK;
}

// ------------------------------------------------------------------------------------------------------
// A new cluster assignment.  The host validates it and lays out the clusters (camera lists, the dense
// blocks of S'_k, the Cholesky step plan: O(m + l + plan) work); the device re-orders the observations
// by (point, cluster, camera), numbers the virtual points (distinct (point, cluster) pairs) and rebuilds
// the camera lists (stba_order.cu), carrying the stored residuals over to the new order.
// The re-ordering kernels of an assignment.  Their launch shapes depend only on q, m and the number of
// camera-graph chunks, and their arguments on which of the two order and residual buffers are current, so
// after the first assignment two captured graphs (one per buffer state) serve every later one and replace
// about 16 dependent launches by one.  Captured on the private stream, launched on the context's.
static void enqueue_reorder(stba_ctx* c, const ReorderArgs& A, bool carry, cudaStream_t st) {
  if (c->mixed)
    launch_reorder<float>(A, c->key, c->tile_sum, c->counts, carry ? (const float*)c->res_cur : nullptr,
                          (float*)c->res_cand, st);
  else
    launch_reorder<double>(A, c->key, c->tile_sum, c->counts, carry ? (const double*)c->res_cur : nullptr,
                           (double*)c->res_cand, st);
}

// The re-ordering of an assignment with the listing of the camera-pair chunks inside clusters on a side
// branch: the listing reads only the new cluster ids, so its five launches overlap the re-ordering's.
static void enqueue_reorder_branches(stba_ctx* c, const ReorderArgs& A, bool carry, cudaStream_t st) {
  const bool chunks = !c->use_pcg && !c->use_spcg && c->pchunks.nchunks > 0;
  if (chunks) {
    cudaEventRecord(c->ev_rfork, st);
    cudaStreamWaitEvent(c->side_stream, c->ev_rfork, 0);
    launch_list_chunks(c->pchunks, c->cam_cluster, c->cl_owned, c->counts + 3, c->side_stream);
    cudaEventRecord(c->ev_rjoin, c->side_stream);
  }
  enqueue_reorder(c, A, carry, st);
  if (chunks) cudaStreamWaitEvent(st, c->ev_rjoin, 0);
}

static stba_status launch_reorder_graph(stba_ctx* c, const ReorderArgs& A, bool carry) {
  if (!c->opt.use_graph) {
    enqueue_reorder_branches(c, A, carry, c->stream);
    CK(cudaGetLastError());
    return STBA_OK;
  }
  // the argument bytes: ReorderArgs (padding after its three ints cleared) and the other arguments
  static_assert(offsetof(ReorderArgs, obs_pt) == 16, "ReorderArgs: three ints, then pointers");
  std::vector<unsigned char> key(sizeof(ReorderArgs));
  std::memcpy(key.data(), &A, sizeof A);
  std::memset(key.data() + 12, 0, 4);
  const void* more[] = {c->key, c->tile_sum, c->counts, carry ? c->res_cur : nullptr, c->res_cand,
                        c->pchunks.chunks, c->pchunks.active, c->pchunks.nactive, c->pchunks.flag,
                        c->pchunks.excl, c->pchunks.tile_sum, c->cam_cluster, c->cl_owned};
  const long long flags[] = {c->mixed, c->use_pcg || c->use_spcg, c->pchunks.nchunks};
  const unsigned char* m1 = reinterpret_cast<const unsigned char*>(more);
  const unsigned char* m2 = reinterpret_cast<const unsigned char*>(flags);
  key.insert(key.end(), m1, m1 + sizeof more);
  key.insert(key.end(), m2, m2 + sizeof flags);
  for (int i = 0; i < 2; ++i)
    if (c->reorder_exec[i] && c->reorder_key[i] == key) {
      CK(cudaGraphLaunch(c->reorder_exec[i], c->stream));
      return STBA_OK;
    }
  CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  enqueue_reorder_branches(c, A, carry, c->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  if (e != cudaSuccess) return fail(c, STBA_ERR_CUDA, "re-ordering capture failed: %s", cudaGetErrorString(e));
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(c, STBA_ERR_CUDA, "re-ordering graph: %s", cudaGetErrorString(e));
  const int slot = c->reorder_next;
  c->reorder_next ^= 1;
  if (c->reorder_exec[slot]) cudaGraphExecDestroy(c->reorder_exec[slot]);
  c->reorder_exec[slot] = x;
  c->reorder_key[slot] = std::move(key);
  CK(cudaGraphLaunch(x, c->stream));
  return STBA_OK;
}

stba_status set_clusters_host(stba_ctx* c, const std::vector<int>& cl) {
  const int m = (int)c->m, n = (int)c->n, q = (int)c->q;
  int l = 0;
  for (int j = 0; j < m; ++j) {
    if (cl[j] < 0 || cl[j] >= m) return fail(c, STBA_ERR_INVALID_ARG, "cluster id %d of camera %d out of range", cl[j], j);
    l = std::max(l, cl[j] + 1);
  }
  std::vector<int> cnt(l, 0);
  for (int j = 0; j < m; ++j) cnt[cl[j]]++;
  for (int k = 0; k < l; ++k)
    if (cnt[k] == 0) return fail(c, STBA_ERR_INVALID_ARG, "cluster %d has no camera (ids must be 0..l-1)", k);
  if (!c->use_pcg && !c->use_spcg) {   // the cluster solve keeps a cluster's vector in shared memory
    int big = 0;
    for (int k = 0; k < l; ++k) big = std::max(big, (9 * cnt[k] + c->tile - 1) / c->tile * c->tile);
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t need = solve_smem_bytes(c->f32f, c->tile, big);
    if (optin > 0 && need > (size_t)optin)
      return fail(c, STBA_ERR_INVALID_ARG,
                  "a cluster of %d unknowns needs %zu bytes of shared memory in the cluster solve (limit %d); "
                  "use smaller clusters or a PCG solver", big, need, optin);
  }

  c->graph_stale = true;   // recaptured by the next iteration (and updated in place when its shape allows)
  c->l = l;
  c->h_clusters = cl;
  // cameras of every cluster, ascending
  c->h_cluster_cam_off.assign(l + 1, 0);
  for (int k = 0; k < l; ++k) c->h_cluster_cam_off[k + 1] = c->h_cluster_cam_off[k] + cnt[k];
  c->h_cluster_cams.assign(m, 0);
  std::vector<int> cam_local(m), fill(l, 0);
  for (int j = 0; j < m; ++j) {
    const int k = cl[j];
    cam_local[j] = fill[k];
    c->h_cluster_cams[c->h_cluster_cam_off[k] + fill[k]] = j;
    fill[k]++;
  }
  // dense layout (padded to the factorisation tile TF)
  const int TF = c->tile;
  c->h_np.assign(l, 0);
  c->h_nk.assign(l, 0);
  c->h_S_off.assign(l, 0);
  c->h_v_off.assign(l, 0);
  int64_t so = 0, vo = 0;
  c->max_np = 0;
  int max_nt = 0;
  for (int k = 0; k < l; ++k) {
    const int nk = 9 * cnt[k];
    const int np = (nk + TF - 1) / TF * TF;
    c->h_nk[k] = nk;
    c->h_np[k] = np;
    c->h_S_off[k] = so;
    c->h_v_off[k] = vo;
    so += (int64_t)np * np;
    vo += np;
    c->max_np = std::max(c->max_np, np);
    max_nt = std::max(max_nt, np / TF);
  }
  c->S_total = so;
  c->v_total = vo;
  // ownership of the clusters (sharded iteration): longest processing time first by the cost model of one
  // iteration per cluster, (9 n_k)^3 / 3 + 2000 x (observations of its cameras); ties go to the lower
  // cluster id and the lower rank.  Every process computes the same owners from the same assignment.
  c->h_owned.assign(l, 1);
  if (c->shard_world > 1) {
    std::vector<double> cost(l, 0.0);
    for (int k = 0; k < l; ++k) cost[k] = std::pow(9.0 * cnt[k], 3) / 3.0;
    for (int j = 0; j < m; ++j) cost[cl[j]] += 2000.0 * c->h_cam_nobs[j];
    std::vector<int> order(l);
    for (int k = 0; k < l; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<double> load(c->shard_world, 0.0);
    for (int k : order) {
      int r = 0;
      for (int t = 1; t < c->shard_world; ++t)
        if (load[t] < load[r]) r = t;
      c->h_owned[k] = r == c->shard_rank ? 1 : 0;
      load[r] += cost[k];
    }
  }
  CK(cudaMemcpyAsync(c->cl_owned, c->h_owned.data(), (size_t)l * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  // panel of the FP32 factor with tile 64: the split panel pays off once a tile step's tiles outnumber the SMs
  // (several waves of panel CTAs per step; each of them would factor its diagonal tile again), the stacked
  // panel when they fit in one wave (a single kernel per step on the critical path)
  c->persistent = c->mixed && TF == 64 && c->panel_choice == STBA_FACTOR_PANEL_PERSISTENT;
  // CTAs per cluster solve: 8 while the solves' CTAs fit in about two waves (more CTAs share each tile step's
  // products), 4 beyond (cheaper barriers and exchanges once the solves queue for SMs anyway)
  c->solve_cs = c->opt.solve_cluster ? c->opt.solve_cluster : ((int64_t)l * 8 <= 2 * (int64_t)num_sms() ? 8 : 4);
  if (c->mixed && TF == 64 && c->panel_choice != STBA_FACTOR_PANEL_STACKED && !c->persistent) {
    int64_t tiles = 0;
    for (int k = 0; k < l; ++k) tiles += c->h_np[k] / TF;
    c->split_panel = c->panel_choice == STBA_FACTOR_PANEL_SPLIT || tiles > num_sms();
  } else {
    c->split_panel = 0;
  }
  c->build_items = c->use_pcg ? 0 : c->pchunks.nchunks;

  // Cholesky step plan (none for the PCG solver)
  if (c->use_pcg) {
    max_nt = 0;
    c->max_np = 0;
    c->S_total = 0;
    c->v_total = 0;
  }
  std::vector<int2> panel, update;
  c->h_panel_off.assign(max_nt + 1, 0);
  c->h_update_off.assign(max_nt + 1, 0);
  c->h_diag_count.assign(max_nt + 1, 0);
  for (int kt = 0; kt < max_nt; ++kt) {
    c->h_panel_off[kt] = (int)panel.size();
    c->h_update_off[kt] = (int)update.size();
    if (c->split_panel)   // the diagonal tiles of the step first
      for (int k = 0; k < l; ++k)
        if (c->h_np[k] / TF > kt && c->h_owned[k]) {
          panel.push_back(make_int2(k, kt));
          c->h_diag_count[kt]++;
        }
    for (int k = 0; k < l; ++k) {
      const int ntk = c->h_np[k] / TF;
      if (ntk <= kt || !c->h_owned[k]) continue;   // sharded: the other processes' clusters
      for (int i = c->split_panel ? kt + 1 : kt; i < ntk; ++i) panel.push_back(make_int2(k, i));
      for (int j = kt + 2; j < ntk; ++j) {   // column kt + 1 is updated by panel kt + 1 itself
        if (c->update_tc)   // tile pairs (i0, i0 + 1) x j, from the diagonal tile down
          for (int i0 = j; i0 < ntk; i0 += 2) update.push_back(make_int2(k, (i0 << 16) | j));
        else
          for (int i = j; i < ntk; ++i) update.push_back(make_int2(k, (i << 16) | j));
      }
    }
  }
  c->h_panel_off[max_nt] = (int)panel.size();
  c->h_update_off[max_nt] = (int)update.size();
  std::vector<int2> res_items, diag_items;
  std::vector<int> cluster_items;   // the clusters this process factors (persistent launch)
  for (int k = 0; k < l; ++k)
    if (c->h_owned[k]) cluster_items.push_back(k);
  for (int k = 0; k < l && !c->use_pcg; ++k)
    if (c->h_owned[k])
      for (int rb = 0; rb < (c->h_nk[k] + 31) / 32; ++rb) res_items.push_back(make_int2(k, rb));
  for (int k = 0; k < l && !c->use_pcg; ++k)
    if (c->h_owned[k])
      for (int t = 0; t < c->h_np[k] / TF; ++t) diag_items.push_back(make_int2(k, t));
  while ((int)c->ev_panel.size() < max_nt) {
    cudaEvent_t e1, e2;
    if (cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&e2, cudaEventDisableTiming) != cudaSuccess)
      return fail(c, STBA_ERR_CUDA, "cudaEventCreate failed");
    c->ev_panel.push_back(e1);
    c->ev_update.push_back(e2);
  }
  {
    int factor_launches = 3;
    for (int kt = 0; kt < max_nt; ++kt)
      factor_launches += (c->h_panel_off[kt + 1] > c->h_panel_off[kt]) + (c->h_update_off[kt + 1] > c->h_update_off[kt]);
    const int build_launches = 1 + (c->pchunks.nchunks > 0 && l < m ? 1 : 0);
    const int solve_launches = 2 + c->set.refine_steps * (2 + (res_items.empty() ? 0 : 1));
    // iter_begin, vp_reduce, pt_acc, vp_finalize | build | factor | solve, count | rhs, update, cam_rt,
    // (cam_df, point_df,) cost, finalize, apply
    c->launches_per_iter = 4 + build_launches + factor_launches + solve_launches + 1 + 6 + (c->mixed ? 3 : 0);
    c->factor_flops = 0;
    for (int k = 0; k < l; ++k) c->factor_flops += std::pow((double)c->h_nk[k], 3) / 3.0;
  }

  // cluster arrays and plan: packed into one pinned staging buffer and copied with one transfer into a
  // device blob; the arrays are views of the blob
  stba_status s;
  {
    size_t bytes = 0;
    auto seg = [&](size_t n_bytes) {
      const size_t o = bytes;
      bytes += (n_bytes + 15) / 16 * 16;
      return o;
    };
    const size_t o_local = seg(4 * (size_t)m), o_cl = seg(4 * (size_t)m), o_ccams = seg(4 * (size_t)m),
                 o_coff = seg(4 * ((size_t)l + 1)), o_np = seg(4 * (size_t)l), o_nk = seg(4 * (size_t)l),
                 o_soff = seg(8 * (size_t)l), o_voff = seg(8 * (size_t)l), o_panel = seg(8 * panel.size()),
                 o_update = seg(8 * update.size()), o_res = seg(8 * res_items.size()),
                 o_diag = seg(8 * diag_items.size()), o_citems = seg(4 * cluster_items.size());
    const int sb = c->stage_cur;
    c->stage_cur = 1 - sb;
    if (c->stage_bytes[sb] < bytes) {
      if (c->stage_h[sb]) {
        CK(cudaEventSynchronize(c->stage_ev[sb]));
        cudaFreeHost(c->stage_h[sb]);
        c->stage_h[sb] = nullptr;
        c->stage_bytes[sb] = 0;
      }
      if (cudaHostAlloc(&c->stage_h[sb], bytes + bytes / 4, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        c->stage_h[sb] = nullptr;
        return fail(c, STBA_ERR_OOM, "pinned host allocation failed");
      }
      c->stage_bytes[sb] = bytes + bytes / 4;
    } else {
      CK(cudaEventSynchronize(c->stage_ev[sb]));   // its previous copy has been consumed
    }
    char* h = (char*)c->stage_h[sb];
    auto pack = [&](size_t o, const void* src, size_t n_bytes) {
      if (n_bytes) std::memcpy(h + o, src, n_bytes);
    };
    pack(o_local, cam_local.data(), 4 * (size_t)m);
    pack(o_cl, cl.data(), 4 * (size_t)m);
    pack(o_ccams, c->h_cluster_cams.data(), 4 * (size_t)m);
    pack(o_coff, c->h_cluster_cam_off.data(), 4 * ((size_t)l + 1));
    pack(o_np, c->h_np.data(), 4 * (size_t)l);
    pack(o_nk, c->h_nk.data(), 4 * (size_t)l);
    pack(o_soff, c->h_S_off.data(), 8 * (size_t)l);
    pack(o_voff, c->h_v_off.data(), 8 * (size_t)l);
    pack(o_panel, panel.data(), 8 * panel.size());
    pack(o_update, update.data(), 8 * update.size());
    pack(o_res, res_items.data(), 8 * res_items.size());
    pack(o_diag, diag_items.data(), 8 * diag_items.size());
    pack(o_citems, cluster_items.data(), 4 * cluster_items.size());
    char* d = nullptr;
    if ((s = ensure(c, c->g_blob, &d, bytes)) != STBA_OK) return s;
    CK(cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, c->stream));
    CK(cudaEventRecord(c->stage_ev[sb], c->stream));
    c->cam_local = (int*)(d + o_local);
    c->cam_cluster = (int*)(d + o_cl);
    c->cluster_cams = (int*)(d + o_ccams);
    c->cluster_cam_off = (int*)(d + o_coff);
    c->cluster_np = (int*)(d + o_np);
    c->cluster_n = (int*)(d + o_nk);
    c->S_off = (int64_t*)(d + o_soff);
    c->v_off = (int64_t*)(d + o_voff);
    c->reorder.cam_cluster = c->cam_cluster;
    const int2 *d_panel = (const int2*)(d + o_panel), *d_update = (const int2*)(d + o_update),
               *d_res = (const int2*)(d + o_res), *d_diag = (const int2*)(d + o_diag);
    c->cplan = CholPlan{d_panel, d_update, d_res, (int)res_items.size(), d_diag, (int)diag_items.size(), max_nt,
                        c->h_panel_off.data(),
                        c->h_update_off.data(), c->max_np, c->side_stream, 0, 0, c->ev_fork, c->ev_join,
                        c->ev_copy, c->ev_panel.data(), c->ev_update.data(), TF, c->update_tc, c->split_panel,
                        c->h_diag_count.data(), c->persistent, (const int*)(d + o_citems),
                        (int)cluster_items.size(), c->solve_cs};
  }
  {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) cudaGetLastError();
    c->cplan.prio_high = greatest;
    c->cplan.prio_low = least;
  }
  // cluster systems and factor storage
  const size_t rs = c->f32f ? sizeof(float) : sizeof(double);   // the factor's reals
  {
    double *S_, *b_;
    char *L_, *Dinv_, *Ldiag_;
    if ((s = ensure(c, c->g_S, &S_, (size_t)c->S_total)) != STBA_OK) return s;
    if ((s = ensure(c, c->g_b, &b_, (size_t)c->v_total)) != STBA_OK) return s;
    if ((s = ensure(c, c->g_L, &L_, (size_t)c->S_total * rs)) != STBA_OK) return s;
    if ((s = ensure(c, c->g_Dinv, &Dinv_, 2 * (size_t)c->v_total * TF * rs)) != STBA_OK) return s;
    if ((s = ensure(c, c->g_Ldiag, &Ldiag_, (size_t)c->v_total * TF * rs)) != STBA_OK) return s;
    if ((s = ensure(c, c->g_scale, &c->fbuf.scale, (size_t)c->v_total)) != STBA_OK) return s;
    if ((s = ensure(c, c->g_x, &c->fbuf.x, (size_t)c->v_total)) != STBA_OK) return s;
    if ((s = ensure(c, c->g_r, &c->fbuf.r, (size_t)c->v_total)) != STBA_OK) return s;
    c->S = S_;
    c->b = b_;
    c->fbuf.L = L_;
    c->fbuf.Dinv = Dinv_;
    c->fbuf.Ldiag = Ldiag_;
  }
  c->fbuf.fail_flags = c->fail_flags;
  c->fbuf.boosted = &c->st->boosted;
  c->fbuf.v_total = c->v_total;

  // observation order, virtual points and camera lists on the device; the stored residuals follow
  {
    ReorderArgs A = c->reorder;
    A.inv_old = c->inv[c->inv_cur];
    A.inv_new = c->inv[1 - c->inv_cur];
    const bool carry = c->have_order;
    if ((s = launch_reorder_graph(c, A, carry)) != STBA_OK) return s;
    if (carry) std::swap(c->res_cur, c->res_cand);
    c->inv_cur = 1 - c->inv_cur;
    c->have_order = true;
    c->counts_known = false;   // read back on demand (refresh_counts); nothing here waits for the device
  }
  (void)n;
  (void)q;
  if (!c->use_pcg) configure_kernels(c->max_np);
  CK(cudaGetLastError());
  return STBA_OK;
}

// ------------------------------------------------------------------------------------------------------
void record_stage(stba_ctx* c, int i) {
  // inside a capture the record becomes an event node of the graph, so every replay times its stages
  cudaEventRecordWithFlags(c->ev[i], c->stream, c->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
}

// The LM step at the current parameters and c->st->lambda: S', the cluster factors, dc and dp (stages 0-3
// and the point update of Algorithm 1).  With stages, records the stage events 0..4.
template <typename real>
void enqueue_step(stba_ctx* c, bool stages) {
  const DevProblem P = dev_problem(c);
  const Scratch<real> W = scratch<real>(c);
  cudaStream_t s = c->stream;
  const size_t rs = sizeof(real);
  auto mark = [&](int i) {
    if (stages) record_stage(c, i);
  };
  mark(0);
  // stage 0: linearisation and virtual points
  launch_iter_begin<real>(c->st, c->set, s);
  if (c->mixed) launch_params_to_float(P, c->cams_f, c->pts_f, s);
  launch_zero_vp(c->vp_acc, c->counts, (int)rs, s);   // 9 nv reals, nv from the device counter
  cudaMemsetAsync(c->S, 0, (size_t)c->S_total * sizeof(double), s);
  cudaMemsetAsync(c->b, 0, (size_t)c->v_total * sizeof(double), s);
  cudaMemsetAsync(c->vgrad, 0, 9 * (size_t)c->m * rs, s);
  cudaMemsetAsync(c->t_acc, 0, 3 * (size_t)c->n * rs, s);
  cudaMemsetAsync(c->fail_flags, 0, (size_t)c->l * sizeof(int), s);
  launch_vp_reduce<real>(P, W, s);
  launch_vp_finalize<real>(P, W, c->st, c->counts, s);
  mark(1);
  // stage 1: S' and b'
  launch_rcs_build<real>(P, W, c->cslots, c->pchunks, (real*)c->Gbuf, c->st, s, c->side_stream, c->ev_sfork,
                         c->ev_sjoin);
  mark(2);
  // stage 2: factorisation (FP32 factor in mixed mode, FP64 factor in FP64 mode)
  if (c->f32f)
    launch_factor<float>(P, W.S, c->fbuf, c->cplan, s);
  else
    launch_factor<double>(P, W.S, c->fbuf, c->cplan, s);
  mark(3);
  // stage 3: cluster solves with FP64 refinement
  if (c->f32f)
    launch_solve<float>(P, W.S, W.b, c->fbuf, c->cplan, c->set.refine_steps, c->dc, c->dcf, s);
  else
    launch_solve<double>(P, W.S, W.b, c->fbuf, c->cplan, c->set.refine_steps, c->dc, c->dcf, s);
  launch_count_failures(c->fail_flags, c->l, c->st, s);
  mark(4);
  // stage 4: points, cost, control
  launch_point_rhs<real>(P, W, s);
  launch_point_update<real>(P, W, s);
}

template <typename real>
void enqueue_iteration(stba_ctx* c) {
  const DevProblem P = dev_problem(c);
  const Scratch<real> W = scratch<real>(c);
  cudaStream_t s = c->stream;
  enqueue_step<real>(c, true);
  launch_cost<real>(P, c->dc, c->dp, c->cam_rt, c->cam_df, c->pt_df, c->partial, c->st, (real*)c->res_cand, s);
  launch_finalize<real>(P, W, c->st, c->set, 1, s);
  launch_apply<real>(P, c->dc, c->dp, c->cams, c->pts, (const real*)c->res_cand, (real*)c->res_cur, c->st, s);
  record_stage(c, 5);
}

// One LM iteration of the full-RCS comparator: the physical point blocks, then S dc = b over all cameras by
// PCG (host-controlled loop), then the same point update, cost and accept / reject as the method.
template <typename real>
int enqueue_pcg_iteration(stba_ctx* c) {
  const DevProblem P = dev_problem(c);
  const Scratch<real> W = scratch<real>(c);
  cudaStream_t s = c->stream;
  record_stage(c, 0);
  launch_iter_begin<real>(c->st, c->set, s);
  if (c->mixed) launch_params_to_float(P, c->cams_f, c->pts_f, s);
  launch_zero_vp(c->vp_acc, c->counts, (int)sizeof(real), s);
  cudaMemsetAsync(c->t_acc, 0, 3 * (size_t)c->n * sizeof(real), s);
  if (c->use_spcg) {
    launch_spcg_zero(P, W.S, s);
    cudaMemsetAsync(c->b, 0, (size_t)c->v_total * sizeof(double), s);
    cudaMemsetAsync(c->vgrad, 0, 9 * (size_t)c->m * sizeof(real), s);
  }
  launch_vp_reduce<real>(P, W, s);
  launch_vp_finalize<real>(P, W, c->st, c->counts, s);
  record_stage(c, 1);
  if (c->use_spcg) {   // the camera pass alone: b', v and the diagonal blocks of S'
    PairChunks none = c->pchunks;
    none.nchunks = 0;
    launch_rcs_build<real>(P, W, c->cslots, none, (real*)c->Gbuf, c->st, s);
  }
  pcg_prepare<real>(P, W, c->cslots, c->pcg, c->st, s);
  record_stage(c, 2);
  record_stage(c, 3);
  const int iters = pcg_iterate<real>(P, W, c->cslots, c->pcg, c->opt.pcg_max_iter, c->opt.pcg_tol, c->st, s);
  record_stage(c, 4);
  launch_point_rhs<real>(P, W, s);
  launch_point_update<real>(P, W, s);
  launch_cost<real>(P, c->dc, c->dp, c->cam_rt, c->cam_df, c->pt_df, c->partial, c->st, (real*)c->res_cand, s);
  launch_finalize<real>(P, W, c->st, c->set, 1, s);
  launch_apply<real>(P, c->dc, c->dp, c->cams, c->pts, (const real*)c->res_cand, (real*)c->res_cur, c->st, s);
  record_stage(c, 5);
  return iters;
}

template <typename real>
void enqueue_cost(stba_ctx* c) {
  const DevProblem P = dev_problem(c);
  const Scratch<real> W = scratch<real>(c);
  launch_iter_begin<real>(c->st, c->set, c->stream);
  launch_cost<real>(P, nullptr, nullptr, c->cam_rt, c->cam_df, c->pt_df, c->partial, c->st, (real*)c->res_cur,
                    c->stream);
  launch_finalize<real>(P, W, c->st, c->set, 0, c->stream);
}

stba_status run_cost(stba_ctx* c, double* F) {
  // lambda_used / corrected are reset by iter_begin; keep lambda itself
  if (c->mixed)
    enqueue_cost<float>(c);
  else
    enqueue_cost<double>(c);
  CK(cudaGetLastError());
  DevState h;
  CK(cudaMemcpyAsync(&h, c->st, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (h.nonfinite) return fail(c, STBA_ERR_NONFINITE, "a point lies at depth <= 1e-9 in front of a camera that sees it");
  if (!std::isfinite(h.F)) return fail(c, STBA_ERR_NONFINITE, "F(x) is not finite");
  if (F) *F = h.F;
  return STBA_OK;
}

// One exchange of the sharded iteration: `count` values (FP64, or the working precision for dtype 1) at the
// device pointer `dev` summed over the processes by the caller's transport.  With host staging the values
// travel through a pinned host buffer and the transport sees host memory (e.g. gloo); otherwise it gets the
// device pointer and the stream (e.g. NCCL).
stba_status shard_exchange(stba_ctx* c, void* dev, int64_t count, int32_t dtype) {
  const size_t bytes = (size_t)count * (dtype == 0 ? 8 : 4);
  if (c->shard_host_staging) {
    if (c->xch_host_bytes < bytes) {
      if (c->xch_host) cudaFreeHost(c->xch_host);
      c->xch_host = nullptr;
      c->xch_host_bytes = 0;
      if (cudaHostAlloc(&c->xch_host, bytes, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, STBA_ERR_OOM, "pinned host allocation of the exchange buffer failed");
      }
      c->xch_host_bytes = bytes;
    }
    CK(cudaMemcpyAsync(c->xch_host, dev, bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (c->shard_fn(c->shard_user, c->xch_host, count, dtype, (void*)c->stream) != 0)
      return fail(c, STBA_ERR_STATE, "the sharded iteration's exchange (all-reduce) failed");
    CK(cudaMemcpyAsync(dev, c->xch_host, bytes, cudaMemcpyHostToDevice, c->stream));
    return STBA_OK;
  }
  if (c->shard_fn(c->shard_user, dev, count, dtype, (void*)c->stream) != 0)
    return fail(c, STBA_ERR_STATE, "the sharded iteration's exchange (all-reduce) failed");
  return STBA_OK;
}

// One LM iteration of the sharded method (stba_set_shard): this process linearises the observations of its
// clusters, builds, factors and solves only those clusters, and three exchanges make the rest identical on
// every process:
//   1. per point, the sums over its virtual points of V and w' (9 values): the physical C_i and w_i of
//      Eq. 15 and the per-point sums of the steepest-descent correction (Sec. 4.3);
//   2. after the cluster solves, Delta c (zero for the other processes' cameras), the camera gradient v and
//      the count of failed cluster factorisations;
// the point update, the cost at x + Delta x and the accept / reject rule then run on complete data in every
// process, which therefore all hold the same parameters, damping and cost.  Enqueued without a graph: the
// exchanges return to the host.
template <typename real>
stba_status run_sharded_iteration(stba_ctx* c) {
  const DevProblem P = dev_problem(c);
  const Scratch<real> W = scratch<real>(c);
  cudaStream_t s = c->stream;
  stba_status st;
  const size_t rs = sizeof(real);
  record_stage(c, 0);
  launch_iter_begin<real>(c->st, c->set, s);
  if (c->mixed) launch_params_to_float(P, c->cams_f, c->pts_f, s);
  launch_zero_vp(c->vp_acc, c->counts, (int)rs, s);
  cudaMemsetAsync(c->S, 0, (size_t)c->S_total * sizeof(double), s);
  cudaMemsetAsync(c->b, 0, (size_t)c->v_total * sizeof(double), s);
  cudaMemsetAsync(c->vgrad, 0, 9 * (size_t)c->m * rs, s);
  cudaMemsetAsync(c->t_acc, 0, 3 * (size_t)c->n * rs, s);
  cudaMemsetAsync(c->fail_flags, 0, (size_t)c->l * sizeof(int), s);
  launch_vp_reduce<real>(P, W, s);   // this process's observations only
  launch_pt_sums<real>(P, W, c->xch, s);
  if ((st = shard_exchange(c, c->xch, 9 * (int64_t)c->n, 0)) != STBA_OK) return st;
  launch_vp_finalize<real>(P, W, c->st, c->counts, s, c->xch);
  record_stage(c, 1);
  launch_rcs_build<real>(P, W, c->cslots, c->pchunks, (real*)c->Gbuf, c->st, s);
  record_stage(c, 2);
  if (c->f32f)
    launch_factor<float>(P, W.S, c->fbuf, c->cplan, s);
  else
    launch_factor<double>(P, W.S, c->fbuf, c->cplan, s);
  record_stage(c, 3);
  if (c->f32f)
    launch_solve<float>(P, W.S, W.b, c->fbuf, c->cplan, c->set.refine_steps, c->dc, c->dcf, s);
  else
    launch_solve<double>(P, W.S, W.b, c->fbuf, c->cplan, c->set.refine_steps, c->dc, c->dcf, s);
  launch_count_failures(c->fail_flags, c->l, c->st, s);
  double* nfail = c->xch + 9 * (size_t)c->n;
  launch_failed_io(c->st, nfail, 1, s);
  if ((st = shard_exchange(c, c->dc, 9 * (int64_t)c->m, 0)) != STBA_OK) return st;
  if ((st = shard_exchange(c, c->vgrad, 9 * (int64_t)c->m, c->mixed ? 1 : 0)) != STBA_OK) return st;
  if ((st = shard_exchange(c, nfail, 1, 0)) != STBA_OK) return st;
  launch_failed_io(c->st, nfail, 0, s);
  if (c->mixed) launch_dc_to_float(c->dc, c->dcf, 9 * (int64_t)c->m, s);
  record_stage(c, 4);
  launch_point_rhs<real>(P, W, s);
  launch_point_update<real>(P, W, s);
  launch_cost<real>(P, c->dc, c->dp, c->cam_rt, c->cam_df, c->pt_df, c->partial, c->st, (real*)c->res_cand, s);
  launch_finalize<real>(P, W, c->st, c->set, 1, s);
  launch_apply<real>(P, c->dc, c->dp, c->cams, c->pts, (const real*)c->res_cand, (real*)c->res_cur, c->st, s);
  record_stage(c, 5);
  CK(cudaGetLastError());
  c->have_stage_times = true;
  return STBA_OK;
}

// Launch structure of the iteration graph: what decides which kernels and dependencies a capture records
// (a wrong guess costs only time: cudaGraphExecUpdate checks the structure itself).
uint64_t graph_signature(const stba_ctx* c) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t v) {
    h ^= v;
    h *= 1099511628211ull;
  };
  const CholPlan& p = c->cplan;
  mix((uint64_t)p.nsteps);
  mix((uint64_t)p.tile);
  mix((uint64_t)(p.split | (p.persistent << 1) | (p.update_tc << 2)));
  mix((uint64_t)p.solve_cs);
  mix((uint64_t)(p.n_res_items > 0));
  mix((uint64_t)c->set.refine_steps);
  mix((uint64_t)(c->mixed ? 1 : 0));
  mix((uint64_t)((c->pchunks.nchunks > 0 && c->l < c->m) ? 1 : 0));
  mix((uint64_t)c->opt.pair_blocks);
  for (int kt = 0; kt < p.nsteps; ++kt) {
    const int npn = p.h_panel_off[kt + 1] - p.h_panel_off[kt];
    const int nu = p.h_update_off[kt + 1] - p.h_update_off[kt];
    const int nd = (p.split && p.h_diag_count) ? p.h_diag_count[kt] : 0;
    mix((uint64_t)((npn > 0) | ((nu > 0) << 1) | ((nd > 0) << 2) | ((npn > nd) << 3)));
  }
  return h;
}

stba_status launch_iteration(stba_ctx* c) {
  if (c->shard_world > 1) return c->mixed ? run_sharded_iteration<float>(c) : run_sharded_iteration<double>(c);
  if (c->use_pcg || c->use_spcg) {
    const int32_t iters = c->mixed ? enqueue_pcg_iteration<float>(c) : enqueue_pcg_iteration<double>(c);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&c->st->info.linear_iterations, &iters, sizeof iters, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->have_stage_times = true;
    return STBA_OK;
  }
  if (!c->opt.use_graph) {
    if (c->mixed)
      enqueue_iteration<float>(c);
    else
      enqueue_iteration<double>(c);
    CK(cudaGetLastError());
    c->have_stage_times = true;
    return STBA_OK;
  }
  if (!c->graph || c->graph_stale) {
    // capture on a private stream (the user's stream may be the legacy default stream)
    cudaStream_t user = c->stream;
    c->stream = c->cap_stream;
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    if (c->mixed)
      enqueue_iteration<float>(c);
    else
      enqueue_iteration<double>(c);
    c->capturing = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    c->stream = user;
    if (e != cudaSuccess) return fail(c, STBA_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    c->graph_stale = false;
    c->graph = nullptr;
    // an executable graph of the same launch structure is updated in place (kernel arguments and launch
    // sizes); instantiating a new one costs far more host time than the device needs for an iteration
    const uint64_t sig = graph_signature(c);
    auto& cache = c->graph_cache;
    for (size_t i = 0; i < cache.size(); ++i) {
      if (cache[i].first != sig) continue;
      cudaGraphExecUpdateResultInfo ri;
      if (cudaGraphExecUpdate(cache[i].second, g, &ri) == cudaSuccess) {
        cudaGraphDestroy(g);
        c->graph = cache[i].second;
        CK(cudaGraphLaunch(c->graph, c->stream));
        c->have_stage_times = true;
        return STBA_OK;
      }
      cudaGetLastError();
      cudaGraphExecDestroy(cache[i].second);
      cache.erase(cache.begin() + (long)i);
      break;
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(c, STBA_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    if (cache.size() >= 8) {   // keep the 8 most recent structures
      cudaGraphExecDestroy(cache.front().second);
      cache.erase(cache.begin());
    }
    cache.emplace_back(sig, ex);
    c->graph = ex;
  }
  CK(cudaGraphLaunch(c->graph, c->stream));
  c->have_stage_times = true;
  return STBA_OK;
}

// One LM iteration; while recording, x_t goes to the tape before it and its record after it (both are
// device-to-device copies on the context stream, outside the captured graph).
stba_status run_iteration(stba_ctx* c) {
  if (c->tape_cap == 0) return launch_iteration(c);
  if (c->tape_len >= c->tape_cap)
    return fail(c, STBA_ERR_STATE, "the tape holds %d iterations; call stba_record again to restart it", c->tape_cap);
  const size_t nx = 9 * (size_t)c->m + 3 * (size_t)c->n;
  double* slot = c->tape_x + nx * (size_t)c->tape_len;
  CK(cudaMemcpyAsync(slot, c->cams, 9 * (size_t)c->m * 8, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(slot + 9 * (size_t)c->m, c->pts, 3 * (size_t)c->n * 8, cudaMemcpyDeviceToDevice, c->stream));
  stba_status s = launch_iteration(c);
  if (s != STBA_OK) return s;
  CK(cudaMemcpyAsync(c->tape_info + c->tape_len, &c->st->info, sizeof(stba_iter_info), cudaMemcpyDeviceToDevice,
                     c->stream));
  if (c->tape_clusters.empty() || c->tape_clusters.back() != c->h_clusters) c->tape_clusters.push_back(c->h_clusters);
  c->tape_cluster_id.push_back((int)c->tape_clusters.size() - 1);
  c->tape_len++;
  return STBA_OK;
}

void free_tape(stba_ctx* c) {
  free_list(c, c->tape_allocs);
  c->tape_x = nullptr;
  c->tape_info = nullptr;
  c->adj = AdjointBuffers{};
  c->adj_save_x = nullptr;
  c->tape_cap = c->tape_len = 0;
  c->tape_broken = false;
  c->tape_clusters.clear();
  c->tape_cluster_id.clear();
}

template <typename real>
void enqueue_adjoint_step(stba_ctx* c, double lam, int corrected, const AdjointBuffers& A) {
  // recompute the forward step at x_t with the recorded damping, then its adjoint (whose launch sizes need
  // the number of virtual points on the host)
  refresh_counts(c);
  launch_set_lambda(c->st, lam, c->stream);
  launch_iter_begin<real>(c->st, c->set, c->stream);
  const DevProblem P = dev_problem(c);
  launch_cost<real>(P, nullptr, nullptr, c->cam_rt, c->cam_df, c->pt_df, c->partial, c->st, (real*)c->res_cur,
                    c->stream);
  enqueue_step<real>(c, false);
  launch_adjoint_step<real>(P, scratch<real>(c), c->clist, c->fbuf, c->cplan, c->set.refine_steps, c->obs_perm, lam,
                            corrected, A, c->stream);
}

stba_status read_info(stba_ctx* c, stba_iter_info* info) {
  DevState h;
  CK(cudaMemcpyAsync(&h, c->st, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (info) *info = h.info;
  if (h.lambda > 1e16) return fail(c, STBA_ERR_STATE, "lambda exceeded 1e16");
  return STBA_OK;
}

bool finite_all(const double* v, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

}  // namespace

// ==========================================================================================================
extern "C" {

void stba_default_options(stba_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->precision = STBA_FP64;
  o->correction = 1;
  o->lambda0 = 1e-4;
  o->lambda_min = 0.0;
  o->correction_lambda = 0.1;
  o->ftol = o->gtol = o->xtol = -1.0;
  o->refine_steps = 1;
  o->use_graph = 1;
  o->linear_solver = STBA_SOLVER_CLUSTERS;
  o->pcg_max_iter = 500;
  o->pcg_tol = 1e-6;
  o->factor_update = STBA_FACTOR_UPDATE_DEFAULT;
  o->factor_panel = STBA_FACTOR_PANEL_DEFAULT;
  o->solve_cluster = 0;
}

const char* stba_status_string(stba_status s) {
  switch (s) {
    case STBA_OK: return "ok";
    case STBA_ERR_INVALID_ARG: return "invalid argument";
    case STBA_ERR_CUDA: return "CUDA error";
    case STBA_ERR_OOM: return "out of device memory";
    case STBA_ERR_NOT_SPD: return "matrix not positive definite";
    case STBA_ERR_NONFINITE: return "non-finite value";
    case STBA_ERR_TIMEOUT: return "timeout";
    case STBA_ERR_STATE: return "invalid state";
  }
  return "unknown status";
}

// ------------------------------------------------------------------------------------------------------
// Camera graph and stochastic graph clustering (host only)
struct stba_graph {
  stba::CameraGraph g;
  int64_t m = 0;
};

stba_status stba_graph_create(int64_t m, int64_t n, const int32_t* obs_cam, const int32_t* obs_pt, int64_t q,
                              stba_graph** out) {
  g_create_error.clear();
  auto bad = [&](const char* msg) {
    g_create_error = msg;
    return STBA_ERR_INVALID_ARG;
  };
  if (!out) return bad("null output pointer");
  *out = nullptr;
  if (!obs_cam || !obs_pt) return bad("null array argument");
  if (m < 1 || n < 1 || q < 0 || m > INT32_MAX / 9 || n > INT32_MAX || q > INT32_MAX - 64) return bad("sizes out of range");
  std::vector<int> pt_off(n + 1, 0);
  for (int64_t o = 0; o < q; ++o) {
    if (obs_cam[o] < 0 || obs_cam[o] >= m || obs_pt[o] < 0 || obs_pt[o] >= n) return bad("observation index out of range");
    pt_off[obs_pt[o] + 1]++;
  }
  for (int64_t i = 0; i < n; ++i) pt_off[i + 1] += pt_off[i];
  std::vector<int> base_cam(q);
  {
    std::vector<int> f(pt_off.begin(), pt_off.end() - 1);
    for (int64_t o = 0; o < q; ++o) base_cam[f[obs_pt[o]]++] = obs_cam[o];
    for (int64_t i = 0; i < n; ++i) {
      std::sort(base_cam.begin() + pt_off[i], base_cam.begin() + pt_off[i + 1]);
      for (int o = pt_off[i] + 1; o < pt_off[i + 1]; ++o)
        if (base_cam[o] == base_cam[o - 1]) return bad("a camera observes a point twice");
    }
  }
  stba_graph* g = new stba_graph();
  g->m = m;
  build_camera_graph((int)m, (int)n, pt_off, base_cam, g->g, false);
  *out = g;
  return STBA_OK;
}

stba_status stba_graph_edges(const stba_graph* g, int64_t* E, int32_t* i, int32_t* j, int64_t* w) {
  if (!g || !E) return STBA_ERR_INVALID_ARG;
  *E = (int64_t)g->g.edge_y.size();
  for (int64_t x = 0; x < g->m; ++x)
    for (int e = g->g.edge_off[x]; e < g->g.edge_off[x + 1]; ++e) {
      if (i) i[e] = g->g.edge_y[e];
      if (j) j[e] = (int32_t)x;
      if (w) w[e] = g->g.edge_w[e];
    }
  return STBA_OK;
}

namespace {
stba_status sgc_args(int32_t gamma, double beta) {
  if (gamma < 1 || !(beta >= 0.0) || !std::isfinite(beta)) {
    g_create_error = "gamma must be >= 1 and beta finite and >= 0";
    return STBA_ERR_INVALID_ARG;
  }
  return STBA_OK;
}
}  // namespace

stba_status stba_graph_cluster(const stba_graph* g, int32_t gamma, double beta, uint64_t seed,
                               int32_t* cluster_assignment, int32_t* l) {
  if (!g || !cluster_assignment || !l) return STBA_ERR_INVALID_ARG;
  stba_status s = sgc_args(gamma, beta);
  if (s != STBA_OK) return s;
  sgc_sample(g->g, (int)g->m, gamma, beta, seed, cluster_assignment, l);
  return STBA_OK;
}

stba_status stba_graph_cluster_batch(const stba_graph* g, int32_t gamma, double beta, uint64_t seed, int32_t count,
                                     int32_t* cluster_assignments, int32_t* l) {
  if (!g || !cluster_assignments || !l || count < 0) return STBA_ERR_INVALID_ARG;
  stba_status s = sgc_args(gamma, beta);
  if (s != STBA_OK) return s;
  sgc_sample_batch(g->g, (int)g->m, gamma, beta, seed, count, cluster_assignments, l);
  return STBA_OK;
}

void stba_graph_destroy(stba_graph* g) { delete g; }

stba_status stba_cluster_sgc(stba_ctx* c, int32_t gamma, double beta, uint64_t seed, int32_t count,
                             int32_t* cluster_assignments, int32_t* l) {
  if (!c || !cluster_assignments || !l || count < 0) return STBA_ERR_INVALID_ARG;
  if (gamma < 1 || !(beta >= 0.0) || !std::isfinite(beta))
    return fail(c, STBA_ERR_INVALID_ARG, "gamma must be >= 1 and beta finite and >= 0");
  sgc_sample_batch(c->cgraph, (int)c->m, gamma, beta, seed, count, cluster_assignments, l);
  return STBA_OK;
}

stba_status stba_autotune(stba_ctx* c, int32_t iterations, int32_t* choice, float* ms) {
  if (!c || iterations < 1) return STBA_ERR_INVALID_ARG;
  if (c->tape_cap > 0) return fail(c, STBA_ERR_STATE, "stba_autotune is not allowed while iterations are recorded");
  constexpr int NCAND = 6;
  const int cand_tile[NCAND] = {64, 64, 64, 32, 64, 64}, cand_tc[NCAND] = {1, 0, 0, 0, 0, 1};
  const int cand_panel[NCAND] = {STBA_FACTOR_PANEL_SPLIT,   STBA_FACTOR_PANEL_SPLIT,      STBA_FACTOR_PANEL_STACKED,
                                 STBA_FACTOR_PANEL_STACKED, STBA_FACTOR_PANEL_PERSISTENT, STBA_FACTOR_PANEL_STACKED};
  if (ms)
    for (int t = 0; t < NCAND; ++t) ms[t] = -1.0f;
  auto report = [&]() {
    if (!choice) return;
    *choice = -1;
    for (int t = 0; t < NCAND; ++t)
      if (cand_tile[t] == c->tile && cand_tc[t] == c->update_tc && cand_panel[t] == c->panel_choice) *choice = t;
  };
  if (!c->f32f || c->use_pcg || c->use_spcg) {   // one candidate (or no factorisation at all)
    report();
    return STBA_OK;
  }
  // state to restore after every trial: parameters, residuals at x (in the order of this assignment, which
  // every trial reproduces), the device LM state
  const size_t nc = 9 * (size_t)c->m, npt = 3 * (size_t)c->n, nr = 2 * (size_t)c->q * sizeof(float);
  double *cams0 = nullptr, *pts0 = nullptr;
  char* res0 = nullptr;
  DevState* st0 = nullptr;
  auto release = [&]() {
    cudaFree(cams0);
    cudaFree(pts0);
    cudaFree(res0);
    cudaFree(st0);
  };
  if (cudaMalloc(&cams0, nc * 8) != cudaSuccess || cudaMalloc(&pts0, npt * 8) != cudaSuccess ||
      cudaMalloc(&res0, nr) != cudaSuccess || cudaMalloc(&st0, sizeof(DevState)) != cudaSuccess) {
    cudaGetLastError();
    release();
    return fail(c, STBA_ERR_OOM, "stba_autotune: no device memory for the saved state");
  }
  auto copy = [&](void* d, const void* s_, size_t b) {
    return cudaMemcpyAsync(d, s_, b, cudaMemcpyDeviceToDevice, c->stream) == cudaSuccess;
  };
  bool ok = copy(cams0, c->cams, nc * 8) && copy(pts0, c->pts, npt * 8) && copy(res0, c->res_cur, nr) &&
            copy(st0, c->st, sizeof(DevState));
  auto restore = [&]() {
    return copy(c->cams, cams0, nc * 8) && copy(c->pts, pts0, npt * 8) && copy(c->res_cur, res0, nr) &&
           copy(c->st, st0, sizeof(DevState));
  };
  const std::vector<int> cl = c->h_clusters;
  float best_ms = 0.f;
  int best = -1;
  stba_status s = STBA_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) ok = false;
  for (int t = 0; t < NCAND && ok && s == STBA_OK; ++t) {
    c->tile = cand_tile[t];
    c->update_tc = cand_tc[t];
    c->panel_choice = cand_panel[t];
    if ((s = set_clusters_host(c, cl)) != STBA_OK) break;
    ok = restore();
    if (ok && (s = run_iteration(c)) != STBA_OK) break;   // warm-up: capture, first launch
    ok = ok && restore() && cudaEventRecord(e0, c->stream) == cudaSuccess;
    for (int i = 0; i < iterations && ok && s == STBA_OK; ++i) s = run_iteration(c);
    if (s != STBA_OK) break;
    ok = ok && cudaEventRecord(e1, c->stream) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
    float el = 0.f;
    ok = ok && cudaEventElapsedTime(&el, e0, e1) == cudaSuccess;
    const float per = el / iterations;
    if (ms) ms[t] = per;
    if (ok && (best < 0 || per < best_ms)) {
      best_ms = per;
      best = t;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s == STBA_OK && ok && best >= 0) {
    c->tile = cand_tile[best];
    c->update_tc = cand_tc[best];
    c->panel_choice = cand_panel[best];
    s = set_clusters_host(c, cl);
    if (s == STBA_OK) ok = restore() && cudaStreamSynchronize(c->stream) == cudaSuccess;
  }
  release();
  if (s != STBA_OK) return s;
  if (!ok) return fail(c, STBA_ERR_CUDA, "stba_autotune: a copy or an event failed");
  c->have_stage_times = false;
  report();
  return STBA_OK;
}

stba_status stba_set_shard(stba_ctx* c, int32_t rank, int32_t world, stba_allreduce_fn fn, void* user,
                           int32_t host_staging) {
  if (!c) return STBA_ERR_INVALID_ARG;
  if (world < 1 || rank < 0 || rank >= world || (world > 1 && !fn))
    return fail(c, STBA_ERR_INVALID_ARG, "stba_set_shard: need 0 <= rank < world and a transport when world > 1");
  if (world > 1 && (c->use_pcg || c->use_spcg))
    return fail(c, STBA_ERR_STATE, "the sharded iteration covers the cluster solver only");
  if (world > 1 && c->tape_cap > 0)
    return fail(c, STBA_ERR_STATE, "the sharded iteration does not record (stba_record / stba_adjoint)");
  if (world > 1 && !c->xch) {
    stba_status s = dalloc(c, &c->xch, 9 * (size_t)c->n + 1);
    if (s != STBA_OK) return s;
  }
  c->shard_rank = world > 1 ? rank : 0;
  c->shard_world = world;
  c->shard_fn = world > 1 ? fn : nullptr;
  c->shard_user = user;
  c->shard_host_staging = host_staging ? 1 : 0;
  c->graph_stale = true;
  const std::vector<int> cl = c->h_clusters;
  return set_clusters_host(c, cl);   // owners and the plan of the current assignment
}

stba_status stba_shard_owned(stba_ctx* c, int32_t* owned, int32_t* l) {
  if (!c || !l) return STBA_ERR_INVALID_ARG;
  *l = c->l;
  if (owned)
    for (int k = 0; k < c->l; ++k) owned[k] = c->h_owned[k];
  return STBA_OK;
}

const char* stba_last_error(stba_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

void stba_destroy(stba_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& e : c->graph_cache) cudaGraphExecDestroy(e.second);
  c->graph_cache.clear();
  c->graph = nullptr;
  free_list(c, c->allocs);
  free_list(c, c->tape_allocs);
  for (GrowBuf* g : {&c->g_panel, &c->g_update, &c->g_res, &c->g_diag, &c->g_S, &c->g_b, &c->g_L, &c->g_Dinv,
                     &c->g_Ldiag, &c->g_scale, &c->g_x, &c->g_r, &c->g_blob})
    if (g->ptr) cudaFree(g->ptr);
  for (int i = 0; i < 2; ++i) {
    if (c->stage_h[i]) cudaFreeHost(c->stage_h[i]);
    if (c->stage_ev[i]) cudaEventDestroy(c->stage_ev[i]);
  }
  if (c->xch_host) cudaFreeHost(c->xch_host);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  for (cudaGraphExec_t& e : c->reorder_exec)
    if (e) cudaGraphExecDestroy(e);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->side_stream) cudaStreamDestroy(c->side_stream);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_rfork) cudaEventDestroy(c->ev_rfork);
  if (c->ev_rjoin) cudaEventDestroy(c->ev_rjoin);
  if (c->ev_sfork) cudaEventDestroy(c->ev_sfork);
  if (c->ev_sjoin) cudaEventDestroy(c->ev_sjoin);
  if (c->ev_copy) cudaEventDestroy(c->ev_copy);
  for (auto e : c->ev_panel) cudaEventDestroy(e);
  for (auto e : c->ev_update) cudaEventDestroy(e);
  delete c;
}

stba_status stba_create(const double* cameras, int64_t m, const double* points, int64_t n, const int32_t* obs_cam,
                        const int32_t* obs_pt, const double* obs_uv, int64_t q, const int32_t* cluster_assignment,
                        const stba_options* opt, void* cuda_stream, stba_ctx** out) {
  if (!out) return STBA_ERR_INVALID_ARG;
  *out = nullptr;
  stba_ctx* c = new stba_ctx();
  g_create_error.clear();
  auto bail = [&](stba_status s) {
    g_create_error = c->err;   // the context is destroyed; stba_last_error(NULL) returns the message
    stba_destroy(c);
    return s;
  };
  if (opt)
    c->opt = *opt;
  else
    stba_default_options(&c->opt);
  if (!cameras || !points || !obs_cam || !obs_pt || !obs_uv || !cluster_assignment)
    return bail(fail(c, STBA_ERR_INVALID_ARG, "null array argument"));
  if (m < 1 || n < 1 || q < 2 || m > INT32_MAX / 9 || n > INT32_MAX / 3 || q > INT32_MAX - 64)
    return bail(fail(c, STBA_ERR_INVALID_ARG, "sizes out of range (m=%lld n=%lld q=%lld)", (long long)m,
                     (long long)n, (long long)q));
  if (!(c->opt.lambda0 > 0) || !std::isfinite(c->opt.lambda0) || c->opt.lambda_min < 0 ||
      (c->opt.precision != STBA_FP64 && c->opt.precision != STBA_MIXED) || c->opt.refine_steps < 0 ||
      c->opt.refine_steps > 8 ||
      (c->opt.linear_solver != STBA_SOLVER_CLUSTERS && c->opt.linear_solver != STBA_SOLVER_PCG_FULL &&
       c->opt.linear_solver != STBA_SOLVER_PCG_CLUSTERS) ||
      (c->opt.linear_solver != STBA_SOLVER_CLUSTERS && (c->opt.pcg_max_iter < 1 || !(c->opt.pcg_tol > 0))) ||
      !(c->opt.huber_a >= 0.0) || !std::isfinite(c->opt.huber_a) ||
      !(c->opt.factor_tile == 0 || c->opt.factor_tile == 32 || (c->opt.factor_tile == 64 && c->opt.precision == STBA_MIXED)) ||
      (c->opt.factor_update != STBA_FACTOR_UPDATE_DEFAULT && c->opt.factor_update != STBA_FACTOR_UPDATE_SIMT &&
       c->opt.factor_update != STBA_FACTOR_UPDATE_TENSOR) ||
      (c->opt.factor_update == STBA_FACTOR_UPDATE_TENSOR &&
       !(c->opt.precision == STBA_MIXED && (c->opt.factor_tile == 0 || c->opt.factor_tile == 64))) ||
      (c->opt.factor_panel != STBA_FACTOR_PANEL_DEFAULT && c->opt.factor_panel != STBA_FACTOR_PANEL_STACKED &&
       c->opt.factor_panel != STBA_FACTOR_PANEL_SPLIT && c->opt.factor_panel != STBA_FACTOR_PANEL_PERSISTENT) ||
      !(c->opt.solve_cluster == 0 || c->opt.solve_cluster == 2 || c->opt.solve_cluster == 4 ||
        c->opt.solve_cluster == 8) ||
      !(c->opt.pair_blocks == STBA_PAIR_BLOCKS_DEFAULT || c->opt.pair_blocks == STBA_PAIR_BLOCKS_STORED ||
        c->opt.pair_blocks == STBA_PAIR_BLOCKS_RECOMPUTE) ||
      ((c->opt.factor_panel == STBA_FACTOR_PANEL_SPLIT || c->opt.factor_panel == STBA_FACTOR_PANEL_PERSISTENT) &&
       !(c->opt.precision == STBA_MIXED && (c->opt.factor_tile == 0 || c->opt.factor_tile == 64))) ||
      !(c->opt.factor_fp64 == 0 || c->opt.factor_fp64 == 1) ||
      (c->opt.factor_fp64 && (c->opt.factor_tile == 64 || c->opt.factor_update == STBA_FACTOR_UPDATE_TENSOR ||
                              c->opt.factor_panel == STBA_FACTOR_PANEL_SPLIT ||
                              c->opt.factor_panel == STBA_FACTOR_PANEL_PERSISTENT)))
    return bail(fail(c, STBA_ERR_INVALID_ARG, "invalid options"));
  c->m = m;
  c->n = n;
  c->q = q;
  c->mixed = c->opt.precision == STBA_MIXED;
  c->f32f = c->mixed && !c->opt.factor_fp64;
  c->tile = c->opt.factor_tile ? c->opt.factor_tile : factor_tile(c->f32f);
  c->update_tc = c->f32f && c->tile == 64 && c->opt.factor_update != STBA_FACTOR_UPDATE_SIMT;
  c->panel_choice = c->opt.factor_panel;
  c->use_pcg = c->opt.linear_solver == STBA_SOLVER_PCG_FULL;
  c->use_spcg = c->opt.linear_solver == STBA_SOLVER_PCG_CLUSTERS;
  c->set.correction = c->opt.correction;
  c->set.correction_lambda = c->opt.correction_lambda;
  c->set.lambda_min = c->opt.lambda_min;
  c->set.ftol = c->opt.ftol;
  c->set.gtol = c->opt.gtol;
  c->set.xtol = c->opt.xtol;
  c->set.refine_steps = c->opt.refine_steps;
  std::vector<double> h_cams(9 * (size_t)m), h_pts(3 * (size_t)n);
  std::vector<int> h_cl(m);
  c->in_cam.resize(q);
  c->in_pt.resize(q);
  c->in_uv.resize(2 * (size_t)q);
  stba_status s;
  if ((s = copy_in(c, h_cams.data(), cameras, h_cams.size() * 8)) != STBA_OK) return bail(s);
  if ((s = copy_in(c, h_pts.data(), points, h_pts.size() * 8)) != STBA_OK) return bail(s);
  if ((s = copy_in(c, c->in_cam.data(), obs_cam, (size_t)q * 4)) != STBA_OK) return bail(s);
  if ((s = copy_in(c, c->in_pt.data(), obs_pt, (size_t)q * 4)) != STBA_OK) return bail(s);
  if ((s = copy_in(c, c->in_uv.data(), obs_uv, (size_t)q * 16)) != STBA_OK) return bail(s);
  if ((s = copy_in(c, h_cl.data(), cluster_assignment, (size_t)m * 4)) != STBA_OK) return bail(s);
  if (!finite_all(h_cams.data(), h_cams.size()) || !finite_all(h_pts.data(), h_pts.size()) ||
      !finite_all(c->in_uv.data(), c->in_uv.size()))
    return bail(fail(c, STBA_ERR_NONFINITE, "non-finite camera, point or observation value"));

  // validate the visibility graph and order observations by (point, camera)
  std::vector<int> pcount(n + 1, 0), ccount(m, 0);
  for (int64_t o = 0; o < q; ++o) {
    const int j = c->in_cam[o], i = c->in_pt[o];
    if (j < 0 || j >= m || i < 0 || i >= n)
      return bail(fail(c, STBA_ERR_INVALID_ARG, "observation %lld has camera %d / point %d out of range", (long long)o, j, i));
    pcount[i + 1]++;
    ccount[j]++;
  }
  for (int64_t i = 0; i < n; ++i)
    if (pcount[i + 1] < 2) return bail(fail(c, STBA_ERR_INVALID_ARG, "point %lld has fewer than 2 observations", (long long)i));
  for (int64_t j = 0; j < m; ++j)
    if (ccount[j] < 1) return bail(fail(c, STBA_ERR_INVALID_ARG, "camera %lld has no observation", (long long)j));
  c->h_cam_nobs = ccount;
  for (int64_t i = 0; i < n; ++i) pcount[i + 1] += pcount[i];
  c->h_pt_off = pcount;
  c->base_order.assign(q, 0);
  {
    std::vector<int> fillp(pcount.begin(), pcount.end() - 1);
    for (int64_t o = 0; o < q; ++o) c->base_order[fillp[c->in_pt[o]]++] = (int)o;
    for (int64_t i = 0; i < n; ++i) {
      auto b = c->base_order.begin() + pcount[i], e = c->base_order.begin() + pcount[i + 1];
      std::sort(b, e, [&](int x, int y) { return c->in_cam[x] < c->in_cam[y]; });
      for (auto it = b + 1; it < e; ++it)
        if (c->in_cam[*it] == c->in_cam[*(it - 1)])
          return bail(fail(c, STBA_ERR_INVALID_ARG, "camera %d observes point %lld twice", c->in_cam[*it], (long long)i));
    }
  }
  for (int j = 0; j < m; ++j) {
    if (h_cl[j] < 0 || h_cl[j] >= m)
      return bail(fail(c, STBA_ERR_INVALID_ARG, "cluster id %d of camera %d out of range", h_cl[j], j));
  }
  {
    std::vector<int> used(m, 0);
    int l = 0;
    for (int j = 0; j < m; ++j) {
      used[h_cl[j]] = 1;
      l = std::max(l, h_cl[j] + 1);
    }
    for (int k = 0; k < l; ++k)
      if (!used[k]) return bail(fail(c, STBA_ERR_INVALID_ARG, "cluster %d has no camera (ids must be 0..l-1)", k));
  }
  // all host-side validation is done; from here on the device is needed
  c->stream = (cudaStream_t)cuda_stream;
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(c, STBA_ERR_CUDA, "cannot create a CUDA stream (is a GPU visible?)"));
  }
  for (auto& e : c->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return bail(fail(c, STBA_ERR_CUDA, "cudaEventCreate failed"));
  if (cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_rfork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_rjoin, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_sfork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_sjoin, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_copy, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->stage_ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->stage_ev[1], cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(c, STBA_ERR_CUDA, "cannot create the factorisation stream or its events"));
  if ((s = dalloc(c, &c->cams, 9 * (size_t)m)) != STBA_OK) return bail(s);
  if ((s = dalloc(c, &c->pts, 3 * (size_t)n)) != STBA_OK) return bail(s);
  if ((s = dalloc(c, &c->dc, 9 * (size_t)m)) != STBA_OK) return bail(s);
  if ((s = dalloc(c, &c->dp, 3 * (size_t)n)) != STBA_OK) return bail(s);
  if ((s = dalloc(c, &c->partial, 6 * (size_t)RED_BLOCKS)) != STBA_OK) return bail(s);
  if ((s = dalloc(c, &c->cam_rt, 15 * (size_t)m)) != STBA_OK) return bail(s);
  if ((s = dalloc(c, &c->cam_df, 28 * (size_t)m)) != STBA_OK) return bail(s);
  if ((s = dalloc(c, &c->pt_df, 6 * (size_t)n)) != STBA_OK) return bail(s);
  if (c->mixed) {
    if ((s = dalloc(c, &c->cams_f, 9 * (size_t)m)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &c->pts_f, 3 * (size_t)n)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &c->dcf, 9 * (size_t)m)) != STBA_OK) return bail(s);
  }
  {
    char *r1, *r2;
    const size_t rsz = 2 * (size_t)q * (c->mixed ? sizeof(float) : sizeof(double));
    if ((s = dalloc(c, &r1, rsz)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &r2, rsz)) != STBA_OK) return bail(s);
    c->res_cur = r1;
    c->res_cand = r2;
  }
  if ((s = dalloc(c, &c->st, 1)) != STBA_OK) return bail(s);
  if (c->use_pcg || c->use_spcg) {
    const size_t rs = c->mixed ? sizeof(float) : sizeof(double);
    char *J, *pw, *tpt, *upt;
    PcgBuffers& B = c->pcg;
    if (c->use_spcg) {   // per-virtual-point vectors at their largest size (nv <= q), zeroed in 16-byte pieces
      char *tv, *uv;
      if ((s = dalloc(c, &tv, 3 * (size_t)q * rs + 16)) != STBA_OK) return bail(s);
      if ((s = dalloc(c, &uv, 3 * (size_t)q * rs + 16)) != STBA_OK) return bail(s);
      B.tvp = tv;
      B.uvp = uv;
      B.split = true;
    }
    if ((s = dalloc(c, &J, 24 * (size_t)q * rs)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &pw, 9 * (size_t)m * rs)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &tpt, 3 * (size_t)n * rs)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &upt, 3 * (size_t)n * rs)) != STBA_OK) return bail(s);
    B.J = J;
    B.pw = pw;
    B.tpt = tpt;
    B.upt = upt;
    double** vecs[] = {&B.x, &B.r, &B.z, &B.p, &B.q};
    for (double** v : vecs)
      if ((s = dalloc(c, v, 9 * (size_t)m)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &B.Mblk, 45 * (size_t)m)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &B.Bdiag, 9 * (size_t)m)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &B.Minv, 81 * (size_t)m)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &B.scal, 8)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &B.partial, 3 * (size_t)RED_BLOCKS)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &B.partial2, 3 * (size_t)RED_BLOCKS)) != STBA_OK) return bail(s);
  }
  {
    cudaError_t e1 = cudaMemcpyAsync(c->cams, h_cams.data(), h_cams.size() * 8, cudaMemcpyHostToDevice, c->stream);
    cudaError_t e2 = cudaMemcpyAsync(c->pts, h_pts.data(), h_pts.size() * 8, cudaMemcpyHostToDevice, c->stream);
    DevState h{};
    h.lambda = c->opt.lambda0;
    cudaError_t e3 = cudaMemcpyAsync(c->st, &h, sizeof h, cudaMemcpyHostToDevice, c->stream);
    cudaError_t e4 = cudaStreamSynchronize(c->stream);
    if (e1 || e2 || e3 || e4) return bail(fail(c, STBA_ERR_CUDA, "upload failed"));
  }
  // camera graph and the chunks of its observation pairs for the off-diagonal S' build
  {
    std::vector<int> base_cam(q);
    for (int64_t o = 0; o < q; ++o) base_cam[o] = c->in_cam[c->base_order[o]];
    build_camera_graph((int)m, (int)n, c->h_pt_off, base_cam, c->cgraph, true);
    const CameraGraph& g = c->cgraph;
    if ((int64_t)g.pairs.size() > INT32_MAX - PAIR_CHUNK)
      return bail(fail(c, STBA_ERR_INVALID_ARG, "more than 2^31 co-visible observation pairs"));
    if (!c->use_pcg && !g.pairs.empty()) {
      std::vector<int4> chunks;
      for (int x = 0; x < (int)m; ++x)
        for (int e = g.edge_off[x]; e < g.edge_off[x + 1]; ++e)
          for (int64_t p0 = g.pair_off[e]; p0 < g.pair_off[e + 1]; p0 += PAIR_CHUNK)
            chunks.push_back(make_int4(x, g.edge_y[e], (int)p0, (int)std::min<int64_t>(PAIR_CHUNK, g.pair_off[e + 1] - p0)));
      int4* d_chunks = nullptr;
      int2* d_pairs = nullptr;
      int *d_active, *d_flag, *d_excl, *d_tiles;
      const size_t nc = chunks.size();
      if ((s = upload(c, &d_chunks, chunks)) != STBA_OK) return bail(s);
      if ((s = upload(c, &d_pairs, g.pairs)) != STBA_OK) return bail(s);
      if ((s = dalloc(c, &d_active, nc)) != STBA_OK) return bail(s);
      if ((s = dalloc(c, &d_flag, nc + 1)) != STBA_OK) return bail(s);
      if ((s = dalloc(c, &d_excl, nc + 1)) != STBA_OK) return bail(s);
      if ((s = dalloc(c, &d_tiles, nc / 2048 + 2)) != STBA_OK) return bail(s);
      c->pchunks = PairChunks{d_chunks, d_pairs, (int)nc, d_active, nullptr, d_flag, d_excl, d_tiles};
    }
  }
  // observation data in the (point, camera) base order, the camera lists, and every buffer whose size does
  // not depend on the cluster assignment
  {
    const size_t Q = (size_t)q;
    std::vector<int> base_cam(Q), base_src(Q), base_pt(Q);
    std::vector<double> base_uv(2 * Q);
    std::vector<float> base_uvf(c->mixed ? 2 * Q : 0);
    std::vector<float4> base_uvdf(c->mixed ? Q : 0);
    for (size_t bo = 0; bo < Q; ++bo) {
      const int src = c->base_order[bo];
      base_cam[bo] = c->in_cam[src];
      base_src[bo] = src;
      base_pt[bo] = c->in_pt[src];
      const double u = c->in_uv[2 * (size_t)src], v = c->in_uv[2 * (size_t)src + 1];
      base_uv[2 * bo] = u;
      base_uv[2 * bo + 1] = v;
      if (c->mixed) {
        const float uh = (float)u, vh = (float)v;
        base_uvf[2 * bo] = uh;
        base_uvf[2 * bo + 1] = vh;
        base_uvdf[bo] = make_float4(uh, (float)(u - (double)uh), vh, (float)(v - (double)vh));
      }
    }
    std::vector<int> cam_off(m + 1, 0), cam_base(Q), ecam(Q), cam_warp_off(m + 1, 0), warp_cam;
    for (size_t bo = 0; bo < Q; ++bo) cam_off[base_cam[bo] + 1]++;
    for (int64_t j = 0; j < m; ++j) cam_off[j + 1] += cam_off[j];
    {
      std::vector<int> f(cam_off.begin(), cam_off.end() - 1);
      for (size_t bo = 0; bo < Q; ++bo) cam_base[f[base_cam[bo]]++] = (int)bo;
      for (int64_t j = 0; j < m; ++j)
        for (int e = cam_off[j]; e < cam_off[j + 1]; ++e) ecam[e] = (int)j;
    }
    // point and observation of every camera-list entry, copied into the slots with each clustering
    std::vector<int> ept(Q);
    std::vector<float2> euvf(c->mixed ? Q : 0);
    std::vector<double2> euvd(c->mixed ? 0 : Q);
    for (size_t e = 0; e < Q; ++e) {
      const int bo = cam_base[e];
      ept[e] = base_pt[bo];
      if (c->mixed)
        euvf[e] = make_float2(base_uvf[2 * (size_t)bo], base_uvf[2 * (size_t)bo + 1]);
      else
        euvd[e] = make_double2(base_uv[2 * (size_t)bo], base_uv[2 * (size_t)bo + 1]);
    }
    for (int64_t j = 0; j < m; ++j) {
      const int nw = (cam_off[j + 1] - cam_off[j] + 31) / 32;
      cam_warp_off[j + 1] = cam_warp_off[j] + nw;
      for (int w = 0; w < nw; ++w) warp_cam.push_back((int)j);
    }
    const int nwarps = cam_warp_off[m];
    ReorderArgs& A = c->reorder;
    A.q = (int)q;
    A.n = (int)n;
    A.m = (int)m;
    int *d_base_cam, *d_base_src, *d_cam_off, *d_cam_base, *d_ecam, *d_eo, *d_nsing, *d_cam_warp_off, *d_warp_cam,
        *d_cam_obs, *d_slots;
    double* d_base_uv;
    if ((s = upload(c, &c->obs_pt, base_pt)) != STBA_OK) return bail(s);
    if ((s = upload(c, &c->pt_off, c->h_pt_off)) != STBA_OK) return bail(s);
    if ((s = upload(c, &d_base_cam, base_cam)) != STBA_OK) return bail(s);
    if ((s = upload(c, &d_base_src, base_src)) != STBA_OK) return bail(s);
    d_base_uv = nullptr;   // FP64 observations in the iteration order: read by the FP64 kernels only
    if (!c->mixed && (s = upload(c, &d_base_uv, base_uv)) != STBA_OK) return bail(s);
    if ((s = upload(c, &d_cam_off, cam_off)) != STBA_OK) return bail(s);
    if ((s = upload(c, &d_cam_base, cam_base)) != STBA_OK) return bail(s);
    if ((s = upload(c, &d_ecam, ecam)) != STBA_OK) return bail(s);
    int* d_ept = nullptr;
    float2* d_euvf = nullptr;
    double2* d_euvd = nullptr;
    int2* d_slot_pv = nullptr;
    float2* d_slot_uvf = nullptr;
    double2* d_slot_uvd = nullptr;
    if ((s = upload(c, &d_ept, ept)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &d_slot_pv, 32 * (size_t)nwarps)) != STBA_OK) return bail(s);
    if (c->mixed) {
      if ((s = upload(c, &d_euvf, euvf)) != STBA_OK) return bail(s);
      if ((s = dalloc(c, &d_slot_uvf, 32 * (size_t)nwarps)) != STBA_OK) return bail(s);
    } else {
      if ((s = upload(c, &d_euvd, euvd)) != STBA_OK) return bail(s);
      if ((s = dalloc(c, &d_slot_uvd, 32 * (size_t)nwarps)) != STBA_OK) return bail(s);
    }
    if ((s = dalloc(c, &d_eo, Q)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &d_nsing, Q)) != STBA_OK) return bail(s);
    if ((s = upload(c, &d_cam_warp_off, cam_warp_off)) != STBA_OK) return bail(s);
    if ((s = upload(c, &d_warp_cam, warp_cam)) != STBA_OK) return bail(s);
    A.base_uvf = nullptr;
    A.base_uvdf = nullptr;
    if (c->mixed) {
      float* d_uvf;
      float4* d_uvdf;
      if ((s = upload(c, &d_uvf, base_uvf)) != STBA_OK) return bail(s);
      if ((s = upload(c, &d_uvdf, base_uvdf)) != STBA_OK) return bail(s);
      A.base_uvf = d_uvf;
      A.base_uvdf = d_uvdf;
      if ((s = dalloc(c, &c->obs_uvf, 2 * Q)) != STBA_OK) return bail(s);
      if ((s = dalloc(c, &c->obs_uvdf, Q)) != STBA_OK) return bail(s);
    }
    int* const* ints_q[] = {&c->obs_cam, &c->obs_vp, &c->obs_perm, &c->obs_base, &c->vp_point, &c->inv[0], &c->inv[1],
                            &c->key};
    for (int* const* pp : ints_q)
      if ((s = dalloc(c, const_cast<int**>(pp), Q)) != STBA_OK) return bail(s);
    int* d_start;   // [q+1] virtual-point starts, then [q+1] the camera-list scan
    if ((s = dalloc(c, &d_start, 2 * (Q + 1))) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &c->vp_off, Q + 1)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &c->pt_vp_off, (size_t)n + 1)) != STBA_OK) return bail(s);
    if (!c->mixed && (s = dalloc(c, &c->obs_uv, 2 * Q)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &d_cam_obs, Q)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &d_slots, 32 * (size_t)nwarps)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &c->tile_sum, Q / 2048 + 2)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &c->counts, 4)) != STBA_OK) return bail(s);   // nv, pairs, singles, active chunks
    // failure flags at their largest size (l <= m); the other cluster arrays live in the assignment blob
    if ((s = dalloc(c, &c->fail_flags, (size_t)m)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &c->cl_owned, (size_t)m)) != STBA_OK) return bail(s);
    {
      const std::vector<int> ones(m, 1);
      CK(cudaMemcpyAsync(c->cl_owned, ones.data(), (size_t)m * sizeof(int), cudaMemcpyHostToDevice, c->stream));
      CK(cudaStreamSynchronize(c->stream));
    }
    // per-iteration scratch (virtual-point arrays at their largest size, nv <= q)
    const size_t rs = c->mixed ? sizeof(float) : sizeof(double);
    char *vpa, *vpi, *pti, *pta, *vg, *ta, *gb;
    if ((s = dalloc(c, &vpa, 9 * Q * rs + 16)) != STBA_OK) return bail(s);   // zeroed in 16-byte pieces
    if ((s = dalloc(c, &vpi, 9 * Q * rs)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &pti, 9 * (size_t)n * rs)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &pta, 9 * (size_t)n * rs)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &vg, 9 * (size_t)m * rs)) != STBA_OK) return bail(s);
    if ((s = dalloc(c, &ta, 3 * (size_t)n * rs)) != STBA_OK) return bail(s);
    // the stored G_o of the camera pass, only when the pair pass reads them (option pair_blocks)
    const bool stored_g = !c->use_pcg && c->opt.pair_blocks == STBA_PAIR_BLOCKS_STORED;
    if ((s = dalloc(c, &gb, (stored_g ? 36 * Q : 1) * rs)) != STBA_OK) return bail(s);
    c->vp_acc = vpa;
    c->vp_info = vpi;
    c->pt_info = pti;
    c->pt_acc = pta;
    c->vgrad = vg;
    c->t_acc = ta;
    c->Gbuf = gb;
    A.obs_pt = c->obs_pt;
    A.pt_off = c->pt_off;
    A.base_cam = d_base_cam;
    A.base_src = d_base_src;
    A.base_uv = d_base_uv;
    A.start = d_start;
    A.obs_base = c->obs_base;
    A.obs_cam = c->obs_cam;
    A.obs_perm = c->obs_perm;
    A.obs_uv = c->obs_uv;
    A.obs_uvf = c->obs_uvf;
    A.obs_uvdf = c->obs_uvdf;
    A.obs_vp = c->obs_vp;
    A.vp_off = c->vp_off;
    A.vp_point = c->vp_point;
    A.pt_vp_off = c->pt_vp_off;
    A.cam_off = d_cam_off;
    A.cam_base = d_cam_base;
    A.ecam = d_ecam;
    A.ept = d_ept;
    A.euvf = d_euvf;
    A.euvd = d_euvd;
    A.slot_pv = d_slot_pv;
    A.slot_uvf = d_slot_uvf;
    A.slot_uvd = d_slot_uvd;
    A.eo = d_eo;
    A.nsing = d_nsing;
    A.cam_warp_off = d_cam_warp_off;
    A.cam_obs = d_cam_obs;
    A.slots = d_slots;
    {   // the padding slots of the camera pass never change
      std::vector<int> pad(32 * (size_t)nwarps, -1);
      if ((s = put(c, d_slots, pad)) != STBA_OK) return bail(s);
    }
    c->pchunks.nactive = c->counts + 3;
    c->pcg.counts = c->counts;
    c->clist = CamLists{d_cam_off, d_cam_obs};
    c->cslots = CamSlots{d_slots, d_warp_cam, nwarps, d_slot_pv, d_slot_uvf, d_slot_uvd};
  }
  if ((s = set_clusters_host(c, h_cl)) != STBA_OK) return bail(s);
  double F;
  if ((s = run_cost(c, &F)) != STBA_OK) return bail(s);
  *out = c;
  return STBA_OK;
}

stba_status stba_set_clusters(stba_ctx* c, const int32_t* cluster_assignment) {
  if (!c || !cluster_assignment) return STBA_ERR_INVALID_ARG;
  std::vector<int> h(c->m);
  stba_status s;
  if ((s = copy_in(c, h.data(), cluster_assignment, (size_t)c->m * 4)) != STBA_OK) return s;
  // the stored residuals follow the observation order; set_clusters_host carries them over
  return set_clusters_host(c, h);
}

stba_status stba_lm_iteration(stba_ctx* c, stba_iter_info* info) {
  if (!c) return STBA_ERR_INVALID_ARG;
  stba_status s = run_iteration(c);
  if (s != STBA_OK) return s;
  if (info) return read_info(c, info);
  return STBA_OK;
}

stba_status stba_solve(stba_ctx* c, int32_t max_iter, stba_iter_info* last) {
  if (!c || max_iter < 0) return STBA_ERR_INVALID_ARG;
  stba_iter_info info{};
  for (int t = 0; t < max_iter; ++t) {
    stba_status s = run_iteration(c);
    if (s != STBA_OK) return s;
    if ((s = read_info(c, &info)) != STBA_OK) return s;
    if (info.stop) break;
  }
  if (last) *last = info;
  return STBA_OK;
}

stba_status stba_cost(stba_ctx* c, double* F) {
  if (!c || !F) return STBA_ERR_INVALID_ARG;
  // recompute without disturbing the accepted-cost state: save and restore st->F
  DevState h;
  CK(cudaMemcpyAsync(&h, c->st, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  stba_status s = run_cost(c, F);
  CK(cudaMemcpyAsync(c->st, &h, sizeof h, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return s;
}

stba_status stba_get_params(stba_ctx* c, double* cameras, double* points) {
  if (!c) return STBA_ERR_INVALID_ARG;
  stba_status s;
  if (cameras && (s = copy_out(c, cameras, c->cams, 9 * (size_t)c->m * 8)) != STBA_OK) return s;
  if (points && (s = copy_out(c, points, c->pts, 3 * (size_t)c->n * 8)) != STBA_OK) return s;
  return STBA_OK;
}

stba_status stba_set_params(stba_ctx* c, const double* cameras, const double* points) {
  if (!c) return STBA_ERR_INVALID_ARG;
  if (c->tape_len > 0) c->tape_broken = true;
  if (cameras) {
    CK(cudaMemcpyAsync(c->cams, cameras, 9 * (size_t)c->m * 8,
                       is_device_ptr(cameras) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  }
  if (points) {
    CK(cudaMemcpyAsync(c->pts, points, 3 * (size_t)c->n * 8,
                       is_device_ptr(points) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  }
  return run_cost(c, nullptr);
}

stba_status stba_get_state(stba_ctx* c, double* lambda, double* F, int64_t* iteration) {
  if (!c) return STBA_ERR_INVALID_ARG;
  DevState h;
  CK(cudaMemcpyAsync(&h, c->st, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (lambda) *lambda = h.lambda;
  if (F) *F = h.F;
  if (iteration) *iteration = h.iteration;
  return STBA_OK;
}

stba_status stba_set_state(stba_ctx* c, double lambda, double F, int64_t iteration) {
  if (!c || !(lambda > 0) || !std::isfinite(lambda)) return STBA_ERR_INVALID_ARG;
  DevState h;
  CK(cudaMemcpyAsync(&h, c->st, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  h.lambda = lambda;
  h.iteration = iteration;
  if (F >= 0) h.F = F;
  CK(cudaMemcpyAsync(c->st, &h, sizeof h, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (F < 0) return run_cost(c, nullptr);
  return STBA_OK;
}

stba_status stba_last_step(stba_ctx* c, double* dc, double* dp) {
  if (!c) return STBA_ERR_INVALID_ARG;
  stba_status s;
  if (dc && (s = copy_out(c, dc, c->dc, 9 * (size_t)c->m * 8)) != STBA_OK) return s;
  if (dp && (s = copy_out(c, dp, c->dp, 3 * (size_t)c->n * 8)) != STBA_OK) return s;
  return STBA_OK;
}

stba_status stba_record(stba_ctx* c, int32_t max_iter) {
  if (!c || max_iter < 0) return STBA_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(c->stream));
  free_tape(c);
  if (max_iter == 0) return STBA_OK;
  const size_t nx = 9 * (size_t)c->m + 3 * (size_t)c->n;
  stba_status s;
  if ((s = dalloc_into(c, &c->tape_x, nx * (size_t)max_iter, c->tape_allocs)) != STBA_OK) return s;
  // the reverse pass's buffers are allocated here, once, so that stba_adjoint allocates nothing
  AdjointBuffers& A = c->adj;
  const size_t q = c->q;
  const bool ok = (s = dalloc_into(c, &c->tape_info, (size_t)max_iter, c->tape_allocs)) == STBA_OK &&
                  (s = dalloc_into(c, &A.a_c, 9 * (size_t)c->m, c->tape_allocs)) == STBA_OK &&
                  (s = dalloc_into(c, &A.a_p, 3 * (size_t)c->n, c->tape_allocs)) == STBA_OK &&
                  (s = dalloc_into(c, &A.u, 3 * (size_t)c->n, c->tape_allocs)) == STBA_OK &&
                  (s = dalloc_into(c, &A.zc, 9 * (size_t)c->m, c->tape_allocs)) == STBA_OK &&
                  (s = dalloc_into(c, &A.vpz, 6 * q, c->tape_allocs)) == STBA_OK &&   // nv <= q
                  (s = dalloc_into(c, &A.T, 12 * q, c->tape_allocs)) == STBA_OK &&
                  (s = dalloc_into(c, &A.qbar, 2 * q, c->tape_allocs)) == STBA_OK &&
                  (s = dalloc_into(c, &A.zeta, 3 * (size_t)c->n, c->tape_allocs)) == STBA_OK &&
                  (s = dalloc_into(c, &A.kappa, 3 * q, c->tape_allocs)) == STBA_OK &&   // nv <= q
                  (s = dalloc_into(c, &c->adj_save_x, nx, c->tape_allocs)) == STBA_OK;
  if (!ok) {
    free_tape(c);
    return s;
  }
  c->tape_cap = max_iter;
  return STBA_OK;
}

stba_status stba_adjoint(stba_ctx* c, const double* dL_dcams, const double* dL_dpts, double* dL_dobs,
                         double* dL_dcams0, double* dL_dpts0) {
  if (!c || !dL_dcams) return STBA_ERR_INVALID_ARG;
  if (c->use_pcg || c->use_spcg) return fail(c, STBA_ERR_STATE, "the adjoint covers the cluster solver only");
  if (c->opt.huber_a > 0) return fail(c, STBA_ERR_STATE, "the adjoint covers the plain least-squares objective only");
  if (c->mixed && !c->f32f) return fail(c, STBA_ERR_STATE, "the adjoint covers the FP32 cluster factor of mixed precision only");
  if (c->tape_len == 0) return fail(c, STBA_ERR_STATE, "no recorded iteration (call stba_record before iterating)");
  if (c->tape_broken)
    return fail(c, STBA_ERR_STATE, "the parameters were replaced between recorded iterations; record again");
  const int T = c->tape_len;
  const int64_t m = c->m, n = c->n, q = c->q;
  std::vector<stba_iter_info> info(T);
  CK(cudaMemcpyAsync(info.data(), c->tape_info, T * sizeof(stba_iter_info), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  // the buffers were allocated with the tape (stba_record): nothing is allocated here
  const AdjointBuffers& A = c->adj;
  double* save_x = c->adj_save_x;
  stba_status s;
  const size_t nx = 9 * (size_t)m + 3 * (size_t)n;
  DevState saved;
  CK(cudaMemcpyAsync(&saved, c->st, sizeof saved, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(save_x, c->cams, 9 * (size_t)m * 8, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(save_x + 9 * m, c->pts, 3 * (size_t)n * 8, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(A.a_c, dL_dcams, 9 * (size_t)m * 8, cudaMemcpyDefault, c->stream));
  if (dL_dpts) {
    CK(cudaMemcpyAsync(A.a_p, dL_dpts, 3 * (size_t)n * 8, cudaMemcpyDefault, c->stream));
  } else {
    CK(cudaMemsetAsync(A.a_p, 0, 3 * (size_t)n * 8, c->stream));
  }
  CK(cudaMemsetAsync(A.qbar, 0, 2 * (size_t)q * 8, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const std::vector<int> final_clusters = c->h_clusters;
  auto reverse_pass = [&]() -> stba_status {
    stba_status s2;
    for (int t = T - 1; t >= 0; --t) {
      if (!info[t].accepted) continue;   // a rejected step leaves x unchanged: the adjoint passes through
      const std::vector<int>& cl = c->tape_clusters[c->tape_cluster_id[t]];
      if (cl != c->h_clusters && (s2 = set_clusters_host(c, cl)) != STBA_OK) return s2;
      const double* slot = c->tape_x + nx * (size_t)t;
      CK(cudaMemcpyAsync(c->cams, slot, 9 * (size_t)m * 8, cudaMemcpyDeviceToDevice, c->stream));
      CK(cudaMemcpyAsync(c->pts, slot + 9 * m, 3 * (size_t)n * 8, cudaMemcpyDeviceToDevice, c->stream));
      if (c->mixed)
        enqueue_adjoint_step<float>(c, info[t].lambda_used, info[t].corrected, A);
      else
        enqueue_adjoint_step<double>(c, info[t].lambda_used, info[t].corrected, A);
      CK(cudaGetLastError());
    }
    CK(cudaStreamSynchronize(c->stream));
    // outputs (qbar is in the input order of the observations)
    if (dL_dcams0) CK(cudaMemcpyAsync(dL_dcams0, A.a_c, 9 * (size_t)m * 8, cudaMemcpyDefault, c->stream));
    if (dL_dpts0) CK(cudaMemcpyAsync(dL_dpts0, A.a_p, 3 * (size_t)n * 8, cudaMemcpyDefault, c->stream));
    if (dL_dobs) CK(cudaMemcpyAsync(dL_dobs, A.qbar, 2 * (size_t)q * 8, cudaMemcpyDefault, c->stream));
    return STBA_OK;
  };
  const stba_status s_pass = reverse_pass();
  const std::string pass_err = c->err;
  // restore the final state on every path: clusters, parameters, their residuals, and the LM state
  if (final_clusters != c->h_clusters && (s = set_clusters_host(c, final_clusters)) != STBA_OK) return s;
  CK(cudaMemcpyAsync(c->cams, save_x, 9 * (size_t)m * 8, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(c->pts, save_x + 9 * m, 3 * (size_t)n * 8, cudaMemcpyDeviceToDevice, c->stream));
  s = run_cost(c, nullptr);
  CK(cudaMemcpyAsync(c->st, &saved, sizeof saved, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (s_pass != STBA_OK) {
    c->err = pass_err;
    return s_pass;
  }
  return s;
}

stba_status stba_problem_info(stba_ctx* c, int64_t* out, int32_t n) {
  if (!c || !out || n < 0) return STBA_ERR_INVALID_ARG;
  stba_status st = refresh_counts(c);
  if (st != STBA_OK) return st;
  int maxn = 0;
  double s_elems = 0;
  for (int v : c->h_nk) {
    maxn = std::max(maxn, v);
    s_elems += 0.5 * (double)v * (v + 1);
  }
  size_t grown = 0;
  for (const GrowBuf* g : {&c->g_panel, &c->g_update, &c->g_res, &c->g_diag, &c->g_S, &c->g_b, &c->g_L, &c->g_Dinv,
                           &c->g_Ldiag, &c->g_scale, &c->g_x, &c->g_r, &c->g_blob})
    grown += g->bytes;
  const int64_t vals[12] = {c->m, c->n, c->q, c->l, c->nv, maxn, (int64_t)(c->bytes_base + grown),
                            c->build_items, c->launches_per_iter, c->n_pairs, (int64_t)c->factor_flops,
                            (int64_t)s_elems};
  for (int i = 0; i < n && i < 12; ++i) out[i] = vals[i];
  return STBA_OK;
}

stba_status stba_get_cluster_system(stba_ctx* c, int32_t k, double* S, double* b, int64_t* dim) {
  if (!c || k < 0 || k >= c->l) return STBA_ERR_INVALID_ARG;
  if (c->use_pcg) return fail(c, STBA_ERR_STATE, "the PCG solver forms no cluster systems");
  if (c->use_spcg) return fail(c, STBA_ERR_STATE, "the split PCG solver forms the diagonal blocks of S' only");
  const int nk = c->h_nk[k], np = c->h_np[k];
  if (dim) *dim = nk;
  if (!S && !b) return STBA_OK;
  const size_t rs = 8;
  std::vector<char> raw((size_t)np * np * rs), rawb((size_t)np * rs);
  CK(cudaMemcpyAsync(raw.data(), (char*)c->S + (size_t)c->h_S_off[k] * rs, raw.size(), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(rawb.data(), (char*)c->b + (size_t)c->h_v_off[k] * rs, rawb.size(), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  auto at = [&](const std::vector<char>& v, size_t i) -> double { return ((const double*)v.data())[i]; };
  if (S) {
    std::vector<double> full((size_t)nk * nk);
    for (int r = 0; r < nk; ++r)
      for (int cc = 0; cc <= r; ++cc) {
        const double a = at(raw, (size_t)r * np + cc);
        full[(size_t)r * nk + cc] = a;
        full[(size_t)cc * nk + r] = a;
      }
    if (is_device_ptr(S)) {
      CK(cudaMemcpy(S, full.data(), full.size() * 8, cudaMemcpyHostToDevice));
    } else {
      std::memcpy(S, full.data(), full.size() * 8);
    }
  }
  if (b) {
    std::vector<double> hb(nk);
    for (int r = 0; r < nk; ++r) hb[r] = at(rawb, r);
    if (is_device_ptr(b)) {
      CK(cudaMemcpy(b, hb.data(), hb.size() * 8, cudaMemcpyHostToDevice));
    } else {
      std::memcpy(b, hb.data(), hb.size() * 8);
    }
  }
  return STBA_OK;
}

stba_status stba_set_timing(stba_ctx* c, int32_t on) {
  if (!c) return STBA_ERR_INVALID_ARG;
  c->timing = on != 0;
  return STBA_OK;
}

stba_status stba_stage_times(stba_ctx* c, float* ms, int32_t n, int32_t* count) {
  if (!c) return STBA_ERR_INVALID_ARG;
  if (count) *count = NSTAGES;
  if (!ms) return STBA_OK;
  if (c->have_stage_times) {
    CK(cudaEventSynchronize(c->ev[NSTAGES]));
    for (int i = 0; i < NSTAGES; ++i) CK(cudaEventElapsedTime(&c->stage_ms[i], c->ev[i], c->ev[i + 1]));
  }
  for (int i = 0; i < n && i < NSTAGES; ++i) ms[i] = c->have_stage_times ? c->stage_ms[i] : -1.0f;
  return STBA_OK;
}

}  // extern "C"
