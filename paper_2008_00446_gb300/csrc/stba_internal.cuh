// Internal declarations shared by the translation units of libstba.so (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <memory>
#include <vector>

#include "../../include/stba.h"

namespace stba {

// ------------------------------------------------------------------------------------------------------
// Device problem description: pointers into the context's device buffers, passed by value to kernels.
// Observations are sorted by (point, cluster of the camera, camera), so every virtual point (a distinct
// (point, cluster) pair, Sec. 4.1-4.2) is a contiguous run and every point is a contiguous run of
// virtual points.
// ------------------------------------------------------------------------------------------------------
struct DevProblem {
  int m, n, q, l, nv;
  const double* cams;      // [m][9] current cameras
  const double* pts;       // [n][3] current points
  const float* cams_f;     // [m][9], [n][3] FP32 copies made once per iteration (mixed precision), so
  const float* pts_f;      //   that the per-observation kernels convert nothing on the FP64 pipe
  const int* obs_cam;      // [q] camera of each sorted observation
  const int* obs_vp;       // [q] virtual point of each sorted observation
  const int* obs_pt;       // [q] point of each sorted observation
  const int* obs_base;     // [q] position of each sorted observation in the (point, camera) order
  const double* obs_uv;    // [q][2] FP64 observations (FP64 mode only; null in mixed precision)
  const float* obs_uvf;    // [q][2] FP32 copy (mixed precision)
  const float4* obs_uvdf;  // [q] double-float copy (u_hi, u_lo, v_hi, v_lo) (mixed precision)
  const int* vp_off;       // [nv+1] observation range of each virtual point
  const int* vp_point;     // [nv] point of each virtual point
  const int* pt_vp_off;    // [n+1] virtual-point range of each point
  const int* pt_off;       // [n+1] observation range of each point
  const int* cam_local;    // [m] index of the camera inside its cluster (cameras ordered by index)
  const int* cam_cluster;  // [m]
  const int* cluster_cams;     // [m] cameras of every cluster, concatenated, ascending per cluster
  const int* cluster_cam_off;  // [l+1]
  const int* cluster_np;       // [l] padded dimension Np_k (multiple of the Cholesky tile)
  const int* cluster_n;        // [l] dimension 9 n_k
  const int64_t* S_off;        // [l] element offset of the dense Np_k x Np_k block of cluster k
  const int64_t* v_off;        // [l] element offset of the length-Np_k vectors of cluster k
  double huber_a;              // Huber scale a (0: plain least squares)
  const float* res_f;          // [q][2] residuals f_o at the current x, computed in FP64, stored in the
  const double* res_d;         //        working precision (res_f in mixed mode, res_d in FP64 mode)
  const int* base_pos;         // [q] sorted position of every base-order observation (current assignment)
  int pair_recompute;          // 1: the pair pass recomputes G_o instead of reading the camera pass's copy
  int sharded;                 // 1: this process owns only some clusters (stba_set_shard)
  const int* cluster_owned;    // [l] 1 where this process builds, factors and solves cluster k (all 1 unless
                               //     sharded)
};

template <typename real> __host__ __device__ inline const real* res_ptr(const DevProblem& P);
template <> __host__ __device__ inline const float* res_ptr<float>(const DevProblem& P) { return P.res_f; }
template <> __host__ __device__ inline const double* res_ptr<double>(const DevProblem& P) { return P.res_d; }

// Device-resident LM state; the captured iteration graph reads and writes it in place.
struct DevState {
  double F;              // F(x) at the current parameters
  double lambda;         // current damping
  double lambda_used;    // damping of the step in flight
  long long iteration;
  unsigned long long grad_max_bits;   // bits of max |J^T f| (non-negative double)
  int failed;            // clusters whose factorisation failed this iteration
  int corrected;         // correction active this iteration
  int nonfinite;         // a non-positive depth was met in the cost at x + dx
  int boosted;           // FP32 pivots raised by static pivoting this iteration
  stba_iter_info info;   // record of the last finished iteration
};

struct Settings {
  double correction_lambda;
  double lambda_min;
  double ftol, gtol, xtol;
  int correction;
  int refine_steps;
};

constexpr int NSTAGES = 5;

// Kernel launchers (explicitly instantiated for float and double in stba_kernels.cu / stba_chol.cu).
template <typename real> struct Scratch {
  real* vp_acc;    // [nv][9]: V = sum Jp^T Jp (6, packed xx xy xz yy yz zz) and w' = -sum Jp^T f (3)
  real* vp_info;   // [nv][9]: L^-1 of V' (6, packed l00 l10 l11 l20 l21 l22) and y = V'^-1 w' (3)
  real* pt_info;   // [n][9]: C^-1 (6, packed symmetric) and w (3) of the physical points
  real* pt_acc;    // [n][9]: C (6, packed) and w (3) of the physical points, summed over their virtual points
  double* S;       // cluster-diagonal S' (dense lower triangles, per-cluster padded blocks); FP64 sums
  double* b;       // b' (per-cluster padded vectors); FP64 sums
  real* vgrad;     // [m][9] camera gradient v = -J_c^T f
  real* t_acc;     // [n][3] sum_o J_p^T J_c dc per point
  double* dc;      // [m][9] camera step
  float* dcf;      // [m][9] FP32 copy of the camera step (mixed precision)
  double* dp;      // [n][3] point step
  double* partial; // reduction partials
};

struct CamLists {     // observations of every camera (sorted positions), host-built per assignment
  const int* cam_obs_off;   // [m+1]
  const int* cam_obs;       // [q]
};

struct CamSlots {     // per-camera observation lists padded to whole warps, for the camera pass
  const int* slots;         // [32 * nwarps] sorted observation position, or -1 (padding)
  const int* warp_cam;      // [nwarps] camera of each warp's 32 slots
  int nwarps;
  // per slot, written with the lists (stba_order.cu), so that the camera pass reads them in its own order
  // instead of gathering them by observation position: (point, virtual point | bit 31 when the virtual
  // point has no other observation) and the observation in the working precision
  const int2* pv;           // [32 * nwarps]
  const float2* uvf;        // [32 * nwarps] FP32 (mixed precision) or null
  const double2* uvd;       // [32 * nwarps] FP64 or null
};

struct PairChunks {   // observation pairs of the camera graph, by edge, cut into chunks (built at create)
  const int4* chunks;       // (camera x, camera y < x, first pair, number of pairs <= PAIR_CHUNK)
  const int2* pairs;        // (base position of the observation by x, base position of the one by y)
  int nchunks;
  const int* active;        // [nchunks] the chunks whose two cameras share a cluster (set per assignment)
  const long long* nactive; // device count of them
  int* flag;                // [nchunks + 1] scratch of the listing
  int* excl;                // [nchunks + 1]
  int* tile_sum;            // [nchunks / 2048 + 2]
};
// lists the chunks inside clusters for the current assignment (cam_cluster on the device)
void launch_list_chunks(const PairChunks& B, const int* cam_cluster, const int* owned, long long* nactive,
                        cudaStream_t stream);
constexpr int PAIR_CHUNK = 64;

// Camera graph (stba_graph.cu): edges (x, y), y < x, grouped by x with y ascending; weight = number of
// common points; the observation pairs of each edge (base positions, observations sorted by (point,
// camera)), ordered by point.
struct SgcBase;   // the initial state of stochastic graph clustering on a graph (stba_graph.cu)
struct CameraGraph {
  std::vector<int> edge_off;       // [m+1]
  std::vector<int> edge_y;         // [E]
  std::vector<int> edge_w;         // [E]
  std::vector<int64_t> pair_off;   // [E+1]
  std::vector<int2> pairs;         // [P]
  mutable std::shared_ptr<const SgcBase> sgc_base;   // built on the first draw
};
void build_camera_graph(int m, int n, const std::vector<int>& pt_off, const std::vector<int>& base_cam,
                        CameraGraph& g, bool with_pairs);
// Stochastic graph clustering (Sec. 4.4, Eq. 16) of the camera graph: labels [m] (0..l-1, numbered by
// smallest camera), *nclusters = l.  The batch form draws count clusterings (seeds seed, seed+1, ...) in
// parallel host threads into labels [count][m].
void sgc_sample(const CameraGraph& g, int m, int gamma, double beta, uint64_t seed, int* labels, int* nclusters);
void sgc_sample_batch(const CameraGraph& g, int m, int gamma, double beta, uint64_t seed, int count, int* labels,
                      int* nclusters);

// Re-ordering for a new cluster assignment (stba_order.cu).  Base = the (point, camera) order of create.
struct ReorderArgs {
  int q, n, m;
  const int* obs_pt;        // [q] point of every position (the same in both orders)
  const int* pt_off;        // [n+1]
  const int* base_cam;      // [q] camera, original index and observation of every base position
  const int* base_src;
  const double* base_uv;    // [q][2]
  const float* base_uvf;    // [q][2] or null
  const float4* base_uvdf;  // [q] or null
  const int* cam_cluster;   // [m] the new assignment
  const int* inv_old;       // [q] new position of every base position under the previous assignment
  int* inv_new;             // [q] ... under the new one
  int* start;               // [q] 1 where a virtual point starts
  int *obs_base, *obs_cam, *obs_perm;
  double* obs_uv;
  float* obs_uvf;
  float4* obs_uvdf;
  int *obs_vp, *vp_off, *vp_point, *pt_vp_off;
  const int* cam_off;       // [m+1] observations of every camera
  const int* cam_base;      // [q]   their base positions, ascending
  const int* ecam;          // [q]   the camera of every entry of cam_base
  const int* ept;           // [q]   the point of every entry of cam_base
  const float2* euvf;       // [q]   its observation in FP32 (mixed precision) or null
  const double2* euvd;      // [q]   its observation in FP64 (FP64 mode) or null
  int2* slot_pv;            // CamSlots::pv, uvf, uvd (written by k_cam_place)
  float2* slot_uvf;
  double2* slot_uvd;
  int* eo;                  // [q]   the new position of every entry of cam_base (scratch of the assignment)
  int* nsing;               // [q]   per base position: its new position, bit 31 set when its virtual point
                            //       has no other observation (scratch of the assignment)
  const int* cam_warp_off;  // [m+1] warps of every camera in the camera pass
  int* cam_obs;             // [q] new positions, single-observation virtual points first
  int* slots;               // [32 * warps] the same padded to whole warps (-1)
};
// key: [q] scratch; tile_sum: [q / 2048 + 1] scratch; A.start: [2 (q + 1)]; counts: [3] -> number of virtual
// points, number of camera-pair instances, number of single-observation virtual points.  With res_old, the residuals are carried over into res_new in the new order.
template <typename real>
void launch_reorder(const ReorderArgs& A, int* key, int* tile_sum, long long* counts, const real* res_old,
                    real* res_new, cudaStream_t stream);

// zeroes the virtual-point accumulators (9 nv reals of real_bytes each; nv = counts[0] on the device)
void launch_zero_vp(void* vp_acc, const long long* counts, int real_bytes, cudaStream_t stream);

constexpr int RED_BLOCKS = 456;    // 3 x 152 SMs: fixed grid of the deterministic reductions
constexpr int RED_THREADS = 256;

template <typename real>
void launch_iter_begin(DevState* st, const Settings& s, cudaStream_t stream);
template <typename real>
void launch_vp_reduce(const DevProblem& P, Scratch<real> W, cudaStream_t stream);
template <typename real>
void launch_vp_finalize(const DevProblem& P, Scratch<real> W, DevState* st, const long long* counts,
                        cudaStream_t stream, const double* pt_sums = nullptr);
// Sharded iteration: per point, the sums over this process's virtual points of V (packed 6) and w' (3), FP64
// [n][9] (the other processes' virtual points are zero here); summed over the processes they are C_i, w_i.
template <typename real>
void launch_pt_sums(const DevProblem& P, Scratch<real> W, double* out, cudaStream_t stream);
// dcf = (float) dc, n values
void launch_dc_to_float(const double* dc, float* dcf, int64_t n, cudaStream_t stream);
// to_double = 1: *x = st->failed; 0: st->failed = (int) *x
void launch_failed_io(DevState* st, double* x, int to_double, cudaStream_t stream);
template <typename real>
void launch_rcs_build(const DevProblem& P, Scratch<real> W, CamSlots CS, PairChunks B, real* Gbuf, DevState* st,
                      cudaStream_t stream, cudaStream_t side = nullptr, cudaEvent_t fork = nullptr,
                      cudaEvent_t join = nullptr);
template <typename real>
void launch_point_rhs(const DevProblem& P, Scratch<real> W, cudaStream_t stream);
// FP32 copies of the cameras and points (mixed precision, once per iteration)
void launch_params_to_float(const DevProblem& P, float* cams_f, float* pts_f, cudaStream_t stream);
template <typename real>
void launch_point_update(const DevProblem& P, Scratch<real> W, cudaStream_t stream);
// k_cam_rt + k_cost: rt is a [m][15] FP64 scratch (R, t, f, k1, k2 of x + dx); residuals go to rout.  In mixed
// mode with a step, the cost runs in double-float arithmetic with the scratch tables cam_df [m][28] and
// pt_df [n][6] (floats).
template <typename real>
void launch_cost(const DevProblem& P, const double* dc, const double* dp, double* rt, float* cam_df, float* pt_df,
                 double* partial, DevState* st, real* rout, cudaStream_t stream);
// with_step = 1: stop tests and accept / reject of the step in W.dc / W.dp; 0: F(x) -> st->F.
template <typename real>
void launch_finalize(const DevProblem& P, Scratch<real> W, DevState* st, const Settings& s, int with_step,
                     cudaStream_t stream);
template <typename real>
void launch_apply(const DevProblem& P, const double* dc, const double* dp, double* cams, double* pts,
                  const real* r_cand, real* r_cur, DevState* st, cudaStream_t stream);
// Sets the dynamic shared-memory limits of the kernels that need more than 48 KB (call outside capture).
void configure_kernels(int max_np);
void configure_solve_kernels(int max_np);
// SM count of the current device (queried once); grids of persistent or grid-stride kernels are sized by it.
int num_sms();
// Shared memory (dynamic and static) of the cluster solve for clusters of up to max_np unknowns (padded).
size_t solve_smem_bytes(bool mixed, int tile, int max_np);

// Cholesky (stba_chol.cu)
struct CholPlan {
  const int2* panel_items;   // (cluster, tile row i) for every step, concatenated
  const int2* update_items;  // (cluster, (i << 16) | j) for every step, concatenated
  const int2* res_items;     // (cluster, 32-row block) of the refinement residual
  int n_res_items;
  const int2* diag_items;    // (cluster, diagonal tile) for the inverses of the diagonal tiles
  int n_diag_items;
  int nsteps;
  const int* h_panel_off;    // host arrays [nsteps + 1] (launch sizes)
  const int* h_update_off;
  int max_np;
  cudaStream_t side_stream;  // second stream of the trailing updates, joined back before the solves
  int prio_high, prio_low;   // launch priorities of the panels and of the trailing updates
  cudaEvent_t ev_fork, ev_join;
  cudaEvent_t ev_copy;            // the scaled copy of the tile columns after the first (side stream), or null
  const cudaEvent_t* ev_panel;    // [nsteps]
  const cudaEvent_t* ev_update;   // [nsteps]
  int tile;                       // factorisation tile T (the dense blocks are padded to it)
  int update_tc;                  // 1: trailing updates on the tensor cores (FP32 factor, T = 64); the update
                                  // items are then (cluster, (i0 << 16) | j) for the tile pair (i0, i0 + 1) x j
  int split;                      // 1: split panel (FP32 factor, T = 64): each step's panel items list the
                                  // diagonal tiles (cluster, kt) first, h_diag_count[kt] of them, then the
                                  // tiles below them
  const int* h_diag_count;        // host [nsteps]
  int persistent;                 // 1: one persistent launch factors every cluster (FP32 factor, T = 64)
  const int* cluster_items;       // [n_cluster_items] the clusters this process factors
  int n_cluster_items;
  int solve_cs;                   // CTAs per thread-block cluster of the cluster solves (2, 4 or 8)
};
struct FactorBuffers {
  void* L;          // factor (F = float or double), same layout as S'
  void* Dinv;       // inverses of the diagonal tiles, T x T per tile, v_off[k] * T offset per cluster;
                    // their transposes follow at offset v_total * T
  void* Ldiag;      // factored diagonal tiles L_kk (same tile layout as Dinv).  Kept out of L: every CTA of a
                    // panel step reads the unfactored A_kk from L, so it must not be overwritten in place
  double* scale;    // [v_total] Jacobi scaling s_i = S_ii^-1/2
  double* x;        // [v_total] solution
  double* r;        // [v_total] refinement residual
  int* fail_flags;  // [l]
  int* boosted;     // counter of raised pivots (in DevState)
  int64_t v_total;
};
int factor_tile(bool mixed);
template <typename F>
void launch_factor(const DevProblem& P, const double* S, const FactorBuffers& fb, const CholPlan& plan,
                   cudaStream_t stream);
// x = S'^-1 b per cluster, scattered to dc [m][9] (and to its FP32 copy dcf when not null)
template <typename F>
void launch_solve(const DevProblem& P, const double* S, const double* b, const FactorBuffers& fb,
                  const CholPlan& plan, int refine_steps, double* dc, float* dcf, cudaStream_t stream);
void launch_count_failures(const int* fail_flags, int l, DevState* st, cudaStream_t stream);

// Adjoint of one accepted step (stba_adjoint.cu).  With the forward step at x_t recomputed in W and fb
// (dc, dp, vp_info, pt_info, S', the cluster factors), maps the upstream adjoint (a_c, a_p) of x_{t+1} in
// place to that of x_t and adds the observation adjoint to qbar, indexed by input order through perm.
// W.b is overwritten (it carries the right-hand side of the adjoint cluster solve).
struct AdjointBuffers {
  double* a_c;    // [m][9] in / out
  double* a_p;    // [n][3] in / out
  double* u;      // [n][3] C^-1 a_p
  double* zc;     // [m][9] S'^-1 a^_c
  double* vpz;    // [nv][6] z_v and the expanded point step of every virtual point
  double* T;      // [q][12] per-observation terms
  double* qbar;   // [q][2] observation adjoint, input order
  double* zeta;   // [n][3] corrected steps: h-weighted mean of the copies' z_v per point
  double* kappa;  // [nv][3] corrected steps: (z_v - zeta_i) o w_i / H_i per virtual point
};
template <typename real>
void launch_adjoint_step(const DevProblem& P, Scratch<real> W, CamLists CL, const FactorBuffers& fb,
                         const CholPlan& plan, int refine_steps, const int* perm, double lam, int corrected,
                         const AdjointBuffers& A, cudaStream_t stream);
void launch_set_lambda(DevState* st, double lam, cudaStream_t stream);

// Full-RCS comparator (stba_pcg.cu): block-Jacobi preconditioned CG on S dc = b over all cameras, matrix-free.
struct PcgBuffers {
  void* J;          // [q][24] J_c and J_p of every observation (working precision)
  double* Mblk;     // [m][45] diagonal blocks of S (lower, undamped B part)
  double* Bdiag;    // [m][9] diag(J_c^T J_c)
  double* Minv;     // [m][81] inverse damped diagonal blocks (the preconditioner)
  double *x, *r, *z, *p, *q;   // [m][9] CG vectors (q also carries the right-hand side at the start)
  void* pw;         // [m][9] p in the working precision
  void* tpt;        // [n][3] E^T p
  void* upt;        // [n][3] C^-1 E^T p
  double* scal;     // b.b, r.z (two parity slots), r.r
  double* partial;  // [3][RED_BLOCKS]
  double* partial2; // [3][RED_BLOCKS]
  bool split;       // STBA_SOLVER_PCG_CLUSTERS: the method's clustered system S' over virtual points
  void* tvp;        // [q][3] (split) E'^T p per virtual point, working precision
  void* uvp;        // [q][3] (split) C'^-1 E'^T p
  const long long* counts;   // (split) device counters, [0] = number of virtual points
};
// split variant: zeroes the diagonal blocks of S' (the camera pass then adds into them)
void launch_spcg_zero(const DevProblem& P, double* S, cudaStream_t stream);
// zeroes the 3 nv reals of a per-virtual-point vector (nv = counts[0] on the device)
void launch_zero_vp3(void* p, const long long* counts, int real_bytes, cudaStream_t stream);
// Jacobians, preconditioner and right-hand side; x = 0, r = b, p = M^-1 b.
template <typename real>
void pcg_prepare(const DevProblem& P, Scratch<real> W, CamSlots CS, const PcgBuffers& B, DevState* st,
                 cudaStream_t stream);
// Iterates until ||r|| <= tol ||b|| or max_iter (the host reads the residual every few iterations), then
// writes dc (and its FP32 copy).  Returns the number of iterations.
template <typename real>
int pcg_iterate(const DevProblem& P, Scratch<real> W, CamSlots CS, const PcgBuffers& B, int max_iter, double tol,
                DevState* st, cudaStream_t stream);

}  // namespace stba
