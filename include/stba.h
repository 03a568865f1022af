/*
 * stba.h -- C ABI of libstba.so: the Levenberg-Marquardt (LM) iteration of Stochastic Bundle Adjustment
 * (Zhou et al., "Stochastic Bundle Adjustment for Efficient and Scalable 3D Reconstruction", ECCV 2020)
 * on one NVIDIA GB300 (sm_103a).
 *
 * Problem (Sec. 3): m cameras c_j in R^9, n points p_i in R^3 and q projections q_o in R^2.  The objective
 * is F(x) = ||f(x)||^2 with f_o = pi(c_cam(o), p_pt(o)) - q_o.  Camera parameters, in this order:
 *   angle-axis rotation w (3), translation t (3), focal length f, radial distortion k1, k2;
 *   Xc = R(w) p + t, (x, y) = Xc.xy / Xc.z, pi = f (1 + k1 r^2 + k2 r^4) (x, y), r^2 = x^2 + y^2.
 * Pixel coordinates are offsets from the image centre.
 *
 * One call of stba_lm_iteration is one pass of Algorithm 1 (Appendix C) for the current cluster
 * assignment: residuals and Jacobians, the clustered reduced camera system S' (Eq. 10) with one virtual
 * copy of each point per cluster that sees it (Sec. 4.1-4.2), the steepest-descent correction when
 * lambda >= correction_lambda (Sec. 4.3), one dense Cholesky solve per cluster (Eq. 13), the point
 * update of Eq. 15, the cost F(x + dx) and the accept / reject rule with lambda /= 3 or *= 3.
 *
 * Conventions
 *   - Every array argument may be a host pointer or a device pointer (detected with
 *     cudaPointerGetAttributes); it is only read (or written) during the call.  The caller keeps
 *     ownership of its arrays.  The library owns all device memory it allocates (freed by stba_destroy).
 *   - All device work is enqueued on the CUDA stream given to stba_create (NULL = legacy default stream).
 *     Calls that return values to the host synchronise that stream.
 *   - A context is not thread safe; use one context per host thread.
 *   - Errors return a status; stba_last_error(ctx) gives a message.  A failed call leaves the
 *     parameters unchanged.
 */
#ifndef STBA_H
#define STBA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stba_ctx stba_ctx;

typedef enum {
  STBA_OK = 0,
  STBA_ERR_INVALID_ARG = 1, /* bad sizes, indices out of range, duplicate projections, empty cluster */
  STBA_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  STBA_ERR_OOM = 3,         /* device allocation failed */
  STBA_ERR_NOT_SPD = 4,     /* reserved: a failed factorisation is reported in stba_iter_info instead */
  STBA_ERR_NONFINITE = 5,   /* non-finite input values, or a point behind a camera (depth <= 1e-9) */
  STBA_ERR_TIMEOUT = 6,     /* reserved for bounded device waits */
  STBA_ERR_STATE = 7        /* wrong call order, or lambda above 1e16 */
} stba_status;

typedef enum { STBA_FP64 = 0, STBA_MIXED = 1 } stba_precision;

typedef enum {
  STBA_SOLVER_CLUSTERS = 0, /* the method: one dense LL^T per cluster system S'_k (Eq. 13) */
  STBA_SOLVER_PCG_FULL = 1, /* the comparator: plain LM on the full reduced camera system of all cameras
                               (Eq. 5, clusters ignored), solved by block-Jacobi preconditioned conjugate
                               gradients, matrix-free; not captured in a graph (the host checks the residual) */
  STBA_SOLVER_PCG_CLUSTERS = 2 /* the method with its split system S' dc = b' (Eq. 10, 13) solved inexactly by
                               the same block-Jacobi PCG, matrix-free over the virtual points, instead of the
                               cluster factorisations (Sec. 6); stops at pcg_tol or pcg_max_iter */
} stba_linear_solver;

typedef struct {
  int32_t precision;        /* STBA_FP64: everything in FP64.  STBA_MIXED: residuals, Jacobians and the
                               Schur accumulation in FP32; factorisation, refinement and cost sums FP64 */
  int32_t correction;       /* 1: steepest-descent correction when lambda >= correction_lambda (Sec. 4.3) */
  double lambda0;           /* initial damping lambda, 1e-4 (Sec. 5.1, Algorithm 1) */
  double lambda_min;        /* floor applied after an accepted step (0 = none; the paper's ablation
                               uses 0.1, Sec. 5.4) */
  double correction_lambda; /* 0.1 (Sec. 4.3) */
  double ftol, gtol, xtol;  /* stop tolerances (Sec. 5.1: 1e-6); <= 0 disables a test */
  int32_t refine_steps;     /* FP64 iterative-refinement steps per cluster solve (default 1) */
  int32_t use_graph;        /* 1: replay each LM iteration as one captured CUDA graph */
  int32_t linear_solver;    /* stba_linear_solver (default STBA_SOLVER_CLUSTERS) */
  int32_t pcg_max_iter;     /* conjugate-gradient iteration limit per LM step (default 500) */
  double pcg_tol;           /* CG stops at ||S dc - b|| <= pcg_tol ||b|| (default 1e-6) */
  double huber_a;           /* Huber loss scale a (Sec. 5.1 uses 0.5); 0 = plain least squares (default).
                               F = sum over observations of rho(||f_o||^2), rho(s) = s for s <= a^2 and
                               2 a sqrt(s) - a^2 beyond (Ceres' HuberLoss); each observation's residual and
                               Jacobian rows enter the normal equations scaled by sqrt(rho'(||f_o||^2)) at
                               the current x.  Not supported by stba_adjoint and stba_cost_noalloc. */
  int32_t factor_tile;      /* tile of the cluster factorisation: 0 = default (64 for the FP32 factor of
                               STBA_MIXED, 32 for FP64); STBA_MIXED also accepts 32.  stba_autotune picks
                               between the candidates by timing. */
  int32_t factor_update;    /* trailing update A_ij -= L_ik L_jk^T of the cluster factorisation (Eq. 13's
                               dense LL^T): 0 = default (STBA_FACTOR_UPDATE_TENSOR where it applies, else
                               STBA_FACTOR_UPDATE_SIMT); STBA_FACTOR_UPDATE_SIMT = FP32/FP64 FMA on the CUDA
                               cores; STBA_FACTOR_UPDATE_TENSOR = tcgen05 tensor cores, TF32 operands split
                               in three products for FP32 accuracy (the FP32 factor of STBA_MIXED with tile
                               64 only; other settings return STBA_ERR_INVALID_ARG). */
  int32_t factor_panel;     /* panel of each tile step of the cluster factorisation: 0 = default (for the
                               FP32 factor with tile 64: STBA_FACTOR_PANEL_SPLIT when the tiles of all
                               clusters outnumber the SMs, i.e. a step runs in several waves, else _STACKED;
                               _STACKED otherwise);
                               STBA_FACTOR_PANEL_STACKED = one kernel per step factors the stacked panel of
                               the diagonal tile and each tile below it (the diagonal tile redundantly per
                               tile row); STBA_FACTOR_PANEL_SPLIT = the diagonal tile is factored and
                               inverted once per cluster, the tiles below are its products with the inverse;
                               STBA_FACTOR_PANEL_PERSISTENT = one launch factors every cluster, a thread-block
                               cluster of 8 CTAs per camera cluster running all its tile steps with cluster
                               barriers between them (SPLIT and PERSISTENT: the FP32 factor of STBA_MIXED
                               with tile 64 only; other settings return STBA_ERR_INVALID_ARG). */
  int32_t solve_cluster;    /* CTAs per thread-block cluster of each camera cluster's triangular solves
                               (2, 4 or 8; 0 = default: 8 while the clusters' solve CTAs fit in two waves on
                               the SMs, else 4): more CTAs share a tile step's products, fewer make its
                               cluster barrier and distributed-shared-memory exchange cheaper. */
  int32_t pair_blocks;      /* off-diagonal camera blocks of S' (Eq. 10, 13), -sum over the observation pairs
                               of a virtual point of G_a^T G_b with G_o = L_v^-1 Jp,o^T Jc,o:
                               STBA_PAIR_BLOCKS_RECOMPUTE (default) = the pair pass recomputes each G_o from
                               the point, the observation, its residual and the virtual point's L_v^-1 (no G
                               buffer, fewer bytes moved);
                               STBA_PAIR_BLOCKS_STORED = the camera pass stores every G_o (36 reals per
                               observation of device memory) and the pair pass reads them.
                               Both give the same S': in FP32 every pass evaluates the Jacobian rows with
                               each operation rounded on its own, so stored and recomputed G_o are bitwise
                               equal (up to the order of the FP64 atomic sums). */
  int32_t factor_fp64;      /* STBA_MIXED only: 1 = factor the cluster systems in FP64 (tile 32, CUDA cores)
                               under the FP32 Jacobians and Schur terms instead of the default FP32 factor
                               with FP64 refinement -- the precision Eq. 13's solve has in the paper's
                               CPU code, at the FP64 rate of this GPU.  Not with factor_tile 64, the tensor-
                               core update, the split or persistent panel (STBA_ERR_INVALID_ARG), nor with
                               stba_adjoint (STBA_ERR_STATE); stba_autotune keeps it as the single
                               configuration.  0 = FP32 factor (default). */
} stba_options;

enum { STBA_PAIR_BLOCKS_DEFAULT = 0, STBA_PAIR_BLOCKS_STORED = 1, STBA_PAIR_BLOCKS_RECOMPUTE = 2 };

enum { STBA_FACTOR_UPDATE_DEFAULT = 0, STBA_FACTOR_UPDATE_SIMT = 1, STBA_FACTOR_UPDATE_TENSOR = 2 };
enum { STBA_FACTOR_PANEL_DEFAULT = 0, STBA_FACTOR_PANEL_STACKED = 1, STBA_FACTOR_PANEL_SPLIT = 2,
       STBA_FACTOR_PANEL_PERSISTENT = 3 };

typedef struct {
  double F_before;      /* F(x) at the start of the iteration */
  double F_after;       /* F(x + dx) of the candidate step; +inf when a cluster factorisation failed */
  double lambda_used;   /* damping used to compute the step */
  double lambda;        /* damping after the accept / reject update */
  double grad_inf;      /* ||J^T f||_inf at x (uncorrected gradient) */
  double dx_norm;       /* ||dx||_2 of the candidate step */
  double x_norm;        /* ||x||_2 at the start of the iteration */
  int32_t accepted;     /* 1 if F(x + dx) < F(x) (strict) and x was updated */
  int32_t stop;         /* 1 if a stop tolerance fired on this step (Algorithm 1) */
  int32_t corrected;    /* 1 if the steepest-descent correction was applied */
  int32_t failed_clusters; /* clusters whose Cholesky factorisation met a pivot <= 0 or non-finite */
  int32_t boosted_pivots;  /* mixed precision: FP32 pivots lost to rounding and raised before FP64
                              refinement (static pivoting); 0 in FP64 mode */
  int32_t linear_iterations; /* conjugate-gradient iterations of the step (the PCG solvers), else 0 */
  int64_t iteration;    /* 1-based count of iterations run on this context */
} stba_iter_info;

/* Fills *opt with the defaults above (FP64, correction on, lambda0 1e-4, tolerances off,
 * refine_steps 1, use_graph 1, cluster solver, pcg_max_iter 500, pcg_tol 1e-6, no Huber loss). */
void stba_default_options(stba_options* opt);

/* Creates a problem (Sec. 3, Algorithm 1 inputs).
 *   cameras [m][9] FP64, points [n][3] FP64 (initial x); obs_cam [q], obs_pt [q] int32 indices;
 *   obs_uv [q][2] FP64 pixel observations; cluster_assignment [m] int32 with values 0..l-1, every
 *   cluster non-empty (the sampled clustering of Sec. 4.2/4.4); opt may be NULL (defaults);
 *   cuda_stream is a cudaStream_t or NULL.
 * Every point needs >= 2 projections and every camera >= 1; a (camera, point) pair may appear once.
 * With the cluster solver the solve of a cluster keeps its vector in one CTA's shared memory: a cluster
 * of more than about 31,500 unknowns (9 per camera; FP32 factor) or 22,100 (FP64) is refused with
 * STBA_ERR_INVALID_ARG and a message naming the limit (the PCG solvers have no such limit).
 * Computes F(x) once.  On success *out owns the context. */
stba_status stba_create(const double* cameras, int64_t m, const double* points, int64_t n,
                        const int32_t* obs_cam, const int32_t* obs_pt, const double* obs_uv, int64_t q,
                        const int32_t* cluster_assignment, const stba_options* opt, void* cuda_stream,
                        stba_ctx** out);

/* Replaces the cluster assignment [m] used by subsequent iterations (the per-iteration resampling of
 * Algorithm 1).  Same validation as stba_create, including the cluster-size limit; after a validation
 * error the previous assignment stays in force.  Enqueues the device re-ordering and returns without
 * waiting. */
stba_status stba_set_clusters(stba_ctx* ctx, const int32_t* cluster_assignment);

/* Runs one LM iteration (Algorithm 1 body).  If info != NULL the stream is synchronised and *info is
 * filled; with info == NULL the call only enqueues work and returns. */
stba_status stba_lm_iteration(stba_ctx* ctx, stba_iter_info* info);

/* Runs up to max_iter iterations, stopping after the first one whose stop flag is set (Algorithm 1).
 * *last (may be NULL) receives the last iteration's record. */
stba_status stba_solve(stba_ctx* ctx, int32_t max_iter, stba_iter_info* last);

/* Recomputes F(x) = ||f(x)||^2 at the current parameters (FP64 sum); synchronises. */
stba_status stba_cost(stba_ctx* ctx, double* F);

/* Copies the current parameters out ([m][9], [n][3], FP64); either pointer may be NULL. */
stba_status stba_get_params(stba_ctx* ctx, double* cameras, double* points);

/* Replaces the parameters ([m][9], [n][3], FP64) and recomputes F(x).  Keeps lambda. */
stba_status stba_set_params(stba_ctx* ctx, const double* cameras, const double* points);

/* Damping / cost state, for checkpoint and resume: reads or overwrites (lambda, F, iteration).
 * stba_set_state with F < 0 recomputes F at the current parameters. */
stba_status stba_get_state(stba_ctx* ctx, double* lambda, double* F, int64_t* iteration);
stba_status stba_set_state(stba_ctx* ctx, double lambda, double F, int64_t iteration);

/* The candidate step of the last iteration, accepted or not: dc [m][9], dp [n][3] (FP64). */
stba_status stba_last_step(stba_ctx* ctx, double* dc, double* dp);

/* Differentiation (the paper has none; the derivative of the solver's executed iterations).
 *
 * stba_record(ctx, max_iter) starts a tape: each of the next max_iter LM iterations (stba_lm_iteration,
 * stba_solve) stores the parameters x_t it starts from ((9m + 3n) FP64 values in device memory, held by
 * the context) and, after it, its record (damping, accept flag, correction flag), with the cluster
 * assignment it used.  It also allocates the reverse pass's buffers (about 184 q + 216 m + 96 n bytes of
 * device memory), so that stba_adjoint allocates nothing.  A further iteration returns STBA_ERR_STATE;
 * stba_record restarts the tape and max_iter = 0 frees it (the buffers with it).  Errors:
 * STBA_ERR_INVALID_ARG (max_iter < 0), STBA_ERR_OOM (the tape or the buffers do not fit; nothing is then
 * recorded). */
stba_status stba_record(stba_ctx* ctx, int32_t max_iter);

/* Reverse-mode derivative of the recorded iterations.  Given the gradient of a loss L at the final
 * parameters, dL_dcams [m][9] and dL_dpts [n][3] (NULL = zero), writes dL/d obs_uv [q][2] (in the order
 * given to stba_create), dL/d cameras [m][9] and dL/d points [n][3] at the start of the tape; any output
 * may be NULL.  FP64 arrays, host or device pointers.
 * Meaning: the derivative of the executed map x_{t+1} = x_t + Delta_t (accepted steps; a rejected step
 * is the identity) with the damping, the cluster assignments and the accept flags held at their recorded
 * values.  Each accepted step is recomputed from its stored x_t with the same kernels and precision as
 * the forward pass; its adjoint solves with that step's cluster factors (z_c = S'^-1 a^_c, the implicit
 * derivative of Eq. 10/13), back-substitutes through the virtual points and Eq. 15, and adds the
 * second-derivative products of the reprojection error.  A step taken with the steepest-descent correction
 * (lambda >= correction_lambda, Sec. 4.3) is differentiated through the closed form of the corrected
 * right-hand side, w~'_v = (h_v / H_i) o w_i (h_v = diag(V_v), H_i their sum over point i's copies, w_i the
 * physical w), including the dependence of h_v / H_i on the parameters.
 * Errors: STBA_ERR_STATE with the PCG solvers or the Huber loss, if nothing was recorded, or if
 * stba_set_params replaced the parameters during the recording.  On return the parameters, the cluster
 * assignment and the LM state are those before the call.  The call synchronises the stream and allocates
 * no memory (its buffers are held with the tape). */
stba_status stba_adjoint(stba_ctx* ctx, const double* dL_dcams, const double* dL_dpts, double* dL_dobs,
                         double* dL_dcams0, double* dL_dpts0);

/* Sizes, first n of: m, n, q, l (clusters), nv (virtual points), max cluster dimension 9 n_k, device
 * bytes held, S' pair-pass work items, kernel launches per LM iteration, camera-pair instances
 * (observation pairs of one virtual point), factorisation flops sum_k (9 n_k)^3 / 3, and elements of the
 * lower triangles of all S'_k. */
stba_status stba_problem_info(stba_ctx* ctx, int64_t* out, int32_t n);

/* The cluster system S'_k Delta c_k = b_k (Eq. 13) of the last iteration, in the order of the cluster's
 * cameras by increasing camera index: S [dim][dim] (FP64, both triangles filled from the lower one) and
 * b [dim]; dim = 9 n_k is written to *dim.  S or b may be NULL (then only dim is returned).
 * STBA_ERR_STATE with the PCG solver (no cluster systems are formed). */
stba_status stba_get_cluster_system(stba_ctx* ctx, int32_t k, double* S, double* b, int64_t* dim);

/* Stage timing: every iteration records CUDA events around its stages on the context stream (inside
 * the captured graph as event nodes).  stba_stage_times waits for the last iteration and copies its
 * stage times (ms) into ms[0..n-1] (stages: 0 linearisation + virtual points, 1 S' build,
 * 2 factorisation, 3 cluster solves with refinement, 4 point update + cost + control); *count gets the
 * number of stages.  stba_set_timing is kept for compatibility and has no effect. */
stba_status stba_set_timing(stba_ctx* ctx, int32_t on);
stba_status stba_stage_times(stba_ctx* ctx, float* ms, int32_t n, int32_t* count);

/* F(x) = ||f(x)||^2 without allocating device memory.  This entry point has no counterpart in the paper;
 * it exists for callers that cannot allocate device memory when they evaluate the cost (a loop with a
 * fixed, pre-reserved memory budget, or code that must not enter the allocator).
 *   cameras [m][9], points [n][3], obs_uv [q][2] (FP64) and obs_cam, obs_pt [q] (int32) are DEVICE
 *   pointers owned by the caller; F_dev is a device double that receives F (FP64 sum, no host sync).
 *   m <= 16384: the scratch (per-camera FP64 rotation table and reduction partials) is one static device
 *   array of 1.97 MB that every GPU loading the library holds until the process exits.  Larger m returns
 *   STBA_ERR_INVALID_ARG.  Indices out of range or a point at depth <= 1e-9 make F NaN.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  The address is kept for the life of the
 * process, so cudaDeviceReset (which unloads the module holding the array) is not supported while the
 * library is loaded.  All calls share the array, so calls that overlap on the GPU (different streams or
 * devices' contexts sharing it) race; serialise them.  An error already pending in the CUDA runtime when
 * the call starts is left in place and returns STBA_ERR_CUDA; so does a failed launch. */
stba_status stba_cost_noalloc(const double* cameras, int64_t m, const double* points, int64_t n,
                              const int32_t* obs_cam, const int32_t* obs_pt, const double* obs_uv, int64_t q,
                              double* F_dev, void* cuda_stream);

/* Camera graph and stochastic graph clustering (Sec. 4.4).  These calls run on the host and use no GPU.
 *
 * The camera graph joins cameras i and j when they observe a common point; the weight w_ij is the number of
 * such points.  Stochastic graph clustering starts from single cameras and joins two neighbouring clusters
 * at a time, drawing the join with probability proportional to exp(beta dQ) (Eq. 16), dQ being the increase
 * of the modularity Q = 1/(2s) sum over edges e_ij of delta(nu_i, nu_j) (w_ij - k_i k_j / (2s)) (the sum runs
 * over the edges of the graph, s = sum of the weights, k_i = weight at camera i).  A join is allowed when
 * the joined cluster has at most gamma cameras; clustering ends when no join is allowed.  The paper uses
 * beta = 10, gamma = 100.  The result is an assignment [m] with ids 0..l-1 numbered by the smallest camera
 * of each cluster; the same seed gives the same assignment.  Errors: STBA_ERR_INVALID_ARG (message from
 * stba_last_error(NULL)). */
typedef struct stba_graph stba_graph;

/* Builds the camera graph of q observations.  obs_cam, obs_pt [q] are HOST arrays (cameras 0..m-1, points
 * 0..n-1); a camera may observe a point at most once.  *out is owned by the caller (stba_graph_destroy). */
stba_status stba_graph_create(int64_t m, int64_t n, const int32_t* obs_cam, const int32_t* obs_pt, int64_t q,
                              stba_graph** out);
/* *E = number of edges; with non-NULL HOST arrays of length *E, the edges (i < j, ordered by j then i) and
 * their weights. */
stba_status stba_graph_edges(const stba_graph* g, int64_t* E, int32_t* i, int32_t* j, int64_t* w);
/* One clustering: cluster_assignment [m] (HOST) and *l.  gamma >= 1, beta finite and >= 0. */
stba_status stba_graph_cluster(const stba_graph* g, int32_t gamma, double beta, uint64_t seed,
                               int32_t* cluster_assignment, int32_t* l);
/* count clusterings with seeds seed, seed + 1, ..., drawn in parallel host threads:
 * cluster_assignments [count][m], l [count] (HOST). */
stba_status stba_graph_cluster_batch(const stba_graph* g, int32_t gamma, double beta, uint64_t seed, int32_t count,
                                     int32_t* cluster_assignments, int32_t* l);
void stba_graph_destroy(stba_graph* g);
/* The same as stba_graph_cluster_batch on the camera graph of a context (built by stba_create). */
stba_status stba_cluster_sgc(stba_ctx* ctx, int32_t gamma, double beta, uint64_t seed, int32_t count,
                             int32_t* cluster_assignments, int32_t* l);

/* Autotuner (the paper has none): times `iterations` LM iterations with every candidate configuration of
 * the cluster factorisation on the current parameters and cluster assignment, restores the parameters,
 * damping and cost after each trial, and keeps the fastest for the following iterations.  Candidates
 * (STBA_MIXED; FP64 has one):
 *   0 = tile 64, split panel, tensor-core trailing update     1 = tile 64, split panel, CUDA-core update
 *   2 = tile 64, stacked panel, CUDA-core update              3 = tile 32, stacked panel, CUDA-core update
 *   4 = tile 64, persistent (one launch of 8-CTA clusters)  5 = tile 64, stacked panel, tensor-core update
 *                                                              (the default on problems of one wave of panels)
 * *choice (optional) receives the index kept (-1 for the single FP64 configuration or the FP64 factor of
 * factor_fp64), ms[0..5] (optional, 6 floats) the
 * time per iteration of each candidate (-1 when not tried).  Synchronises the context stream.  Errors:
 * STBA_ERR_STATE while iterations are being recorded (stba_record), STBA_ERR_INVALID_ARG for
 * iterations < 1. */
stba_status stba_autotune(stba_ctx* ctx, int32_t iterations, int32_t* choice, float* ms);

/* Measured arithmetic peaks of the current GPU, the denominators of the factorisation's roofline.  The
 * paper has no counterpart: this is measurement infrastructure.  *fp32_tflops (optional): FP32 FMA rate of
 * the CUDA cores (16 independent FMA chains per thread, 4 CTAs of 256 threads per SM).  *tf32_tflops
 * (optional): dense TF32 rate of the tensor cores (tcgen05.mma kind::tf32, M = 128, N = 256, K = 8, back to
 * back into one TMEM accumulator, one CTA per SM); a 3xTF32 product of FP32 accuracy runs at a third of it.
 * Each kernel runs once untimed, then `reps` times between events on cuda_stream.  Allocates (and frees) a
 * few bytes of device memory; synchronises the stream.  Errors: STBA_ERR_INVALID_ARG (reps < 1, both outputs
 * NULL), STBA_ERR_CUDA (a CUDA error, also one already pending), STBA_ERR_TIMEOUT (the tensor-core kernel's
 * bounded wait gave up). */
stba_status stba_measure_peaks(void* cuda_stream, int32_t reps, double* fp32_tflops, double* tf32_tflops);

/* Sharded iteration over several processes, one context each (the paper's cluster-parallel, distributed
 * execution, Sec. 1 and the distributed runs of Sec. 5): after point splitting and binding (Sec. 4.1-4.2) the
 * cluster systems of Eq. 13 are independent, so each process linearises the observations of, builds,
 * factors and solves only the clusters it owns, and sums what spans clusters with the caller's transport.
 *   rank, world: this process and the number of processes; every process creates its context from the same
 *     problem and applies the same cluster assignments (stba_set_clusters) in the same order.  A cluster
 *     belongs to one process, chosen on every assignment by the same deterministic rule everywhere: longest
 *     processing time first by the cost model (9 n_k)^3 / 3 + 2000 x (observations of its cameras), ties to
 *     the lower cluster id and the lower rank.  stba_shard_owned reports the owned clusters.
 *   fn: the transport: sums `count` values (dtype 0 = FP64, 1 = FP32) over all processes, in place, and
 *     returns 0 on success.  host_staging = 1: the library copies the values to a pinned host buffer,
 *     synchronises its stream, calls fn with the host pointer, and copies the sums back (CPU transports such
 *     as gloo); host_staging = 0: fn gets the device pointer and the context stream, and must order its work
 *     on that stream (device transports such as NCCL).  user is passed to fn unchanged.
 * Per LM iteration fn is called four times: the per-point sums of the virtual-point blocks (9 n FP64: C_i
 * and w_i of Eq. 15, which also carry the per-point sums of the steepest-descent correction, Sec. 4.3);
 * after the cluster solves Delta c (9 m FP64, zero for the other processes' cameras), the camera gradient
 * (9 m, working precision) and the number of failed factorisations (1 FP64).  The point update, F(x + Delta
 * x) and the accept rule then run on complete data in every process, so all hold the same parameters,
 * damping and cost.  Sharded iterations are not captured in a CUDA graph and are not recorded for the
 * adjoint.  world = 1 returns to the single-process iteration.
 * Errors: STBA_ERR_INVALID_ARG (rank out of range, no transport), STBA_ERR_STATE (a PCG solver, a recording
 * tape; a transport call that returned non-zero fails the iteration with STBA_ERR_STATE). */
typedef int32_t (*stba_allreduce_fn)(void* user, void* data, int64_t count, int32_t dtype, void* cuda_stream);
stba_status stba_set_shard(stba_ctx* ctx, int32_t rank, int32_t world, stba_allreduce_fn fn, void* user,
                           int32_t host_staging);
/* *l = clusters of the current assignment; owned [l] (optional, HOST) = 1 where this process owns cluster k. */
stba_status stba_shard_owned(stba_ctx* ctx, int32_t* owned, int32_t* l);

/* Frees every device allocation of the context.  NULL is allowed. */
void stba_destroy(stba_ctx* ctx);

const char* stba_status_string(stba_status s);
const char* stba_last_error(stba_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* STBA_H */
