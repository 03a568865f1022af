// Adjoint of one accepted STBA step (reverse mode through the executed LM iteration).
//
// The paper has no derivative of its solver; the adjoint differentiates the computed map x_{t+1} = x_t + Delta_t
// with the damping lambda, the cluster assignment and the accept flag held at their forward values.  An
// accepted step is defined implicitly by the damped, cluster-split normal equations (Eq. 10, Eq. 13):
//   camera part   Delta c = the camera part of H' dx' = -J'^T f, H' = J'^T J' + lambda diag(J'^T J')
//                 (virtual points p', one per (point, cluster) pair),
//   point part    Delta p = C^-1 (w - E^T Delta c) (Eq. 15, physical uncorrected C, E, w).
// For an upstream adjoint a = (a_c, a_p) of x_{t+1}, with every forward quantity recomputed at x_t:
//   u   = C^-1 a_p                       a^_c = a_c - E u
//   z_c = S'^-1 a^_c (same cluster factors as the forward solve)
//   z_v = -C'_v^-1 E'_v^T z_c            (z' = [z_c; z_v] = H'^-1 [a^_c; 0])
//   q_bar_o += g_o = J_o (z'_o + U_o)    (f_o = pi_o - q_o, so the observation enters with a minus sign
//                                         that cancels the one of Delta = -M f)
//   x_bar = a - sum_o [J_o^T g_o + second-derivative terms]
// where, per observation, with local 12-vectors (camera 9, point 3) z'_o, dx'_o = [Delta c; Delta p'_v],
// U_o = [0; u], DP_o = [0; Delta p], DC_o = [Delta c; 0], rho_o = f_o + J_c Delta c, and
// (alpha, beta) = sum_s alpha_s H_s beta (H_s the Hessian of residual component s), the terms are
//   (f + J dx', z') + (J z', dx') + (J DP + rho, U) + (J U, DP + DC)
//   + sum_s (e_s, 2 lambda J[s,:] o (z' o dx' + U o DP))          (the lambda diag(J^T J) damping)
// The (alpha, beta) products come from the Jacobian evaluated on dual numbers (stba_dual.cuh).  The
// per-observation products run in the working precision (FP32 in mixed mode, as the forward step's
// Jacobians do); the adjoint vectors and every sum over observations are FP64.
//
// A step taken with the steepest-descent correction (Sec. 4.3; lambda >= the threshold) solves H' dx' = g~'
// with w~'_v = (h_v / H_i) o w_i for the virtual points v of point i (the closed form of the correction:
// h_v = diag(V_v) undamped, H_i = sum over the copies of h_v, w_i the physical w).  The recomputed forward
// step already carries w~' in dx'; its adjoint differs in two places:
//   - where z' meets the right-hand side (the (f, .) term, J^T g and q_bar), the copies' z_v are replaced by
//     zeta_i = sum_v h_v o z_v / H_i, so (f + J dx', z') splits into (f, z~) + (J dx', z');
//   - the derivative of h_v / H_i adds sum_s (e_s, J[s,:] o [0; -2 kappa_v]), kappa_v = (z_v - zeta_i) o w_i / H_i,
//     which joins the damping directions' weights.
#include <climits>

#include "stba_camera.cuh"
#include "stba_device.cuh"
#include "stba_dual.cuh"
#include "stba_internal.cuh"

namespace stba {

namespace {

constexpr int ADJ_THREADS = 128;

// One observation's camera, point and measurement in the working precision: FP64 from the parameters, or
// the per-iteration FP32 copies in mixed precision (the forward step's Jacobians are FP32 there too).
template <typename real>
__device__ __forceinline__ void load_obs_w(const DevProblem& P, int o, Cam<real>& C, real X[3], real& uo,
                                           real& vo) {
  C = load_cam_w<real>(P, P.obs_cam[o]);
  load_point_w<real>(P, P.obs_pt[o], X);
  load_uv<real>(P, o, uo, vo);
}

template <typename real>
__global__ void k_adj_point_u(int n, const real* __restrict__ pt_info, const double* __restrict__ a_p,
                              double* __restrict__ u) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const real* in = pt_info + 9 * (size_t)i;   // C^-1, packed symmetric 00 01 02 11 12 22
    const double* a = a_p + 3 * (size_t)i;
    const double c00 = in[0], c01 = in[1], c02 = in[2], c11 = in[3], c12 = in[4], c22 = in[5];
    double* o = u + 3 * (size_t)i;
    o[0] = c00 * a[0] + c01 * a[1] + c02 * a[2];
    o[1] = c01 * a[0] + c11 * a[1] + c12 * a[2];
    o[2] = c02 * a[0] + c12 * a[1] + c22 * a[2];
  }
}

// Block sum of NV per-thread values; thread i < NV of the block gets sum i in the return value.
template <int NV>
__device__ __forceinline__ double block_sum_to_thread(const double (&v)[NV]) {
  __shared__ double red[ADJ_THREADS / 32][NV];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double x = v[i];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(FULL_MASK, x, d);
    if (lane == 0) red[warp][i] = x;
  }
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < NV)
    for (int w = 0; w < ADJ_THREADS / 32; ++w) s += red[w][threadIdx.x];
  return s;
}

// a^_c = a_c - E u, one CTA per camera, written into the per-cluster padded vector layout of b'.
template <typename real>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_cam_rhs(DevProblem P, CamLists CL, const double* __restrict__ u,
                                                             const double* __restrict__ a_c, double* __restrict__ bhat) {
  const int j = blockIdx.x;
  double acc[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) acc[i] = 0.0;
  for (int e = CL.cam_obs_off[j] + threadIdx.x; e < CL.cam_obs_off[j + 1]; e += blockDim.x) {
    const int o = CL.cam_obs[e];
    Cam<real> C;
    real X[3], uo, vo, r[2], Jc[2][9], Jp[2][3];
    load_obs_w<real>(P, o, C, X, uo, vo);
    project_jacobian<real, true>(C, X, uo, vo, r, Jc, Jp);
    const double* up = u + 3 * (size_t)P.obs_pt[o];
    const real u0 = (real)up[0], u1 = (real)up[1], u2 = (real)up[2];
    const real t0 = Jp[0][0] * u0 + Jp[0][1] * u1 + Jp[0][2] * u2;
    const real t1 = Jp[1][0] * u0 + Jp[1][1] * u1 + Jp[1][2] * u2;
#pragma unroll
    for (int i = 0; i < 9; ++i) acc[i] += (double)(Jc[0][i] * t0 + Jc[1][i] * t1);
  }
  const double s = block_sum_to_thread<9>(acc);
  if (threadIdx.x < 9) {
    const int k = P.cam_cluster[j], lc = P.cam_local[j];
    bhat[P.v_off[k] + 9 * lc + threadIdx.x] = a_c[9 * (size_t)j + threadIdx.x] - s;
  }
}

// Per observation, warp-segmented by virtual point: E'_v^T z_c and E'_v^T Delta c (3 + 3 sums).
template <typename real>
__global__ void __launch_bounds__(256) k_adj_vp(DevProblem P, const double* __restrict__ zc,
                                                const double* __restrict__ dc, double* __restrict__ vpz) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool act = o < P.q;
  int v = INT_MAX;
  double val[6] = {0, 0, 0, 0, 0, 0};
  if (act) {
    v = P.obs_vp[o];
    Cam<real> C;
    real X[3], uo, vo, r[2], Jc[2][9], Jp[2][3];
    load_obs_w<real>(P, o, C, X, uo, vo);
    project_jacobian<real, true>(C, X, uo, vo, r, Jc, Jp);
    const double* z = zc + 9 * (size_t)P.obs_cam[o];
    const double* d = dc + 9 * (size_t)P.obs_cam[o];
    real jz0 = 0, jz1 = 0, jd0 = 0, jd1 = 0;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      const real zcv = (real)z[c], dcv = (real)d[c];
      jz0 += Jc[0][c] * zcv;
      jz1 += Jc[1][c] * zcv;
      jd0 += Jc[0][c] * dcv;
      jd1 += Jc[1][c] * dcv;
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      val[s] = (double)(Jp[0][s] * jz0 + Jp[1][s] * jz1);
      val[3 + s] = (double)(Jp[0][s] * jd0 + Jp[1][s] * jd1);
    }
  }
  segmented_scan<6>(val, v, lane);
  segmented_store<6>(val, v, act, lane, o, P.vp_off, vpz);
}

// Per virtual point: z_v = -C'_v^-1 (E'^T z_c)_v and the expanded point step dp'_v = C'_v^-1 (w'_v - (E'^T dc)_v)
// = y_v - C'_v^-1 (E'^T dc)_v (uncorrected w').
template <typename real>
__global__ void k_adj_vp_final(int nv, const real* __restrict__ vp_info, double* __restrict__ vpz) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    const real* in = vp_info + 9 * (size_t)v;
    double Li[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) Li[c] = (double)in[c];
    double* e = vpz + 6 * (size_t)v;
    const double e1[3] = {e[0], e[1], e[2]}, e2[3] = {e[3], e[4], e[5]};
    double x1[3], x2[3];
    chol3_apply(Li, e1, x1);
    chol3_apply(Li, e2, x2);
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      e[s] = -x1[s];
      e[3 + s] = (double)in[6 + s] - x2[s];
    }
  }
}

// Corrected steps: per point, zeta_i = sum_v h_v o z_v / H_i, and per virtual point kappa_v = (z_v - zeta_i) o
// w_i / H_i, from the undamped V_v and uncorrected w'_v the forward pass accumulated (vp_acc) and z_v (vpz).
template <typename real>
__global__ void k_adj_zeta(DevProblem P, const real* __restrict__ vp_acc, const double* __restrict__ vpz,
                           double* __restrict__ zeta, double* __restrict__ kappa) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
    const int vb = P.pt_vp_off[i], ve = P.pt_vp_off[i + 1];
    double H[3] = {0, 0, 0}, w[3] = {0, 0, 0}, hz[3] = {0, 0, 0};
    for (int v = vb; v < ve; ++v) {
      const real* a = vp_acc + 9 * (size_t)v;
      const double h[3] = {(double)a[0], (double)a[3], (double)a[5]};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        H[k] += h[k];
        w[k] += (double)a[6 + k];
        hz[k] += h[k] * vpz[6 * (size_t)v + k];
      }
    }
    double z[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      z[k] = hz[k] / H[k];
      zeta[3 * (size_t)i + k] = z[k];
    }
    for (int v = vb; v < ve; ++v)
#pragma unroll
      for (int k = 0; k < 3; ++k) kappa[3 * (size_t)v + k] = (vpz[6 * (size_t)v + k] - z[k]) * w[k] / H[k];
  }
}

// out += sum_s alpha_s d/de J_s(theta + e beta) (12 entries: camera 9, point 3) for one observation, on
// dual numbers of the working precision.
template <typename real>
__device__ __forceinline__ void hess_vec(const Cam<real>& C0, const real X0[3], real uo, real vo, real al0, real al1,
                                         const real beta[12], real out[12]) {
  using D = DualT<real>;
  Cam<D> C;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    C.w[k] = D(C0.w[k], beta[k]);
    C.t[k] = D(C0.t[k], beta[3 + k]);
  }
  C.f = D(C0.f, beta[6]);
  C.k1 = D(C0.k1, beta[7]);
  C.k2 = D(C0.k2, beta[8]);
  const D X[3] = {D(X0[0], beta[9]), D(X0[1], beta[10]), D(X0[2], beta[11])};
  D r[2], Jc[2][9], Jp[2][3];
  project_jacobian<D, true>(C, X, D(uo), D(vo), r, Jc, Jp);
#pragma unroll
  for (int c = 0; c < 9; ++c) out[c] += al0 * Jc[0][c].d + al1 * Jc[1][c].d;
#pragma unroll
  for (int c = 0; c < 3; ++c) out[9 + c] += al0 * Jp[0][c].d + al1 * Jp[1][c].d;
}

// Per observation: g_o (added to q_bar in input order) and the 12 local terms T_o of x_bar.  The products
// run in the working precision (FP32 in mixed mode, like the forward step's Jacobians), from the adjoint
// vectors held in FP64; f_o is the stored residual the forward step linearised with.
template <typename real>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_obs(DevProblem P, const int* __restrict__ perm, double lam,
                                                         const double* __restrict__ dc, const double* __restrict__ dp,
                                                         const double* __restrict__ zc, const double* __restrict__ u,
                                                         const double* __restrict__ vpz, int corr,
                                                         const double* __restrict__ zeta,
                                                         const double* __restrict__ kappa, double* __restrict__ T,
                                                         double* __restrict__ qbar) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= P.q) return;
  const int cam = P.obs_cam[o], pt = P.obs_pt[o], v = P.obs_vp[o];
  Cam<real> C;
  real X[3], uo, vo, f[2], Jc[2][9], Jp[2][3];
  load_obs_w<real>(P, o, C, X, uo, vo);
  project_jacobian<real, true>(C, X, uo, vo, f, Jc, Jp);
  f[0] = res_ptr<real>(P)[2 * (size_t)o];
  f[1] = res_ptr<real>(P)[2 * (size_t)o + 1];
  real z[12], dx[12], uu[3], dpp[3];
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    z[c] = (real)zc[9 * (size_t)cam + c];
    dx[c] = (real)dc[9 * (size_t)cam + c];
  }
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    z[9 + s] = (real)vpz[6 * (size_t)v + s];
    dx[9 + s] = (real)vpz[6 * (size_t)v + 3 + s];
    uu[s] = (real)u[3 * (size_t)pt + s];
    dpp[s] = (real)dp[3 * (size_t)pt + s];
  }
  // z~: z' with the point part replaced by zeta of the physical point on a corrected step
  real zp[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) zp[s] = corr ? (real)zeta[3 * (size_t)pt + s] : z[9 + s];
  // J z', J z~, J dx', J U, J DP, rho = f + J_c dc
  real Jz[2], Jzt[2], Jdx[2], JU[2], JDP[2], rho[2];
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    real a = 0, cdc = 0;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      a += Jc[t][c] * z[c];
      cdc += Jc[t][c] * dx[c];
    }
    real pz = 0, pzt = 0, pdx = 0, pu = 0, pdp = 0;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      pz += Jp[t][s] * z[9 + s];
      pzt += Jp[t][s] * zp[s];
      pdx += Jp[t][s] * dx[9 + s];
      pu += Jp[t][s] * uu[s];
      pdp += Jp[t][s] * dpp[s];
    }
    Jz[t] = a + pz;
    Jzt[t] = a + pzt;
    Jdx[t] = cdc + pdx;
    JU[t] = pu;
    JDP[t] = pdp;
    rho[t] = f[t] + cdc;
  }
  const real g0 = Jzt[0] + JU[0], g1 = Jzt[1] + JU[1];
  {
    double* qb = qbar + 2 * (size_t)perm[o];
    qb[0] += (double)g0;
    qb[1] += (double)g1;
  }
  real acc[12];
#pragma unroll
  for (int c = 0; c < 9; ++c) acc[c] = Jc[0][c] * g0 + Jc[1][c] * g1;
#pragma unroll
  for (int s = 0; s < 3; ++s) acc[9 + s] = Jp[0][s] * g0 + Jp[1][s] * g1;
  // damping weights 2 lambda (z' o dx' + U o DP), times the rows of J below
  const real lam2 = (real)(2.0 * lam);
  real wdm[12];
#pragma unroll
  for (int c = 0; c < 9; ++c) wdm[c] = lam2 * z[c] * dx[c];
#pragma unroll
  for (int s = 0; s < 3; ++s)
    wdm[9 + s] = lam2 * (z[9 + s] * dx[9 + s] + uu[s] * dpp[s]) - (corr ? real(2) * (real)kappa[3 * (size_t)v + s] : real(0));
  real al0, al1, beta[12];
  const int ndir = corr ? 7 : 6;
#pragma unroll 1
  for (int dir = 0; dir < ndir; ++dir) {
    switch (dir) {
      case 0:   // (f + J dx', z'), or (f, z~) on a corrected step
        al0 = f[0] + (corr ? real(0) : Jdx[0]);
        al1 = f[1] + (corr ? real(0) : Jdx[1]);
#pragma unroll
        for (int c = 0; c < 9; ++c) beta[c] = z[c];
#pragma unroll
        for (int s = 0; s < 3; ++s) beta[9 + s] = zp[s];
        break;
      case 6:   // corrected step: (J dx', z')
        al0 = Jdx[0];
        al1 = Jdx[1];
#pragma unroll
        for (int c = 0; c < 12; ++c) beta[c] = z[c];
        break;
      case 1:   // (J z', dx')
        al0 = Jz[0];
        al1 = Jz[1];
#pragma unroll
        for (int c = 0; c < 12; ++c) beta[c] = dx[c];
        break;
      case 2:   // (J DP + rho, U)
        al0 = JDP[0] + rho[0];
        al1 = JDP[1] + rho[1];
#pragma unroll
        for (int c = 0; c < 9; ++c) beta[c] = real(0);
#pragma unroll
        for (int s = 0; s < 3; ++s) beta[9 + s] = uu[s];
        break;
      case 3:   // (J U, DP + DC)
        al0 = JU[0];
        al1 = JU[1];
#pragma unroll
        for (int c = 0; c < 9; ++c) beta[c] = dx[c];
#pragma unroll
        for (int s = 0; s < 3; ++s) beta[9 + s] = dpp[s];
        break;
      default: {   // (e_s, J[s,:] o wdm), s = dir - 4: the damping (and, corrected, the kappa) terms
        const int s = dir - 4;
        al0 = s == 0 ? real(1) : real(0);
        al1 = s == 0 ? real(0) : real(1);
#pragma unroll
        for (int c = 0; c < 9; ++c) beta[c] = (s == 0 ? Jc[0][c] : Jc[1][c]) * wdm[c];
#pragma unroll
        for (int k = 0; k < 3; ++k) beta[9 + k] = (s == 0 ? Jp[0][k] : Jp[1][k]) * wdm[9 + k];
      }
    }
    hess_vec<real>(C, X, uo, vo, al0, al1, beta, acc);
  }
  double* To = T + 12 * (size_t)o;
#pragma unroll
  for (int c = 0; c < 12; ++c) To[c] = (double)acc[c];
}

// a_c -= sum_o T_o[0:9] over the camera's observations (one CTA per camera, fixed-order reduction).
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_cam_reduce(CamLists CL, const double* __restrict__ T,
                                                                double* __restrict__ a_c) {
  const int j = blockIdx.x;
  double acc[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) acc[i] = 0.0;
  for (int e = CL.cam_obs_off[j] + threadIdx.x; e < CL.cam_obs_off[j + 1]; e += blockDim.x) {
    const double* t = T + 12 * (size_t)CL.cam_obs[e];
#pragma unroll
    for (int i = 0; i < 9; ++i) acc[i] += t[i];
  }
  const double s = block_sum_to_thread<9>(acc);
  if (threadIdx.x < 9) a_c[9 * (size_t)j + threadIdx.x] -= s;
}

// a_p -= sum_o T_o[9:12] over the point's observations (contiguous in the sorted order).
__global__ void k_adj_pt_reduce(DevProblem P, const double* __restrict__ T, double* __restrict__ a_p) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
    double s0 = 0, s1 = 0, s2 = 0;
    for (int o = P.pt_off[i]; o < P.pt_off[i + 1]; ++o) {
      const double* t = T + 12 * (size_t)o + 9;
      s0 += t[0];
      s1 += t[1];
      s2 += t[2];
    }
    double* a = a_p + 3 * (size_t)i;
    a[0] -= s0;
    a[1] -= s1;
    a[2] -= s2;
  }
}

__global__ void k_adj_set_lambda(DevState* st, double lam) {
  if (threadIdx.x == 0 && blockIdx.x == 0) st->lambda = lam;
}

}  // namespace

void launch_set_lambda(DevState* st, double lam, cudaStream_t stream) {
  k_adj_set_lambda<<<1, 32, 0, stream>>>(st, lam);
}

template <typename real>
void launch_adjoint_step(const DevProblem& P, Scratch<real> W, CamLists CL, const FactorBuffers& fb,
                         const CholPlan& plan, int refine_steps, const int* perm, double lam, int corrected,
                         const AdjointBuffers& A, cudaStream_t stream) {
  const int pblocks = std::min((P.n + 255) / 256, 4096);
  k_adj_point_u<real><<<pblocks, 256, 0, stream>>>(P.n, W.pt_info, A.a_p, A.u);
  // a^_c into the padded layout of b' (its padding rows stay zero), then z_c = S'^-1 a^_c
  int64_t v_total = fb.v_total;
  cudaMemsetAsync(W.b, 0, (size_t)v_total * sizeof(double), stream);
  k_adj_cam_rhs<real><<<P.m, ADJ_THREADS, 0, stream>>>(P, CL, A.u, A.a_c, W.b);
  launch_solve<real>(P, W.S, W.b, fb, plan, refine_steps, A.zc, nullptr, stream);
  cudaMemsetAsync(A.vpz, 0, 6 * (size_t)P.nv * sizeof(double), stream);
  k_adj_vp<real><<<(P.q + 255) / 256, 256, 0, stream>>>(P, A.zc, W.dc, A.vpz);
  k_adj_vp_final<real><<<std::min((P.nv + 255) / 256, 4096), 256, 0, stream>>>(P.nv, W.vp_info, A.vpz);
  if (corrected) k_adj_zeta<real><<<pblocks, 256, 0, stream>>>(P, W.vp_acc, A.vpz, A.zeta, A.kappa);
  k_adj_obs<real><<<(P.q + ADJ_THREADS - 1) / ADJ_THREADS, ADJ_THREADS, 0, stream>>>(
      P, perm, lam, W.dc, W.dp, A.zc, A.u, A.vpz, corrected, A.zeta, A.kappa, A.T, A.qbar);
  k_adj_cam_reduce<<<P.m, ADJ_THREADS, 0, stream>>>(CL, A.T, A.a_c);
  k_adj_pt_reduce<<<pblocks, 256, 0, stream>>>(P, A.T, A.a_p);
}

template void launch_adjoint_step<float>(const DevProblem&, Scratch<float>, CamLists, const FactorBuffers&,
                                         const CholPlan&, int, const int*, double, int, const AdjointBuffers&,
                                         cudaStream_t);
template void launch_adjoint_step<double>(const DevProblem&, Scratch<double>, CamLists, const FactorBuffers&,
                                          const CholPlan&, int, const int*, double, int, const AdjointBuffers&,
                                          cudaStream_t);

}  // namespace stba
