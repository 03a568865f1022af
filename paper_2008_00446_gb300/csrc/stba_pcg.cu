// Comparator of the method: plain LM with the full reduced camera system of all cameras (Eq. 5-6,
// S dc = b, S = B - E C^-1 E^T with the physical points; no clusters), solved by block-Jacobi
// preconditioned conjugate gradients, matrix-free.
//
//   k_pcg_jac      per observation: J_c (2x9) and J_p (2x3) at the current x, stored once per LM iteration
//   k_pcg_precond  per camera (one warp per 32 of its observations): the diagonal block
//                  S_jj = B_jj - sum_o J_c^T J_p C^-1 J_p^T J_c (undamped B part), diag(J_c^T J_c) and
//                  v = -J_c^T f; k_pcg_invert adds lambda diag(B) and inverts S_jj (9x9 Cholesky, FP64)
//   S p            k_pcg_Et (per observation, segmented by point: t = E^T p), k_pcg_u (u = C^-1 t), then
//                  k_pcg_cam (per camera: y = sum_o J_c^T (J_c p_j - J_p u) + lambda diag(B) p_j)
//   CG vectors     one thread per camera (9 entries and the 9x9 preconditioner), FP64; the scalars
//                  alpha, beta and the residual norms stay on the device (k_pcg_update, k_pcg_dir).
// The right-hand side b = v - E C^-1 w is S applied to nothing but the point part: k_pcg_cam with p = 0
// and u = C^-1 w.
//
// Split variant (STBA_SOLVER_PCG_CLUSTERS; Sec. 6, the inexact solve of the split RCS): the method's own
// clustered system S' dc = b' (Eq. 10, 13, virtual points, correction) solved by the same PCG instead of the
// cluster factorisations.  The camera pass provides b' and the diagonal blocks of S' (the preconditioner);
// S' p = B p - E' C'^-1 E'^T p runs over the virtual points (k_spcg_Et, k_spcg_u), and a virtual point with
// one observation enters through its cancellation-free form J_c^T (I + J_p L^-1 J_p^T)^-1 J_c (the camera
// pass's Woodbury form) (k_spcg_cam).  One CG runs over the block-diagonal system of all clusters at once
// (shared step lengths; its solution is every cluster's).
#include <climits>

#include "stba_camera.cuh"
#include "stba_device.cuh"
#include "stba_internal.cuh"

namespace stba {

namespace {

constexpr int JSTRIDE = 24;   // J_c (18) + J_p (6) per observation, working precision

template <typename real>
__global__ void __launch_bounds__(256) k_pcg_jac(DevProblem P, real* __restrict__ J) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < P.q; o += gridDim.x * blockDim.x) {
    const Cam<real> C = load_cam_w<real>(P, P.obs_cam[o]);
    real X[3];
    load_point_w(P, P.obs_pt[o], X);
    real uo, vo, r[2], Jc[2][9], Jp[2][3];
    load_uv(P, o, uo, vo);
    project_jacobian<real, true>(C, X, uo, vo, r, Jc, Jp);
    r[0] = res_ptr<real>(P)[2 * (size_t)o];
    r[1] = res_ptr<real>(P)[2 * (size_t)o + 1];
    scale_rows(huber_sqrt_weight<real>(P.huber_a, r[0], r[1]), r, Jc, Jp);   // robust loss: sqrt(rho') rows
    real v[JSTRIDE];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      v[c] = Jc[0][c];
      v[9 + c] = Jc[1][c];
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      v[18 + s] = Jp[0][s];
      v[21 + s] = Jp[1][s];
    }
    real* out = J + (size_t)JSTRIDE * o;
    if constexpr (sizeof(real) == 4) {
#pragma unroll
      for (int q4 = 0; q4 < JSTRIDE / 4; ++q4)
        reinterpret_cast<float4*>(out)[q4] = make_float4(v[4 * q4], v[4 * q4 + 1], v[4 * q4 + 2], v[4 * q4 + 3]);
    } else {
#pragma unroll
      for (int q2 = 0; q2 < JSTRIDE / 2; ++q2) reinterpret_cast<double2*>(out)[q2] = make_double2(v[2 * q2], v[2 * q2 + 1]);
    }
  }
}

template <typename real>
__device__ __forceinline__ void load_j(const real* J, int o, real (&Jc)[2][9], real (&Jp)[2][3]) {
  const real* p = J + (size_t)JSTRIDE * o;
  real v[JSTRIDE];
  if constexpr (sizeof(real) == 4) {
#pragma unroll
    for (int q4 = 0; q4 < JSTRIDE / 4; ++q4) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(p) + q4);
      v[4 * q4] = t.x;
      v[4 * q4 + 1] = t.y;
      v[4 * q4 + 2] = t.z;
      v[4 * q4 + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int q2 = 0; q2 < JSTRIDE / 2; ++q2) {
      const double2 t = __ldg(reinterpret_cast<const double2*>(p) + q2);
      v[2 * q2] = t.x;
      v[2 * q2 + 1] = t.y;
    }
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    Jc[0][c] = v[c];
    Jc[1][c] = v[9 + c];
  }
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    Jp[0][s] = v[18 + s];
    Jp[1][s] = v[21 + s];
  }
}

// Sum over the warp of v[0..N-1]; lane i < N receives sum i.
template <int N, typename real>
__device__ __forceinline__ real warp_sums_to_lanes(real (&v)[N]) {
  const int lane = threadIdx.x & 31;
  real mine = real(0);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    real x = v[i];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(FULL_MASK, x, d);
    if (lane == i) mine = x;
  }
  return mine;
}

// Per camera diagonal block of S (45 lower entries, without the damping), diag(B) and v = -J_c^T f.
template <typename real>
__global__ void __launch_bounds__(256) k_pcg_precond(DevProblem P, CamSlots CS, const real* __restrict__ J,
                                                     const real* __restrict__ pt_info, double* __restrict__ Mblk,
                                                     double* __restrict__ Bdiag, real* __restrict__ vgrad) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= CS.nwarps) return;
  const int lane = threadIdx.x & 31;
  const int j = CS.warp_cam[gw];
  const int o = CS.slots[32 * (size_t)gw + lane];
  real Jc[2][9], Jp[2][3], f[2] = {0, 0};
  real H[3][9];   // C^-1 J_p^T J_c
#pragma unroll
  for (int c = 0; c < 9; ++c) Jc[0][c] = Jc[1][c] = H[0][c] = H[1][c] = H[2][c] = real(0);
#pragma unroll
  for (int s = 0; s < 3; ++s) Jp[0][s] = Jp[1][s] = real(0);
  if (o >= 0) {
    load_j(J, o, Jc, Jp);   // rows already scaled by sqrt(rho') under a robust loss
    f[0] = res_ptr<real>(P)[2 * (size_t)o];
    f[1] = res_ptr<real>(P)[2 * (size_t)o + 1];
    const real sw = huber_sqrt_weight<real>(P.huber_a, f[0], f[1]);
    f[0] *= sw;
    f[1] *= sw;
    const real* ci = pt_info + 9 * (size_t)P.obs_pt[o];   // C^-1 packed 00 01 02 11 12 22
    const real Ci[3][3] = {{ci[0], ci[1], ci[2]}, {ci[1], ci[3], ci[4]}, {ci[2], ci[4], ci[5]}};
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      real g[3];
#pragma unroll
      for (int s = 0; s < 3; ++s) g[s] = Jp[0][s] * Jc[0][c] + Jp[1][s] * Jc[1][c];
#pragma unroll
      for (int s = 0; s < 3; ++s) H[s][c] = Ci[s][0] * g[0] + Ci[s][1] * g[1] + Ci[s][2] * g[2];
    }
  }
  // 45 + 9 + 9 terms, summed over the warp in two groups of 32 (transposed reduction)
  real sums[2];
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    real v[32];
    int t = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
      for (int jj = 0; jj <= i; ++jj, ++t) {
        if (t / 32 == half) {
          // (J_c^T J_c)_ij - (J_p^T J_c)_:i . H_:j
          real g0 = Jp[0][0] * Jc[0][i] + Jp[1][0] * Jc[1][i];
          real g1 = Jp[0][1] * Jc[0][i] + Jp[1][1] * Jc[1][i];
          real g2 = Jp[0][2] * Jc[0][i] + Jp[1][2] * Jc[1][i];
          v[t - 32 * half] = Jc[0][i] * Jc[0][jj] + Jc[1][i] * Jc[1][jj] - (g0 * H[0][jj] + g1 * H[1][jj] + g2 * H[2][jj]);
        }
      }
    if (half == 1) {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        v[45 - 32 + i] = Jc[0][i] * Jc[0][i] + Jc[1][i] * Jc[1][i];
        v[54 - 32 + i] = -(Jc[0][i] * f[0] + Jc[1][i] * f[1]);
      }
      v[31] = real(0);
    }
    // same transposed reduction as the camera pass
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
      const bool up = (lane & s) != 0;
#pragma unroll
      for (int i = 0; i < s; ++i) {
        const real send = up ? v[i] : v[i + s];
        const real keep = up ? v[i + s] : v[i];
        v[i] = keep + __shfl_xor_sync(FULL_MASK, send, s);
      }
    }
    sums[half] = v[0];
  }
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int e = lane + 32 * half;
    if (e < 45)
      atomicAdd(Mblk + 45 * (size_t)j + e, (double)sums[half]);
    else if (e < 54)
      atomicAdd(Bdiag + 9 * (size_t)j + (e - 45), (double)sums[half]);
    else if (e < 63)
      atomicAdd(vgrad + 9 * (size_t)j + (e - 54), sums[half]);
  }
}

// Minv_j = (S_jj + lambda diag(B_j))^-1, dense 9x9 (row-major), FP64 Cholesky; a non-positive pivot falls back
// to the inverse of the damped diagonal.
__global__ void k_pcg_invert(int m, const double* __restrict__ Mblk, const double* __restrict__ Bdiag,
                             const DevState* st, double* __restrict__ Minv) {
  const double lam = st->lambda_used;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    double A[9][9];
    int t = 0;
    for (int r = 0; r < 9; ++r)
      for (int c = 0; c <= r; ++c, ++t) {
        double v = Mblk[45 * (size_t)j + t];
        if (r == c) v += lam * Bdiag[9 * (size_t)j + r];
        A[r][c] = v;
        A[c][r] = v;
      }
    double Lf[9][9] = {};
    bool ok = true;
    for (int c = 0; c < 9 && ok; ++c) {
      double d = A[c][c];
      for (int k2 = 0; k2 < c; ++k2) d -= Lf[c][k2] * Lf[c][k2];
      if (!(d > 0.0)) {
        ok = false;
        break;
      }
      Lf[c][c] = sqrt(d);
      for (int r = c + 1; r < 9; ++r) {
        double s = A[r][c];
        for (int k2 = 0; k2 < c; ++k2) s -= Lf[r][k2] * Lf[c][k2];
        Lf[r][c] = s / Lf[c][c];
      }
    }
    double* out = Minv + 81 * (size_t)j;
    if (!ok) {
      for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) out[9 * r + c] = (r == c && A[r][r] > 0.0) ? 1.0 / A[r][r] : 0.0;
      continue;
    }
    // inverse = L^-T L^-1, column by column
    for (int c = 0; c < 9; ++c) {
      double y[9];
      for (int r = 0; r < 9; ++r) {
        double s = (r == c) ? 1.0 : 0.0;
        for (int k2 = 0; k2 < r; ++k2) s -= Lf[r][k2] * y[k2];
        y[r] = s / Lf[r][r];
      }
      for (int r = 8; r >= 0; --r) {
        double s = y[r];
        for (int k2 = r + 1; k2 < 9; ++k2) s -= Lf[k2][r] * out[9 * k2 + c];
        out[9 * r + c] = s / Lf[r][r];
      }
    }
  }
}

// t_i = sum_{o in point i} J_p^T (J_c p_cam(o)), segmented by point (observations are sorted by point)
template <typename real>
__global__ void __launch_bounds__(256) k_pcg_Et(DevProblem P, const real* __restrict__ J, const real* __restrict__ p,
                                                real* __restrict__ t) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool act = o < P.q;
  int pt = INT_MAX;
  real val[3] = {0, 0, 0};
  if (act) {
    pt = P.obs_pt[o];
    real Jc[2][9], Jp[2][3];
    load_j(J, o, Jc, Jp);
    const real* pc = p + 9 * (size_t)P.obs_cam[o];
    real a0 = 0, a1 = 0;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      const real x = pc[c];
      a0 += Jc[0][c] * x;
      a1 += Jc[1][c] * x;
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) val[s] = Jp[0][s] * a0 + Jp[1][s] * a1;
  }
  segmented_scan<3>(val, pt, lane);
  segmented_store<3>(val, pt, act, lane, o, P.pt_off, t);
}

// u_i = C_i^-1 t_i
template <typename real>
__global__ void k_pcg_u(int n, const real* __restrict__ pt_info, const real* __restrict__ t, real* __restrict__ u) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const real* ci = pt_info + 9 * (size_t)i;
    const real* ti = t + 3 * (size_t)i;
    real* ui = u + 3 * (size_t)i;
    ui[0] = ci[0] * ti[0] + ci[1] * ti[1] + ci[2] * ti[2];
    ui[1] = ci[1] * ti[0] + ci[3] * ti[1] + ci[4] * ti[2];
    ui[2] = ci[2] * ti[0] + ci[4] * ti[1] + ci[5] * ti[2];
  }
}

// y_j += sum_{o in camera j} J_c^T (J_c p_j - J_p u_pt(o)) (+ lambda diag(B_j) p_j, added by the camera's first
// warp).  With p = null the J_c p term is absent (right-hand side pass).
template <typename real>
__global__ void __launch_bounds__(256) k_pcg_cam(DevProblem P, CamSlots CS, const real* __restrict__ J,
                                                 const real* __restrict__ p, const real* __restrict__ u,
                                                 const double* __restrict__ Bdiag, const DevState* st,
                                                 double* __restrict__ y) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= CS.nwarps) return;
  const int lane = threadIdx.x & 31;
  const int j = CS.warp_cam[gw];
  const int o = CS.slots[32 * (size_t)gw + lane];
  real v[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) v[c] = real(0);
  if (o >= 0) {
    real Jc[2][9], Jp[2][3];
    load_j(J, o, Jc, Jp);
    const real* ui = u + 3 * (size_t)P.obs_pt[o];
    real a0 = -(Jp[0][0] * ui[0] + Jp[0][1] * ui[1] + Jp[0][2] * ui[2]);
    real a1 = -(Jp[1][0] * ui[0] + Jp[1][1] * ui[1] + Jp[1][2] * ui[2]);
    if (p) {
      const real* pj = p + 9 * (size_t)j;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        a0 += Jc[0][c] * pj[c];
        a1 += Jc[1][c] * pj[c];
      }
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) v[c] = Jc[0][c] * a0 + Jc[1][c] * a1;
  }
  const real s = warp_sums_to_lanes<9>(v);
  if (lane < 9) {
    double add = (double)s;
    if (p && (gw == 0 || CS.warp_cam[gw - 1] != j))
      add += st->lambda_used * Bdiag[9 * (size_t)j + lane] * (double)p[9 * (size_t)j + lane];
    atomicAdd(y + 9 * (size_t)j + lane, add);
  }
}

// split variant: zero the diagonal blocks of S' before the camera pass accumulates into them
__global__ void k_spcg_zero(DevProblem P, double* __restrict__ S) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 81 * P.m; e += gridDim.x * blockDim.x) {
    const int j = e / 81, rc = e - 81 * (e / 81), r = rc / 9, c = rc - 9 * (rc / 9);
    const int k = P.cam_cluster[j], lc = P.cam_local[j], np = P.cluster_np[k];
    S[P.S_off[k] + (size_t)(9 * lc + r) * np + 9 * lc + c] = 0.0;
  }
}

// split variant: the damped diagonal blocks of S' (45 lower entries) and b' of every camera, from the
// cluster layout filled by the camera pass
__global__ void k_spcg_blocks(DevProblem P, const double* __restrict__ S, const double* __restrict__ b,
                              double* __restrict__ Mblk, double* __restrict__ rhs) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P.m; j += gridDim.x * blockDim.x) {
    const int k = P.cam_cluster[j], lc = P.cam_local[j], np = P.cluster_np[k];
    const double* Sk = S + P.S_off[k] + (size_t)(9 * lc) * np + 9 * lc;
    int t = 0;
    for (int r = 0; r < 9; ++r)
      for (int c = 0; c <= r; ++c, ++t) Mblk[45 * (size_t)j + t] = Sk[(size_t)r * np + c];
    for (int r = 0; r < 9; ++r) rhs[9 * (size_t)j + r] = b[P.v_off[k] + 9 * lc + r];
  }
}

// t_v = sum_{o in v} J_p^T (J_c p_cam(o)), segmented by virtual point
template <typename real>
__global__ void __launch_bounds__(256) k_spcg_Et(DevProblem P, const real* __restrict__ J, const real* __restrict__ p,
                                                 real* __restrict__ t) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool act = o < P.q;
  int v = INT_MAX;
  real val[3] = {0, 0, 0};
  if (act) {
    v = P.obs_vp[o];
    real Jc[2][9], Jp[2][3];
    load_j(J, o, Jc, Jp);
    const real* pc = p + 9 * (size_t)P.obs_cam[o];
    real a0 = 0, a1 = 0;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      a0 += Jc[0][c] * pc[c];
      a1 += Jc[1][c] * pc[c];
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) val[s] = Jp[0][s] * a0 + Jp[1][s] * a1;
  }
  segmented_scan<3>(val, v, lane);
  segmented_store<3>(val, v, act, lane, o, P.vp_off, t);
}

// u_v = V'_v^-1 t_v with V' = L L^T (L^-1 packed in vp_info); nv from the device counter
template <typename real>
__global__ void k_spcg_u(const long long* __restrict__ counts, const real* __restrict__ vp_info,
                         const real* __restrict__ t, real* __restrict__ u) {
  const long long nv = counts[0];
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
    real Li[6], tv[3], uv[3];
#pragma unroll
    for (int c = 0; c < 6; ++c) Li[c] = vp_info[9 * v + c];
#pragma unroll
    for (int c = 0; c < 3; ++c) tv[c] = t[3 * v + c];
    chol3_apply(Li, tv, uv);
#pragma unroll
    for (int c = 0; c < 3; ++c) u[3 * v + c] = uv[c];
  }
}

// y_j += sum over the camera's observations of J_c^T N J_c p_j (single-observation virtual points, N =
// (I + J_p Lambda^-1 J_p^T)^-1, Lambda = lambda diag(J_p^T J_p)) or J_c^T (J_c p_j - J_p u_v) (the others),
// plus lambda diag(J_c^T J_c) p_j: S' p for the cameras of every cluster
template <typename real>
__global__ void __launch_bounds__(256) k_spcg_cam(DevProblem P, CamSlots CS, const real* __restrict__ J,
                                                  const real* __restrict__ p, const real* __restrict__ u,
                                                  const DevState* st, double* __restrict__ y) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= CS.nwarps) return;
  const int lane = threadIdx.x & 31;
  const int j = CS.warp_cam[gw];
  const int o = CS.slots[32 * (size_t)gw + lane];
  const real lam = (real)st->lambda_used;
  real vsum[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) vsum[c] = real(0);
  if (o >= 0) {
    real Jc[2][9], Jp[2][3];
    load_j(J, o, Jc, Jp);
    const real* pj = p + 9 * (size_t)j;
    real a0 = 0, a1 = 0;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      a0 += Jc[0][c] * pj[c];
      a1 += Jc[1][c] * pj[c];
    }
    const int v = P.obs_vp[o];
    real b0, b1;
    if (P.vp_off[v + 1] - P.vp_off[v] == 1) {
      real K00 = 0, K01 = 0, K11 = 0;
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        const real il = real(1) / (lam * (Jp[0][s] * Jp[0][s] + Jp[1][s] * Jp[1][s]));
        K00 += Jp[0][s] * Jp[0][s] * il;
        K01 += Jp[0][s] * Jp[1][s] * il;
        K11 += Jp[1][s] * Jp[1][s] * il;
      }
      const real idet = real(1) / ((real(1) + K00) * (real(1) + K11) - K01 * K01);
      b0 = ((real(1) + K11) * a0 - K01 * a1) * idet;
      b1 = (-K01 * a0 + (real(1) + K00) * a1) * idet;
    } else {
      const real* uv = u + 3 * (size_t)v;
      b0 = a0 - (Jp[0][0] * uv[0] + Jp[0][1] * uv[1] + Jp[0][2] * uv[2]);
      b1 = a1 - (Jp[1][0] * uv[0] + Jp[1][1] * uv[1] + Jp[1][2] * uv[2]);
    }
#pragma unroll
    for (int c = 0; c < 9; ++c)
      vsum[c] = Jc[0][c] * b0 + Jc[1][c] * b1 + lam * (Jc[0][c] * Jc[0][c] + Jc[1][c] * Jc[1][c]) * pj[c];
  }
  const real sv = warp_sums_to_lanes<9>(vsum);
  if (lane < 9) atomicAdd(y + 9 * (size_t)j + lane, (double)sv);
}

// Block sums of up to three per-thread values into partial[c * RED_BLOCKS + block].
__device__ __forceinline__ void block_partials3(double a, double b, double c, double* partial) {
  __shared__ double red[3][RED_THREADS / 32];
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    a += __shfl_xor_sync(FULL_MASK, a, d);
    b += __shfl_xor_sync(FULL_MASK, b, d);
    c += __shfl_xor_sync(FULL_MASK, c, d);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[0][w] = a;
    red[1][w] = b;
    red[2][w] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s[3] = {0, 0, 0};
    for (int i = 0; i < RED_THREADS / 32; ++i)
      for (int k = 0; k < 3; ++k) s[k] += red[k][i];
    for (int k = 0; k < 3; ++k) partial[k * RED_BLOCKS + blockIdx.x] = s[k];
  }
}

__device__ __forceinline__ double sum_partials(const double* partial) {
  double s = 0.0;
  for (int i = 0; i < RED_BLOCKS; ++i) s += partial[i];
  return s;
}

// z_j = Minv_j r_j (9 entries of camera j)
__device__ __forceinline__ void apply_minv(const double* __restrict__ Minv, int j, const double* r, double* z) {
  const double* M = Minv + 81 * (size_t)j;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    double s = 0.0;
#pragma unroll
    for (int b = 0; b < 9; ++b) s += M[9 * a + b] * r[b];
    z[a] = s;
  }
}

// r = b (= v + y from the right-hand-side pass), x = 0, z = Minv r, p = z; partials of r.z and r.r and b.b
template <typename real>
__global__ void __launch_bounds__(RED_THREADS) k_pcg_init(int m, const real* __restrict__ vgrad,
                                                          const double* __restrict__ yrhs,
                                                          const double* __restrict__ Minv, double* x, double* r,
                                                          double* pvec, real* pw, double* partial) {
  double rz = 0, rr = 0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    double rj[9], zj[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      rj[a] = (vgrad ? (double)vgrad[9 * (size_t)j + a] : 0.0) + yrhs[9 * (size_t)j + a];
      x[9 * (size_t)j + a] = 0.0;
      r[9 * (size_t)j + a] = rj[a];
    }
    apply_minv(Minv, j, rj, zj);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      pvec[9 * (size_t)j + a] = zj[a];
      pw[9 * (size_t)j + a] = (real)zj[a];
      rz += rj[a] * zj[a];
      rr += rj[a] * rj[a];
    }
  }
  block_partials3(rz, rr, 0.0, partial);
}

// scalars: s[0] = b.b, s[1 + parity] = r.z, s[3] = r.r
__global__ void k_pcg_start(const double* partial, double* s) {
  if (threadIdx.x == 0) {
    s[1] = sum_partials(partial);
    s[2] = 0.0;
    s[3] = sum_partials(partial + RED_BLOCKS);
    s[0] = s[3];
  }
}

// partials of p.q
__global__ void __launch_bounds__(RED_THREADS) k_pcg_pq(int m9, const double* __restrict__ pvec,
                                                        const double* __restrict__ q, double* partial) {
  double a = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m9; i += gridDim.x * blockDim.x) a += pvec[i] * q[i];
  block_partials3(a, 0.0, 0.0, partial);
}

// alpha = r.z / p.q; x += alpha p; r -= alpha q; z = Minv r; partials of the new r.z and r.r
__global__ void __launch_bounds__(RED_THREADS) k_pcg_update(int m, const double* __restrict__ pq_part,
                                                            const double* __restrict__ s, int parity,
                                                            const double* __restrict__ pvec,
                                                            const double* __restrict__ q,
                                                            const double* __restrict__ Minv, double* x, double* r,
                                                            double* z, double* partial) {
  const double pq = sum_partials(pq_part);
  const double alpha = (pq != 0.0) ? s[1 + parity] / pq : 0.0;
  double rz = 0, rr = 0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    double rj[9], zj[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const size_t i = 9 * (size_t)j + a;
      x[i] += alpha * pvec[i];
      rj[a] = r[i] - alpha * q[i];
      r[i] = rj[a];
    }
    apply_minv(Minv, j, rj, zj);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      z[9 * (size_t)j + a] = zj[a];
      rz += rj[a] * zj[a];
      rr += rj[a] * rj[a];
    }
  }
  block_partials3(rz, rr, 0.0, partial);
}

// beta = r.z_new / r.z_old; p = z + beta p (and its working-precision copy); the new scalars go to the
// other parity slot
template <typename real>
__global__ void __launch_bounds__(RED_THREADS) k_pcg_dir(int m9, const double* __restrict__ partial, double* s,
                                                         int parity, const double* __restrict__ z, double* pvec,
                                                         real* pw) {
  const double rz_new = sum_partials(partial);
  const double rz_old = s[1 + parity];
  const double beta = (rz_old != 0.0) ? rz_new / rz_old : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m9; i += gridDim.x * blockDim.x) {
    const double pn = z[i] + beta * pvec[i];
    pvec[i] = pn;
    pw[i] = (real)pn;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    s[1 + (1 - parity)] = rz_new;
    s[3] = sum_partials(partial + RED_BLOCKS);
  }
}

template <typename real>
__global__ void k_pcg_finish(int m9, const double* __restrict__ x, double* dc, float* dcf) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m9; i += gridDim.x * blockDim.x) {
    dc[i] = x[i];
    if (dcf) dcf[i] = (float)x[i];
  }
}

// u_i = C_i^-1 w_i (the point part of the right-hand side; w is stored after C^-1 in pt_info)
template <typename real>
__global__ void k_pcg_uw(int n, const real* __restrict__ pt_info, real* __restrict__ u) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const real* ci = pt_info + 9 * (size_t)i;
    real* ui = u + 3 * (size_t)i;
    ui[0] = ci[0] * ci[6] + ci[1] * ci[7] + ci[2] * ci[8];
    ui[1] = ci[1] * ci[6] + ci[3] * ci[7] + ci[4] * ci[8];
    ui[2] = ci[2] * ci[6] + ci[4] * ci[7] + ci[5] * ci[8];
  }
}

}  // namespace

template <typename real>
void pcg_prepare(const DevProblem& P, Scratch<real> W, CamSlots CS, const PcgBuffers& B, DevState* st,
                 cudaStream_t stream) {
  const int m = P.m, m9 = 9 * P.m;
  real* J = reinterpret_cast<real*>(B.J);
  real* pw = reinterpret_cast<real*>(B.pw);
  real* upt = reinterpret_cast<real*>(B.upt);
  const int obs_blocks = std::min((P.q + 255) / 256, num_sms() * 16);
  const int cam_blocks = (CS.nwarps + 7) / 8;
  const int pt_blocks = std::min((P.n + 255) / 256, 4096);
  const int vec_blocks = std::min((m + RED_THREADS - 1) / RED_THREADS, RED_BLOCKS);
  k_pcg_jac<real><<<obs_blocks, 256, 0, stream>>>(P, J);
  cudaMemsetAsync(B.Bdiag, 0, 9 * (size_t)m * sizeof(double), stream);
  if (B.split) {
    // the camera pass has filled the diagonal blocks of S' (damped) and b'
    k_spcg_blocks<<<(m + 127) / 128, 128, 0, stream>>>(P, W.S, W.b, B.Mblk, B.q);
    k_pcg_invert<<<(m + 127) / 128, 128, 0, stream>>>(m, B.Mblk, B.Bdiag, st, B.Minv);   // Bdiag = 0: no more damping
    cudaMemsetAsync(B.partial, 0, 3 * RED_BLOCKS * sizeof(double), stream);
    cudaMemsetAsync(B.partial2, 0, 3 * RED_BLOCKS * sizeof(double), stream);
    k_pcg_init<real><<<vec_blocks, RED_THREADS, 0, stream>>>(m, nullptr, B.q, B.Minv, B.x, B.r, B.p, pw, B.partial);
    k_pcg_start<<<1, 32, 0, stream>>>(B.partial, B.scal);
    return;
  }
  cudaMemsetAsync(B.Mblk, 0, 45 * (size_t)m * sizeof(double), stream);
  cudaMemsetAsync(W.vgrad, 0, 9 * (size_t)m * sizeof(real), stream);
  k_pcg_precond<real><<<cam_blocks, 256, 0, stream>>>(P, CS, J, W.pt_info, B.Mblk, B.Bdiag, W.vgrad);
  k_pcg_invert<<<(m + 127) / 128, 128, 0, stream>>>(m, B.Mblk, B.Bdiag, st, B.Minv);
  // right-hand side b = v - E C^-1 w: the camera pass with p = 0 and u = C^-1 w
  k_pcg_uw<real><<<pt_blocks, 256, 0, stream>>>(P.n, W.pt_info, upt);
  cudaMemsetAsync(B.q, 0, (size_t)m9 * sizeof(double), stream);
  k_pcg_cam<real><<<cam_blocks, 256, 0, stream>>>(P, CS, J, nullptr, upt, B.Bdiag, st, B.q);
  // partial slots beyond the launched blocks stay zero
  cudaMemsetAsync(B.partial, 0, 3 * RED_BLOCKS * sizeof(double), stream);
  cudaMemsetAsync(B.partial2, 0, 3 * RED_BLOCKS * sizeof(double), stream);
  k_pcg_init<real><<<vec_blocks, RED_THREADS, 0, stream>>>(m, W.vgrad, B.q, B.Minv, B.x, B.r, B.p, pw, B.partial);
  k_pcg_start<<<1, 32, 0, stream>>>(B.partial, B.scal);
}

void launch_spcg_zero(const DevProblem& P, double* S, cudaStream_t stream) {
  k_spcg_zero<<<std::min((81 * P.m + 255) / 256, 4 * RED_BLOCKS), 256, 0, stream>>>(P, S);
}

template <typename real>
int pcg_iterate(const DevProblem& P, Scratch<real> W, CamSlots CS, const PcgBuffers& B, int max_iter, double tol,
                DevState* st, cudaStream_t stream) {
  const int m = P.m, m9 = 9 * P.m;
  real* J = reinterpret_cast<real*>(B.J);
  real* pw = reinterpret_cast<real*>(B.pw);
  real* tpt = reinterpret_cast<real*>(B.tpt);
  real* upt = reinterpret_cast<real*>(B.upt);
  const int seg_blocks = (P.q + 255) / 256;
  const int cam_blocks = (CS.nwarps + 7) / 8;
  const int pt_blocks = std::min((P.n + 255) / 256, 4096);
  const int vec_blocks = std::min((m + RED_THREADS - 1) / RED_THREADS, RED_BLOCKS);
  const int vec9_blocks = std::min((m9 + RED_THREADS - 1) / RED_THREADS, RED_BLOCKS);
  int it = 0;
  const double tol2 = tol * tol;
  constexpr int CHECK_EVERY = 4;
  while (it < max_iter) {
    const int upto = std::min(it + CHECK_EVERY, max_iter);
    for (; it < upto; ++it) {
      const int parity = it & 1;
      // q = S p
      cudaMemsetAsync(B.q, 0, (size_t)m9 * sizeof(double), stream);
      if (B.split) {   // S' p over the virtual points
        real* tvp = reinterpret_cast<real*>(B.tvp);
        real* uvp = reinterpret_cast<real*>(B.uvp);
        launch_zero_vp3(tvp, B.counts, (int)sizeof(real), stream);
        k_spcg_Et<real><<<seg_blocks, 256, 0, stream>>>(P, J, pw, tvp);
        k_spcg_u<real><<<2 * RED_BLOCKS, 256, 0, stream>>>(B.counts, W.vp_info, tvp, uvp);
        k_spcg_cam<real><<<cam_blocks, 256, 0, stream>>>(P, CS, J, pw, uvp, st, B.q);
      } else {
        cudaMemsetAsync(tpt, 0, 3 * (size_t)P.n * sizeof(real), stream);
        k_pcg_Et<real><<<seg_blocks, 256, 0, stream>>>(P, J, pw, tpt);
        k_pcg_u<real><<<pt_blocks, 256, 0, stream>>>(P.n, W.pt_info, tpt, upt);
        k_pcg_cam<real><<<cam_blocks, 256, 0, stream>>>(P, CS, J, pw, upt, B.Bdiag, st, B.q);
      }
      k_pcg_pq<<<vec9_blocks, RED_THREADS, 0, stream>>>(m9, B.p, B.q, B.partial2);
      k_pcg_update<<<vec_blocks, RED_THREADS, 0, stream>>>(m, B.partial2, B.scal, parity, B.p, B.q, B.Minv, B.x, B.r,
                                                           B.z, B.partial);
      k_pcg_dir<real><<<vec9_blocks, RED_THREADS, 0, stream>>>(m9, B.partial, B.scal, parity, B.z, B.p, pw);
    }
    double hs[4];
    if (cudaMemcpyAsync(hs, B.scal, sizeof hs, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
      break;
    if (!(hs[3] > tol2 * hs[0])) break;   // converged (or the residual is not finite)
  }
  k_pcg_finish<real><<<vec9_blocks, RED_THREADS, 0, stream>>>(m9, B.x, W.dc, W.dcf);
  return it;
}

#define PCG_INSTANTIATE(real)                                                                                  \
  template void pcg_prepare<real>(const DevProblem&, Scratch<real>, CamSlots, const PcgBuffers&, DevState*,   \
                                  cudaStream_t);                                                              \
  template int pcg_iterate<real>(const DevProblem&, Scratch<real>, CamSlots, const PcgBuffers&, int, double,  \
                                 DevState*, cudaStream_t);
PCG_INSTANTIATE(float)
PCG_INSTANTIATE(double)

}  // namespace stba
