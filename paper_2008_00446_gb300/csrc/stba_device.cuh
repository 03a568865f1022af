// Device helpers shared by the per-iteration kernels and the adjoint kernels: observation loads, warp
// segmented sums over runs of equal keys, and 3x3 Cholesky inverses.
#pragma once
#include <cuda_runtime.h>

#include "stba_camera.cuh"
#include "stba_internal.cuh"

namespace stba {

#define FULL_MASK 0xffffffffu

template <typename real>
__device__ __forceinline__ void load_uv(const DevProblem& P, int o, real& u, real& v) {
  if constexpr (sizeof(real) == 8) {
    double2 t = reinterpret_cast<const double2*>(P.obs_uv)[o];
    u = t.x;
    v = t.y;
  } else {
    float2 t = reinterpret_cast<const float2*>(P.obs_uvf)[o];
    u = t.x;
    v = t.y;
  }
}

template <typename real>
__device__ __forceinline__ void load_point(const double* p, real X[3]) {
  X[0] = (real)p[0];
  X[1] = (real)p[1];
  X[2] = (real)p[2];
}

// Camera and point in the working precision: FP64 from the parameters, FP32 from the per-iteration copies.
template <typename real>
__device__ __forceinline__ Cam<real> load_cam_w(const DevProblem& P, int j) {
  Cam<real> C;
  if constexpr (sizeof(real) == 8) {
    C = load_cam<real>(P.cams + 9 * (size_t)j);
  } else {
    const float* c = P.cams_f + 9 * (size_t)j;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      C.w[k] = c[k];
      C.t[k] = c[3 + k];
    }
    C.f = c[6];
    C.k1 = c[7];
    C.k2 = c[8];
  }
  return C;
}
template <typename real>
__device__ __forceinline__ void load_point_w(const DevProblem& P, int i, real X[3]) {
  if constexpr (sizeof(real) == 8) {
    load_point(P.pts + 3 * (size_t)i, X);
  } else {
    const float* p = P.pts_f + 3 * (size_t)i;
    X[0] = p[0];
    X[1] = p[1];
    X[2] = p[2];
  }
}

// Records of 9 reals, one per lane, of cnt <= 32 consecutive records r0.. (r0 a multiple of 32), staged
// through the warp's 288-real shared buffer sm (16-byte aligned): a full block of 32 records is one
// contiguous, 16-byte aligned span, moved with 16-byte vector accesses by the whole warp instead of nine
// strided scalar accesses per lane.  Lanes >= cnt get / store nothing.
template <typename real>
__device__ __forceinline__ void warp_load_rec9(const real* __restrict__ g, long long r0, int cnt, real* sm, int lane,
                                               real (&x)[9]) {
  const real* blk = g + 9 * r0;
  if (cnt == 32 && ((reinterpret_cast<size_t>(blk) & 15) == 0)) {
    constexpr int NQ = 9 * 32 * (int)sizeof(real) / 16;
    for (int k = lane; k < NQ; k += 32) reinterpret_cast<float4*>(sm)[k] = reinterpret_cast<const float4*>(blk)[k];
  } else {
    for (int k = lane; k < 9 * cnt; k += 32) sm[k] = blk[k];
  }
  __syncwarp();
  if (lane < cnt) {
#pragma unroll
    for (int c = 0; c < 9; ++c) x[c] = sm[9 * lane + c];
  }
  __syncwarp();
}

template <typename real>
__device__ __forceinline__ void warp_store_rec9(real* __restrict__ g, long long r0, int cnt, real* sm, int lane,
                                                const real (&x)[9]) {
  if (lane < cnt) {
#pragma unroll
    for (int c = 0; c < 9; ++c) sm[9 * lane + c] = x[c];
  }
  __syncwarp();
  real* blk = g + 9 * r0;
  if (cnt == 32 && ((reinterpret_cast<size_t>(blk) & 15) == 0)) {
    constexpr int NQ = 9 * 32 * (int)sizeof(real) / 16;
    for (int k = lane; k < NQ; k += 32) reinterpret_cast<float4*>(blk)[k] = reinterpret_cast<const float4*>(sm)[k];
  } else {
    for (int k = lane; k < 9 * cnt; k += 32) blk[k] = sm[k];
  }
  __syncwarp();
}

// Inclusive warp scan of NV values restricted to runs of equal (non-decreasing) keys.
template <int NV, typename real>
__device__ __forceinline__ void segmented_scan(real (&val)[NV], int key, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int ku = __shfl_up_sync(FULL_MASK, key, d);
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      real y = __shfl_up_sync(FULL_MASK, val[c], d);
      if (lane >= d && ku == key) val[c] += y;
    }
  }
}

// The last lane of each run writes the run's sum.  A run lying wholly inside this warp's 32
// observations is stored; a run that continues into a neighbouring warp is added atomically
// (the destination was zeroed before the launch).
template <int NV, typename real>
__device__ __forceinline__ void segmented_store(const real (&val)[NV], int key, bool act, int lane, int o,
                                                const int* seg_off, real* dst_base) {
  int knext = __shfl_down_sync(FULL_MASK, key, 1);
  if (act && (lane == 31 || knext != key)) {
    int w0 = o - lane;
    bool whole = seg_off[key] >= w0 && seg_off[key + 1] <= w0 + 32;
    real* dst = dst_base + (size_t)NV * key;
    if (whole) {
#pragma unroll
      for (int c = 0; c < NV; ++c) dst[c] = val[c];
    } else {
#pragma unroll
      for (int c = 0; c < NV; ++c) atomicAdd(dst + c, val[c]);
    }
  }
}

// 3x3 symmetric positive-definite helpers (packed lower/symmetric storage xx xy xz yy yz zz).
template <typename real>
__device__ __forceinline__ real safe_pivot(real d) {
  return d > real(0) ? d : (real)(sizeof(real) == 8 ? 1e-300 : 1e-30);
}

// Cholesky V = L L^T and the inverse of L (packed l00 l10 l11 l20 l21 l22).
template <typename real>
__device__ __forceinline__ void chol3_inv(const real V[6], real Li[6]) {
  real l00 = sqrt(safe_pivot(V[0]));
  real l10 = V[1] / l00;
  real l20 = V[2] / l00;
  real l11 = sqrt(safe_pivot(V[3] - l10 * l10));
  real l21 = (V[4] - l20 * l10) / l11;
  real l22 = sqrt(safe_pivot(V[5] - l20 * l20 - l21 * l21));
  real i00 = real(1) / l00, i11 = real(1) / l11, i22 = real(1) / l22;
  real i10 = -l10 * i00 * i11;
  real i21 = -l21 * i11 * i22;
  real i20 = -(l20 * i00 + l21 * i10) * i22;
  Li[0] = i00;
  Li[1] = i10;
  Li[2] = i11;
  Li[3] = i20;
  Li[4] = i21;
  Li[5] = i22;
}

// x = (L L^T)^-1 w = L^-T (L^-1 w)
template <typename real>
__device__ __forceinline__ void chol3_apply(const real Li[6], const real w[3], real x[3]) {
  real z0 = Li[0] * w[0];
  real z1 = Li[1] * w[0] + Li[2] * w[1];
  real z2 = Li[3] * w[0] + Li[4] * w[1] + Li[5] * w[2];
  x[0] = Li[0] * z0 + Li[1] * z1 + Li[3] * z2;
  x[1] = Li[2] * z1 + Li[4] * z2;
  x[2] = Li[5] * z2;
}

// Huber loss (Ceres' HuberLoss(a) on s = ||f_o||^2): the residual and Jacobian rows of an observation enter
// the normal equations scaled by sqrt(rho'(s)) = 1 for s <= a^2 and sqrt(a / sqrt(s)) beyond.
template <typename real>
__device__ __forceinline__ real huber_sqrt_weight(double a, real r0, real r1) {
  if (!(a > 0.0)) return real(1);
  const real s = r0 * r0 + r1 * r1, ar = (real)a;
  return s <= ar * ar ? real(1) : sqrt(ar / sqrt(s));
}

template <typename real>
__device__ __forceinline__ void scale_rows(real sw, real (&r)[2], real (&Jc)[2][9], real (&Jp)[2][3]) {
  r[0] *= sw;
  r[1] *= sw;
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    Jc[0][c] *= sw;
    Jc[1][c] *= sw;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Jp[0][c] *= sw;
    Jp[1][c] *= sw;
  }
}

// rho(s) of the cost, in FP64
__device__ __forceinline__ double huber_rho(double a, double s) {
  if (!(a > 0.0) || s <= a * a) return s;
  return 2.0 * a * sqrt(s) - a * a;
}

}  // namespace stba
