// Reprojection error and its analytic Jacobian (Sec. 3), hand-derived for the device.
//
//   Y = R(w) X = X + a (w x X) + b (w (w.X) - s X),  s = |w|^2, a = sin(th)/th, b = (1 - cos th)/s
//   Xc = Y + t,  x = Xc0/Xc2, y = Xc1/Xc2,  r2 = x^2 + y^2,  d = 1 + k1 r2 + k2 r2^2
//   pi = f d (x, y),  f_o = pi - q_o
// Derivatives:
//   d pi / d(x, y) = f [[d + 2 x^2 e, 2 x y e], [2 x y e, d + 2 y^2 e]],  e = k1 + 2 k2 r2
//   d(x, y) / d Xc = [[1/z, 0, -x/z], [0, 1/z, -y/z]]        -> P = d pi / d Xc (2x3)
//   d pi / d t = P,   d pi / d X = P R(w)
//   d Y / d w = 2 a' (w x X) w^T - a [X]x + 2 b' (w (w.X) - s X) w^T + b ((w.X) I + w X^T - 2 X w^T)
//   with a' = da/ds = (cos th - a) / (2 s) and b' = db/ds = (a/2 - b) / s;
//   d pi / d f = d (x, y),  d pi / d k1 = f r2 (x, y),  d pi / d k2 = f r2^2 (x, y).
// Near th = 0 the Taylor series of a, b, a', b' in s replace the quotients.
#pragma once
#include <cuda_runtime.h>

namespace stba {

template <typename real> struct RodSeries;
template <> struct RodSeries<double> { static constexpr double cut = 1e-4; };
template <> struct RodSeries<float> { static constexpr float cut = 1e-1f; };

// sqrt and sincos in the working precision; rodrigues_coeffs calls them unqualified, so other number
// types (the dual numbers of the adjoint) supply their own overloads, found by argument-dependent lookup.
__device__ __forceinline__ float sq_root(float x) { return sqrtf(x); }
__device__ __forceinline__ double sq_root(double x) { return sqrt(x); }
__device__ __forceinline__ void sin_cos(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sin_cos(double x, double* s, double* c) { sincos(x, s, c); }

template <typename real>
__device__ __forceinline__ void rodrigues_coeffs(real s, real& a, real& b, real& da, real& db) {
  if (s < RodSeries<real>::cut) {
    // a = sum (-s)^k / (2k+1)!,  b = sum (-s)^k / (2k+2)!  (to s^3) and their s-derivatives
    a = real(1) - s * (real(1) / 6 - s * (real(1) / 120 - s * (real(1) / 5040)));
    b = real(0.5) - s * (real(1) / 24 - s * (real(1) / 720 - s * (real(1) / 40320)));
    da = -real(1) / 6 + s * (real(1) / 60 - s * (real(1) / 1680 - s * (real(1) / 90720)));
    db = -real(1) / 24 + s * (real(1) / 360 - s * (real(1) / 13440 - s * (real(1) / 907200)));
  } else {
    real th = sq_root(s);
    real sn, cs, sh, ch;
    sin_cos(th, &sn, &cs);
    sin_cos(real(0.5) * th, &sh, &ch);
    a = sn / th;
    b = real(2) * sh * sh / s;
    da = (cs - a) / (real(2) * s);
    db = (real(0.5) * a - b) / s;
  }
}

// Camera parameters converted to the working precision.
template <typename real> struct Cam {
  real w[3], t[3], f, k1, k2;
};

template <typename real>
__device__ __forceinline__ Cam<real> load_cam(const double* c) {
  Cam<real> C;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    C.w[k] = (real)c[k];
    C.t[k] = (real)c[3 + k];
  }
  C.f = (real)c[6];
  C.k1 = (real)c[7];
  C.k2 = (real)c[8];
  return C;
}

template <typename real>
__device__ __forceinline__ Cam<real> load_cam_step(const double* c, const double* dc) {
  Cam<real> C;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    C.w[k] = (real)(c[k] + dc[k]);
    C.t[k] = (real)(c[3 + k] + dc[3 + k]);
  }
  C.f = (real)(c[6] + dc[6]);
  C.k1 = (real)(c[7] + dc[7]);
  C.k2 = (real)(c[8] + dc[8]);
  return C;
}

// Residual only (cost evaluation).  Returns the depth Xc.z in *z.
template <typename real>
__device__ __forceinline__ void project_residual(const Cam<real>& C, const real X[3], real u_obs, real v_obs,
                                                 real r[2], real* z) {
  const real* w = C.w;
  real s = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  real a, b, da, db;
  rodrigues_coeffs(s, a, b, da, db);
  real wx[3] = {w[1] * X[2] - w[2] * X[1], w[2] * X[0] - w[0] * X[2], w[0] * X[1] - w[1] * X[0]};
  real wd = w[0] * X[0] + w[1] * X[1] + w[2] * X[2];
  real Xc[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) Xc[i] = X[i] + a * wx[i] + b * (w[i] * wd - s * X[i]) + C.t[i];
  real iz = real(1) / Xc[2];
  real x = Xc[0] * iz, y = Xc[1] * iz;
  real r2 = x * x + y * y;
  real d = real(1) + r2 * (C.k1 + C.k2 * r2);
  r[0] = C.f * d * x - u_obs;
  r[1] = C.f * d * y - v_obs;
  *z = Xc[2];
}

// Residual and Jacobian blocks: Jc (2x9, row-major) and Jp (2x3).  With want_cam = false only Jp.
template <typename real, bool want_cam>
__device__ __forceinline__ void project_jacobian(const Cam<real>& C, const real X[3], real u_obs, real v_obs,
                                                 real r[2], real Jc[2][9], real Jp[2][3]) {
  const real* w = C.w;
  real s = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  real a, b, da, db;
  rodrigues_coeffs(s, a, b, da, db);
  real wx[3] = {w[1] * X[2] - w[2] * X[1], w[2] * X[0] - w[0] * X[2], w[0] * X[1] - w[1] * X[0]};
  real wd = w[0] * X[0] + w[1] * X[1] + w[2] * X[2];
  real Xc[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) Xc[i] = X[i] + a * wx[i] + b * (w[i] * wd - s * X[i]) + C.t[i];
  real iz = real(1) / Xc[2];
  real x = Xc[0] * iz, y = Xc[1] * iz;
  real r2 = x * x + y * y;
  real d = real(1) + r2 * (C.k1 + C.k2 * r2);
  real fd = C.f * d;
  r[0] = fd * x - u_obs;
  r[1] = fd * y - v_obs;
  real e = C.k1 + real(2) * C.k2 * r2;
  real fe2 = real(2) * C.f * e;
  real dux = fd + fe2 * x * x, duy = fe2 * x * y;
  real dvx = duy, dvy = fd + fe2 * y * y;
  real P[2][3];
  P[0][0] = dux * iz;
  P[0][1] = duy * iz;
  P[0][2] = -(dux * x + duy * y) * iz;
  P[1][0] = dvx * iz;
  P[1][1] = dvy * iz;
  P[1][2] = -(dvx * x + dvy * y) * iz;
  // R(w) = I + a [w]x + b (w w^T - s I)
  real R[3][3];
  R[0][0] = real(1) + b * (w[0] * w[0] - s);
  R[1][1] = real(1) + b * (w[1] * w[1] - s);
  R[2][2] = real(1) + b * (w[2] * w[2] - s);
  R[0][1] = -a * w[2] + b * w[0] * w[1];
  R[1][0] = a * w[2] + b * w[0] * w[1];
  R[0][2] = a * w[1] + b * w[0] * w[2];
  R[2][0] = -a * w[1] + b * w[0] * w[2];
  R[1][2] = -a * w[0] + b * w[1] * w[2];
  R[2][1] = a * w[0] + b * w[1] * w[2];
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int j = 0; j < 3; ++j) Jp[t][j] = P[t][0] * R[0][j] + P[t][1] * R[1][j] + P[t][2] * R[2][j];
  if constexpr (want_cam) {
    // dY/dw
    real u1[3], u2[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      u1[i] = real(2) * da * wx[i];
      u2[i] = real(2) * db * (w[i] * wd - s * X[i]);
    }
    real Xh[3][3] = {{0, -X[2], X[1]}, {X[2], 0, -X[0]}, {-X[1], X[0], 0}};
    real dY[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        dY[i][j] = (u1[i] + u2[i]) * w[j] - a * Xh[i][j] +
                   b * ((i == j ? wd : real(0)) + w[i] * X[j] - real(2) * X[i] * w[j]);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Jc[t][j] = P[t][0] * dY[0][j] + P[t][1] * dY[1][j] + P[t][2] * dY[2][j];
        Jc[t][3 + j] = P[t][j];
      }
    }
    Jc[0][6] = d * x;
    Jc[1][6] = d * y;
    Jc[0][7] = C.f * r2 * x;
    Jc[1][7] = C.f * r2 * y;
    Jc[0][8] = C.f * r2 * r2 * x;
    Jc[1][8] = C.f * r2 * r2 * y;
  }
}

}  // namespace stba
