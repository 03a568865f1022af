// Forward-mode dual numbers v + e d (e^2 = 0) in FP64 (Dual) or FP32 (DualF).  Evaluating the analytic
// reprojection Jacobian (project_jacobian) on duals whose tangents are a direction beta in the 12 local
// parameters (camera 9, point 3) of one observation gives the directional derivative of that Jacobian along
// beta, i.e. the second-derivative products sum_s alpha_s H_s beta of the adjoint, without truncation error.
// The FP32 form serves the mixed-precision adjoint: this GPU's FP64 pipe runs at 1/64 of the FP32 rate.
#pragma once
#include <cuda_runtime.h>

#include "stba_camera.cuh"

namespace stba {

// The operators are hidden friends (non-template functions of each instantiation), so that a constant of
// another arithmetic type (an int literal) converts to R and takes the cheaper mixed form.
template <typename R> struct DualT {
  R v, d;
  DualT() = default;
  __host__ __device__ constexpr DualT(R x) : v(x), d(R(0)) {}
  __host__ __device__ constexpr DualT(R x, R t) : v(x), d(t) {}

  friend __device__ __forceinline__ DualT operator+(DualT a, DualT b) { return DualT(a.v + b.v, a.d + b.d); }
  friend __device__ __forceinline__ DualT operator-(DualT a, DualT b) { return DualT(a.v - b.v, a.d - b.d); }
  friend __device__ __forceinline__ DualT operator-(DualT a) { return DualT(-a.v, -a.d); }
  friend __device__ __forceinline__ DualT operator*(DualT a, DualT b) {
    return DualT(a.v * b.v, a.d * b.v + a.v * b.d);
  }
  friend __device__ __forceinline__ DualT operator/(DualT a, DualT b) {
    const R q = a.v / b.v;
    return DualT(q, (a.d - q * b.d) / b.v);
  }
  // mixed forms with a constant (no tangent), so constants cost no extra arithmetic
  friend __device__ __forceinline__ DualT operator+(DualT a, R b) { return DualT(a.v + b, a.d); }
  friend __device__ __forceinline__ DualT operator+(R a, DualT b) { return DualT(a + b.v, b.d); }
  friend __device__ __forceinline__ DualT operator-(DualT a, R b) { return DualT(a.v - b, a.d); }
  friend __device__ __forceinline__ DualT operator-(R a, DualT b) { return DualT(a - b.v, -b.d); }
  friend __device__ __forceinline__ DualT operator*(DualT a, R b) { return DualT(a.v * b, a.d * b); }
  friend __device__ __forceinline__ DualT operator*(R a, DualT b) { return DualT(a * b.v, a * b.d); }
  friend __device__ __forceinline__ DualT operator/(DualT a, R b) { return DualT(a.v / b, a.d / b); }
  friend __device__ __forceinline__ DualT operator/(R a, DualT b) {
    const R q = a / b.v;
    return DualT(q, -q * b.d / b.v);
  }
  friend __device__ __forceinline__ bool operator<(DualT a, R b) { return a.v < b; }

  friend __device__ __forceinline__ DualT sq_root(DualT a) {
    const R r = sq_root(a.v);
    return DualT(r, R(0.5) * a.d / r);
  }
  friend __device__ __forceinline__ void sin_cos(DualT x, DualT* s, DualT* c) {
    R sv, cv;
    sin_cos(x.v, &sv, &cv);
    *s = DualT(sv, cv * x.d);
    *c = DualT(cv, -sv * x.d);
  }
};

using Dual = DualT<double>;
using DualF = DualT<float>;

// the series threshold of the rotation coefficients is that of the value part's precision
template <> struct RodSeries<Dual> { static constexpr double cut = RodSeries<double>::cut; };
template <> struct RodSeries<DualF> { static constexpr float cut = RodSeries<float>::cut; };

}  // namespace stba
