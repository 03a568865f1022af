// Forward-mode dual numbers v + e d (e^2 = 0) in FP64.  Evaluating the analytic reprojection Jacobian
// (project_jacobian) on duals whose tangents are a direction beta in the 12 local parameters (camera 9,
// point 3) of one observation gives the directional derivative of that Jacobian along beta, i.e. the
// second-derivative products sum_s alpha_s H_s beta of the adjoint, without truncation error.
#pragma once
#include <cuda_runtime.h>

#include "stba_camera.cuh"

namespace stba {

struct Dual {
  double v, d;
  Dual() = default;
  __host__ __device__ constexpr Dual(double x) : v(x), d(0.0) {}
  __host__ __device__ constexpr Dual(double x, double t) : v(x), d(t) {}
};

__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
// mixed forms with a constant (no tangent), so constants cost no extra arithmetic
__device__ __forceinline__ Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
__device__ __forceinline__ Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
__device__ __forceinline__ Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
__device__ __forceinline__ Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
__device__ __forceinline__ Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
__device__ __forceinline__ Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
__device__ __forceinline__ Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
__device__ __forceinline__ Dual operator/(double a, Dual b) {
  const double q = a / b.v;
  return Dual(q, -q * b.d / b.v);
}
__device__ __forceinline__ bool operator<(Dual a, double b) { return a.v < b; }

__device__ __forceinline__ Dual sq_root(Dual a) {
  const double r = sqrt(a.v);
  return Dual(r, 0.5 * a.d / r);
}
__device__ __forceinline__ void sin_cos(Dual x, Dual* s, Dual* c) {
  double sv, cv;
  sincos(x.v, &sv, &cv);
  *s = Dual(sv, cv * x.d);
  *c = Dual(cv, -sv * x.d);
}

// the FP64 series threshold of the rotation coefficients applies to the value part
template <> struct RodSeries<Dual> { static constexpr double cut = 1e-4; };

}  // namespace stba
