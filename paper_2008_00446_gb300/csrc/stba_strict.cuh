// FP32 numbers whose rounding is fixed by the source: a product is held unrounded (SFProd) and fused with
// the addition or subtraction it meets (one fused multiply-add, __fmaf_rn), every other operation is rounded
// on its own (__fadd_rn, __fmul_rn, ...), and the compiler contracts or re-associates nothing.  The
// arithmetic of an expression is then the same in every kernel that evaluates it.  The FP32 kernels that form
// V_v, the diagonal and the off-diagonal blocks of S'_k (Eq. 10, 13) all evaluate the reprojection Jacobian
// of an observation (Sec. 3) on this type, so that they see bitwise the same J_c, J_p (and G_o =
// L_v^-1 J_p^T J_c, whether the pair pass reads the camera pass's copy or recomputes it).
#pragma once
#include <cuda_runtime.h>

#include "stba_camera.cuh"

namespace stba {

struct SFProd;

struct SF {
  float v;
  SF() = default;
  __host__ __device__ constexpr SF(float x) : v(x) {}
  __device__ __forceinline__ SF(const SFProd& p);   // the product, rounded

  friend __device__ __forceinline__ SF operator+(SF a, SF b) { return SF(__fadd_rn(a.v, b.v)); }
  friend __device__ __forceinline__ SF operator-(SF a, SF b) { return SF(__fsub_rn(a.v, b.v)); }
  friend __device__ __forceinline__ SF operator-(SF a) { return SF(-a.v); }
  friend __device__ __forceinline__ SFProd operator*(SF a, SF b);
  friend __device__ __forceinline__ SF operator/(SF a, SF b) { return SF(__fdiv_rn(a.v, b.v)); }
  friend __device__ __forceinline__ bool operator<(SF a, SF b) { return a.v < b.v; }

  friend __device__ __forceinline__ SF sq_root(SF a) { return SF(__fsqrt_rn(a.v)); }
  friend __device__ __forceinline__ void sin_cos(SF x, SF* s, SF* c) {
    float sv, cv;
    sincosf(x.v, &sv, &cv);
    *s = SF(sv);
    *c = SF(cv);
  }
};

// a * b, not yet rounded
struct SFProd {
  float a, b;
  __device__ __forceinline__ float rounded() const { return __fmul_rn(a, b); }

  friend __device__ __forceinline__ SF operator+(SFProd p, SF c) { return SF(__fmaf_rn(p.a, p.b, c.v)); }
  friend __device__ __forceinline__ SF operator+(SF c, SFProd p) { return SF(__fmaf_rn(p.a, p.b, c.v)); }
  friend __device__ __forceinline__ SF operator+(SFProd p, SFProd q) { return SF(__fmaf_rn(p.a, p.b, q.rounded())); }
  friend __device__ __forceinline__ SF operator-(SFProd p, SF c) { return SF(__fmaf_rn(p.a, p.b, -c.v)); }
  friend __device__ __forceinline__ SF operator-(SF c, SFProd p) { return SF(__fmaf_rn(-p.a, p.b, c.v)); }
  friend __device__ __forceinline__ SF operator-(SFProd p, SFProd q) { return SF(__fmaf_rn(p.a, p.b, -q.rounded())); }
  friend __device__ __forceinline__ SFProd operator-(SFProd p) { return SFProd{-p.a, p.b}; }
  friend __device__ __forceinline__ SFProd operator*(SFProd p, SF c) { return SFProd{p.rounded(), c.v}; }
  friend __device__ __forceinline__ SFProd operator*(SF c, SFProd p) { return SFProd{c.v, p.rounded()}; }
  friend __device__ __forceinline__ SFProd operator*(SFProd p, SFProd q) { return SFProd{p.rounded(), q.rounded()}; }
  friend __device__ __forceinline__ SF operator/(SFProd p, SF d) { return SF(__fdiv_rn(p.rounded(), d.v)); }
  friend __device__ __forceinline__ SF operator/(SF n, SFProd p) { return SF(__fdiv_rn(n.v, p.rounded())); }
};

__device__ __forceinline__ SF::SF(const SFProd& p) : v(p.rounded()) {}
__device__ __forceinline__ SFProd operator*(SF a, SF b) { return SFProd{a.v, b.v}; }

template <> struct RodSeries<SF> { static constexpr float cut = RodSeries<float>::cut; };

// Residual-free Jacobian rows J_c (2 x 9, want_cam only) and J_p (2 x 3) of one observation in FP32, every
// operation rounded on its own (J_p does not depend on want_cam).
template <bool want_cam = true>
__device__ __forceinline__ void project_jacobian_strict(const Cam<float>& C, const float X[3], float u_obs,
                                                        float v_obs, float Jc[2][9], float Jp[2][3]) {
  Cam<SF> Cs;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    Cs.w[k] = SF(C.w[k]);
    Cs.t[k] = SF(C.t[k]);
  }
  Cs.f = SF(C.f);
  Cs.k1 = SF(C.k1);
  Cs.k2 = SF(C.k2);
  const SF Xs[3] = {SF(X[0]), SF(X[1]), SF(X[2])};
  SF r[2], Jcs[2][9], Jps[2][3];
  project_jacobian<SF, want_cam>(Cs, Xs, SF(u_obs), SF(v_obs), r, Jcs, Jps);
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    if constexpr (want_cam) {
#pragma unroll
      for (int c = 0; c < 9; ++c) Jc[t][c] = Jcs[t][c].v;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) Jp[t][c] = Jps[t][c].v;
  }
}

// sqrt(rho'(|f|^2)) of the Huber loss (1 without a robust loss), every operation rounded on its own.
__device__ __forceinline__ float huber_sqrt_weight_strict(double a, float r0, float r1) {
  if (!(a > 0.0)) return 1.f;
  const float s = __fadd_rn(__fmul_rn(r0, r0), __fmul_rn(r1, r1)), ar = (float)a;
  return s <= __fmul_rn(ar, ar) ? 1.f : __fsqrt_rn(__fdiv_rn(ar, __fsqrt_rn(s)));
}

}  // namespace stba
