// Per-iteration kernels of the STBA LM step (Algorithm 1), except the dense cluster factorisation.
//
//   k_vp_reduce      per observation, warp-segmented by virtual point: V = sum Jp^T Jp, w' = -sum Jp^T f
//                    (Eq. 10: C' and w' of the split points).
//   k_pt_acc         per point (a warp per 32 points): C and w of the physical point, summed over its
//                    virtual points.
//   k_vp_finalize    per virtual point: steepest-descent correction of w' (Sec. 4.3, closed form below),
//                    damped V', its Cholesky inverse, y = V'^-1 w'; per point: physical C^-1 and w (Eq. 4)
//                    for Eq. 15.
//   k_cam_pass       per camera (a warp per 32 of its observations): the diagonal blocks of S'_k, b' and the
//                    camera gradient (Eq. 10/13).
//   k_pair_build     per camera pair of the camera graph inside a cluster: the off-diagonal blocks of S'_k.
//   k_point_rhs      per observation, warp-segmented by point: sum_o Jp^T Jc dc.
//   k_point_update   per point: dp = C^-1 (w - E^T dc) (Eq. 6 = Eq. 15).
//   k_cost(_df)      F(x + dx) with FP64 sums; k_finalize: stop tests and the accept rule of Algorithm 1.
//
// Correction closed form: A has no camera columns and H~ = diag(H_lambda) is diagonal, so
// nu = (A H~^-1 A^T)^-1 A H~^-1 g makes H~^-1 (g - A^T nu) the H~-weighted projection of H~^-1 g on the
// steps where all virtual copies of a point are equal.  Per point and coordinate a:
//   dbar_a = sum_k w'_k,a / sum_k H~_k,a,  corrected w'_k,a = H~_k,a dbar_a,
// with H~_k = (1 + lambda) diag(V_k); the factor (1 + lambda) cancels.
#include <cfloat>
#include <climits>

#include "stba_camera.cuh"
#include "stba_device.cuh"
#include "stba_strict.cuh"
#include "stba_internal.cuh"

namespace stba {

// ------------------------------------------------------------------------------------------------------
template <typename real>
__global__ void k_iter_begin(DevState* st, Settings s) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    st->lambda_used = st->lambda;
    st->corrected = (s.correction && st->lambda >= s.correction_lambda) ? 1 : 0;
    st->grad_max_bits = 0ull;
    st->failed = 0;
    st->nonfinite = 0;
    st->boosted = 0;
  }
}

template <typename real>
void launch_iter_begin(DevState* st, const Settings& s, cudaStream_t stream) {
  k_iter_begin<real><<<1, 32, 0, stream>>>(st, s);
}

// ------------------------------------------------------------------------------------------------------
template <typename real>
__global__ void __launch_bounds__(256) k_vp_reduce(DevProblem P, real* vp_acc) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  // sharded: only the observations of this process's clusters (a virtual point lies in one cluster, so its
  // observations are all in or all out)
  const bool act = o < P.q && (!P.sharded || P.cluster_owned[P.cam_cluster[P.obs_cam[o]]]);
  int v = INT_MAX;
  real val[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) val[c] = 0;
  if (act) {
    v = P.obs_vp[o];
    const int cam = P.obs_cam[o];
    const int pt = P.vp_point[v];
    Cam<real> C = load_cam_w<real>(P, cam);
    real X[3];
    load_point_w(P, pt, X);
    real uo, vo;
    load_uv(P, o, uo, vo);
    real r[2], Jc[2][9], Jp[2][3];
    // FP32: the strict rows, bitwise those of the camera and pair passes
    if constexpr (sizeof(real) == 4)
      project_jacobian_strict<false>(C, X, uo, vo, Jc, Jp);
    else
      project_jacobian<real, false>(C, X, uo, vo, r, Jc, Jp);
    r[0] = res_ptr<real>(P)[2 * (size_t)o];
    r[1] = res_ptr<real>(P)[2 * (size_t)o + 1];
    real sw;   // 1 without a robust loss
    if constexpr (sizeof(real) == 4)
      sw = huber_sqrt_weight_strict(P.huber_a, r[0], r[1]);
    else
      sw = huber_sqrt_weight<real>(P.huber_a, r[0], r[1]);
    r[0] *= sw;
    r[1] *= sw;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Jp[0][c] *= sw;
      Jp[1][c] *= sw;
    }
    val[0] = Jp[0][0] * Jp[0][0] + Jp[1][0] * Jp[1][0];
    val[1] = Jp[0][0] * Jp[0][1] + Jp[1][0] * Jp[1][1];
    val[2] = Jp[0][0] * Jp[0][2] + Jp[1][0] * Jp[1][2];
    val[3] = Jp[0][1] * Jp[0][1] + Jp[1][1] * Jp[1][1];
    val[4] = Jp[0][1] * Jp[0][2] + Jp[1][1] * Jp[1][2];
    val[5] = Jp[0][2] * Jp[0][2] + Jp[1][2] * Jp[1][2];
#pragma unroll
    for (int j = 0; j < 3; ++j) val[6 + j] = -(Jp[0][j] * r[0] + Jp[1][j] * r[1]);
  }
  segmented_scan<9>(val, v, lane);
  segmented_store<9>(val, v, act, lane, o, P.vp_off, vp_acc);
}

template <typename real>
void launch_vp_reduce(const DevProblem& P, Scratch<real> W, cudaStream_t stream) {
  int blocks = (P.q + 255) / 256;
  k_vp_reduce<real><<<blocks, 256, 0, stream>>>(P, W.vp_acc);
}

// ------------------------------------------------------------------------------------------------------
template <typename real>
__device__ __forceinline__ double block_max(double v) {
  __shared__ double red[32];
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v = fmax(v, __shfl_xor_sync(FULL_MASK, v, d));
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) r = fmax(r, __shfl_xor_sync(FULL_MASK, r, d));
  }
  return r;
}

// Per point, the sums over its virtual points of V_v and w'_v: C and w of the physical point (Eq. 15).  A warp
// takes 32 consecutive points; their virtual points are one contiguous range of records, which the warp
// moves through shared memory 32 records at a time with coalesced loads, each lane adding up its own
// point's records in order (no atomics: the sums do not depend on the launch).
template <typename real>
__global__ void __launch_bounds__(256) k_pt_acc(DevProblem P, const real* __restrict__ vp_acc,
                                                real* __restrict__ pt_acc) {
  __shared__ __align__(16) real stage[8][288];
  const int lane = threadIdx.x & 31;
  real* sm = stage[threadIdx.x >> 5];
  const long long wstride = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; w * 32 < P.n; w += wstride) {
    const long long i0 = w * 32;
    const int cnt = (int)(P.n - i0 < 32 ? P.n - i0 : 32);
    const int i = (int)i0 + lane;
    const long long vb = lane < cnt ? P.pt_vp_off[i] : 0, ve = lane < cnt ? P.pt_vp_off[i + 1] : 0;
    const long long r0 = __shfl_sync(FULL_MASK, vb, 0), r1 = __shfl_sync(FULL_MASK, ve, cnt - 1);
    real acc[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) acc[c] = real(0);
    for (long long r = r0; r < r1; r += 32) {   // records [r, r + nr) of the warp's range
      const int nr = (int)(r1 - r < 32 ? r1 - r : 32);
      const real* blk = vp_acc + 9 * r;
      for (int k = lane; k < 9 * nr; k += 32) sm[k] = blk[k];
      __syncwarp();
      const long long ub = vb > r ? vb : r, ue = ve < r + nr ? ve : r + nr;
      for (long long u = ub; u < ue; ++u)
#pragma unroll
        for (int c = 0; c < 9; ++c) acc[c] += sm[9 * (u - r) + c];
      __syncwarp();
    }
    warp_store_rec9(pt_acc, i0, cnt, sm, lane, acc);
  }
}

// Warp chunks of 32 virtual points (the first ceil(nv / 32)), then of 32 points; records move through shared
// memory as whole 16-byte vectors.  Virtual point v: L_v^-1 of V'_v = V_v + lambda diag(V_v) and
// y_v = V'_v^-1 w'_v, where on a corrected step w'_v = diag(V_v) dbar_i, dbar_i = w_i / diag(C_i) (Sec. 4.3).
// Point i: C_i^-1 of C_i + lambda diag(C_i), the uncorrected w_i, and max |w| for the stop test.  C_i and w_i
// come from k_pt_acc, or from pt_sums (FP64, summed over every process's virtual points) when the iteration
// is sharded.
template <typename real>
__global__ void __launch_bounds__(256) k_vp_finalize(DevProblem P, Scratch<real> W, DevState* st,
                                                     const double* __restrict__ pt_sums,
                                                     const long long* __restrict__ counts) {
  __shared__ __align__(16) real stage[8][288];
  const real lam = (real)st->lambda_used;
  const bool corr = st->corrected != 0;
  const long long nv = counts[0];
  const int lane = threadIdx.x & 31;
  real* sm = stage[threadIdx.x >> 5];
  double gmax = 0.0;
  // C_i (6 packed) and w_i (3) of point i, read directly (corrected steps)
  auto point_sums = [&](int i, real (&a)[9]) {
    if (pt_sums) {
#pragma unroll
      for (int c = 0; c < 9; ++c) a[c] = (real)pt_sums[9 * (size_t)i + c];
    } else if (P.pt_vp_off[i] == P.pt_vp_off[i + 1]) {   // no observation
#pragma unroll
      for (int c = 0; c < 9; ++c) a[c] = real(0);
    } else {
#pragma unroll
      for (int c = 0; c < 9; ++c) a[c] = W.pt_acc[9 * (size_t)i + c];
    }
  };
  const long long nvc = (nv + 31) / 32, npc = ((long long)P.n + 31) / 32;
  const long long wstride = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long ch = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; ch < nvc + npc; ch += wstride) {
    real a[9], o[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) a[c] = o[c] = real(0);
    if (ch < nvc) {
      const long long v0 = ch * 32, v = v0 + lane;
      const int cnt = (int)(nv - v0 < 32 ? nv - v0 : 32);
      warp_load_rec9(W.vp_acc, v0, cnt, sm, lane, a);
      const bool other = pt_sums && a[0] == real(0) && a[3] == real(0) && a[5] == real(0);   // another process's
      if (lane < cnt && !other) {
        real V[6] = {a[0], a[1], a[2], a[3], a[4], a[5]}, wv[3] = {a[6], a[7], a[8]};
        if (corr) {
          real s[9];
          point_sums(P.vp_point[v], s);
          wv[0] = V[0] * (s[6] / s[0]);
          wv[1] = V[3] * (s[7] / s[3]);
          wv[2] = V[5] * (s[8] / s[5]);
        }
        V[0] += lam * V[0];
        V[3] += lam * V[3];
        V[5] += lam * V[5];
        real Li[6], y[3];
        chol3_inv(V, Li);
        chol3_apply(Li, wv, y);
#pragma unroll
        for (int c = 0; c < 6; ++c) o[c] = Li[c];
#pragma unroll
        for (int c = 0; c < 3; ++c) o[6 + c] = y[c];
      }
      warp_store_rec9(W.vp_info, v0, cnt, sm, lane, o);
    } else {
      // physical point: C + lambda diag(C), its inverse, uncorrected w
      const long long i0 = (ch - nvc) * 32;
      const int i = (int)(i0 + lane);
      const int cnt = (int)(P.n - i0 < 32 ? P.n - i0 : 32);
      if (pt_sums) {
        if (lane < cnt) point_sums(i, a);
      } else {
        warp_load_rec9(W.pt_acc, i0, cnt, sm, lane, a);
        if (lane < cnt && P.pt_vp_off[i] == P.pt_vp_off[i + 1]) {   // no observation
#pragma unroll
          for (int c = 0; c < 9; ++c) a[c] = real(0);
        }
      }
      if (lane < cnt) {
        const real Cd[6] = {a[0] * (1 + lam), a[1], a[2], a[3] * (1 + lam), a[4], a[5] * (1 + lam)};
        real Li[6];
        chol3_inv(Cd, Li);
        // C^-1 = L^-T L^-1 (symmetric packed 00 01 02 11 12 22)
        o[0] = Li[0] * Li[0] + Li[1] * Li[1] + Li[3] * Li[3];
        o[1] = Li[1] * Li[2] + Li[3] * Li[4];
        o[2] = Li[3] * Li[5];
        o[3] = Li[2] * Li[2] + Li[4] * Li[4];
        o[4] = Li[4] * Li[5];
        o[5] = Li[5] * Li[5];
        o[6] = a[6];
        o[7] = a[7];
        o[8] = a[8];
        gmax = fmax(gmax, fmax(fabs((double)a[6]), fmax(fabs((double)a[7]), fabs((double)a[8]))));
      }
      warp_store_rec9(W.pt_info, i0, cnt, sm, lane, o);
    }
  }
  double bm = block_max<real>(gmax);
  if (threadIdx.x == 0) atomicMax(&st->grad_max_bits, (unsigned long long)__double_as_longlong(bm));
}

template <typename real>
void launch_vp_finalize(const DevProblem& P, Scratch<real> W, DevState* st, const long long* counts,
                        cudaStream_t stream, const double* pt_sums) {
  // grids sized by the largest nv (q); the kernels read nv from the device counter
  const long long nmax = (long long)P.q + P.n + 31;
  const long long cap = 8LL * num_sms();
  if (!pt_sums)
    k_pt_acc<real><<<(int)std::min<long long>(((long long)P.n + 255) / 256, cap), 256, 0, stream>>>(P, W.vp_acc,
                                                                                                 W.pt_acc);
  k_vp_finalize<real><<<(int)std::min<long long>((nmax + 255) / 256, cap), 256, 0, stream>>>(P, W, st, pt_sums,
                                                                                            counts);
}

template <typename real>
__global__ void k_pt_sums(DevProblem P, const real* __restrict__ vp_acc, double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
    double s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int v = P.pt_vp_off[i]; v < P.pt_vp_off[i + 1]; ++v)
#pragma unroll
      for (int c = 0; c < 9; ++c) s[c] += (double)vp_acc[9 * (size_t)v + c];
#pragma unroll
    for (int c = 0; c < 9; ++c) out[9 * (size_t)i + c] = s[c];
  }
}

template <typename real>
void launch_pt_sums(const DevProblem& P, Scratch<real> W, double* out, cudaStream_t stream) {
  k_pt_sums<real><<<std::min((P.n + 255) / 256, 4096), 256, 0, stream>>>(P, W.vp_acc, out);
}

__global__ void k_dc_to_float(const double* __restrict__ dc, float* __restrict__ dcf, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dcf[i] = (float)dc[i];
}

void launch_dc_to_float(const double* dc, float* dcf, int64_t n, cudaStream_t stream) {
  k_dc_to_float<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, stream>>>(dc, dcf, n);
}

__global__ void k_failed_io(DevState* st, double* x, int to_double) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    if (to_double)
      *x = (double)st->failed;
    else
      st->failed = (int)(*x + 0.5);
  }
}

void launch_failed_io(DevState* st, double* x, int to_double, cudaStream_t stream) {
  k_failed_io<<<1, 32, 0, stream>>>(st, x, to_double);
}

// ------------------------------------------------------------------------------------------------------
// S' build (Eq. 10/13), in two passes.  With V' = L L^T the Cholesky factor of a virtual point's damped
// block and G_o = L^-1 Jp,o^T Jc,o (3x9) for each of its observations, E' C'^-1 E'^T = G^T G, so
//   off-diagonal camera blocks   S(a, b) = - sum_v G_a^T G_b                       (k_pair_build)
//   diagonal camera block        S(a, a) = sum_o [Jc^T Jc + lambda diag(Jc^T Jc) - G_o^T G_o]  (k_cam_pass)
//   right-hand side              b(a)    = - sum_o Jc^T (f_o + Jp,o y_v),  y_v = V'^-1 w'_v
//   camera gradient              v(a)    = - sum_o Jc^T f_o
// For a virtual point with one observation, Jc^T Jc - G^T G = Jc^T (I - Jp V'^-1 Jp^T) Jc cancels by a
// factor ~ lambda; it is evaluated in the equivalent Woodbury form Jc^T (I + Jp Lambda^-1 Jp^T)^-1 Jc with
// Lambda = lambda diag(Jp^T Jp), and without correction b(a) gets -Jc^T (I + Jp Lambda^-1 Jp^T)^-1 f_o.
//
// k_cam_pass: one warp per 32 observations of one camera (each camera's observation list is padded to
// whole warps on the host, single-observation virtual points first so that warps mostly run one branch).
// Every thread forms the 45 + 9 + 9 terms of its observation; the warp sums them in the working precision
// with a transposed reduction (62 shuffles leave lane L with the sums of terms L and 32 + L; a tree sum of
// 32 terms, error <= 5 ulp of the sum of magnitudes) and adds them atomically into the FP64 S', b' and v
// (zeroed before the launch): FP32 terms, FP64 accumulation across warps.  The per-observation arithmetic
// stays off the FP64 pipe, which on this GPU runs at 1/64 of the FP32 rate.  It also stores G_o of every
// observation of a multi-observation virtual point for the pair pass, unless the pair pass recomputes G_o.
// In FP32 both passes evaluate the Jacobian rows with every operation rounded on its own (stba_strict.cuh):
// the diagonal and off-diagonal blocks of a virtual point then come from bitwise the same J_c, J_p and G_o
// whether G_o is stored or recomputed, and the FP32 S' does not change with the compiler's choice of
// fused multiply-adds in the surrounding code.
// G_o is stored column by column, four reals per camera-parameter column c (G[0][c], G[1][c], G[2][c], 0),
// so that the pair pass reads a column with one 16-byte (FP32) load.
constexpr int GSTRIDE = 36;   // reals per stored G_o

// one stored G column from 16-byte aligned shared memory
template <typename real>
__device__ __forceinline__ void load_gcol_s(const real* p, real (&v)[3]) {
  if constexpr (sizeof(real) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
  } else {
    const double2 t = *reinterpret_cast<const double2*>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = p[2];
  }
}

template <typename real>
__device__ __forceinline__ void load_gcol(const real* p, real (&v)[3]) {
  if constexpr (sizeof(real) == 4) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
  } else {
    const double2 t = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = t.x;
    v[1] = t.y;
    v[2] = __ldg(p + 2);
  }
}

// On return lane L holds the sum over the warp's lanes of v[L].  Each halving step keeps one half of the
// values (lanes whose bit s is set keep the upper half) and adds the partner's copy of it.
template <typename real>
__device__ __forceinline__ real warp_transpose_sum32(real (&v)[32]) {
  const int lane = threadIdx.x & 31;
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
  return v[0];
}

// P = L^-1 Jp^T (3 x 2) and G = P Jc (3 x 9) of one observation, with every product and sum rounded by explicit
// fma / mul intrinsics, so that the camera pass and the pair pass form bitwise the same G from the same inputs
// (the S' of a virtual point then stays consistent between its diagonal and off-diagonal camera blocks).
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

template <typename real>
__device__ __forceinline__ void g_of_obs(const real* Li, const real (&Jc)[2][9], const real (&Jp)[2][3], real (&Pm)[3][2],
                                         real (&G)[3][9]) {
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    Pm[0][t] = mul_rn(Li[0], Jp[t][0]);
    Pm[1][t] = fma_rn(Li[2], Jp[t][1], mul_rn(Li[1], Jp[t][0]));
    Pm[2][t] = fma_rn(Li[5], Jp[t][2], fma_rn(Li[4], Jp[t][1], mul_rn(Li[3], Jp[t][0])));
  }
#pragma unroll
  for (int c = 0; c < 9; ++c)
#pragma unroll
    for (int s = 0; s < 3; ++s) G[s][c] = fma_rn(Pm[s][1], Jc[1][c], mul_rn(Pm[s][0], Jc[0][c]));
}

// J_c and J_p of the observation at sorted position o, seen by camera C, scaled by the Huber weight of the
// stored residual f_o (returned, scaled, in r).  STRICT (FP32 only): every operation rounded on its own, so
// that the camera pass and the pair pass form bitwise the same rows.
template <typename real, bool STRICT>
__device__ __forceinline__ void obs_jacobian_at(const DevProblem& P, const Cam<real>& C, int o, int pt, real uo,
                                                real vo, real (&r)[2], real (&Jc)[2][9], real (&Jp)[2][3]) {
  static_assert(!STRICT || sizeof(real) == 4, "the strict rounding mode is FP32 only");
  real X[3];
  load_point_w(P, pt, X);
  if constexpr (STRICT)
    project_jacobian_strict(C, X, uo, vo, Jc, Jp);
  else
    project_jacobian<real, true>(C, X, uo, vo, r, Jc, Jp);
  r[0] = res_ptr<real>(P)[2 * (size_t)o];
  r[1] = res_ptr<real>(P)[2 * (size_t)o + 1];
  real sw;
  if constexpr (STRICT)
    sw = huber_sqrt_weight_strict(P.huber_a, r[0], r[1]);
  else
    sw = huber_sqrt_weight<real>(P.huber_a, r[0], r[1]);
  scale_rows(sw, r, Jc, Jp);
}

template <typename real, bool STRICT>
__device__ __forceinline__ void obs_jacobian(const DevProblem& P, const Cam<real>& C, int o, real (&r)[2],
                                             real (&Jc)[2][9], real (&Jp)[2][3]) {
  real uo, vo;
  load_uv(P, o, uo, vo);
  obs_jacobian_at<real, STRICT>(P, C, o, P.obs_pt[o], uo, vo, r, Jc, Jp);
}

// STRICT (the FP32 pass): the Jacobian rows with every operation rounded on its own, as in the pair pass.
template <typename real, bool STRICT>
__global__ void __launch_bounds__(256, sizeof(real) == 4 ? 4 : 3) k_cam_pass(DevProblem P, Scratch<real> W, CamSlots CS, real* Gbuf,
                                                  const DevState* st) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= CS.nwarps) return;   // uniform per warp
  const int lane = threadIdx.x & 31;
  const int j = CS.warp_cam[gw];
  if (P.sharded && !P.cluster_owned[P.cam_cluster[j]]) return;   // another process's cluster (uniform per warp)
  const int o = CS.slots[32 * (size_t)gw + lane];
  const real lam = (real)st->lambda_used;
  const bool corr = st->corrected != 0;
  real Jc[2][9], N00 = 0, N01 = 0, N11 = 0, br[2] = {0, 0}, r[2] = {0, 0};
#pragma unroll
  for (int c = 0; c < 9; ++c) Jc[0][c] = Jc[1][c] = 0;
  if (o >= 0) {
    const Cam<real> C = load_cam_w<real>(P, j);
    // point, virtual point and observation of the slot, stored in slot order with the camera lists
    const size_t sl = 32 * (size_t)gw + lane;
    const int2 pv = CS.pv[sl];
    const int v = pv.y & INT_MAX;
    const bool single = pv.y < 0;
    real uo, vo;
    if constexpr (sizeof(real) == 4) {
      const float2 t = CS.uvf[sl];
      uo = t.x;
      vo = t.y;
    } else {
      const double2 t = CS.uvd[sl];
      uo = t.x;
      vo = t.y;
    }
    real Jp[2][3];
    obs_jacobian_at<real, STRICT>(P, C, o, pv.x, uo, vo, r, Jc, Jp);
    const real* vi = W.vp_info + 9 * (size_t)v;
    // Both cases reduce to Jc^T N Jc with a 2x2 N:
    //   single observation  N = (I + Jp Lambda^-1 Jp^T)^-1                 (Woodbury, no cancellation)
    //   several             N = I - Jp V'^-1 Jp^T = I - P^T P, P = L^-1 Jp^T  (V' = L L^T)
    if (single) {
      real il[3];
#pragma unroll
      for (int s = 0; s < 3; ++s) il[s] = real(1) / (lam * (Jp[0][s] * Jp[0][s] + Jp[1][s] * Jp[1][s]));
      real K00 = 0, K01 = 0, K11 = 0;
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        K00 += Jp[0][s] * Jp[0][s] * il[s];
        K01 += Jp[0][s] * Jp[1][s] * il[s];
        K11 += Jp[1][s] * Jp[1][s] * il[s];
      }
      const real idet = real(1) / ((real(1) + K00) * (real(1) + K11) - K01 * K01);
      N00 = (real(1) + K11) * idet;
      N01 = -K01 * idet;
      N11 = (real(1) + K00) * idet;
      if (corr) {
        br[0] = r[0] + Jp[0][0] * vi[6] + Jp[0][1] * vi[7] + Jp[0][2] * vi[8];
        br[1] = r[1] + Jp[1][0] * vi[6] + Jp[1][1] * vi[7] + Jp[1][2] * vi[8];
      } else {
        br[0] = N00 * r[0] + N01 * r[1];
        br[1] = N01 * r[0] + N11 * r[1];
      }
    } else {
      real Pm[3][2], Gm[3][9];   // P = L^-1 Jp^T (3x2), G = P Jc
      g_of_obs<real>(vi, Jc, Jp, Pm, Gm);
      N00 = real(1) - (Pm[0][0] * Pm[0][0] + Pm[1][0] * Pm[1][0] + Pm[2][0] * Pm[2][0]);
      N01 = -(Pm[0][0] * Pm[0][1] + Pm[1][0] * Pm[1][1] + Pm[2][0] * Pm[2][1]);
      N11 = real(1) - (Pm[0][1] * Pm[0][1] + Pm[1][1] * Pm[1][1] + Pm[2][1] * Pm[2][1]);
      // G = L^-1 Jp^T Jc = P Jc (3x9), stored by columns with 16-byte vector stores (unless the pair pass
      // recomputes it)
      real* Gs = Gbuf + (size_t)GSTRIDE * P.obs_base[o];   // indexed like the camera graph's pairs
#pragma unroll
      for (int c = 0; c < 9 && !P.pair_recompute; ++c) {
        const real g0 = Gm[0][c], g1 = Gm[1][c], g2 = Gm[2][c];
        if constexpr (sizeof(real) == 4) {
          reinterpret_cast<float4*>(Gs)[c] = make_float4(g0, g1, g2, 0.f);
        } else {
          reinterpret_cast<double2*>(Gs)[2 * c] = make_double2(g0, g1);
          reinterpret_cast<double2*>(Gs)[2 * c + 1] = make_double2(g2, 0.0);
        }
      }
      br[0] = r[0] + Jp[0][0] * vi[6] + Jp[0][1] * vi[7] + Jp[0][2] * vi[8];
      br[1] = r[1] + Jp[1][0] * vi[6] + Jp[1][1] * vi[7] + Jp[1][2] * vi[8];
    }
  }
  // terms: 0..44 diagonal block (packed lower, row-major), 45..53 b', 54..62 v, 63 unused
  real NJ[2][9];
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    NJ[0][c] = N00 * Jc[0][c] + N01 * Jc[1][c];
    NJ[1][c] = N01 * Jc[0][c] + N11 * Jc[1][c];
  }
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
          real d = Jc[0][i] * NJ[0][jj] + Jc[1][i] * NJ[1][jj];
          if (i == jj) d += lam * (Jc[0][i] * Jc[0][i] + Jc[1][i] * Jc[1][i]);
          v[t - 32 * half] = d;
        }
      }
    if (half == 1) {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        v[45 - 32 + i] = -(Jc[0][i] * br[0] + Jc[1][i] * br[1]);
        v[54 - 32 + i] = -(Jc[0][i] * r[0] + Jc[1][i] * r[1]);
      }
      v[31] = real(0);
    }
    sums[half] = warp_transpose_sum32(v);
  }
  const int k = P.cam_cluster[j], lc = P.cam_local[j];
  const int np = P.cluster_np[k];
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int e = lane + 32 * half;
    const double x = (double)sums[half];
    if (e < 45) {
      int row = 0;
      while ((row + 1) * (row + 2) / 2 <= e) ++row;
      const int col = e - row * (row + 1) / 2;
      atomicAdd(W.S + P.S_off[k] + (size_t)(9 * lc + row) * np + 9 * lc + col, x);
    } else if (e < 54) {
      atomicAdd(W.b + P.v_off[k] + 9 * lc + (e - 45), x);
    } else if (e < 63) {
      atomicAdd(W.vgrad + 9 * (size_t)j + (e - 54), sums[half]);
    }
  }
}

// k_pair_build: the off-diagonal blocks S'_k(la, lb) = -sum over the points seen by both cameras x > y of
// one cluster of G_x^T G_y (Eq. 10, 13).  The observation pairs of the camera graph are listed once, at
// create, by edge (x, y) and cut into chunks of at most PAIR_CHUNK; under a cluster assignment an edge
// contributes exactly when both cameras are in one cluster (its two observations of a point are then in
// one virtual point), and a chunk adds to one block only.  The re-ordering of an assignment lists the
// chunks whose edge lies inside a cluster; a fixed grid of warps walks that list.  A warp's work is a
// sequence of pieces of CH pairs (the chunks it takes, cut into pieces); the G rows of the next piece are
// copied into shared memory (cp.async, one row per lane) while 27 lanes accumulate the current one: lane
// (g, rb, cb) takes every third pair (slot g) and the 3 x 3 sub-block (rb, cb) of the 9 x 9 block, in
// registers; the three slots are summed by two shuffles and the block is added once per chunk into the
// FP64 S'_k.
constexpr int PB_WARPS = 8;

template <typename real> struct PairStage {
  static constexpr int CH = 64 / (int)sizeof(real);                   // pairs per piece
  static constexpr int PIECES = 2;                                      // double buffer
  static constexpr size_t bytes = sizeof(real) * (size_t)PB_WARPS * PIECES * CH * 2 * GSTRIDE;
};

__device__ __forceinline__ void cp_async_16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// G_o = L_v^-1 Jp,o^T Jc,o (3 x 9) of the observation at sorted position pos by camera cam, written by columns
// (G[0][c], G[1][c], G[2][c], 0) to dst: the camera pass's arithmetic (Jacobians at the current x, Huber
// weights from the stored residual, L_v^-1 of the virtual point's damped block); STRICT as in the camera pass.
template <typename real, bool STRICT>
__device__ __forceinline__ void obs_G(const DevProblem& P, const Scratch<real>& W, int cam, int pos, real* dst) {
  const Cam<real> C = load_cam_w<real>(P, cam);
  real r[2], Jc[2][9], Jp[2][3];
  obs_jacobian<real, STRICT>(P, C, pos, r, Jc, Jp);
  real Pm[3][2], Gm[3][9];
  g_of_obs<real>(W.vp_info + 9 * (size_t)P.obs_vp[pos], Jc, Jp, Pm, Gm);
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    const real g0 = Gm[0][c], g1 = Gm[1][c], g2 = Gm[2][c];
    if constexpr (sizeof(real) == 4) {
      reinterpret_cast<float4*>(dst)[c] = make_float4(g0, g1, g2, 0.f);
    } else {
      reinterpret_cast<double2*>(dst)[2 * c] = make_double2(g0, g1);
      reinterpret_cast<double2*>(dst)[2 * c + 1] = make_double2(g2, 0.0);
    }
  }
}

template <typename real, bool RECOMPUTE>
__global__ void __launch_bounds__(32 * PB_WARPS) k_pair_build(DevProblem P, Scratch<real> W, PairChunks B,
                                                              const real* __restrict__ Gbuf) {
  constexpr int CH = PairStage<real>::CH;
  constexpr int ROWQ = GSTRIDE * (int)sizeof(real) / 16;   // 16-byte pieces of one G row
  extern __shared__ __align__(16) unsigned char pb_smem[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  real* stage = reinterpret_cast<real*>(pb_smem) + (size_t)wib * 2 * CH * 2 * GSTRIDE;   // [2][CH][2][GSTRIDE]
  const long long nactive = *B.nactive;
  const long long wstride = ((long long)gridDim.x * blockDim.x) >> 5;
  long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (w >= nactive) return;   // uniform per warp
  // lanes 0..26: pair slot g = lane / 9 of every three, and the 3 x 3 sub-block (rb, cb) of the 9 x 9 block
  const int g = lane / 9, sub = lane - 9 * (lane / 9), rb = sub / 3, cb = sub - 3 * (sub / 3);
  const bool act = lane < 27;
  const int j = lane % CH, side = lane / CH;
  // the piece (chunk record, first pair) being copied and the one being accumulated
  int4 ch = B.chunks[B.active[w]];
  int c0 = 0;
  auto issue = [&](const int4& chunk, int first, int buf) {
    const int cn = min(CH, chunk.w - first);
    if (side < 2 && j < cn) {
      const int2 pr = B.pairs[chunk.z + first + j];
      real* dst = stage + ((size_t)(buf * CH + j) * 2 + side) * GSTRIDE;
      if constexpr (RECOMPUTE) {   // computed here: no G buffer, about 90 bytes read per pair instead of 288
        const int b = side ? pr.y : pr.x;
        obs_G<real, sizeof(real) == 4>(P, W, side ? chunk.y : chunk.x, P.base_pos[b], dst);
      } else {
        const real* src = Gbuf + (size_t)GSTRIDE * (side ? pr.y : pr.x);
#pragma unroll
        for (int q = 0; q < ROWQ; ++q)
          cp_async_16(dst + q * (16 / (int)sizeof(real)), src + q * (16 / (int)sizeof(real)));
      }
    }
    cp_async_commit();
  };
  issue(ch, 0, 0);
  int buf = 0;
  real acc[3][3];
#pragma unroll
  for (int x = 0; x < 3; ++x) acc[x][0] = acc[x][1] = acc[x][2] = real(0);
  for (;;) {
    // the next piece: the rest of this chunk, else the warp's next chunk
    int4 nch = ch;
    int n0 = c0 + CH;
    bool more = true;
    if (n0 >= ch.w) {
      const long long nw = w + wstride;
      if (nw < nactive) {
        nch = B.chunks[B.active[nw]];
        n0 = 0;
      } else {
        more = false;
      }
    }
    if (more) {
      issue(nch, n0, buf ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    if (act) {
      const int cn = min(CH, ch.w - c0);
      const real* base = stage + (size_t)buf * CH * 2 * GSTRIDE;
      for (int jj = g; jj < cn; jj += 3) {   // pair slot g of every three
        const real* ga = base + (size_t)jj * 2 * GSTRIDE;
        const real* gb = ga + GSTRIDE;
        real a[3][3], b[3][3];
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          load_gcol_s(ga + 4 * (3 * rb + x), a[x]);
          load_gcol_s(gb + 4 * (3 * cb + x), b[x]);
        }
#pragma unroll
        for (int x = 0; x < 3; ++x)
#pragma unroll
          for (int y = 0; y < 3; ++y) acc[x][y] += a[x][0] * b[y][0] + a[x][1] * b[y][1] + a[x][2] * b[y][2];
      }
    }
    __syncwarp();   // every lane is done with this buffer before it is refilled
    if (c0 + CH >= ch.w) {   // the chunk is complete: sum the three pair slots, one add per block entry
#pragma unroll
      for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int y = 0; y < 3; ++y) {
          // lane L < 9 adds slots 1 and 2 from lanes L + 9 and L + 18 (source lanes wrap mod 32 for the rest)
          const real v = acc[x][y];
          acc[x][y] = v + __shfl_sync(FULL_MASK, v, lane + 9) + __shfl_sync(FULL_MASK, v, lane + 18);
        }
      if (lane < 9) {
        const int k = P.cam_cluster[ch.x];
        const int la = P.cam_local[ch.x], lb = P.cam_local[ch.y];   // la > lb: local order follows camera order
        const int np = P.cluster_np[k];
        double* dst = W.S + P.S_off[k] + (size_t)(9 * la + 3 * rb) * np + 9 * lb + 3 * cb;
#pragma unroll
        for (int x = 0; x < 3; ++x)
#pragma unroll
          for (int y = 0; y < 3; ++y) atomicAdd(dst + (size_t)x * np + y, -(double)acc[x][y]);
      }
#pragma unroll
      for (int x = 0; x < 3; ++x) acc[x][0] = acc[x][1] = acc[x][2] = real(0);
      if (!more) break;
      w += wstride;
    }
    ch = nch;
    c0 = n0;
    buf ^= 1;
  }
}

template <typename real>
void launch_rcs_build(const DevProblem& P, Scratch<real> W, CamSlots CS, PairChunks B, real* Gbuf, DevState* st,
                      cudaStream_t stream, cudaStream_t side, cudaEvent_t fork, cudaEvent_t join) {
  const bool pairs = B.nchunks > 0 && P.l < P.m;
  // a pair pass that recomputes G_o depends on nothing the camera pass writes (they add to different
  // blocks of S'), so with a second stream the two run side by side
  const bool beside = pairs && P.pair_recompute && side != nullptr;
  if (beside) {
    cudaEventRecord(fork, stream);
    cudaStreamWaitEvent(side, fork, 0);
  }
  cudaStream_t ps = beside ? side : stream;
  // FP32: both passes take the strict Jacobian rows, so that stored and recomputed G_o are bitwise equal
  k_cam_pass<real, sizeof(real) == 4><<<(CS.nwarps + 7) / 8, 256, 0, stream>>>(P, W, CS, Gbuf, st);
  if (pairs) {   // a fixed grid walks the list of chunks inside clusters
    const int grid = std::min((B.nchunks + PB_WARPS - 1) / PB_WARPS, 3 * num_sms());
    if (P.pair_recompute)
      k_pair_build<real, true><<<grid, 32 * PB_WARPS, PairStage<real>::bytes, ps>>>(P, W, B, Gbuf);
    else
      k_pair_build<real, false><<<grid, 32 * PB_WARPS, PairStage<real>::bytes, ps>>>(P, W, B, Gbuf);
  }
  if (beside) {
    cudaEventRecord(join, side);
    cudaStreamWaitEvent(stream, join, 0);
  }
}

// ------------------------------------------------------------------------------------------------------
template <typename real>
__global__ void __launch_bounds__(256) k_point_rhs(DevProblem P, const double* dc, const float* dcf, real* t_acc) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool act = o < P.q;
  int pt = INT_MAX;
  real val[3] = {0, 0, 0};
  if (act) {
    pt = P.obs_pt[o];
    const int cam = P.obs_cam[o];
    Cam<real> C = load_cam_w<real>(P, cam);
    real X[3];
    load_point_w(P, pt, X);
    real uo, vo;
    load_uv(P, o, uo, vo);
    real r[2], Jc[2][9], Jp[2][3];
    project_jacobian<real, true>(C, X, uo, vo, r, Jc, Jp);
    real jd0 = 0, jd1 = 0;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      const real dcc = (sizeof(real) == 4) ? (real)dcf[9 * (size_t)cam + c] : (real)dc[9 * (size_t)cam + c];
      jd0 += Jc[0][c] * dcc;
      jd1 += Jc[1][c] * dcc;
    }
    // with a robust loss both Jacobians carry sqrt(rho'): the product carries rho'
    real wgt = real(1);
    if (P.huber_a > 0.0) {
      const real sw = huber_sqrt_weight<real>(P.huber_a, res_ptr<real>(P)[2 * (size_t)o], res_ptr<real>(P)[2 * (size_t)o + 1]);
      wgt = sw * sw;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) val[j] = wgt * (Jp[0][j] * jd0 + Jp[1][j] * jd1);
  }
  segmented_scan<3>(val, pt, lane);
  segmented_store<3>(val, pt, act, lane, o, P.pt_off, t_acc);
}

// dp = C^-1 (w - t) per point; the same grid also forms the partial sums of the stop tests: |dp|^2, |p|^2,
// |dc|^2, |c|^2 and max |v| (camera gradient), one partial per block at partial[RED_BLOCKS * (1..5) + block].
template <typename real>
__global__ void __launch_bounds__(256) k_point_update(DevProblem P, const real* pt_info, const real* t_acc,
                                                      const double* dc, const real* vgrad, double* dp,
                                                      double* partial) {
  double s_dp = 0.0, s_p = 0.0, s_dc = 0.0, s_c = 0.0;
  real gmax = real(0);   // max |v| in the working precision (exact)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
    const real* in = pt_info + 9 * (size_t)i;
    const real* t = t_acc + 3 * (size_t)i;
    real g0 = in[6] - t[0], g1 = in[7] - t[1], g2 = in[8] - t[2];
    real d0 = in[0] * g0 + in[1] * g1 + in[2] * g2;
    real d1 = in[1] * g0 + in[3] * g1 + in[4] * g2;
    real d2 = in[2] * g0 + in[4] * g1 + in[5] * g2;
    double* out = dp + 3 * (size_t)i;
    out[0] = d0;
    out[1] = d1;
    out[2] = d2;
    s_dp += (double)d0 * d0 + (double)d1 * d1 + (double)d2 * d2;
    const double* p = P.pts + 3 * (size_t)i;
    s_p += p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 9 * P.m; i += gridDim.x * blockDim.x) {
    const double d = dc[i], c = P.cams[i];
    s_dc += d * d;
    s_c += c * c;
    gmax = fmax(gmax, fabs(vgrad[i]));
  }
  __shared__ double red[4][8];
  __shared__ real redm[8];
  for (int d = 16; d > 0; d >>= 1) {
    s_dp += __shfl_xor_sync(FULL_MASK, s_dp, d);
    s_p += __shfl_xor_sync(FULL_MASK, s_p, d);
    s_dc += __shfl_xor_sync(FULL_MASK, s_dc, d);
    s_c += __shfl_xor_sync(FULL_MASK, s_c, d);
    gmax = fmax(gmax, __shfl_xor_sync(FULL_MASK, gmax, d));
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[0][w] = s_dp;
    red[1][w] = s_p;
    red[2][w] = s_dc;
    red[3][w] = s_c;
    redm[w] = gmax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a[4] = {0, 0, 0, 0};
    real mx = real(0);
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      for (int c = 0; c < 4; ++c) a[c] += red[c][i];
      mx = fmax(mx, redm[i]);
    }
    for (int c = 0; c < 4; ++c) partial[(1 + c) * RED_BLOCKS + blockIdx.x] = a[c];
    partial[5 * RED_BLOCKS + blockIdx.x] = (double)mx;
  }
}

// ------------------------------------------------------------------------------------------------------
// Residuals in FP64 (both precisions): the cost F(x + dx) and the accept test need them to FP64 accuracy,
// and the stored residuals drive the next linearisation (FP32 projections of pixel coordinates of a few
// hundred px carry ~3e-5 px of rounding, which the conditioning of S' amplifies in the step).
// k_cam_rt precomputes per camera R(w + dw) (Rodrigues in FP64), t + dt and the intrinsics.
__global__ void k_cam_rt(int m, const double* cams, const double* dc, double* rt) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    double c[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) c[i] = cams[9 * (size_t)j + i] + (dc ? dc[9 * (size_t)j + i] : 0.0);
    const double s = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    double a, b, da, db;
    rodrigues_coeffs(s, a, b, da, db);
    const double* w = c;
    double* o = rt + 15 * (size_t)j;
    o[0] = 1.0 + b * (w[0] * w[0] - s);
    o[1] = -a * w[2] + b * w[0] * w[1];
    o[2] = a * w[1] + b * w[0] * w[2];
    o[3] = a * w[2] + b * w[0] * w[1];
    o[4] = 1.0 + b * (w[1] * w[1] - s);
    o[5] = -a * w[0] + b * w[1] * w[2];
    o[6] = -a * w[1] + b * w[0] * w[2];
    o[7] = a * w[0] + b * w[1] * w[2];
    o[8] = 1.0 + b * (w[2] * w[2] - s);
#pragma unroll
    for (int i = 0; i < 6; ++i) o[9 + i] = c[3 + i];
  }
}

// F = sum |f_o|^2 at the parameters described by rt and pts (+ dp); writes f_o to rout (working precision).
template <typename real>
__global__ void __launch_bounds__(RED_THREADS) k_cost(DevProblem P, const double* rt, const double* dp,
                                                      double* partial, DevState* st, real* rout) {
  double s = 0.0;
  int bad = 0;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < P.q; o += gridDim.x * blockDim.x) {
    const int cam = P.obs_cam[o];
    const int pt = P.obs_pt[o];
    const double* C = rt + 15 * (size_t)cam;
    const double* p = P.pts + 3 * (size_t)pt;
    double X0 = p[0], X1 = p[1], X2 = p[2];
    if (dp) {
      const double* q = dp + 3 * (size_t)pt;
      X0 += q[0];
      X1 += q[1];
      X2 += q[2];
    }
    const double xc = C[0] * X0 + C[1] * X1 + C[2] * X2 + C[9];
    const double yc = C[3] * X0 + C[4] * X1 + C[5] * X2 + C[10];
    const double zc = C[6] * X0 + C[7] * X1 + C[8] * X2 + C[11];
    const double iz = 1.0 / zc;
    const double x = xc * iz, y = yc * iz;
    const double r2 = x * x + y * y;
    const double fd = C[12] * (1.0 + r2 * (C[13] + C[14] * r2));
    const double2 uv = reinterpret_cast<const double2*>(P.obs_uv)[o];
    const double r0 = fd * x - uv.x, r1 = fd * y - uv.y;
    if (!(zc > 1e-9)) bad = 1;
    s += huber_rho(P.huber_a, r0 * r0 + r1 * r1);   // rho(s) = s without a robust loss
    rout[2 * (size_t)o] = (real)r0;
    rout[2 * (size_t)o + 1] = (real)r1;
  }
  __shared__ double red[RED_THREADS / 32];
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(FULL_MASK, s, d);
  bad = __any_sync(FULL_MASK, bad);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = s;
  if (lane == 0 && bad) st->nonfinite = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0;
    for (int i = 0; i < RED_THREADS / 32; ++i) a += red[i];
    partial[blockIdx.x] = a;
  }
}

// ------------------------------------------------------------------------------------------------------
// Cost of the candidate step in mixed mode, in double-float arithmetic (a value is an unevaluated sum
// hi + lo of two floats, ~48-bit significand; Dekker's and Knuth's error-free transformations, with the
// product error taken by an FMA).  The FP64 pipe of this GPU runs at 1/64 of the FP32 rate; double-float
// keeps the residuals accurate to ~1e-12 px at pixel offsets of a few hundred px on the FP32 pipe.
// Per camera the FP64 table of k_cam_rt is split into double-float (R, t, f; k1 and k2 as floats, since
// they scale the small distortion term only); per point the candidate p + dp is split in k_point_df.
__device__ __forceinline__ float2 df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return make_float2(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ float2 df_fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = a + b;
  return make_float2(s, b - (s - a));
}
__device__ __forceinline__ float2 df_add(float2 x, float2 y) {
  const float2 s = df_two_sum(x.x, y.x);
  return df_fast_two_sum(s.x, s.y + (x.y + y.y));
}
__device__ __forceinline__ float2 df_sub(float2 x, float2 y) { return df_add(x, make_float2(-y.x, -y.y)); }
__device__ __forceinline__ float2 df_mul(float2 x, float2 y) {
  const float p = x.x * y.x;
  const float e = fmaf(x.x, y.y, fmaf(x.y, y.x, fmaf(x.x, y.x, -p)));
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ float2 df_rcp(float2 y) {   // one Newton correction of the FP32 reciprocal
  const float q = __frcp_rn(y.x);
  const float2 r = df_sub(make_float2(1.f, 0.f), df_mul(make_float2(q, 0.f), y));
  return df_fast_two_sum(q, r.x * q);
}
__device__ __forceinline__ float2 df_split(double d) {
  const float hi = __double2float_rn(d);
  return make_float2(hi, __double2float_rn(d - (double)hi));
}

constexpr int CAM_DF = 28;   // floats per camera: R (9 x 2), t (3 x 2), f (2), k1, k2

__global__ void k_cam_df(int m, const double* __restrict__ rt, float* __restrict__ cdf) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    const double* c = rt + 15 * (size_t)j;
    float* o = cdf + CAM_DF * (size_t)j;
#pragma unroll
    for (int i = 0; i < 13; ++i) {
      const float2 v = df_split(c[i]);
      o[2 * i] = v.x;
      o[2 * i + 1] = v.y;
    }
    o[26] = (float)c[13];
    o[27] = (float)c[14];
  }
}

__global__ void k_point_df(int n, const double* __restrict__ pts, const double* __restrict__ dp,
                           float* __restrict__ pdf) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n; i += gridDim.x * blockDim.x) {
    const float2 v = df_split(dp ? pts[i] + dp[i] : pts[i]);
    reinterpret_cast<float2*>(pdf)[i] = v;
  }
}

__global__ void __launch_bounds__(RED_THREADS) k_cost_df(DevProblem P, const float* __restrict__ cdf,
                                                         const float* __restrict__ pdf, double* partial,
                                                         DevState* st, float* rout) {
  float2 acc = make_float2(0.f, 0.f);
  double acc_rho = 0.0;
  int bad = 0;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < P.q; o += gridDim.x * blockDim.x) {
    const float4* C4 = reinterpret_cast<const float4*>(cdf + CAM_DF * (size_t)P.obs_cam[o]);
    float cv[CAM_DF];
#pragma unroll
    for (int q4 = 0; q4 < CAM_DF / 4; ++q4) {
      const float4 t4 = __ldg(C4 + q4);
      cv[4 * q4] = t4.x;
      cv[4 * q4 + 1] = t4.y;
      cv[4 * q4 + 2] = t4.z;
      cv[4 * q4 + 3] = t4.w;
    }
    const float2* X2 = reinterpret_cast<const float2*>(pdf) + 3 * (size_t)P.obs_pt[o];
    const float2 X[3] = {X2[0], X2[1], X2[2]};
    float2 Xc[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float2 a = df_mul(make_float2(cv[6 * r], cv[6 * r + 1]), X[0]);
      const float2 b = df_mul(make_float2(cv[6 * r + 2], cv[6 * r + 3]), X[1]);
      const float2 c = df_mul(make_float2(cv[6 * r + 4], cv[6 * r + 5]), X[2]);
      Xc[r] = df_add(df_add(a, b), df_add(c, make_float2(cv[18 + 2 * r], cv[19 + 2 * r])));
    }
    if (!(Xc[2].x > 1e-9f)) bad = 1;
    const float2 iz = df_rcp(Xc[2]);
    const float2 x = df_mul(Xc[0], iz), y = df_mul(Xc[1], iz);
    const float r2 = x.x * x.x + y.x * y.x;
    const float2 d = df_fast_two_sum(1.f, r2 * (cv[26] + cv[27] * r2));
    const float2 fd = df_mul(make_float2(cv[24], cv[25]), d);
    const float4 uv = P.obs_uvdf[o];
    const float2 r0 = df_sub(df_mul(fd, x), make_float2(uv.x, uv.y));
    const float2 r1 = df_sub(df_mul(fd, y), make_float2(uv.z, uv.w));
    const float2 sq = df_add(df_mul(r0, r0), df_mul(r1, r1));
    if (P.huber_a > 0.0)   // robust loss: rho of the FP64 value of the double-float square
      acc_rho += huber_rho(P.huber_a, (double)sq.x + (double)sq.y);
    else
      acc = df_add(acc, sq);
    rout[2 * (size_t)o] = r0.x + r0.y;
    rout[2 * (size_t)o + 1] = r1.x + r1.y;
  }
  double s = (double)acc.x + (double)acc.y + acc_rho;
  __shared__ double red[RED_THREADS / 32];
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(FULL_MASK, s, d);
  bad = __any_sync(FULL_MASK, bad);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = s;
  if (lane == 0 && bad) st->nonfinite = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0;
    for (int i = 0; i < RED_THREADS / 32; ++i) a += red[i];
    partial[blockIdx.x] = a;
  }
}

// ------------------------------------------------------------------------------------------------------
// Stop tests and accept / reject (Algorithm 1), one block; fixed-order sums of the partials.
template <typename real>
__global__ void __launch_bounds__(1024) k_finalize(DevProblem P, const real* vgrad, const double* dc,
                                                   const double* partial, DevState* st, Settings s,
                                                   int with_step) {
  __shared__ double red[4][32];
  double F_new = 0, dpn = 0, pn = 0, dcn = 0, cn = 0, gmax = 0;
  for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) {
    F_new += partial[i];
    if (with_step) {
      dpn += partial[RED_BLOCKS + i];
      pn += partial[2 * RED_BLOCKS + i];
      dcn += partial[3 * RED_BLOCKS + i];
      cn += partial[4 * RED_BLOCKS + i];
      gmax = fmax(gmax, partial[5 * RED_BLOCKS + i]);
    }
  }
  double vals[4] = {F_new, dpn + dcn, pn + cn, gmax};
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < 3; ++c)
    for (int d = 16; d > 0; d >>= 1) vals[c] += __shfl_xor_sync(FULL_MASK, vals[c], d);
  for (int d = 16; d > 0; d >>= 1) vals[3] = fmax(vals[3], __shfl_xor_sync(FULL_MASK, vals[3], d));
  if (lane == 0)
    for (int c = 0; c < 4; ++c) red[c][w] = vals[c];
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot[4] = {0, 0, 0, 0};
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      tot[0] += red[0][i];
      tot[1] += red[1][i];
      tot[2] += red[2][i];
      tot[3] = fmax(tot[3], red[3][i]);
    }
    if (!with_step) {
      st->F = tot[0];
      st->info.F_before = tot[0];
      return;
    }
    double Fn = tot[0];
    const double F = st->F;
    const double lam = st->lambda_used;
    if (st->failed > 0 || st->nonfinite || !isfinite(Fn)) Fn = __longlong_as_double(0x7ff0000000000000ll);
    const double grad = fmax(tot[3], __longlong_as_double((long long)st->grad_max_bits));
    const double dxn = sqrt(tot[1]), xn = sqrt(tot[2]);
    int stop = 0;
    if (s.ftol > 0 && F > 0 && fabs(F - Fn) / F < s.ftol) stop = 1;
    if (s.gtol > 0 && grad < s.gtol) stop = 1;
    if (s.xtol > 0 && dxn < s.xtol * (xn + s.xtol)) stop = 1;
    const int accepted = (Fn < F) ? 1 : 0;
    const double lam_new = accepted ? fmax(lam / 3.0, s.lambda_min) : lam * 3.0;
    st->lambda = lam_new;
    if (accepted) st->F = Fn;
    st->iteration += 1;
    stba_iter_info& I = st->info;
    I.F_before = F;
    I.F_after = Fn;
    I.lambda_used = lam;
    I.lambda = lam_new;
    I.grad_inf = grad;
    I.dx_norm = dxn;
    I.x_norm = xn;
    I.accepted = accepted;
    I.stop = stop;
    I.corrected = st->corrected;
    I.failed_clusters = st->failed;
    I.boosted_pivots = st->boosted;
    I.linear_iterations = 0;
    I.iteration = st->iteration;
  }
}

template <typename real>
__global__ void k_apply(int m, int n, int q, const double* dc, const double* dp, double* cams, double* pts,
                        const real* r_cand, real* r_cur, const DevState* st) {
  if (!st->info.accepted) return;
  const int total = 9 * m + 3 * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    if (i < 9 * m)
      cams[i] += dc[i];
    else
      pts[i - 9 * m] += dp[i - 9 * m];
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * q; i += gridDim.x * blockDim.x) r_cur[i] = r_cand[i];
}

// ------------------------------------------------------------------------------------------------------
// launchers
template <typename real>
void launch_point_update(const DevProblem& P, Scratch<real> W, cudaStream_t stream) {
  k_point_update<real><<<RED_BLOCKS, RED_THREADS, 0, stream>>>(P, W.pt_info, W.t_acc, W.dc, W.vgrad, W.dp,
                                                               W.partial);
}

template <typename real>
void launch_finalize(const DevProblem& P, Scratch<real> W, DevState* st, const Settings& s, int with_step,
                     cudaStream_t stream) {
  k_finalize<real><<<1, 1024, 0, stream>>>(P, W.vgrad, W.dc, W.partial, st, s, with_step);
}

template <typename real>
void launch_apply(const DevProblem& P, const double* dc, const double* dp, double* cams, double* pts,
                  const real* r_cand, real* r_cur, DevState* st, cudaStream_t stream) {
  int total = std::max(9 * P.m + 3 * P.n, 2 * P.q);
  int blocks = (total + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  k_apply<real><<<blocks, 256, 0, stream>>>(P.m, P.n, P.q, dc, dp, cams, pts, r_cand, r_cur, st);
}

template <typename real>
void launch_point_rhs(const DevProblem& P, Scratch<real> W, cudaStream_t stream) {
  int blocks = (P.q + 255) / 256;
  k_point_rhs<real><<<blocks, 256, 0, stream>>>(P, W.dc, W.dcf, W.t_acc);
}

template <typename real>
void launch_cost(const DevProblem& P, const double* dc, const double* dp, double* rt, float* cam_df, float* pt_df,
                 double* partial, DevState* st, real* rout, cudaStream_t stream) {
  k_cam_rt<<<(P.m + 127) / 128, 128, 0, stream>>>(P.m, P.cams, dc, rt);
  // FP32 working precision: always the double-float kernels (cam_df, pt_df and the double-float observations
  // are required; the FP64 observations are not kept in that mode); dc, dp null: F(x) itself
  if constexpr (sizeof(real) == 4) {
    k_cam_df<<<(P.m + 127) / 128, 128, 0, stream>>>(P.m, rt, cam_df);
    k_point_df<<<std::min((3 * P.n + 255) / 256, 2048), 256, 0, stream>>>(P.n, P.pts, dp, pt_df);
    k_cost_df<<<RED_BLOCKS, RED_THREADS, 0, stream>>>(P, cam_df, pt_df, partial, st, (float*)rout);
  } else {
    k_cost<real><<<RED_BLOCKS, RED_THREADS, 0, stream>>>(P, rt, dp, partial, st, rout);
  }
}


__global__ void k_params_to_float(int m, int n, const double* __restrict__ cams, const double* __restrict__ pts,
                                  float* __restrict__ cams_f, float* __restrict__ pts_f) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 9 * m + 3 * n; i += gridDim.x * blockDim.x) {
    if (i < 9 * m)
      cams_f[i] = (float)cams[i];
    else
      pts_f[i - 9 * m] = (float)pts[i - 9 * m];
  }
}

void launch_params_to_float(const DevProblem& P, float* cams_f, float* pts_f, cudaStream_t stream) {
  const int total = 9 * P.m + 3 * P.n;
  k_params_to_float<<<std::min((total + 255) / 256, 2048), 256, 0, stream>>>(P.m, P.n, P.cams, P.pts, cams_f, pts_f);
}

void configure_kernels(int max_np) {
  configure_solve_kernels(max_np);
  cudaFuncSetAttribute(k_pair_build<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)PairStage<float>::bytes);
  cudaFuncSetAttribute(k_pair_build<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)PairStage<float>::bytes);
  cudaFuncSetAttribute(k_pair_build<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)PairStage<double>::bytes);
  cudaFuncSetAttribute(k_pair_build<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)PairStage<double>::bytes);
}

#define INSTANTIATE(real)                                                                                  \
  template void launch_iter_begin<real>(DevState*, const Settings&, cudaStream_t);                        \
  template void launch_vp_reduce<real>(const DevProblem&, Scratch<real>, cudaStream_t);                   \
  template void launch_vp_finalize<real>(const DevProblem&, Scratch<real>, DevState*, const long long*,   \
                                         cudaStream_t, const double*);                                     \
  template void launch_pt_sums<real>(const DevProblem&, Scratch<real>, double*, cudaStream_t);              \
  template void launch_rcs_build<real>(const DevProblem&, Scratch<real>, CamSlots, PairChunks, real*,     \
                                       DevState*, cudaStream_t, cudaStream_t, cudaEvent_t, cudaEvent_t);  \
  template void launch_point_update<real>(const DevProblem&, Scratch<real>, cudaStream_t);                \
  template void launch_finalize<real>(const DevProblem&, Scratch<real>, DevState*, const Settings&, int,  \
                                      cudaStream_t);                                                      \
  template void launch_point_rhs<real>(const DevProblem&, Scratch<real>, cudaStream_t);                  \
  template void launch_cost<real>(const DevProblem&, const double*, const double*, double*, float*, float*, \
                                  double*, DevState*, real*, cudaStream_t);                               \
  template void launch_apply<real>(const DevProblem&, const double*, const double*, double*, double*,     \
                                   const real*, real*, DevState*, cudaStream_t);                          \


INSTANTIATE(float)
INSTANTIATE(double)

}  // namespace stba
