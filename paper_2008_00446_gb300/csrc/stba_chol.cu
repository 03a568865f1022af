// Batched dense LL^T factorisation and solve of the per-cluster systems S'_k dc_k = b_k (Eq. 13; the
// paper solves them with dense LL^T, Sec. 5.1), for clusters of uneven size, one launch per step.
//
// Storage: cluster k owns an Np_k x Np_k row-major block (Np_k = 9 n_k rounded up to the tile T) whose
// lower triangle is significant.  Padding rows and columns are zero and their diagonal is treated as 1,
// so the padded system is block diagonal with an identity block and solves to zero there.
//
// The factorised matrix is the Jacobi-scaled  S~ = D^-1/2 S D^-1/2, D = diag(S) (s_i = S_ii^-1/2), so that
// S x = b becomes S~ z = s o b, x = s o z.  Right-looking tiled algorithm, step kt:
//   panel   for every tile row i >= kt: factor the diagonal tile (kt, kt) in shared memory (redundantly in
//           each CTA, T^3/3 flops); the CTA of i = kt also stores the inverse of L_kt,kt; the CTAs of
//           i > kt solve L_i,kt L_kt,kt^T = A_i,kt;
//   update  for every kt < j <= i: A_i,j -= L_i,kt L_j,kt^T.
// FP64 factor (FP64 mode): a pivot that is not positive and finite marks the cluster as failed, and the
// LM step is rejected (lambda *= 3).  FP32 factor (mixed mode): a pivot that rounding has made vanish
// (below 2^-20 of the unit scaled diagonal; legitimate pivots of the damped system are about lambda or
// more) is raised to 2^-12 and counted -- static pivoting, as in Li & Demmel's SuperLU_DIST -- and the
// FP64 iterative refinement that follows solves the unmodified system.  A non-finite pivot fails.
//
// Solves: one CTA per cluster; with the inverted diagonal tiles every tile step is two parallel
// matrix-vector products.  Refinement: r = b - S x in FP64 over many CTAs (S symmetric, lower stored),
// then x += D^-1/2 (L L^T)^-1 D^-1/2 r.
#include "stba_internal.cuh"

namespace stba {

#define FULL_MASK 0xffffffffu

template <typename F> struct FactorCfg;
template <> struct FactorCfg<double> { static constexpr int T = 32; };
template <> struct FactorCfg<float> { static constexpr int T = 64; };

int factor_tile(bool mixed) { return mixed ? FactorCfg<float>::T : FactorCfg<double>::T; }

// s_i = 1 / sqrt(S_ii) (1 on padding)
template <typename Sreal>
__global__ void k_diag_scale(DevProblem P, const Sreal* S, double* scale) {
  const int k = blockIdx.y;
  const int np = P.cluster_np[k], nk = P.cluster_n[k];
  const Sreal* Sk = S + P.S_off[k];
  double* sk = scale + P.v_off[k];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
    double d = i < nk ? (double)Sk[(size_t)i * np + i] : 1.0;
    sk[i] = d > 0.0 ? 1.0 / sqrt(d) : 1.0;
  }
}

// L = s_i s_j S_ij (lower triangle and diagonal blocks' contents; the upper part is never read)
template <typename Sreal, typename F>
__global__ void k_scaled_copy(DevProblem P, const Sreal* S, const double* scale, F* L) {
  const int k = blockIdx.y;
  const int np = P.cluster_np[k];
  const Sreal* Sk = S + P.S_off[k];
  F* Lk = L + P.S_off[k];
  const double* sk = scale + P.v_off[k];
  for (int r = blockIdx.x; r < np; r += gridDim.x) {
    const double sr = sk[r];
    for (int c = threadIdx.x; c <= r; c += blockDim.x)
      Lk[(size_t)r * np + c] = (F)((double)Sk[(size_t)r * np + c] * sr * sk[c]);
  }
}

// Unblocked LL^T of the diagonal tile in shared memory (lower triangle).
template <typename F, int T>
__device__ void factor_diag_tile(F (*D)[T + 1], int row0, int nk, int* fail, int* boosted) {
  for (int j = 0; j < T; ++j) {
    if (threadIdx.x == 0) {
      F d = D[j][j];
      if (row0 + j >= nk) {
        d = F(1);
      } else if (!isfinite(d)) {
        *fail = 1;
        d = F(1);
      } else if (sizeof(F) == 8) {
        if (!(d > F(0))) {
          *fail = 1;
          d = F(1);
        }
      } else if (d < F(1.0 / 1048576)) {
        atomicAdd(boosted, 1);
        d = F(1.0 / 4096);
      }
      D[j][j] = sqrt(d);
    }
    __syncthreads();
    const F djj = D[j][j];
    for (int r = j + 1 + threadIdx.x; r < T; r += blockDim.x) D[r][j] /= djj;
    __syncthreads();
    for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
      const int r = idx / T, c = idx - (idx / T) * T;
      if (c > j && r >= c) D[r][c] -= D[r][j] * D[c][j];
    }
    __syncthreads();
  }
}

template <typename F, int T>
__global__ void __launch_bounds__(256) k_chol_panel(F* L, F* Dinv, DevProblem P, const int2* items, int kt,
                                                    int* fail_flags, int* boosted) {
  __shared__ F D[T][T + 1];
  __shared__ F X[T][T + 1];
  const int2 it = items[blockIdx.x];
  const int k = it.x, i = it.y;
  const int np = P.cluster_np[k], nk = P.cluster_n[k];
  F* A = L + P.S_off[k];
  const size_t base_kk = (size_t)(kt * T) * np + kt * T;
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
    const int r = idx / T, c = idx - (idx / T) * T;
    D[r][c] = (c <= r) ? A[base_kk + (size_t)r * np + c] : F(0);
  }
  __syncthreads();
  factor_diag_tile<F, T>(D, kt * T, nk, fail_flags + k, boosted);
  if (i == kt) {
    for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
      const int r = idx / T, c = idx - (idx / T) * T;
      if (c <= r) A[base_kk + (size_t)r * np + c] = D[r][c];
    }
    // inverse of the lower-triangular tile, one column per thread: L Y = I
    for (int c = threadIdx.x; c < T; c += blockDim.x) {
      for (int r = 0; r < T; ++r) {
        if (r < c) {
          X[r][c] = F(0);
          continue;
        }
        F s = (r == c) ? F(1) : F(0);
        for (int j = c; j < r; ++j) s -= D[r][j] * X[j][c];
        X[r][c] = s / D[r][r];
      }
    }
    __syncthreads();
    F* Di = Dinv + (size_t)P.v_off[k] * T + (size_t)kt * T * T;
    for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
      const int r = idx / T, c = idx - (idx / T) * T;
      Di[idx] = X[r][c];
    }
    return;
  }
  const size_t base_ik = (size_t)(i * T) * np + kt * T;
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
    const int r = idx / T, c = idx - (idx / T) * T;
    X[r][c] = A[base_ik + (size_t)r * np + c];
  }
  __syncthreads();
  // X L_kk^T = A  ->  X[r][c] = (A[r][c] - sum_{j<c} X[r][j] L[c][j]) / L[c][c], rows independent
  for (int r = threadIdx.x; r < T; r += blockDim.x) {
    for (int c = 0; c < T; ++c) {
      F s = X[r][c];
      for (int j = 0; j < c; ++j) s -= X[r][j] * D[c][j];
      X[r][c] = s / D[c][c];
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
    const int r = idx / T, c = idx - (idx / T) * T;
    A[base_ik + (size_t)r * np + c] = X[r][c];
  }
}

// A_ij -= L_i,kt L_j,kt^T on a T x T tile; 256 threads, each an (T/16) x (T/16) register block.
template <typename F, int T>
__global__ void __launch_bounds__(256) k_chol_update(F* L, DevProblem P, const int2* items, int kt) {
  constexpr int R = T / 16;
  constexpr int LD = T + (sizeof(F) == 4 ? 4 : 2);
  __shared__ __align__(16) F LiT[T][LD];
  __shared__ __align__(16) F LjT[T][LD];
  const int2 it = items[blockIdx.x];
  const int k = it.x, i = it.y >> 16, j = it.y & 0xffff;
  const int np = P.cluster_np[k];
  F* A = L + P.S_off[k];
  const size_t bi = (size_t)(i * T) * np + kt * T, bj = (size_t)(j * T) * np + kt * T;
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
    const int r = idx / T, c = idx - (idx / T) * T;
    LiT[c][r] = A[bi + (size_t)r * np + c];
    LjT[c][r] = A[bj + (size_t)r * np + c];
  }
  __syncthreads();
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
  F acc[R][R];
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int b = 0; b < R; ++b) acc[a][b] = F(0);
#pragma unroll 4
  for (int kk = 0; kk < T; ++kk) {
    F av[R], bv[R];
#pragma unroll
    for (int a = 0; a < R; ++a) av[a] = LiT[kk][tr * R + a];
#pragma unroll
    for (int b = 0; b < R; ++b) bv[b] = LjT[kk][tc * R + b];
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int b = 0; b < R; ++b) acc[a][b] += av[a] * bv[b];
  }
  const size_t bij = (size_t)(i * T) * np + j * T;
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int b = 0; b < R; ++b) A[bij + (size_t)(tr * R + a) * np + tc * R + b] -= acc[a][b];
}

// ------------------------------------------------------------------------------------------------------
template <typename F>
__device__ F warp_sum(F v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(FULL_MASK, v, d);
  return v;
}

// x := D^-1/2 (L L^T)^-1 D^-1/2 rhs  (accumulate = 0) or x += ... (accumulate = 1); one CTA per cluster.
template <typename F, int T, typename Rreal>
__global__ void __launch_bounds__(256) k_tri_solve(DevProblem P, const F* L, const F* Dinv, const double* scale,
                                                   const Rreal* rhs, double* x, int accumulate) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  F* y = reinterpret_cast<F*>(smem_raw);
  __shared__ F t[T];
  __shared__ F part[8][T];
  const int k = blockIdx.x;
  const int np = P.cluster_np[k];
  const F* A = L + P.S_off[k];
  const F* Di = Dinv + (size_t)P.v_off[k] * T;
  const double* sk = scale + P.v_off[k];
  const Rreal* rk = rhs + P.v_off[k];
  double* xk = x + P.v_off[k];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int nt = np / T;
  for (int i = threadIdx.x; i < np; i += blockDim.x) y[i] = (F)((double)rk[i] * sk[i]);
  __syncthreads();
  // forward: L y = s o rhs
  for (int it = 0; it < nt; ++it) {
    const int r0 = it * T;
    for (int rr = warp; rr < T; rr += nwarps) {
      const F* row = A + (size_t)(r0 + rr) * np;
      F s = F(0);
      for (int c = lane; c < r0; c += 32) s += row[c] * y[c];
      s = warp_sum(s);
      if (lane == 0) t[rr] = y[r0 + rr] - s;
    }
    __syncthreads();
    const F* Dt = Di + (size_t)it * T * T;
    for (int rr = warp; rr < T; rr += nwarps) {
      F s = F(0);
      for (int c = lane; c <= rr; c += 32) s += Dt[rr * T + c] * t[c];
      s = warp_sum(s);
      if (lane == 0) y[r0 + rr] = s;
    }
    __syncthreads();
  }
  // backward: L^T z = y
  for (int it = nt - 1; it >= 0; --it) {
    const int r0 = it * T;
    for (int cc = lane; cc < T; cc += 32) {
      F p = F(0);
      for (int c = r0 + T + warp; c < np; c += nwarps) p += A[(size_t)c * np + r0 + cc] * y[c];
      part[warp][cc] = p;
    }
    __syncthreads();
    for (int cc = threadIdx.x; cc < T; cc += blockDim.x) {
      F s = F(0);
      for (int w = 0; w < nwarps; ++w) s += part[w][cc];
      t[cc] = y[r0 + cc] - s;
    }
    __syncthreads();
    const F* Dt = Di + (size_t)it * T * T;
    // z_tile = Dinv^T t: z[c] = sum_{r >= c} Dinv[r][c] t[r]
    for (int cc = threadIdx.x; cc < T; cc += blockDim.x) {
      F s = F(0);
      for (int r = cc; r < T; ++r) s += Dt[r * T + cc] * t[r];
      y[r0 + cc] = s;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    const double v = (double)y[i] * sk[i];
    xk[i] = accumulate ? xk[i] + v : v;
  }
}

// r = b - S x (FP64), rows [r0, r0 + 32) of one cluster per CTA; r was set to b before.
template <typename Sreal>
__global__ void __launch_bounds__(256) k_residual(DevProblem P, const Sreal* S, const double* x, double* r,
                                                  const int2* items) {
  __shared__ double colacc[4096];
  const int2 it = items[blockIdx.x];
  const int k = it.x, r0 = it.y * 32;
  const int np = P.cluster_np[k], nk = P.cluster_n[k];
  const Sreal* Sk = S + P.S_off[k];
  const double* xk = x + P.v_off[k];
  double* rk = r + P.v_off[k];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int rend = min(r0 + 32, nk);
  // lower part: rk[row] -= sum_{c <= row} S[row][c] x[c]; transposed part: rk[c] -= S[row][c] x[row], c < row
  for (int cb = 0; cb < rend; cb += 4096) {
    const int cend = min(cb + 4096, rend);
    for (int i = threadIdx.x; i < cend - cb; i += blockDim.x) colacc[i] = 0.0;
    __syncthreads();
    for (int row = r0 + warp; row < rend; row += nwarps) {
      const Sreal* srow = Sk + (size_t)row * np;
      const double xr = xk[row];
      double s = 0.0;
      const int cmax = min(row, cend - 1);
      for (int c = cb + lane; c <= cmax; c += 32) {
        const double a = (double)srow[c];
        s += a * xk[c];
        if (c < row) atomicAdd(colacc + (c - cb), a * xr);
      }
      s = warp_sum(s);
      if (lane == 0) atomicAdd(rk + row, -s);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cend - cb; i += blockDim.x)
      if (colacc[i] != 0.0) atomicAdd(rk + cb + i, -colacc[i]);
    __syncthreads();
  }
}

template <typename Rreal>
__global__ void k_copy_vec(const Rreal* src, double* dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

__global__ void k_scatter_dc(DevProblem P, const double* x, double* dc) {
  const int k = blockIdx.x;
  const int nk = P.cluster_n[k], cbase = P.cluster_cam_off[k];
  const double* xk = x + P.v_off[k];
  for (int i = threadIdx.x; i < nk; i += blockDim.x) {
    const int cam = P.cluster_cams[cbase + i / 9];
    dc[9 * (size_t)cam + i % 9] = xk[i];
  }
}

__global__ void k_count_failures(const int* fail_flags, int l, DevState* st) {
  int c = 0;
  for (int i = threadIdx.x; i < l; i += blockDim.x) c += fail_flags[i] != 0;
  for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(FULL_MASK, c, d);
  __shared__ int red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    st->failed = t;
  }
}

// ------------------------------------------------------------------------------------------------------
// Host launchers
template <typename Sreal, typename F>
void launch_factor(const DevProblem& P, const Sreal* S, const FactorBuffers& fb, const CholPlan& plan,
                   cudaStream_t stream) {
  constexpr int T = FactorCfg<F>::T;
  F* L = reinterpret_cast<F*>(fb.L);
  F* Dinv = reinterpret_cast<F*>(fb.Dinv);
  dim3 g1(std::max(1, std::min(plan.max_np / 256 + 1, 64)), P.l);
  k_diag_scale<Sreal><<<g1, 256, 0, stream>>>(P, S, fb.scale);
  dim3 g2(std::min(plan.max_np, 1024), P.l);
  k_scaled_copy<Sreal, F><<<g2, 256, 0, stream>>>(P, S, fb.scale, L);
  for (int kt = 0; kt < plan.nsteps; ++kt) {
    const int npn = plan.h_panel_off[kt + 1] - plan.h_panel_off[kt];
    if (npn > 0)
      k_chol_panel<F, T><<<npn, 256, 0, stream>>>(L, Dinv, P, plan.panel_items + plan.h_panel_off[kt], kt,
                                                   fb.fail_flags, fb.boosted);
    const int nu = plan.h_update_off[kt + 1] - plan.h_update_off[kt];
    if (nu > 0) k_chol_update<F, T><<<nu, 256, 0, stream>>>(L, P, plan.update_items + plan.h_update_off[kt], kt);
  }
}

template <typename Sreal, typename F>
void launch_solve(const DevProblem& P, const Sreal* S, const Sreal* b, const FactorBuffers& fb, const CholPlan& plan,
                  int refine_steps, double* dc, cudaStream_t stream) {
  constexpr int T = FactorCfg<F>::T;
  const F* L = reinterpret_cast<const F*>(fb.L);
  const F* Dinv = reinterpret_cast<const F*>(fb.Dinv);
  const size_t smem = sizeof(F) * (size_t)plan.max_np;
  k_tri_solve<F, T, Sreal><<<P.l, 256, smem, stream>>>(P, L, Dinv, fb.scale, b, fb.x, 0);
  const int nblk = (int)std::min<int64_t>(fb.v_total / 256 + 1, 152 * 8);
  for (int s = 0; s < refine_steps; ++s) {
    k_copy_vec<Sreal><<<nblk, 256, 0, stream>>>(b, fb.r, fb.v_total);
    if (plan.n_res_items > 0) k_residual<Sreal><<<plan.n_res_items, 256, 0, stream>>>(P, S, fb.x, fb.r, plan.res_items);
    k_tri_solve<F, T, double><<<P.l, 256, smem, stream>>>(P, L, Dinv, fb.scale, fb.r, fb.x, 1);
  }
  k_scatter_dc<<<P.l, 256, 0, stream>>>(P, fb.x, dc);
}

void configure_solve_kernels(int max_np) {
  const int s32 = (int)(sizeof(float) * (size_t)max_np), s64 = (int)(sizeof(double) * (size_t)max_np);
  cudaFuncSetAttribute(k_tri_solve<float, 64, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32);
  cudaFuncSetAttribute(k_tri_solve<float, 64, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32);
  cudaFuncSetAttribute(k_tri_solve<double, 32, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64);
}

void launch_count_failures(const int* fail_flags, int l, DevState* st, cudaStream_t stream) {
  k_count_failures<<<1, 256, 0, stream>>>(fail_flags, l, st);
}

template void launch_factor<float, float>(const DevProblem&, const float*, const FactorBuffers&, const CholPlan&,
                                          cudaStream_t);
template void launch_factor<double, double>(const DevProblem&, const double*, const FactorBuffers&,
                                            const CholPlan&, cudaStream_t);
template void launch_solve<float, float>(const DevProblem&, const float*, const float*, const FactorBuffers&,
                                         const CholPlan&, int, double*, cudaStream_t);
template void launch_solve<double, double>(const DevProblem&, const double*, const double*, const FactorBuffers&,
                                           const CholPlan&, int, double*, cudaStream_t);

}  // namespace stba
