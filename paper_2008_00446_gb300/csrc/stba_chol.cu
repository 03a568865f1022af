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

// Register-blocked tile kernels.  256 threads form a 16 x 16 grid; thread (bi, bj) holds the R x R block
// (R = T / 16) of rows bi R .. and columns bj R .. in registers.  Column j is broadcast through a double
// buffer in shared memory, so each of the T steps costs one barrier.
//
// factor_tile_regs: right-looking LL^T of the diagonal tile with the unscaled column,
// a_rc -= a_rj a_cj / a_jj; the pivots a_jj are kept and the columns scaled at the end.
template <typename F, int T>
__device__ __forceinline__ void factor_tile_regs(F (&a)[T / 16][T / 16], int bi, int bj, F* colbuf, F* piv, int row0, int nk,
                                 int* fail, int* boosted) {
  constexpr int R = T / 16;
  for (int j = 0; j < T; ++j) {
    F* col = colbuf + (j & 1) * T;
    if (bj == j / R) {
#pragma unroll
      for (int ii = 0; ii < R; ++ii) {
        const int jr = j % R;
        F v = a[ii][0];
#pragma unroll
        for (int jj = 1; jj < R; ++jj) v = (jj == jr) ? a[ii][jj] : v;
        col[bi * R + ii] = v;
      }
    }
    __syncthreads();
    F d = col[j];
    bool bad = false, boost = false;
    if (row0 + j >= nk) {
      d = F(1);
    } else if (!isfinite(d)) {
      bad = true;
      d = F(1);
    } else if (sizeof(F) == 8) {
      if (!(d > F(0))) {
        bad = true;
        d = F(1);
      }
    } else if (d < F(1.0 / 1048576)) {
      boost = true;
      d = F(1.0 / 4096);
    }
    if (threadIdx.x == 0) {
      piv[j] = d;
      if (bad) *fail = 1;
      if (boost && boosted) atomicAdd(boosted, 1);
    }
    const F inv = F(1) / d;
    if (bi >= bj) {
      F cr[R], cc[R];
#pragma unroll
      for (int ii = 0; ii < R; ++ii) cr[ii] = col[bi * R + ii] * inv;
#pragma unroll
      for (int jj = 0; jj < R; ++jj) cc[jj] = col[bj * R + jj];
#pragma unroll
      for (int ii = 0; ii < R; ++ii)
#pragma unroll
        for (int jj = 0; jj < R; ++jj) {
          const int r = bi * R + ii, cl = bj * R + jj;
          if (cl > j && r >= cl) a[ii][jj] -= cr[ii] * cc[jj];
        }
    }
  }
  __syncthreads();
#pragma unroll
  for (int ii = 0; ii < R; ++ii)
#pragma unroll
    for (int jj = 0; jj < R; ++jj) {
      const int r = bi * R + ii, cl = bj * R + jj;
      a[ii][jj] = (r > cl) ? a[ii][jj] / sqrt(piv[cl]) : ((r == cl) ? sqrt(piv[cl]) : F(0));
    }
}

// trsm_tile_regs: X L^T = A for a full tile X (registers), L lower triangular in shared memory; the
// columns of X are finished left to right and each finished column updates the ones to its right.
template <typename F, int T>
__device__ __forceinline__ void trsm_tile_regs(F (&x)[T / 16][T / 16], int bi, int bj, const F (*Ls)[T + 1], F* colbuf) {
  constexpr int R = T / 16;
  for (int c = 0; c < T; ++c) {
    F* col = colbuf + (c & 1) * T;
    if (bj == c / R) {
      const F inv = F(1) / Ls[c][c];
      const int cr_ = c % R;
#pragma unroll
      for (int ii = 0; ii < R; ++ii) {
        F v = F(0);
#pragma unroll
        for (int jj = 0; jj < R; ++jj) {
          const F nv = x[ii][jj] * inv;
          x[ii][jj] = (jj == cr_) ? nv : x[ii][jj];
          v = (jj == cr_) ? nv : v;
        }
        col[bi * R + ii] = v;
      }
    }
    __syncthreads();
    F cr[R], lc[R];
#pragma unroll
    for (int ii = 0; ii < R; ++ii) cr[ii] = col[bi * R + ii];
#pragma unroll
    for (int jj = 0; jj < R; ++jj) lc[jj] = Ls[bj * R + jj][c];
#pragma unroll
    for (int ii = 0; ii < R; ++ii)
#pragma unroll
      for (int jj = 0; jj < R; ++jj)
        if (bj * R + jj > c) x[ii][jj] -= cr[ii] * lc[jj];
  }
}

template <typename F, int T>
__global__ void __launch_bounds__(256) k_chol_panel(F* L, DevProblem P, const int2* items, int kt,
                                                    int* fail_flags, int* boosted) {
  constexpr int R = T / 16;
  __shared__ F Ls[T][T + 1];
  __shared__ F colbuf[2 * T];
  __shared__ F piv[T];
  const int2 it = items[blockIdx.x];
  const int k = it.x, i = it.y;
  const int np = P.cluster_np[k], nk = P.cluster_n[k];
  F* A = L + P.S_off[k];
  const int bi = threadIdx.x >> 4, bj = threadIdx.x & 15;
  const size_t base_kk = (size_t)(kt * T) * np + kt * T;
  F a[R][R];
#pragma unroll
  for (int ii = 0; ii < R; ++ii)
#pragma unroll
    for (int jj = 0; jj < R; ++jj) {
      const int r = bi * R + ii, cl = bj * R + jj;
      a[ii][jj] = (cl <= r) ? A[base_kk + (size_t)r * np + cl] : F(0);
    }
  F x[R][R];
  const size_t base_ik = (size_t)(i * T) * np + kt * T;
  if (i != kt) {
#pragma unroll
    for (int ii = 0; ii < R; ++ii)
#pragma unroll
      for (int jj = 0; jj < R; ++jj) x[ii][jj] = A[base_ik + (size_t)(bi * R + ii) * np + bj * R + jj];
  }
  factor_tile_regs<F, T>(a, bi, bj, colbuf, piv, kt * T, nk, fail_flags + k, (i == kt) ? boosted : nullptr);
  if (i == kt) {
#pragma unroll
    for (int ii = 0; ii < R; ++ii)
#pragma unroll
      for (int jj = 0; jj < R; ++jj) {
        const int r = bi * R + ii, cl = bj * R + jj;
        if (cl <= r) A[base_kk + (size_t)r * np + cl] = a[ii][jj];
      }
    return;
  }
#pragma unroll
  for (int ii = 0; ii < R; ++ii)
#pragma unroll
    for (int jj = 0; jj < R; ++jj) Ls[bi * R + ii][bj * R + jj] = a[ii][jj];
  __syncthreads();
  trsm_tile_regs<F, T>(x, bi, bj, Ls, colbuf);
#pragma unroll
  for (int ii = 0; ii < R; ++ii)
#pragma unroll
    for (int jj = 0; jj < R; ++jj) A[base_ik + (size_t)(bi * R + ii) * np + bj * R + jj] = x[ii][jj];
}

// Inverse of every diagonal tile of the factor (for the solves), one CTA per tile: L Y = I column by
// column, four threads per column splitting each dot product.
template <typename F, int T>
__global__ void __launch_bounds__(256) k_diag_inverse(const F* L, F* Dinv, DevProblem P, const int2* items) {
  __shared__ F D[T][T + 1];
  __shared__ F Y[T][T + 1];
  const int2 it = items[blockIdx.x];
  const int k = it.x, t = it.y;
  const int np = P.cluster_np[k];
  const F* A = L + P.S_off[k];
  const size_t base = (size_t)(t * T) * np + t * T;
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
    const int r = idx / T, c = idx - (idx / T) * T;
    D[r][c] = (c <= r) ? A[base + (size_t)r * np + c] : F(0);
  }
  __syncthreads();
  const int cl = threadIdx.x >> 2, part = threadIdx.x & 3;
  for (int cb = cl; cb < T; cb += blockDim.x >> 2) {
    for (int r = 0; r < T; ++r) {
      F s = F(0);
      for (int j = cb + part; j < r; j += 4) s += D[r][j] * Y[j][cb];
      s += __shfl_xor_sync(FULL_MASK, s, 1);
      s += __shfl_xor_sync(FULL_MASK, s, 2);
      const F v = (r < cb) ? F(0) : (((r == cb) ? F(1) : F(0)) - s) / D[r][r];
      __syncwarp();
      if (part == 0) Y[r][cb] = v;
      __syncwarp();
    }
  }
  __syncthreads();
  F* Di = Dinv + (size_t)P.v_off[k] * T + (size_t)t * T * T;
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) Di[idx] = Y[idx / T][idx - (idx / T) * T];
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
// Each tile step: the off-diagonal part as a matrix-vector product (every warp keeps T / 8 rows in
// flight), then the diagonal tile through its stored inverse, staged in shared memory.
template <typename F, int T, typename Rreal>
__global__ void __launch_bounds__(256) k_tri_solve(DevProblem P, const F* L, const F* Dinv, const double* scale,
                                                   const Rreal* rhs, double* x, int accumulate) {
  constexpr int RW = T / 8;   // rows per warp
  extern __shared__ __align__(16) unsigned char smem_raw[];
  F* y = reinterpret_cast<F*>(smem_raw);
  __shared__ F Ds[T][T + 1];
  __shared__ F t[T];
  __shared__ F part[8][T];
  const int k = blockIdx.x;
  const int np = P.cluster_np[k];
  const F* A = L + P.S_off[k];
  const F* Di = Dinv + (size_t)P.v_off[k] * T;
  const double* sk = scale + P.v_off[k];
  const Rreal* rk = rhs + P.v_off[k];
  double* xk = x + P.v_off[k];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nt = np / T;
  for (int i = threadIdx.x; i < np; i += blockDim.x) y[i] = (F)((double)rk[i] * sk[i]);
  __syncthreads();
  // forward: L y = s o rhs
  for (int it = 0; it < nt; ++it) {
    const int r0 = it * T;
    const F* Dt = Di + (size_t)it * T * T;
    for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) Ds[idx / T][idx - (idx / T) * T] = Dt[idx];
    F acc[RW];
#pragma unroll
    for (int q = 0; q < RW; ++q) acc[q] = F(0);
    const F* rows = A + (size_t)(r0 + warp * RW) * np;
    int c = lane;
    for (; c + 32 < r0; c += 64) {
      const F y0 = y[c], y1 = y[c + 32];
#pragma unroll
      for (int q = 0; q < RW; ++q) acc[q] += rows[(size_t)q * np + c] * y0 + rows[(size_t)q * np + c + 32] * y1;
    }
    for (; c < r0; c += 32) {
      const F yc = y[c];
#pragma unroll
      for (int q = 0; q < RW; ++q) acc[q] += rows[(size_t)q * np + c] * yc;
    }
#pragma unroll
    for (int q = 0; q < RW; ++q) {
      const F s = warp_sum(acc[q]);
      if (lane == 0) t[warp * RW + q] = y[r0 + warp * RW + q] - s;
    }
    __syncthreads();
    for (int rr = warp; rr < T; rr += 8) {
      F s = F(0);
      for (int c = lane; c <= rr; c += 32) s += Ds[rr][c] * t[c];
      s = warp_sum(s);
      if (lane == 0) y[r0 + rr] = s;
    }
    __syncthreads();
  }
  // backward: L^T z = y
  for (int it = nt - 1; it >= 0; --it) {
    const int r0 = it * T;
    const F* Dt = Di + (size_t)it * T * T;
    for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) Ds[idx / T][idx - (idx / T) * T] = Dt[idx];
    {
      constexpr int NC = T / 32;   // columns per lane
      F p[NC][4];
#pragma unroll
      for (int u = 0; u < NC; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) p[u][v] = F(0);
      int c = r0 + T + warp;
      for (; c + 24 < np; c += 32) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const F yc = y[c + 8 * v];
          const F* row = A + (size_t)(c + 8 * v) * np + r0 + lane;
#pragma unroll
          for (int u = 0; u < NC; ++u) p[u][v] += row[32 * u] * yc;
        }
      }
      for (; c < np; c += 8) {
        const F yc = y[c];
        const F* row = A + (size_t)c * np + r0 + lane;
#pragma unroll
        for (int u = 0; u < NC; ++u) p[u][0] += row[32 * u] * yc;
      }
#pragma unroll
      for (int u = 0; u < NC; ++u) part[warp][lane + 32 * u] = (p[u][0] + p[u][1]) + (p[u][2] + p[u][3]);
    }
    __syncthreads();
    for (int cc = threadIdx.x; cc < T; cc += blockDim.x) {
      F s = F(0);
#pragma unroll
      for (int w = 0; w < 8; ++w) s += part[w][cc];
      t[cc] = y[r0 + cc] - s;
    }
    __syncthreads();
    // z_tile = Dinv^T t: z[c] = sum_{r >= c} Dinv[r][c] t[r]
    for (int cc = warp; cc < T; cc += 8) {
      F s = F(0);
      for (int r = cc + lane; r < T; r += 32) s += Ds[r][cc] * t[r];
      s = warp_sum(s);
      if (lane == 0) y[r0 + cc] = s;
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
template <typename F>
void launch_factor(const DevProblem& P, const double* S, const FactorBuffers& fb, const CholPlan& plan,
                   cudaStream_t stream) {
  using Sreal = double;
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
      k_chol_panel<F, T><<<npn, 256, 0, stream>>>(L, P, plan.panel_items + plan.h_panel_off[kt], kt, fb.fail_flags,
                                                   fb.boosted);
    const int nu = plan.h_update_off[kt + 1] - plan.h_update_off[kt];
    if (nu > 0) k_chol_update<F, T><<<nu, 256, 0, stream>>>(L, P, plan.update_items + plan.h_update_off[kt], kt);
  }
  if (plan.n_diag_items > 0) k_diag_inverse<F, T><<<plan.n_diag_items, 256, 0, stream>>>(L, Dinv, P, plan.diag_items);
}

template <typename F>
void launch_solve(const DevProblem& P, const double* S, const double* b, const FactorBuffers& fb,
                  const CholPlan& plan, int refine_steps, double* dc, cudaStream_t stream) {
  using Sreal = double;
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
  cudaFuncSetAttribute(k_tri_solve<float, 64, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32);
  cudaFuncSetAttribute(k_tri_solve<double, 32, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64);
}

void launch_count_failures(const int* fail_flags, int l, DevState* st, cudaStream_t stream) {
  k_count_failures<<<1, 256, 0, stream>>>(fail_flags, l, st);
}

template void launch_factor<float>(const DevProblem&, const double*, const FactorBuffers&, const CholPlan&,
                                   cudaStream_t);
template void launch_factor<double>(const DevProblem&, const double*, const FactorBuffers&, const CholPlan&,
                                    cudaStream_t);
template void launch_solve<float>(const DevProblem&, const double*, const double*, const FactorBuffers&,
                                  const CholPlan&, int, double*, cudaStream_t);
template void launch_solve<double>(const DevProblem&, const double*, const double*, const FactorBuffers&,
                                   const CholPlan&, int, double*, cudaStream_t);

}  // namespace stba
