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
#include <cooperative_groups.h>

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

// Correctly rounded reciprocal (one special-function instruction plus fix-up instead of a division).
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }

// Named barriers: the producer warp arrives without waiting, the consumer warps wait.
__device__ __forceinline__ void named_arrive(int id, int nthreads) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Register-blocked tile kernels.  256 threads form a 16 x 16 grid; thread (bi, bj) = (tid % 16, tid / 16)
// holds the R x R block (R = T / 16) of rows bi R .. and columns bj R .. in registers.  Warp w therefore
// owns the 2R consecutive columns 2R w ..; lane l of it holds rows R (l % 16) .. of half l / 16 of them.
// Both kernels sweep the tile in T / 2R blocked steps: warp w finishes its own columns with shuffles only,
// publishes them in shared memory (one buffer per step) and arrives on named barrier 1 + w; the warps to
// its right wait on that barrier and apply a rank-2R update from registers.  A warp starts its own step
// as soon as it has applied the steps before it, so the updates of distant warps overlap the next step.
//
// factor_tile_regs: LL^T of the diagonal tile.  Inside a block the updates use the unscaled columns,
// a_rc -= a_rj a_cj / a_jj; the pivots a_jj are kept, the published columns are scaled by a_jj^-1/2, and
// every column is scaled once at the end.
template <typename F, int T>
__device__ __forceinline__ void factor_tile_regs(F (&a)[T / 16][T / 16], F (*U)[T][T / 8], F* piv, F* tab,
                                                 int row0, int nk, int* fail, int* boosted) {
  constexpr int R = T / 16, W = 2 * R;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int bi = threadIdx.x & 15, bj = threadIdx.x >> 4, h = lane >> 4;
  for (int w = 0; w < 8; ++w) {
    const int c0 = W * w;
    if (warp == w) {
#pragma unroll
      for (int jj = 0; jj < W; ++jj) {
        const int hj = jj / R, cj = jj % R;
        const int cg = c0 + jj;
        F d = __shfl_sync(0xffffffffu, a[cj][cj], hj * 16 + 2 * w + hj);
        bool bad = false, boost = false;
        if (row0 + cg >= nk) {
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
        if (lane == 0) {
          piv[cg] = d;
          if (bad) *fail = 1;
          if (boost && boosted) atomicAdd(boosted, 1);
        }
        const F inv = rcp_rn(d);
        F colr[R], rowc[R];
#pragma unroll
        for (int ii = 0; ii < R; ++ii) colr[ii] = __shfl_sync(0xffffffffu, a[ii][cj], bi + 16 * hj);
#pragma unroll
        for (int j2 = 0; j2 < R; ++j2) rowc[j2] = __shfl_sync(0xffffffffu, a[j2][cj], (2 * w + h) + 16 * hj);
#pragma unroll
        for (int ii = 0; ii < R; ++ii)
#pragma unroll
          for (int j2 = 0; j2 < R; ++j2) {
            const int r = R * bi + ii, cl = c0 + R * h + j2;
            if (cl > cg && r >= cl) a[ii][j2] -= colr[ii] * rowc[j2] * inv;
          }
      }
      __syncwarp();
#pragma unroll
      for (int ii = 0; ii < R; ++ii)
#pragma unroll
        for (int j2 = 0; j2 < R; ++j2) {
          const int cl = c0 + R * h + j2;
          U[w][R * bi + ii][R * h + j2] = a[ii][j2] * rsqrt(piv[cl]);
        }
      if (w < 7) named_arrive(1 + w, 32 * (8 - w));
    } else if (warp > w) {
      named_sync(1 + w, 32 * (8 - w));
      if (bi >= bj) {
        F ur[R][W], uc[R][W];
#pragma unroll
        for (int ii = 0; ii < R; ++ii)
#pragma unroll
          for (int k = 0; k < W; ++k) {
            ur[ii][k] = U[w][R * bi + ii][k];
            uc[ii][k] = U[w][R * bj + ii][k];
          }
        if (bi > bj) {
#pragma unroll
          for (int ii = 0; ii < R; ++ii)
#pragma unroll
            for (int jj = 0; jj < R; ++jj) {
              F s = F(0);
#pragma unroll
              for (int k = 0; k < W; ++k) s += ur[ii][k] * uc[jj][k];
              a[ii][jj] -= s;
            }
        } else {
#pragma unroll
          for (int ii = 0; ii < R; ++ii)
#pragma unroll
            for (int jj = 0; jj <= ii; ++jj) {
              F s = F(0);
#pragma unroll
              for (int k = 0; k < W; ++k) s += ur[ii][k] * uc[jj][k];
              a[ii][jj] -= s;
            }
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < T) {
    const F sq = sqrt(piv[threadIdx.x]);
    tab[threadIdx.x] = rcp_rn(sq);
    tab[T + threadIdx.x] = sq;
  }
  __syncthreads();
#pragma unroll
  for (int ii = 0; ii < R; ++ii)
#pragma unroll
    for (int jj = 0; jj < R; ++jj) {
      const int r = R * bi + ii, cl = R * bj + jj;
      a[ii][jj] = (r > cl) ? a[ii][jj] * tab[cl] : ((r == cl) ? tab[T + cl] : F(0));
    }
  __syncthreads();
}

// trsm_tile_regs: X L^T = A for a full tile X (registers), L lower triangular in shared memory (Ls) with
// the reciprocals of its diagonal in rcp.  Warp w solves its 2R columns (rows are independent; the two
// halves of the warp exchange their solved values by shuffles), publishes them, and the warps to its
// right subtract X[:, block] L[c, block]^T.
template <typename F, int T>
__device__ __forceinline__ void trsm_tile_regs(F (&x)[T / 16][T / 16], const F (*Ls)[T + 1], const F* rcp,
                                               F (*U)[T][T / 8]) {
  constexpr int R = T / 16, W = 2 * R;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int bi = threadIdx.x & 15, bj = threadIdx.x >> 4, h = lane >> 4;
  for (int w = 0; w < 8; ++w) {
    const int c0 = W * w;
    if (warp == w) {
#pragma unroll
      for (int jj = 0; jj < W; ++jj) {
        const int hj = jj / R, cj = jj % R;
        const int cg = c0 + jj;
        if (h == hj) {
#pragma unroll
          for (int ii = 0; ii < R; ++ii) x[ii][cj] *= rcp[cg];
        }
        F xs[R];
#pragma unroll
        for (int ii = 0; ii < R; ++ii) xs[ii] = __shfl_sync(0xffffffffu, x[ii][cj], bi + 16 * hj);
#pragma unroll
        for (int j2 = 0; j2 < R; ++j2) {
          const int cl = c0 + R * h + j2;
          if (cl > cg) {
            const F l = Ls[cl][cg];
#pragma unroll
            for (int ii = 0; ii < R; ++ii) x[ii][j2] -= xs[ii] * l;
          }
        }
      }
#pragma unroll
      for (int ii = 0; ii < R; ++ii)
#pragma unroll
        for (int j2 = 0; j2 < R; ++j2) U[w][R * bi + ii][R * h + j2] = x[ii][j2];
      if (w < 7) named_arrive(1 + w, 32 * (8 - w));
    } else if (warp > w) {
      named_sync(1 + w, 32 * (8 - w));
      F ux[R][W], lc[R][W];
#pragma unroll
      for (int ii = 0; ii < R; ++ii)
#pragma unroll
        for (int k = 0; k < W; ++k) {
          ux[ii][k] = U[w][R * bi + ii][k];
          lc[ii][k] = Ls[R * bj + ii][c0 + k];
        }
#pragma unroll
      for (int ii = 0; ii < R; ++ii)
#pragma unroll
        for (int jj = 0; jj < R; ++jj) {
          F s = F(0);
#pragma unroll
          for (int k = 0; k < W; ++k) s += ux[ii][k] * lc[jj][k];
          x[ii][jj] -= s;
        }
    }
  }
}

template <typename F, int T>
__global__ void __launch_bounds__(256) k_chol_panel(F* L, DevProblem P, const int2* items, int kt,
                                                    int* fail_flags, int* boosted) {
  constexpr int R = T / 16;
  __shared__ F Ls[T][T + 1];
  __shared__ __align__(16) F U[8][T][T / 8];
  __shared__ F piv[T];
  __shared__ F tab[2 * T];
  const int2 it = items[blockIdx.x];
  const int k = it.x, i = it.y;
  const int np = P.cluster_np[k], nk = P.cluster_n[k];
  F* A = L + P.S_off[k];
  const int bj = threadIdx.x >> 4, bi = threadIdx.x & 15;
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
  factor_tile_regs<F, T>(a, U, piv, tab, kt * T, nk, fail_flags + k, (i == kt) ? boosted : nullptr);
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
  trsm_tile_regs<F, T>(x, Ls, tab, U);
#pragma unroll
  for (int ii = 0; ii < R; ++ii)
#pragma unroll
    for (int jj = 0; jj < R; ++jj) A[base_ik + (size_t)(bi * R + ii) * np + bj * R + jj] = x[ii][jj];
}

// Inverse of every diagonal tile of the factor (for the solves), one CTA per tile: L Y = I column by
// column, four threads per column splitting each dot product.
template <typename F, int T>
__global__ void __launch_bounds__(256) k_diag_inverse(const F* L, F* Dinv, DevProblem P, const int2* items,
                                                      int64_t v_total) {
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
  F* DiT = Di + v_total * T;   // transposed copy in the second half of the buffer
  for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
    const int r = idx / T, c = idx - (idx / T) * T;
    Di[idx] = Y[r][c];
    DiT[idx] = Y[c][r];
  }
}

// R consecutive elements from 16-byte aligned shared memory in one vector load where the width allows.
template <typename F, int R>
__device__ __forceinline__ void load_vec(const F* p, F (&v)[R]) {
  if constexpr (sizeof(F) == 4 && R == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  } else if constexpr (sizeof(F) == 8 && R == 2) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    v[0] = t.x;
    v[1] = t.y;
  } else {
#pragma unroll
    for (int a = 0; a < R; ++a) v[a] = p[a];
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
    load_vec<F, R>(&LiT[kk][tr * R], av);
    load_vec<F, R>(&LjT[kk][tc * R], bv);
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

// x := D^-1/2 (L L^T)^-1 D^-1/2 rhs  (accumulate = 0) or x += ... (accumulate = 1).
// One thread-block cluster of CS CTAs per camera cluster.  Each CTA keeps the whole vector in shared
// memory; at tile step `it` CTA `rank` forms the partial product of the tiles it owns (tile columns j <
// it with j = rank mod CS for the forward pass, tile rows j > it for the backward pass), the partials are
// exchanged through distributed shared memory after one cluster barrier, and every CTA applies the stored
// inverse of the diagonal tile redundantly, so the next step needs no further synchronisation.
constexpr int SOLVE_CS = 8;

// out[r] = sum_c M[r][c] v[c] for a T x T row-major tile M (global) and v in shared memory; 256 threads,
// 256 / T threads per row, each a contiguous slice of the row.
template <typename F, int T>
__device__ __forceinline__ void tile_matvec(const F* __restrict__ M, const F* v, F* out) {
  constexpr int PARTS = 256 / T, LEN = T / PARTS;
  const int r = threadIdx.x / PARTS, part = threadIdx.x - (threadIdx.x / PARTS) * PARTS;
  const F* row = M + (size_t)r * T + part * LEN;
  F s = F(0);
#pragma unroll
  for (int c = 0; c < LEN; ++c) s += __ldg(row + c) * v[part * LEN + c];
#pragma unroll
  for (int d = PARTS / 2; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
  if (part == 0) out[r] = s;
}

template <typename F, int T, typename Rreal>
__global__ void __launch_bounds__(256) k_tri_solve(DevProblem P, const F* L, const F* Dinv, const double* scale,
                                                   const Rreal* rhs, double* x, int accumulate, int64_t v_total) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  F* y = reinterpret_cast<F*>(smem_raw);
  __shared__ F partial[2][T];
  __shared__ F t[T];
  __shared__ F part8[8][T];
  const int rank = (int)cluster.block_rank();
  const int k = blockIdx.x / SOLVE_CS;
  const int np = P.cluster_np[k];
  const F* A = L + P.S_off[k];
  const F* Di = Dinv + (size_t)P.v_off[k] * T;
  const double* sk = scale + P.v_off[k];
  const Rreal* rk = rhs + P.v_off[k];
  double* xk = x + P.v_off[k];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nt = np / T;
  constexpr int RW = T / 8;   // rows per warp within a tile
  for (int i = threadIdx.x; i < np; i += blockDim.x) y[i] = (F)((double)rk[i] * sk[i]);
  __syncthreads();
  int step = 0;
  // forward: L y = s o rhs
  for (int it = 0; it < nt; ++it, ++step) {
    const int r0 = it * T;
    F acc[RW];
#pragma unroll
    for (int q = 0; q < RW; ++q) acc[q] = F(0);
    for (int j = rank; j < it; j += SOLVE_CS) {
      const F* blk = A + (size_t)(r0 + warp * RW) * np + j * T;
#pragma unroll
      for (int cc = 0; cc < T; cc += 32) {
        const F yc = y[j * T + cc + lane];
#pragma unroll
        for (int q = 0; q < RW; ++q) acc[q] += blk[(size_t)q * np + cc + lane] * yc;
      }
    }
#pragma unroll
    for (int q = 0; q < RW; ++q) {
      const F s = warp_sum(acc[q]);
      if (lane == 0) partial[step & 1][warp * RW + q] = s;
    }
    cluster.sync();
    for (int r = threadIdx.x; r < T; r += blockDim.x) {
      F s = F(0);
#pragma unroll
      for (int c = 0; c < SOLVE_CS; ++c) s += cluster.map_shared_rank(&partial[step & 1][0], c)[r];
      t[r] = y[r0 + r] - s;
    }
    __syncthreads();
    tile_matvec<F, T>(Di + (size_t)it * T * T, t, y + r0);
    __syncthreads();
  }
  // backward: L^T z = y
  for (int it = nt - 1; it >= 0; --it, ++step) {
    const int r0 = it * T;
    constexpr int NC = T / 32;
    F p[NC];
#pragma unroll
    for (int u = 0; u < NC; ++u) p[u] = F(0);
    for (int j = it + 1 + rank; j < nt; j += SOLVE_CS) {
      const F* blk = A + (size_t)(j * T) * np + r0;
#pragma unroll 4
      for (int rr = warp; rr < T; rr += 8) {
        const F zc = y[j * T + rr];
#pragma unroll
        for (int u = 0; u < NC; ++u) p[u] += blk[(size_t)rr * np + lane + 32 * u] * zc;
      }
    }
#pragma unroll
    for (int u = 0; u < NC; ++u) part8[warp][lane + 32 * u] = p[u];
    __syncthreads();
    for (int cc = threadIdx.x; cc < T; cc += blockDim.x) {
      F s = F(0);
#pragma unroll
      for (int w = 0; w < 8; ++w) s += part8[w][cc];
      partial[step & 1][cc] = s;
    }
    cluster.sync();
    for (int r = threadIdx.x; r < T; r += blockDim.x) {
      F s = F(0);
#pragma unroll
      for (int c = 0; c < SOLVE_CS; ++c) s += cluster.map_shared_rank(&partial[step & 1][0], c)[r];
      t[r] = y[r0 + r] - s;
    }
    __syncthreads();
    // z_tile = Dinv^T t through the stored transpose
    tile_matvec<F, T>(Di + v_total * T + (size_t)it * T * T, t, y + r0);
    __syncthreads();
  }
  if (rank == 0)
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
      const double v = (double)y[i] * sk[i];
      xk[i] = accumulate ? xk[i] + v : v;
    }
  cluster.sync();   // keep this CTA's shared memory alive until every peer has read it
}

template <typename F, int T, typename Rreal>
void launch_tri_solve(const DevProblem& P, const F* L, const F* Dinv, const double* scale, const Rreal* rhs,
                      double* x, int accumulate, int max_np, int64_t v_total, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P.l * SOLVE_CS);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = sizeof(F) * (size_t)max_np;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = SOLVE_CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_tri_solve<F, T, Rreal>, P, L, Dinv, scale, rhs, x, accumulate, v_total);
}

// r = b - S x (FP64) with S symmetric, lower triangle stored; r was set to b before.  One CTA per
// (cluster, 32-row tile row I); its 4 warps take the tiles (I, J), J <= I, in turn.  A warp stages the
// 32 x 32 tile in shared memory with coalesced row loads, then lane l forms both the row sum of tile row l
// (S_IJ x_J, kept in registers over the warp's tiles) and the column sum of tile column l (S_IJ^T x_I,
// added atomically to r_J; on the diagonal tile only below the diagonal).
constexpr int RES_WARPS = 4;

template <typename Sreal>
__global__ void __launch_bounds__(32 * RES_WARPS) k_residual(DevProblem P, const Sreal* S, const double* x,
                                                             double* r, const int2* items) {
  __shared__ double T[RES_WARPS][32][33];
  __shared__ double xs[RES_WARPS][32];
  __shared__ double xi[32];
  __shared__ double red[RES_WARPS][32];
  const int2 it = items[blockIdx.x];
  const int k = it.x, I = it.y;
  const int np = P.cluster_np[k], nk = P.cluster_n[k];
  const Sreal* Sk = S + P.S_off[k];
  const double* xk = x + P.v_off[k];
  double* rk = r + P.v_off[k];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = 32 * I;
  if (warp == 0) xi[lane] = (i0 + lane < nk) ? xk[i0 + lane] : 0.0;
  __syncthreads();
  double rowacc = 0.0;
  for (int J = warp; J <= I; J += RES_WARPS) {
    const int j0 = 32 * J;
    const int col = j0 + lane;
    for (int rr = 0; rr < 32; ++rr) {
      const int row = i0 + rr;
      T[warp][rr][lane] = (row < nk && col < nk && col <= row) ? (double)Sk[(size_t)row * np + col] : 0.0;
    }
    xs[warp][lane] = (col < nk) ? xk[col] : 0.0;
    __syncwarp();
    double rs = 0.0, cs = 0.0;
#pragma unroll 8
    for (int c = 0; c < 32; ++c) rs += T[warp][lane][c] * xs[warp][c];
    if (J < I) {
#pragma unroll 8
      for (int rr = 0; rr < 32; ++rr) cs += T[warp][rr][lane] * xi[rr];
    } else {
      for (int rr = lane + 1; rr < 32; ++rr) cs += T[warp][rr][lane] * xi[rr];
    }
    rowacc += rs;
    if (col < nk && cs != 0.0) atomicAdd(rk + col, -cs);
    __syncwarp();
  }
  red[warp][lane] = rowacc;
  __syncthreads();
  if (warp == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < RES_WARPS; ++w) t += red[w][lane];
    if (i0 + lane < nk) atomicAdd(rk + i0 + lane, -t);
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
  if (plan.n_diag_items > 0)
    k_diag_inverse<F, T><<<plan.n_diag_items, 256, 0, stream>>>(L, Dinv, P, plan.diag_items, fb.v_total);
}

template <typename F>
void launch_solve(const DevProblem& P, const double* S, const double* b, const FactorBuffers& fb,
                  const CholPlan& plan, int refine_steps, double* dc, cudaStream_t stream) {
  using Sreal = double;
  constexpr int T = FactorCfg<F>::T;
  const F* L = reinterpret_cast<const F*>(fb.L);
  const F* Dinv = reinterpret_cast<const F*>(fb.Dinv);
  launch_tri_solve<F, T, Sreal>(P, L, Dinv, fb.scale, b, fb.x, 0, plan.max_np, fb.v_total, stream);
  const int nblk = (int)std::min<int64_t>(fb.v_total / 256 + 1, 152 * 8);
  for (int s = 0; s < refine_steps; ++s) {
    k_copy_vec<Sreal><<<nblk, 256, 0, stream>>>(b, fb.r, fb.v_total);
    if (plan.n_res_items > 0)
      k_residual<Sreal><<<plan.n_res_items, 32 * RES_WARPS, 0, stream>>>(P, S, fb.x, fb.r, plan.res_items);
    launch_tri_solve<F, T, double>(P, L, Dinv, fb.scale, fb.r, fb.x, 1, plan.max_np, fb.v_total, stream);
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
