// Batched dense LL^T factorisation and solve of the per-cluster systems S'_k dc_k = b_k (Eq. 13; the
// paper solves them with dense LL^T, Sec. 5.1), for clusters of uneven size, one launch per step.
//
// Storage: cluster k owns an Np_k x Np_k row-major block (Np_k = 9 n_k rounded up to the tile T) whose
// lower triangle is significant.  Padding rows and columns are zero and their diagonal is treated as 1,
// so the padded system is block diagonal with an identity block and solves to zero there.
//
// The factorised matrix is the Jacobi-scaled  S~ = D^-1/2 S D^-1/2, D = diag(S) (s_i = S_ii^-1/2), so that
// S x = b becomes S~ z = s o b, x = s o z.  Right-looking tiled algorithm with a look-ahead of one column,
// step kt:
//   panel   for every tile row i >= kt: apply step kt - 1's update to tiles (kt, kt) and (i, kt), factor
//           the diagonal tile with its inverse (redundantly in each CTA); the CTA of i = kt stores
//           L_kt,kt and L_kt,kt^-1 (for the solves), the others L_i,kt = A_i,kt L_kt,kt^-T;
//   update  for every kt + 1 < j <= i: A_i,j -= L_i,kt L_j,kt^T, on a second stream, overlapping the
//           next panel.
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

#include <map>
#include <mutex>

#include "stba_internal.cuh"
#include "stba_tc.cuh"

namespace stba {

#define FULL_MASK 0xffffffffu

// default tile of the factorisation: 64 for the FP32 factor (32 is the other candidate of stba_autotune),
// 32 for the FP64 factor
int factor_tile(bool mixed) { return mixed ? 64 : 32; }

// s_i = 1 / sqrt(S_ii) (1 on padding)
template <typename Sreal>
__global__ void k_diag_scale(DevProblem P, const Sreal* S, double* scale) {
  const int k = blockIdx.y;
  if (P.sharded && !P.cluster_owned[k]) return;
  const int np = P.cluster_np[k], nk = P.cluster_n[k];
  const Sreal* Sk = S + P.S_off[k];
  double* sk = scale + P.v_off[k];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
    double d = i < nk ? (double)Sk[(size_t)i * np + i] : 1.0;
    sk[i] = d > 0.0 ? 1.0 / sqrt(d) : 1.0;
  }
}

// L = s_i s_j S_ij (lower triangle and diagonal blocks' contents; the upper part is never read), for the
// columns [c_lo, c_hi) of the lower triangle (rows from c_lo on)
template <typename Sreal, typename F>
__global__ void k_scaled_copy(DevProblem P, const Sreal* S, const double* scale, F* L, int c_lo, int c_hi) {
  const int k = blockIdx.y;
  if (P.sharded && !P.cluster_owned[k]) return;
  const int np = P.cluster_np[k];
  const Sreal* Sk = S + P.S_off[k];
  F* Lk = L + P.S_off[k];
  const double* sk = scale + P.v_off[k];
  for (int r = c_lo + blockIdx.x; r < np; r += gridDim.x) {
    const double sr = sk[r];
    const int ce = min(r, c_hi - 1);
    for (int c = c_lo + threadIdx.x; c <= ce; c += blockDim.x)
      Lk[(size_t)r * np + c] = (F)((double)Sk[(size_t)r * np + c] * sr * sk[c]);
  }
}

// Correctly rounded reciprocal (one special-function instruction plus fix-up instead of a division).
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }

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

// Asynchronous global -> shared copies of one element (4 or 8 bytes), so that all the loads of a tile are
// in flight at once and may land at transposed positions.
template <typename F>
__device__ __forceinline__ void cp_async_elem(F* smem_dst, const F* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  if constexpr (sizeof(F) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}
// one 16-byte asynchronous global -> shared copy (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}

__device__ __forceinline__ float rsqrt_w(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_w(double x) { return rsqrt(x); }

// LL^T of the 8 x 8 diagonal block at (b0, b0) of a shared-memory tile, by one thread in registers; the
// reciprocal pivots go to rinv.  Pivot rules: padding rows (global row >= nk) get 1; FP64 -- a pivot that is
// not positive and finite fails the cluster; FP32 -- a non-finite pivot fails it, and a pivot that
// rounding made vanish (< 2^-20 of the unit scaled diagonal) is raised to 2^-12 and counted (static
// pivoting; the FP64 refinement solves the unmodified system).
template <typename F, int LDA>
__device__ __forceinline__ void chol8(F (*Ad)[LDA], int b0, int row0, int nk, F* rinv, int* fail, int* boosted) {
  F d[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) d[r][c] = (c <= r) ? Ad[b0 + r][b0 + c] : F(0);
  int bad = 0, nboost = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    F pv = d[j][j];
    if (row0 + b0 + j >= nk) {
      pv = F(1);
    } else if (!isfinite(pv)) {
      bad = 1;
      pv = F(1);
    } else if (sizeof(F) == 8) {
      if (!(pv > F(0))) {
        bad = 1;
        pv = F(1);
      }
    } else if (pv < F(1.0 / 1048576)) {
      ++nboost;
      pv = F(1.0 / 4096);
    }
    const F is = rsqrt_w(pv);
    d[j][j] = pv * is;
    rinv[j] = is;
#pragma unroll
    for (int r = j + 1; r < 8; ++r) d[r][j] *= is;
#pragma unroll
    for (int c = j + 1; c < 8; ++c)
#pragma unroll
      for (int r = c; r < 8; ++r) d[r][c] -= d[r][j] * d[c][j];
  }
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c <= r; ++c) Ad[b0 + r][b0 + c] = d[r][c];
  if (bad) *fail = 1;
  if (nboost && boosted) atomicAdd(boosted, nboost);
}

// ------------------------------------------------------------------------------------------------------
// Panel of tile step kt, one CTA per tile row i >= kt of a cluster (512 threads: the diagonal tile's work on
// threads 0..255, the row tile's on threads 256..511, wherever the two are independent):
//   1. fused update from step kt - 1 (kt > 0):  A_kt,kt -= L_kt,kt-1 L_kt,kt-1^T,  A_i,kt -= L_i,kt-1 L_kt,kt-1^T
//      (the trailing update of the other tiles of step kt - 1 runs concurrently in k_chol_update);
//   2. LL^T of the stacked panel [A_kt,kt; A_i,kt] in blocks of 8 columns (the diagonal tile redundantly
//      in every CTA of the step): per block one thread factors the 8 x 8 diagonal block, the block
//      column below is solved against it row by row (forward substitution), and the columns to its
//      right get the rank-8 update; rows of A_i,kt are just more rows below the diagonal, so they come
//      out as L_i,kt.  The CTA of i = kt stores L_kt,kt, the others L_i,kt.
// Dynamic shared memory: Ad, Ax (T x (T + 1)) and two T x LDV buffers for the transposed tiles of the
// fused update.
constexpr int PANEL_THREADS = 512;

template <typename F, int T>
struct PanelLayout {
  static constexpr int LDA = T + 1;
  static constexpr int LDV = T + (sizeof(F) == 4 ? 4 : 2);   // 16-byte rows for vector loads
  static constexpr size_t bytes = sizeof(F) * (2 * (size_t)T * LDA + 2 * (size_t)T * LDV);
};

template <typename F, int T>
__global__ void __launch_bounds__(PANEL_THREADS) k_chol_panel(F* L, F* Ldiag, DevProblem P, const int2* items, int kt,
                                                    int* fail_flags, int* boosted) {
  using PL = PanelLayout<F, T>;
  constexpr int R = T / 16, LDA = PL::LDA, LDV = PL::LDV, NB = T / 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  F(*Ad)[LDA] = reinterpret_cast<F(*)[LDA]>(smem_raw);
  F(*Ax)[LDA] = Ad + T;
  F* bufV = reinterpret_cast<F*>(Ax + T);
  F(*LkT)[LDV] = reinterpret_cast<F(*)[LDV]>(bufV);
  F(*LiT)[LDV] = LkT + T;
  __shared__ F rinv2[2][8];   // reciprocal pivots of block b in rinv2[b & 1]
  const int2 it = items[blockIdx.x];
  const int k = it.x, i = it.y;
  const bool diag = (i == kt);
  const int np = P.cluster_np[k], nk = P.cluster_n[k];
  F* A = L + P.S_off[k];
  const int tid = threadIdx.x;
  // fused update: threads 0..255 form the diagonal tile's product, threads 256..511 the row tile's
  const int half = tid >> 8, bi = tid & 15, bj = (tid & 255) >> 4;
  const size_t base_kk = (size_t)(kt * T) * np + kt * T;
  const size_t base_ik = (size_t)(i * T) * np + kt * T;
  // 1. loads; the upper part of the diagonal tile is never stored, so it is set to zero
  for (int idx = tid; idx < T * T; idx += PANEL_THREADS) {
    const int r = idx / T, c = idx - (idx / T) * T;
    if (c <= r)
      cp_async_elem(&Ad[r][c], A + base_kk + (size_t)r * np + c);
    else
      Ad[r][c] = F(0);
    if (!diag) cp_async_elem(&Ax[r][c], A + base_ik + (size_t)r * np + c);
    if (kt > 0) {
      cp_async_elem(&LkT[c][r], A + base_kk - T + (size_t)r * np + c);
      if (!diag) cp_async_elem(&LiT[c][r], A + base_ik - T + (size_t)r * np + c);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  if (kt > 0) {
    // half 0: A_kt,kt -= L_kt,kt-1 L_kt,kt-1^T (lower part); half 1: A_i,kt -= L_i,kt-1 L_kt,kt-1^T
    if (half == 0 || !diag) {
      F acc[R][R];
#pragma unroll
      for (int a = 0; a < R; ++a)
#pragma unroll
        for (int b = 0; b < R; ++b) acc[a][b] = F(0);
      F(*Lr)[LDV] = half ? LiT : LkT;
#pragma unroll 4
      for (int m = 0; m < T; ++m) {
        F lr[R], lc[R];
        load_vec<F, R>(&Lr[m][bi * R], lr);
        load_vec<F, R>(&LkT[m][bj * R], lc);
#pragma unroll
        for (int a = 0; a < R; ++a)
#pragma unroll
          for (int b = 0; b < R; ++b) acc[a][b] += lr[a] * lc[b];
      }
#pragma unroll
      for (int a = 0; a < R; ++a)
#pragma unroll
        for (int b = 0; b < R; ++b) {
          const int r = bi * R + a, c = bj * R + b;
          if (half)
            Ax[r][c] -= acc[a][b];
          else if (c <= r)
            Ad[r][c] -= acc[a][b];
        }
    }
    __syncthreads();
  }
  // 2. blocked LL^T of the stacked panel.  Per block b: the rows below are solved against L_bb; then warp 0
  //    applies block b's rank-8 update to the next 8 x 8 diagonal block and lane 0 factors it, while warps
  //    1..7 apply the update to the rest of the diagonal tile and warps 8..15 to the row tile (look-ahead
  //    of one block).
  if (tid == 0) chol8<F, LDA>(Ad, 0, kt * T, nk, rinv2[0], fail_flags + k, diag ? boosted : nullptr);
  __syncthreads();
  for (int b = 0; b < NB; ++b) {
    const int b0 = 8 * b;
    const F* rinv = rinv2[b & 1];
    // block column below the diagonal block: L_rb L_bb^T = A_rb, one row per thread (Ad rows, then Ax rows)
    const int rows_d = T - b0 - 8;
    const int rows_tot = rows_d + (diag ? 0 : T);
    if (tid < rows_tot) {
      F* row = (tid < rows_d) ? &Ad[b0 + 8 + tid][0] : &Ax[tid - rows_d][0];
      F o8[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        F s = row[b0 + c];
#pragma unroll
        for (int t = 0; t < c; ++t) s -= o8[t] * Ad[b0 + c][b0 + t];
        o8[c] = s * rinv[c];
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) row[b0 + c] = o8[c];
    }
    __syncthreads();
    if (b + 1 == NB) break;
    const int n0 = b0 + 8;   // first column of the next block
    if (tid < 32) {
      // next diagonal block: entries (r, c), n0 <= c <= r < n0 + 8 (36 of them)
      for (int e = tid; e < 36; e += 32) {
        int rr = 0;
        while ((rr + 1) * (rr + 2) / 2 <= e) ++rr;
        const int cc = e - rr * (rr + 1) / 2;
        F s = F(0);
#pragma unroll
        for (int t = 0; t < 8; ++t) s += Ad[n0 + rr][b0 + t] * Ad[n0 + cc][b0 + t];
        Ad[n0 + rr][n0 + cc] -= s;
      }
      __syncwarp();
      if (tid == 0) chol8<F, LDA>(Ad, n0, kt * T, nk, rinv2[(b + 1) & 1], fail_flags + k, diag ? boosted : nullptr);
    } else {
      // rank-8 update of the other columns right of the block, register-blocked R x R cells: warps 1..7
      // take the diagonal tile's cells, warps 8..15 the row tile's
      const bool xpart = tid >= 256;
      for (int cell = xpart ? tid - 256 : tid - 32; cell < 256; cell += xpart ? 256 : 224) {
        const int ci = cell & 15, cj = cell >> 4;
        const int c0 = cj * R, r0 = ci * R;
        if (c0 + R <= n0 || (xpart && diag)) continue;
        F lc[R][8];
#pragma unroll
        for (int cc = 0; cc < R; ++cc)
#pragma unroll
          for (int t = 0; t < 8; ++t) lc[cc][t] = Ad[c0 + cc][b0 + t];
        if (!xpart && cj <= ci && r0 + R > n0) {
#pragma unroll
          for (int a = 0; a < R; ++a) {
            F lr[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) lr[t] = Ad[r0 + a][b0 + t];
#pragma unroll
            for (int cc = 0; cc < R; ++cc) {
              const int r = r0 + a, c = c0 + cc;
              if (c <= r && c >= n0 && r >= n0 + 8) {
                F s = F(0);
#pragma unroll
                for (int t = 0; t < 8; ++t) s += lr[t] * lc[cc][t];
                Ad[r][c] -= s;
              }
            }
          }
        }
        if (xpart) {
#pragma unroll
          for (int a = 0; a < R; ++a) {
            F xr[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) xr[t] = Ax[r0 + a][b0 + t];
#pragma unroll
            for (int cc = 0; cc < R; ++cc) {
              const int c = c0 + cc;
              if (c >= n0) {
                F s = F(0);
#pragma unroll
                for (int t = 0; t < 8; ++t) s += xr[t] * lc[cc][t];
                Ax[r0 + a][c] -= s;
              }
            }
          }
        }
      }
    }
    __syncthreads();
  }
  // 3. outputs.  L_kk goes to its own buffer: later CTAs of this step may still be loading A_kk from L.
  if (diag) {
    F* Lkk = Ldiag + (size_t)P.v_off[k] * T + (size_t)kt * T * T;
    for (int idx = tid; idx < T * T; idx += PANEL_THREADS) {
      const int r = idx / T, c = idx - (idx / T) * T;
      Lkk[idx] = (c <= r) ? Ad[r][c] : F(0);
    }
    return;
  }
  for (int idx = tid; idx < T * T; idx += PANEL_THREADS) {
    const int r = idx / T, c = idx - (idx / T) * T;
    A[base_ik + (size_t)r * np + c] = Ax[r][c];
  }
}

// Inverse Y of a lower-triangular T x T tile D in shared memory (Y zeroed, D's upper part zero, both visible
// to every thread), by recursive doubling, 256 threads: the inverses of the 8 x 8 diagonal blocks by forward
// substitution (8 threads per block), then for h = 8, 16, .. T/2 the off-diagonal block of every 2h x 2h
// diagonal block, Y21 = -Y22 (L21 Y11), as two parallel products (Z: T * T / 2 scratch).  Ends synchronised.
template <typename F, int T>
__device__ __forceinline__ void tile_inverse(const F (*D)[T + 1], F (*Y)[T + 1], F* Z) {
  const int tid = threadIdx.x;
  if (tid < T) {   // column j of the inverse of diagonal block blk
    const int blk = tid >> 3, j = tid & 7, b0 = 8 * blk;
    F y[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      F s = (r == j) ? F(1) : F(0);
#pragma unroll
      for (int m = 0; m < r; ++m) s -= D[b0 + r][b0 + m] * y[m];
      y[r] = (r < j) ? F(0) : s / D[b0 + r][b0 + r];
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) Y[b0 + r][b0 + j] = y[r];
  }
  __syncthreads();
  for (int h = 8; h < T; h *= 2) {
    const int n_out = T * h / 2;   // (T / 2h) pairs x h x h
    for (int e = tid; e < n_out; e += 256) {
      const int p = e / (h * h), rr = (e / h) % h, cc = e % h;
      const int r2 = (2 * p + 1) * h + rr, c1 = 2 * p * h + cc;
      F s = F(0);
      for (int q = cc; q < h; ++q) s += D[r2][2 * p * h + q] * Y[2 * p * h + q][c1];
      Z[e] = s;   // (L21 Y11)[rr][cc]
    }
    __syncthreads();
    for (int e = tid; e < n_out; e += 256) {
      const int p = e / (h * h), rr = (e / h) % h, cc = e % h;
      const int r2 = (2 * p + 1) * h + rr, c1 = 2 * p * h + cc;
      F s = F(0);
      for (int q = 0; q <= rr; ++q) s += Y[r2][(2 * p + 1) * h + q] * Z[p * h * h + q * h + cc];
      Y[r2][c1] = -s;
    }
    __syncthreads();
  }
}

// Inverse Y of every diagonal tile of the factor (for the solves), one CTA per tile (tile_inverse).  Writes
// Y row-major and its transpose at offset v_total * T.
template <typename F, int T>
__global__ void __launch_bounds__(256) k_diag_inverse(const F* Ldiag, F* Dinv, DevProblem P, const int2* items,
                                                      int64_t v_total) {
  __shared__ F D[T][T + 1];
  __shared__ F Y[T][T + 1];
  __shared__ F Z[T * T / 2];
  const int2 it = items[blockIdx.x];
  const int k = it.x, t = it.y;
  const F* Lkk = Ldiag + (size_t)P.v_off[k] * T + (size_t)t * T * T;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < T * T; idx += 256) {
    const int r = idx / T, c = idx - (idx / T) * T;
    D[r][c] = (c <= r) ? Lkk[idx] : F(0);
    Y[r][c] = F(0);
  }
  __syncthreads();
  tile_inverse<F, T>(D, Y, Z);
  F* Di = Dinv + (size_t)P.v_off[k] * T + (size_t)t * T * T;
  F* DiT = Di + v_total * T;
  for (int idx = tid; idx < T * T; idx += 256) {
    const int r = idx / T, c = idx - (idx / T) * T;
    Di[idx] = Y[r][c];
    DiT[idx] = Y[c][r];
  }
}

// ------------------------------------------------------------------------------------------------------
// Split panel of tile step kt (the FP32 factor with T = 64): the diagonal tile is factored once per cluster,
// the tiles below it by a product with its inverse, so that a step's critical path is two short kernels.
//
// k_chol_diag, one CTA per cluster with a tile step kt:  A_kt,kt -= L_kt,kt-1 L_kt,kt-1^T (step kt - 1's
// update of the diagonal tile), LL^T of the tile in blocks of 8 columns (as the panel, 64 rows), and its
// inverse Y = L_kt,kt^-1 (tile_inverse), written to Dinv (row-major) and its transpose (for the solves and
// for k_chol_trsm).  Pivot rules as in chol8.
// LL^T of a T x T diagonal tile Ad (lower part; upper part zero) in shared memory, in place, 256 threads, in
// blocks of 8 columns: per block one thread factors the 8 x 8 diagonal block (chol8), the rows below are
// solved against it, and the columns to its right get the rank-8 update, warp 0 updating and factoring the
// next diagonal block meanwhile (one block of look-ahead).  row0: global row of the tile's first row (pivot
// rules of chol8 for padding rows); fail, boosted as in chol8.  Ends synchronised.
template <typename F, int T>
__device__ __forceinline__ void factor_diag_tile(F (*Ad)[T + 1], F (*rinv2)[8], int row0, int nk, int* fail,
                                                 int* boosted) {
  constexpr int R = T / 16, LDA = T + 1, NB = T / 8;
  const int tid = threadIdx.x;
  if (tid == 0) chol8<F, LDA>(Ad, 0, row0, nk, rinv2[0], fail, boosted);
  __syncthreads();
  for (int b = 0; b < NB; ++b) {
    const int b0 = 8 * b;
    const F* rinv = rinv2[b & 1];
    const int rows_d = T - b0 - 8;
    if (tid < rows_d) {
      F* row = &Ad[b0 + 8 + tid][0];
      F o8[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        F s = row[b0 + c];
#pragma unroll
        for (int t = 0; t < c; ++t) s -= o8[t] * Ad[b0 + c][b0 + t];
        o8[c] = s * rinv[c];
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) row[b0 + c] = o8[c];
    }
    __syncthreads();
    if (b + 1 == NB) break;
    const int n0 = b0 + 8;
    if (tid < 32) {
      for (int e = tid; e < 36; e += 32) {
        int rr = 0;
        while ((rr + 1) * (rr + 2) / 2 <= e) ++rr;
        const int cc = e - rr * (rr + 1) / 2;
        F s = F(0);
#pragma unroll
        for (int t = 0; t < 8; ++t) s += Ad[n0 + rr][b0 + t] * Ad[n0 + cc][b0 + t];
        Ad[n0 + rr][n0 + cc] -= s;
      }
      __syncwarp();
      if (tid == 0) chol8<F, LDA>(Ad, n0, row0, nk, rinv2[(b + 1) & 1], fail, boosted);
    } else {
      for (int cell = tid - 32; cell < 256; cell += 224) {
        const int ci = cell & 15, cj = cell >> 4;
        const int c0 = cj * R, r0 = ci * R;
        if (c0 + R <= n0 || cj > ci || r0 + R <= n0 + 8) continue;
        F lc[R][8];
#pragma unroll
        for (int cc = 0; cc < R; ++cc)
#pragma unroll
          for (int t = 0; t < 8; ++t) lc[cc][t] = Ad[c0 + cc][b0 + t];
#pragma unroll
        for (int a = 0; a < R; ++a) {
          F lr[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) lr[t] = Ad[r0 + a][b0 + t];
#pragma unroll
          for (int cc = 0; cc < R; ++cc) {
            const int r = r0 + a, c = c0 + cc;
            if (c <= r && c >= n0 && r >= n0 + 8) {
              F s = F(0);
#pragma unroll
              for (int t = 0; t < 8; ++t) s += lr[t] * lc[cc][t];
              Ad[r][c] -= s;
            }
          }
        }
      }
    }
    __syncthreads();
  }
}

template <typename F, int T>
struct DiagLayout {
  static constexpr int LDA = T + 1;
  static constexpr int LDV = T + (sizeof(F) == 4 ? 4 : 2);
  static constexpr size_t bytes = sizeof(F) * (2 * (size_t)T * LDA + (size_t)T * LDV + (size_t)T * T / 2);
};

template <typename F, int T>
__global__ void __launch_bounds__(256) k_chol_diag(const F* L, F* Dinv, DevProblem P, const int2* items, int kt,
                                                   int* fail_flags, int* boosted, int64_t v_total) {
  using DL = DiagLayout<F, T>;
  constexpr int R = T / 16, LDA = DL::LDA, LDV = DL::LDV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  F(*Ad)[LDA] = reinterpret_cast<F(*)[LDA]>(smem_raw);
  F(*Y)[LDA] = Ad + T;
  F(*LkT)[LDV] = reinterpret_cast<F(*)[LDV]>(Y + T);
  F* Z = reinterpret_cast<F*>(LkT + T);
  __shared__ F rinv2[2][8];
  const int k = items[blockIdx.x].x;
  const int np = P.cluster_np[k], nk = P.cluster_n[k];
  const F* A = L + P.S_off[k];
  const int tid = threadIdx.x;
  const int bi = tid & 15, bj = tid >> 4;
  const size_t base_kk = (size_t)(kt * T) * np + kt * T;
  for (int idx = tid; idx < T * T; idx += 256) {
    const int r = idx / T, c = idx - (idx / T) * T;
    if (c <= r)
      cp_async_elem(&Ad[r][c], A + base_kk + (size_t)r * np + c);
    else
      Ad[r][c] = F(0);
    Y[r][c] = F(0);
    if (kt > 0) cp_async_elem(&LkT[c][r], A + base_kk - T + (size_t)r * np + c);
  }
  cp_async_wait_all();
  __syncthreads();
  if (kt > 0) {   // A_kk -= L_k,kt-1 L_k,kt-1^T (lower part)
    F acc[R][R];
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int b = 0; b < R; ++b) acc[a][b] = F(0);
#pragma unroll 4
    for (int m = 0; m < T; ++m) {
      F lr[R], lc[R];
      load_vec<F, R>(&LkT[m][bi * R], lr);
      load_vec<F, R>(&LkT[m][bj * R], lc);
#pragma unroll
      for (int a = 0; a < R; ++a)
#pragma unroll
        for (int b = 0; b < R; ++b) acc[a][b] += lr[a] * lc[b];
    }
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int b = 0; b < R; ++b) {
        const int r = bi * R + a, c = bj * R + b;
        if (c <= r) Ad[r][c] -= acc[a][b];
      }
    __syncthreads();
  }
  factor_diag_tile<F, T>(Ad, rinv2, kt * T, nk, fail_flags + k, boosted);
  tile_inverse<F, T>(Ad, Y, Z);
  F* Di = Dinv + (size_t)P.v_off[k] * T + (size_t)kt * T * T;
  F* DiT = Di + v_total * T;
  for (int idx = tid; idx < T * T; idx += 256) {
    const int r = idx / T, c = idx - (idx / T) * T;
    Di[idx] = Y[r][c];
    DiT[idx] = Y[c][r];
  }
}

// k_chol_trsm, one CTA per tile row i > kt of a cluster with a tile step kt:
//   A_i,kt -= L_i,kt-1 L_kt,kt-1^T   (step kt - 1's update of the tile)
//   L_i,kt  = A_i,kt Y^T              (Y = L_kt,kt^-1 from k_chol_diag: the triangular solve as a product)
// both as 64 x 64 x 64 register-blocked products (4 x 4 per thread) over transposed shared-memory tiles.
template <typename F, int T>
struct TrsmLayout {
  static constexpr int LD = T + (sizeof(F) == 4 ? 4 : 2);
  static constexpr size_t bytes = sizeof(F) * 4 * (size_t)T * LD;
};

template <typename F, int T>
__global__ void __launch_bounds__(256) k_chol_trsm(F* L, const F* Dinv, DevProblem P, const int2* items, int kt,
                                                   int64_t v_total) {
  constexpr int R = T / 16, LD = TrsmLayout<F, T>::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  F(*AT)[LD] = reinterpret_cast<F(*)[LD]>(smem_raw);   // A_i,kt transposed
  F(*YT)[LD] = AT + T;                                   // Y^T (row m, column c = Y[c][m])
  F(*LiT)[LD] = YT + T;                                  // L_i,kt-1 transposed
  F(*LkT)[LD] = LiT + T;                                 // L_kt,kt-1 transposed
  const int2 it = items[blockIdx.x];
  const int k = it.x, i = it.y;
  const int np = P.cluster_np[k];
  F* A = L + P.S_off[k];
  const F* DiT = Dinv + v_total * T + (size_t)P.v_off[k] * T + (size_t)kt * T * T;
  const size_t base_ik = (size_t)(i * T) * np + kt * T, base_kk = (size_t)(kt * T) * np + kt * T;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < T * T; idx += 256) {
    const int r = idx / T, c = idx - (idx / T) * T;
    cp_async_elem(&AT[c][r], A + base_ik + (size_t)r * np + c);
    if (kt > 0) {
      cp_async_elem(&LiT[c][r], A + base_ik - T + (size_t)r * np + c);
      cp_async_elem(&LkT[c][r], A + base_kk - T + (size_t)r * np + c);
    }
  }
  {
    constexpr int CH = T * (int)sizeof(F) / 16;   // 16-byte chunks per row of Y^T
    for (int q = tid; q < T * CH; q += 256) {
      const int r = q / CH, c = q - (q / CH) * CH;
      cp_async16(&YT[r][c * (16 / (int)sizeof(F))], DiT + (size_t)r * T + c * (16 / (int)sizeof(F)));
    }
  }
  cp_async_wait_all();
  __syncthreads();
  const int tr = tid >> 4, tc = tid & 15;
  if (kt > 0) {
    F acc[R][R];
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int b = 0; b < R; ++b) acc[a][b] = F(0);
#pragma unroll 4
    for (int m = 0; m < T; ++m) {
      F av[R], bv[R];
      load_vec<F, R>(&LiT[m][tr * R], av);
      load_vec<F, R>(&LkT[m][tc * R], bv);
#pragma unroll
      for (int a = 0; a < R; ++a)
#pragma unroll
        for (int b = 0; b < R; ++b) acc[a][b] += av[a] * bv[b];
    }
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int b = 0; b < R; ++b) AT[tc * R + b][tr * R + a] -= acc[a][b];
    __syncthreads();
  }
  F acc[R][R];
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int b = 0; b < R; ++b) acc[a][b] = F(0);
#pragma unroll 4
  for (int m = 0; m < T; ++m) {
    F av[R], bv[R];
    load_vec<F, R>(&AT[m][tr * R], av);
    load_vec<F, R>(&YT[m][tc * R], bv);
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int b = 0; b < R; ++b) acc[a][b] += av[a] * bv[b];
  }
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int b = 0; b < R; ++b) A[base_ik + (size_t)(tr * R + a) * np + tc * R + b] = acc[a][b];
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
    cp_async_elem(&LiT[c][r], A + bi + (size_t)r * np + c);
    cp_async_elem(&LjT[c][r], A + bj + (size_t)r * np + c);
  }
  cp_async_wait_all();
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
// Trailing update on the fifth-generation tensor cores (FP32 factor, T = 64).  One CTA per item (k, i0, j)
// updates the two tiles (i0, j) and (i0 + 1, j) of cluster k:  [A_i0,j; A_i0+1,j] -= [L_i0,kt; L_i0+1,kt] L_j,kt^T,
// one 128 x 64 x 64 product D = A B^T by tcgen05.mma (kind::tf32, FP32 accumulation in tensor memory).
// FP32 accuracy from TF32 operands: every value x is split into hi = tf32(x) and lo = tf32(x - hi), and
// D = A_hi B_lo + A_lo B_hi + A_hi B_hi (3xTF32; the dropped A_lo B_lo is below FP32 rounding), 24 MMAs
// of K = 8 issued by one thread.  The operands are converted by all threads into the no-swizzle K-major
// core-matrix layout (stba_tc.cuh); while the MMAs run, each thread loads the 32 old values it will
// update (one row, 32 columns), then subtracts its 32 accumulator columns read from TMEM.  The wait for
// the MMAs is bounded: a CTA that gives up marks the cluster failed (the LM step is rejected), frees its
// tensor memory and returns.  When i0 + 1 is past the cluster's last tile, the second half of A is zero and
// its rows are not written.
constexpr int TCU_THREADS = 256;
constexpr size_t TCU_SMEM = sizeof(uint32_t) * (2 * 128 * 64 + 2 * 64 * 64);   // A hi/lo, B hi/lo: 96 KB
constexpr int TCU_MAX_POLLS = 1 << 26;

__device__ __forceinline__ void split_store(uint32_t* hi, uint32_t* lo, int off, float4 v) {
  const uint32_t h0 = tc::to_tf32(v.x), h1 = tc::to_tf32(v.y), h2 = tc::to_tf32(v.z), h3 = tc::to_tf32(v.w);
  *reinterpret_cast<uint4*>(hi + off) = make_uint4(h0, h1, h2, h3);
  *reinterpret_cast<uint4*>(lo + off) =
      make_uint4(tc::to_tf32(v.x - __uint_as_float(h0)), tc::to_tf32(v.y - __uint_as_float(h1)),
                 tc::to_tf32(v.z - __uint_as_float(h2)), tc::to_tf32(v.w - __uint_as_float(h3)));
}

__global__ void __launch_bounds__(TCU_THREADS, 2) k_chol_update_tc(float* L, DevProblem P, const int2* items, int kt,
                                                                  int* fail_flags) {
  constexpr int T = 64;
  extern __shared__ __align__(128) uint32_t tsm[];
  uint32_t* Ah = tsm;   // 128 x 64 TF32, core-matrix layout
  uint32_t* Al = tsm + 128 * 64;
  uint32_t* Bh = tsm + 2 * 128 * 64;   // 64 x 64
  uint32_t* Bl = Bh + 64 * 64;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t taddr_s;
  const int2 it = items[blockIdx.x];
  const int k = it.x, i0 = it.y >> 16, j = it.y & 0xffff;
  const int np = P.cluster_np[k];
  float* A = L + P.S_off[k];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rows_valid = min(128, np - i0 * T);   // 64 or 128
  const float* srcA = A + (size_t)(i0 * T) * np + kt * T;
  const float* srcB = A + (size_t)(j * T) * np + kt * T;
  // 16-byte chunk q = tid + 256 u: row (q >> 7) * 8 + (q & 7), columns 4 ((q >> 3) & 15) ..: the 8 threads of a
  // shared-memory store phase write one whole core matrix (no bank conflicts).  Every load of the thread (its
  // 12 operand chunks and the 32 old values it will update) is issued before any of them is used.
  const int R = 32 * (warp & 3) + lane, c0 = 32 * (warp >> 2);   // epilogue: row R, columns c0 .. c0 + 31
  const bool valid = R < rows_valid;
  float* dst = A + (size_t)(i0 * T + R) * np + j * T + c0;
  float4 va[8], vb[4], old[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int q = tid + TCU_THREADS * u;
    const int r = ((q >> 7) << 3) | (q & 7), kc = (q >> 3) & 15;
    va[u] = r < rows_valid ? *reinterpret_cast<const float4*>(srcA + (size_t)r * np + 4 * kc)
                           : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int q = tid + TCU_THREADS * u;
    const int r = ((q >> 7) << 3) | (q & 7), kc = (q >> 3) & 15;
    vb[u] = *reinterpret_cast<const float4*>(srcB + (size_t)r * np + 4 * kc);
  }
#pragma unroll
  for (int v = 0; v < 8; ++v) old[v] = valid ? *reinterpret_cast<const float4*>(dst + 4 * v) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int q = tid + TCU_THREADS * u;
    split_store(Ah, Al, tc::core_off<64>(((q >> 7) << 3) | (q & 7), 4 * ((q >> 3) & 15)), va[u]);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int q = tid + TCU_THREADS * u;
    split_store(Bh, Bl, tc::core_off<64>(((q >> 7) << 3) | (q & 7), 4 * ((q >> 3) & 15)), vb[u]);
  }
  tc::fence_async_smem();
  if (tid == 0) tc::mbar_init(&mbar, 1);
  if (warp == 0) tc::tmem_alloc(&taddr_s, 64);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = taddr_s;
  if (tid == 0) {
    constexpr uint32_t idesc = tc::idesc_tf32(128, 64);
    const uint32_t pa[3] = {tc::smem_u32(Ah), tc::smem_u32(Al), tc::smem_u32(Ah)};
    const uint32_t pb[3] = {tc::smem_u32(Bl), tc::smem_u32(Bh), tc::smem_u32(Bh)};
#pragma unroll
    for (int pass = 0; pass < 3; ++pass)
#pragma unroll
      for (int ks = 0; ks < 8; ++ks)
        tc::mma_tf32(tmem, tc::smem_desc(pa[pass] + ks * 256, 128, 2048), tc::smem_desc(pb[pass] + ks * 256, 128, 2048),
                     idesc, (pass | ks) != 0);
    tc::mma_commit(&mbar);
  }
  // thread (lane quarter warp & 3, column half warp >> 2): row R of the 128, columns c0 .. c0 + 31 of tile j
  const bool done = __all_sync(0xffffffffu, tc::mbar_wait_bounded(&mbar, 0, TCU_MAX_POLLS));
  if (done) {
    tc::fence_after_sync();
    float d[32];
    tc::tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0, d);
    if (valid) {
#pragma unroll
      for (int v = 0; v < 8; ++v)
        *reinterpret_cast<float4*>(dst + 4 * v) =
            make_float4(old[v].x - d[4 * v], old[v].y - d[4 * v + 1], old[v].z - d[4 * v + 2], old[v].w - d[4 * v + 3]);
    }
  } else if (lane == 0) {
    atomicExch(fail_flags + k, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 64);
}


// ------------------------------------------------------------------------------------------------------
// Persistent factorisation (FP32 factor, T = 64): one thread-block cluster of FCS CTAs per camera cluster
// runs every tile step of that cluster in one launch.  Tile (i, j) of the lower triangle belongs to CTA
// (i (i + 1) / 2 + j) mod FCS for the whole factorisation (round robin over the tiles, so every step's work
// spreads over the CTAs).  Step kt:
//   1. the owner of (kt, kt) factors the tile (factor_diag_tile; every update of it has been applied by the
//      same CTA) and inverts it (tile_inverse), writing Y = L_kt,kt^-1 and Y^T to Dinv for the solves;
//   2. cluster barrier; every CTA forms its tiles below the diagonal, L_i,kt = A_i,kt Y^T;
//   3. cluster barrier; every CTA applies A_i,j -= L_i,kt L_j,kt^T to its tiles kt < j <= i.
// Between CTAs only the finished column kt (after barrier 2) and Y (after barrier 1) travel, through L2: they
// are read with L1-bypassing loads, after a device-scope fence and the cluster barrier.  Every CTA runs the
// same number of barriers (2 per step).  Replaces the per-step panel / update launches and the separate
// inverses of the diagonal tiles.
constexpr int FCS = 8;

template <int T>
struct ClusterFactorLayout {
  static constexpr int LDA = T + 1;             // diagonal phase: Ad, Y [T][LDA], Z [T * T / 2]
  static constexpr int LD = T + 4;              // product phases: two [T][LD] tiles (16-byte rows)
  static constexpr size_t diag_bytes = sizeof(float) * (2 * (size_t)T * LDA + (size_t)T * T / 2);
  static constexpr size_t prod_bytes = sizeof(float) * 2 * (size_t)T * LD;
  static constexpr size_t bytes = diag_bytes > prod_bytes ? diag_bytes : prod_bytes;
};

__device__ __forceinline__ int factor_tile_owner(int i, int j) { return (i * (i + 1) / 2 + j) % FCS; }

// The 16-byte pieces of a T x T tile that thread t loads (T * T / 4 / 256 of them): piece u is row
// (t + 256 u) % T, columns 4 ((t + 256 u) / T) .. + 3.  Loads first (all in flight at once), stores after.
template <int T>
struct TilePieces {
  static constexpr int N = T * T / 4 / 256;
  float4 v[N];
};
template <int T, bool CG>
__device__ __forceinline__ void tile_pieces_load(TilePieces<T>& t, const float* src, size_t ld) {
#pragma unroll
  for (int u = 0; u < TilePieces<T>::N; ++u) {
    const int q = threadIdx.x + 256 * u, r = q % T, c4 = 4 * (q / T);
    const float4* p = reinterpret_cast<const float4*>(src + (size_t)r * ld + c4);
    t.v[u] = CG ? __ldcg(p) : *p;
  }
}
// dst[c][r] = tile[r][c] (consecutive threads write consecutive r: consecutive banks)
template <int T, int LD>
__device__ __forceinline__ void tile_pieces_store_transposed(float (*dst)[LD], const TilePieces<T>& t) {
#pragma unroll
  for (int u = 0; u < TilePieces<T>::N; ++u) {
    const int q = threadIdx.x + 256 * u, r = q % T, c4 = 4 * (q / T);
    dst[c4][r] = t.v[u].x;
    dst[c4 + 1][r] = t.v[u].y;
    dst[c4 + 2][r] = t.v[u].z;
    dst[c4 + 3][r] = t.v[u].w;
  }
}
// the R x R block (rows tr R + a, columns tc R ..) that the thread updates, as R 16-byte pieces
template <int T>
__device__ __forceinline__ void block_load(float4 (&b)[T / 16], const float* dst, size_t ld) {
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
#pragma unroll
  for (int a = 0; a < T / 16; ++a) b[a] = *reinterpret_cast<const float4*>(dst + (size_t)(tr * (T / 16) + a) * ld + tc * (T / 16));
}

// acc[a][b] = sum_m X[m][tr R + a] Y[m][tc R + b] over the T rows m of two transposed tiles
template <int T, int LD>
__device__ __forceinline__ void tile_product(const float (*X)[LD], const float (*Y)[LD], float (&acc)[T / 16][T / 16]) {
  constexpr int R = T / 16;
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int b = 0; b < R; ++b) acc[a][b] = 0.f;
#pragma unroll 4
  for (int m = 0; m < T; ++m) {
    float xv[R], yv[R];
    load_vec<float, R>(&X[m][tr * R], xv);
    load_vec<float, R>(&Y[m][tc * R], yv);
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int b = 0; b < R; ++b) acc[a][b] += xv[a] * yv[b];
  }
}

template <int T>
__global__ void __launch_bounds__(256) k_chol_cluster(float* L, float* Dinv, DevProblem P, const int* cluster_items,
                                                      int* fail_flags, int* boosted, int64_t v_total) {
  namespace cg = cooperative_groups;
  using CL = ClusterFactorLayout<T>;
  constexpr int R = T / 16, LDA = CL::LDA, LD = CL::LD;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float(*Ad)[LDA] = reinterpret_cast<float(*)[LDA]>(smem_raw);   // diagonal phase
  float(*Y)[LDA] = Ad + T;
  float* Z = reinterpret_cast<float*>(Y + T);
  float(*X1)[LD] = reinterpret_cast<float(*)[LD]>(smem_raw);   // product phases (alias the diagonal phase)
  float(*X2)[LD] = X1 + T;
  __shared__ float rinv2[2][8];
  const int rank = (int)cluster.block_rank();
  const int k = cluster_items[blockIdx.x / FCS];
  const int np = P.cluster_np[k], nk = P.cluster_n[k], nt = np / T;
  float* A = L + P.S_off[k];
  float* Di = Dinv + (size_t)P.v_off[k] * T;
  float* DiT = Di + v_total * T;
  const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
  auto tile = [&](int i, int j) { return A + (size_t)(i * T) * np + j * T; };
  // the diagonal tile kt and its inverse, by its owner (every update of the tile is this CTA's own)
  auto diagonal = [&](int kt) {
    const float* src = tile(kt, kt);
    for (int idx = tid; idx < T * T; idx += 256) {
      const int r = idx / T, c = idx - (idx / T) * T;
      Ad[r][c] = c <= r ? src[(size_t)r * np + c] : 0.f;
      Y[r][c] = 0.f;
    }
    __syncthreads();
    factor_diag_tile<float, T>(Ad, rinv2, kt * T, nk, fail_flags + k, boosted);
    tile_inverse<float, T>(Ad, Y, Z);
    float* d = Di + (size_t)kt * T * T;
    float* dT = DiT + (size_t)kt * T * T;
    for (int idx = tid; idx < T * T; idx += 256) {
      const int r = idx / T, c = idx - (idx / T) * T;
      d[idx] = Y[r][c];
      dT[idx] = Y[c][r];
    }
    __syncthreads();
  };
  if (factor_tile_owner(0, 0) == rank) diagonal(0);
  for (int kt = 0; kt < nt; ++kt) {
    // 1. the diagonal tile kt is factored: at the start (kt = 0) or, one step ahead, by its owner during the
    //    trailing update of step kt - 1 (look-ahead)
    __threadfence();
    cluster.sync();
    // 2. the tiles below the diagonal: L_i,kt = A_i,kt Y^T
    bool have_yt = false;
    for (int i = kt + 1; i < nt; ++i) {
      if (factor_tile_owner(i, kt) != rank) continue;
      TilePieces<T> a_ik, yt;
      tile_pieces_load<T, false>(a_ik, tile(i, kt), np);   // this CTA's own tile
      if (!have_yt) tile_pieces_load<T, true>(yt, DiT + (size_t)kt * T * T, T);   // Y^T, row-major in DiT
      tile_pieces_store_transposed<T, LD>(X1, a_ik);
      if (!have_yt) {   // X2[m][c] = (Y^T)[m][c]: the pieces go in untransposed
#pragma unroll
        for (int u = 0; u < TilePieces<T>::N; ++u) {
          const int q = tid + 256 * u, r = q % T, c4 = 4 * (q / T);
          *reinterpret_cast<float4*>(&X2[r][c4]) = yt.v[u];
        }
        have_yt = true;
      }
      __syncthreads();
      float acc[R][R];
      tile_product<T, LD>(X1, X2, acc);
      float* dst = tile(i, kt);
#pragma unroll
      for (int a = 0; a < R; ++a)
        *reinterpret_cast<float4*>(dst + (size_t)(tr * R + a) * np + tc * R) =
            make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
      __syncthreads();   // X1 is reloaded next
    }
    __threadfence();
    cluster.sync();
    // 3. trailing update of this CTA's tiles kt < j <= i; the owner of the next diagonal tile updates it first
    //    and factors it before its other tiles (look-ahead)
    if (kt + 1 < nt && factor_tile_owner(kt + 1, kt + 1) == rank) {
      TilePieces<T> l1;
      float4 old[R];
      float* dst = tile(kt + 1, kt + 1);
      tile_pieces_load<T, true>(l1, tile(kt + 1, kt), np);
      block_load<T>(old, dst, np);
      tile_pieces_store_transposed<T, LD>(X1, l1);
      __syncthreads();
      float acc[R][R];
      tile_product<T, LD>(X1, X1, acc);
#pragma unroll
      for (int a = 0; a < R; ++a)
        *reinterpret_cast<float4*>(dst + (size_t)(tr * R + a) * np + tc * R) =
            make_float4(old[a].x - acc[a][0], old[a].y - acc[a][1], old[a].z - acc[a][2], old[a].w - acc[a][3]);
      __syncthreads();
      diagonal(kt + 1);
    }
    for (int i = kt + 1; i < nt; ++i) {
      bool have_li = false;
      for (int j = kt + 1; j <= i; ++j) {
        if (factor_tile_owner(i, j) != rank || (i == kt + 1 && j == kt + 1)) continue;
        TilePieces<T> li, lj;
        float4 old[R];
        float* dst = tile(i, j);
        if (!have_li) tile_pieces_load<T, true>(li, tile(i, kt), np);
        tile_pieces_load<T, true>(lj, tile(j, kt), np);
        block_load<T>(old, dst, np);
        if (!have_li) {
          tile_pieces_store_transposed<T, LD>(X1, li);
          have_li = true;
        }
        tile_pieces_store_transposed<T, LD>(X2, lj);
        __syncthreads();
        float acc[R][R];
        tile_product<T, LD>(X1, X2, acc);
#pragma unroll
        for (int a = 0; a < R; ++a)
          *reinterpret_cast<float4*>(dst + (size_t)(tr * R + a) * np + tc * R) =
              make_float4(old[a].x - acc[a][0], old[a].y - acc[a][1], old[a].z - acc[a][2], old[a].w - acc[a][3]);
        __syncthreads();   // X2 (and X1 at the next i) are reloaded
      }
    }
  }
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
// inverse of the diagonal tile redundantly, so the next step needs no further synchronisation.  The tiles
// do not depend on the vector: the owned tiles of the next steps (up to SOLVE_PF of them each) and their
// diagonal inverses are copied into shared memory (cp.async) while step it computes, `nst` stages deep:
// three (two steps ahead) when the launch is one wave of CTAs, two otherwise, where the smaller shared
// memory lets two CTAs share an SM and the waves halve.
constexpr int SOLVE_PF = 2;

template <typename F, int T>
struct SolveLayout {
  static constexpr int LDT = T + 16 / (int)sizeof(F);   // padded rows, 16-byte aligned
  static constexpr size_t tile_elems = (size_t)T * LDT;
  // per stage [SOLVE_PF tiles + 1 diagonal inverse][T][LDT]; the stages are followed by the vector y
  static constexpr size_t stage_bytes = sizeof(F) * (SOLVE_PF + 1) * tile_elems;
};

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait2() { asm volatile("cp.async.wait_group 2;\n" ::: "memory"); }

// T x T tile at src (row stride ld elements) into padded shared rows
template <typename F, int T>
__device__ __forceinline__ void prefetch_tile(F* dst, const F* src, size_t ld) {
  constexpr int CH = T * (int)sizeof(F) / 16;   // 16-byte chunks per row
  constexpr int LDT = SolveLayout<F, T>::LDT;
  for (int q = threadIdx.x; q < T * CH; q += blockDim.x) {
    const int r = q / CH, c = q - (q / CH) * CH;
    cp_async16(dst + (size_t)r * LDT + c * (16 / sizeof(F)), src + (size_t)r * ld + c * (16 / sizeof(F)));
  }
}

// out[r] = sum_c M[r][c] v[c], M a padded shared tile; 256 / T threads per row
template <typename F, int T>
__device__ __forceinline__ void smem_matvec(const F* M, const F* v, F* out) {
  constexpr int PARTS = 256 / T, LEN = T / PARTS, LDT = SolveLayout<F, T>::LDT;
  const int r = threadIdx.x / PARTS, part = threadIdx.x - (threadIdx.x / PARTS) * PARTS;
  const F* row = M + (size_t)r * LDT + part * LEN;
  F s = F(0);
#pragma unroll
  for (int c = 0; c < LEN; ++c) s += row[c] * v[part * LEN + c];
#pragma unroll
  for (int d = PARTS / 2; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
  if (part == 0) out[r] = s;
}

template <typename F, int T, typename Rreal, int CS>
__global__ void __launch_bounds__(256) k_tri_solve(DevProblem P, const F* L, const F* Dinv, const double* scale,
                                                   const Rreal* rhs, double* x, int accumulate, int64_t v_total,
                                                   int nst) {
  namespace cg = cooperative_groups;
  using SL = SolveLayout<F, T>;
  constexpr int PARTS = 256 / T, LEN = T / PARTS, LDT = SL::LDT;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  F* buf = reinterpret_cast<F*>(smem_raw);                   // [nst][SOLVE_PF + 1][T][LDT]
  F* y = buf + nst * (SOLVE_PF + 1) * SL::tile_elems;
  __shared__ F partial[2][T];
  __shared__ F t[T];
  __shared__ F pcol[PARTS][T];
  const int rank = (int)cluster.block_rank();
  const int k = blockIdx.x / CS;
  if (P.sharded && !P.cluster_owned[k]) return;   // the whole thread-block cluster leaves, before any barrier
  const int np = P.cluster_np[k];
  const F* A = L + P.S_off[k];
  const F* Di = Dinv + (size_t)P.v_off[k] * T;
  const F* DiT = Di + v_total * T;
  const double* sk = scale + P.v_off[k];
  const Rreal* rk = rhs + P.v_off[k];
  double* xk = x + P.v_off[k];
  const int nt = np / T;
  const int tid = threadIdx.x;
  auto tile_buf = [&](int stage, int slot) { return buf + ((size_t)stage * (SOLVE_PF + 1) + slot) * SL::tile_elems; };
  // step s = 0 .. 2 nt - 1: forward steps it = s, backward steps it = 2 nt - 1 - s
  auto issue = [&](int s) {
    if (s < 2 * nt) {
      const bool fwd = s < nt;
      const int it = fwd ? s : 2 * nt - 1 - s;
      int m = 0;
      if (fwd) {
        for (int j = rank; j < it && m < SOLVE_PF; j += CS, ++m)
          prefetch_tile<F, T>(tile_buf(s % nst, m), A + (size_t)(it * T) * np + j * T, np);
      } else {
        for (int j = it + 1 + rank; j < nt && m < SOLVE_PF; j += CS, ++m)
          prefetch_tile<F, T>(tile_buf(s % nst, m), A + (size_t)(j * T) * np + it * T, np);
      }
      prefetch_tile<F, T>(tile_buf(s % nst, SOLVE_PF), (fwd ? Di : DiT) + (size_t)it * T * T, T);
    }
    cp_async_commit();
  };
  issue(0);
  if (nst == 3) issue(1);
  for (int i = tid; i < np; i += blockDim.x) y[i] = (F)((double)rk[i] * sk[i]);
  for (int s = 0; s < 2 * nt; ++s) {
    issue(s + nst - 1);   // into the stage step s - 1 used; every thread passed its last barrier
    if (nst == 3)
      cp_async_wait2();
    else
      cp_async_wait1();
    __syncthreads();
    const int st = s % nst;
    const bool fwd = s < nt;
    const int it = fwd ? s : 2 * nt - 1 - s;
    const int r0 = it * T;
    if (fwd) {
      // partial[r] = sum over owned tiles j of L[it][j] y_j: thread (row, part)
      const int r = tid / PARTS, part = tid - (tid / PARTS) * PARTS;
      F acc = F(0);
      int m = 0;
      for (int j = rank; j < it; j += CS, ++m) {
        const F* yj = y + j * T + part * LEN;
        if (m < SOLVE_PF) {
          const F* row = tile_buf(st, m) + (size_t)r * LDT + part * LEN;
#pragma unroll
          for (int c = 0; c < LEN; ++c) acc += row[c] * yj[c];
        } else {
          const F* row = A + (size_t)(r0 + r) * np + j * T + part * LEN;
#pragma unroll
          for (int c = 0; c < LEN; ++c) acc += __ldg(row + c) * yj[c];
        }
      }
#pragma unroll
      for (int d = PARTS / 2; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
      if (part == 0) partial[s & 1][r] = acc;
    } else {
      // partial[c] = sum over owned tiles j of L[j][it]^T z_j: thread (column, part of the rows)
      const int c = tid % T, part = tid / T;
      F acc = F(0);
      int m = 0;
      for (int j = it + 1 + rank; j < nt; j += CS, ++m) {
        const F* zj = y + j * T + part * LEN;
        if (m < SOLVE_PF) {
          const F* col = tile_buf(st, m) + (size_t)(part * LEN) * LDT + c;
#pragma unroll
          for (int rr = 0; rr < LEN; ++rr) acc += col[(size_t)rr * LDT] * zj[rr];
        } else {
          const F* col = A + (size_t)(j * T + part * LEN) * np + r0 + c;
#pragma unroll
          for (int rr = 0; rr < LEN; ++rr) acc += __ldg(col + (size_t)rr * np) * zj[rr];
        }
      }
      pcol[part][c] = acc;
      __syncthreads();
      if (tid < T) {
        F v = F(0);
#pragma unroll
        for (int q = 0; q < PARTS; ++q) v += pcol[q][tid];
        partial[s & 1][tid] = v;
      }
    }
    cluster.sync();
    for (int r = tid; r < T; r += blockDim.x) {
      F sum = F(0);
#pragma unroll
      for (int q = 0; q < CS; ++q) sum += cluster.map_shared_rank(&partial[s & 1][0], q)[r];
      t[r] = y[r0 + r] - sum;
    }
    __syncthreads();
    // y_it = D_it^-1 t (forward) or D_it^-T t (backward, through the stored transpose)
    smem_matvec<F, T>(tile_buf(st, SOLVE_PF), t, y + r0);
    __syncthreads();
  }
  if (rank == 0)
    for (int i = tid; i < np; i += blockDim.x) {
      const double v = (double)y[i] * sk[i];
      xk[i] = accumulate ? xk[i] + v : v;
    }
  cluster.sync();   // keep this CTA's shared memory alive until every peer has read it
}

// Device figures, read by configure_solve_kernels.
static int g_num_sms = 0, g_smem_optin = 0;

// Shared memory of one solve CTA: nst stages, the vector, and the static arrays (partial[2][T], t[T],
// pcol[256 / T][T]).
template <typename F, int T>
size_t solve_cta_bytes(int nst, int max_np) {
  return nst * SolveLayout<F, T>::stage_bytes +
         sizeof(F) * ((size_t)max_np + (3 + 256 / T) * (size_t)T);
}

template <typename F, int T>
int solve_stages(int l, int max_np, int cs) {
  const bool one_wave = (int64_t)l * cs <= g_num_sms;
  return one_wave && solve_cta_bytes<F, T>(3, max_np) <= (size_t)g_smem_optin ? 3 : 2;
}

template <typename F, int T, typename Rreal>
void launch_tri_solve(const DevProblem& P, const F* L, const F* Dinv, const double* scale, const Rreal* rhs,
                      double* x, int accumulate, int max_np, int64_t v_total, int cs, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P.l * cs);
  cfg.blockDim = dim3(256);
  const int nst = solve_stages<F, T>(P.l, max_np, cs);
  cfg.dynamicSmemBytes = nst * SolveLayout<F, T>::stage_bytes + sizeof(F) * (size_t)max_np;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cs == 2)
    cudaLaunchKernelEx(&cfg, k_tri_solve<F, T, Rreal, 2>, P, L, Dinv, scale, rhs, x, accumulate, v_total, nst);
  else if (cs == 4)
    cudaLaunchKernelEx(&cfg, k_tri_solve<F, T, Rreal, 4>, P, L, Dinv, scale, rhs, x, accumulate, v_total, nst);
  else
    cudaLaunchKernelEx(&cfg, k_tri_solve<F, T, Rreal, 8>, P, L, Dinv, scale, rhs, x, accumulate, v_total, nst);
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

// sharded: another process's clusters scatter zeros (their steps arrive by the exchange of dc)
__global__ void k_scatter_dc(DevProblem P, const double* x, double* dc, float* dcf) {
  const int k = blockIdx.x;
  const int nk = P.cluster_n[k], cbase = P.cluster_cam_off[k];
  const bool own = !P.sharded || P.cluster_owned[k];
  const double* xk = x + P.v_off[k];
  for (int i = threadIdx.x; i < nk; i += blockDim.x) {
    const int cam = P.cluster_cams[cbase + i / 9];
    const double v = own ? xk[i] : 0.0;
    dc[9 * (size_t)cam + i % 9] = v;
    if (dcf) dcf[9 * (size_t)cam + i % 9] = (float)v;
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

// A launch of `threads` threads (256 for launch_prio) with a scheduling priority (kept by graph capture as a
// node attribute): the panels on the critical path go first, the trailing updates fill the remaining SMs.
template <typename... KArgs, typename... Args>
void launch_prio_n(void (*kernel)(KArgs...), int grid, int threads, size_t smem, cudaStream_t stream, int prio,
                   Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = prio;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename... KArgs, typename... Args>
void launch_prio(void (*kernel)(KArgs...), int grid, size_t smem, cudaStream_t stream, int prio, Args... args) {
  launch_prio_n(kernel, grid, 256, smem, stream, prio, args...);
}
// A panel CTA is bound by the latency of its column chain: a second panel CTA on the same SM would halve
// the speed of both.  When a tile step's panels fit on the SMs one each, their dynamic shared memory is
// raised above half of an SM's so that they do take one SM each; a step with more panels than SMs keeps
// the plain size, so that the SMs hold several and the waves stay few (figures set by
// configure_solve_kernels).
static size_t g_panel_min_smem = 0;

template <typename F, int T>
size_t panel_smem(int npn = 0) {
  return npn <= g_num_sms ? std::max(PanelLayout<F, T>::bytes, g_panel_min_smem) : PanelLayout<F, T>::bytes;
}

template <typename F, int T>
void launch_factor_t(const DevProblem& P, const double* S, const FactorBuffers& fb, const CholPlan& plan,
                     cudaStream_t stream) {
  using Sreal = double;
  F* L = reinterpret_cast<F*>(fb.L);
  F* Dinv = reinterpret_cast<F*>(fb.Dinv);
  dim3 g1(std::max(1, std::min(plan.max_np / 256 + 1, 64)), P.l);
  k_diag_scale<Sreal><<<g1, 256, 0, stream>>>(P, S, fb.scale);
  dim3 g2(std::min(plan.max_np, 1024), P.l);
  // the first tile column now (the first panels read it); with more tile steps, the rest of the copy runs
  // on the side stream beside panel 0, and panel 1 waits for it
  bool copy_beside = plan.nsteps > 1 && plan.ev_copy != nullptr;
  if constexpr (sizeof(F) == 4 && T == 64) copy_beside = copy_beside && !plan.persistent;
  k_scaled_copy<Sreal, F><<<g2, 256, 0, stream>>>(P, S, fb.scale, L, 0, copy_beside ? T : INT_MAX);
  // panels on `stream`; the trailing updates (all tiles but the next column, which the next panel updates
  // itself) on the side stream, so that update kt overlaps panel kt + 1.  Panel kt + 2 waits for update kt.
  if constexpr (sizeof(F) == 4 && T == 64) {
    if (plan.persistent) {   // every tile step of every cluster in one launch of 8-CTA thread-block clusters
      if (plan.n_cluster_items > 0) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(plan.n_cluster_items * FCS);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = ClusterFactorLayout<T>::bytes;
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = FCS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, k_chol_cluster<T>, reinterpret_cast<float*>(L), reinterpret_cast<float*>(Dinv), P,
                           plan.cluster_items, fb.fail_flags, fb.boosted, fb.v_total);
      }
      return;
    }
  }
  cudaStream_t side = plan.side_stream;
  cudaEventRecord(plan.ev_fork, stream);
  cudaStreamWaitEvent(side, plan.ev_fork, 0);
  if (copy_beside) {
    k_scaled_copy<Sreal, F><<<g2, 256, 0, side>>>(P, S, fb.scale, L, T, INT_MAX);
    cudaEventRecord(plan.ev_copy, side);
  }
  for (int kt = 0; kt < plan.nsteps; ++kt) {
    if (kt >= 2) cudaStreamWaitEvent(stream, plan.ev_update[kt - 2], 0);
    if (kt == 1 && copy_beside) cudaStreamWaitEvent(stream, plan.ev_copy, 0);
    const int npn = plan.h_panel_off[kt + 1] - plan.h_panel_off[kt];
    const int2* pitems = plan.panel_items + plan.h_panel_off[kt];
    bool stacked = true;
    if constexpr (sizeof(F) == 4 && T == 64) {
      if (plan.split) {   // diagonal tiles (factor + inverse), then the tiles below them
        stacked = false;
        const int nd = plan.h_diag_count[kt];
        if (nd > 0)
          launch_prio(k_chol_diag<F, T>, nd, DiagLayout<F, T>::bytes, stream, plan.prio_high, (const F*)L, Dinv, P,
                      pitems, kt, fb.fail_flags, fb.boosted, fb.v_total);
        if (npn > nd)
          launch_prio(k_chol_trsm<F, T>, npn - nd, TrsmLayout<F, T>::bytes, stream, plan.prio_high, L,
                      (const F*)Dinv, P, pitems + nd, kt, fb.v_total);
      }
    }
    if (stacked && npn > 0)
      launch_prio_n(k_chol_panel<F, T>, npn, PANEL_THREADS, panel_smem<F, T>(npn), stream, plan.prio_high, L,
                    reinterpret_cast<F*>(fb.Ldiag), P, pitems, kt, fb.fail_flags, fb.boosted);
    cudaEventRecord(plan.ev_panel[kt], stream);
    cudaStreamWaitEvent(side, plan.ev_panel[kt], 0);
    const int nu = plan.h_update_off[kt + 1] - plan.h_update_off[kt];
    if (nu > 0) {
      if constexpr (sizeof(F) == 4 && T == 64) {
        if (plan.update_tc) {
          launch_prio(k_chol_update_tc, nu, TCU_SMEM, side, plan.prio_low, reinterpret_cast<float*>(L), P,
                      plan.update_items + plan.h_update_off[kt], kt, fb.fail_flags);
        } else {
          launch_prio(k_chol_update<F, T>, nu, 0, side, plan.prio_low, L, P, plan.update_items + plan.h_update_off[kt], kt);
        }
      } else {
        launch_prio(k_chol_update<F, T>, nu, 0, side, plan.prio_low, L, P, plan.update_items + plan.h_update_off[kt], kt);
      }
    }
    cudaEventRecord(plan.ev_update[kt], side);
  }
  cudaEventRecord(plan.ev_join, side);
  cudaStreamWaitEvent(stream, plan.ev_join, 0);
  if (plan.n_diag_items > 0 && !plan.split)   // the split panel's diagonal kernels wrote the inverses
    k_diag_inverse<F, T><<<plan.n_diag_items, 256, 0, stream>>>(reinterpret_cast<const F*>(fb.Ldiag), Dinv, P,
                                                                plan.diag_items, fb.v_total);
}

template <typename F, int T>
void launch_solve_t(const DevProblem& P, const double* S, const double* b, const FactorBuffers& fb,
                    const CholPlan& plan, int refine_steps, double* dc, float* dcf, cudaStream_t stream) {
  using Sreal = double;
  const F* L = reinterpret_cast<const F*>(fb.L);
  const F* Dinv = reinterpret_cast<const F*>(fb.Dinv);
  launch_tri_solve<F, T, Sreal>(P, L, Dinv, fb.scale, b, fb.x, 0, plan.max_np, fb.v_total, plan.solve_cs, stream);
  const int nblk = (int)std::min<int64_t>(fb.v_total / 256 + 1, (int64_t)num_sms() * 8);
  for (int s = 0; s < refine_steps; ++s) {
    k_copy_vec<Sreal><<<nblk, 256, 0, stream>>>(b, fb.r, fb.v_total);
    if (plan.n_res_items > 0)
      k_residual<Sreal><<<plan.n_res_items, 32 * RES_WARPS, 0, stream>>>(P, S, fb.x, fb.r, plan.res_items);
    launch_tri_solve<F, T, double>(P, L, Dinv, fb.scale, fb.r, fb.x, 1, plan.max_np, fb.v_total, plan.solve_cs,
                                   stream);
  }
  k_scatter_dc<<<P.l, 256, 0, stream>>>(P, fb.x, dc, dcf);
}

// the tile size of the plan: FP32 factors 32 or 64 (chosen by stba_autotune), FP64 factors 32
template <typename F>
void launch_factor(const DevProblem& P, const double* S, const FactorBuffers& fb, const CholPlan& plan,
                   cudaStream_t stream) {
  if (sizeof(F) == 4 && plan.tile == 64)
    launch_factor_t<F, 64>(P, S, fb, plan, stream);
  else
    launch_factor_t<F, 32>(P, S, fb, plan, stream);
}

template <typename F>
void launch_solve(const DevProblem& P, const double* S, const double* b, const FactorBuffers& fb,
                  const CholPlan& plan, int refine_steps, double* dc, float* dcf, cudaStream_t stream) {
  if (sizeof(F) == 4 && plan.tile == 64)
    launch_solve_t<F, 64>(P, S, b, fb, plan, refine_steps, dc, dcf, stream);
  else
    launch_solve_t<F, 32>(P, S, b, fb, plan, refine_steps, dc, dcf, stream);
}

size_t solve_smem_bytes(bool mixed, int tile, int max_np) {   // with the smallest stage count
  if (!mixed) return solve_cta_bytes<double, 32>(2, max_np);
  return tile == 64 ? solve_cta_bytes<float, 64>(2, max_np) : solve_cta_bytes<float, 32>(2, max_np);
}

int num_sms() {
  if (g_num_sms <= 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

// The largest dynamic shared memory of a kernel is a per-function attribute shared by every context of the
// process.  It is only ever raised: a context with smaller clusters must not lower it below what another
// live context's next launch asks for.
static void raise_smem_attr(const void* fn, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> set_to;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  int& cur = set_to[{dev, fn}];
  if (bytes > cur && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess)
    cur = bytes;
}

void configure_solve_kernels(int max_np) {
  int dev = 0, per_sm = 0, reserved = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
  g_smem_optin = optin;
  const int spread = per_sm / 2 - reserved + 128;   // two CTAs asking this much exceed one SM
  g_panel_min_smem = (per_sm > 0 && spread > 0 && spread <= optin) ? (size_t)spread : 0;
  raise_smem_attr((const void*)k_chol_panel<float, 64>, (int)panel_smem<float, 64>());
  raise_smem_attr((const void*)k_chol_panel<float, 32>, (int)panel_smem<float, 32>());
  raise_smem_attr((const void*)k_chol_panel<double, 32>, (int)panel_smem<double, 32>());
  raise_smem_attr((const void*)k_chol_update_tc, (int)TCU_SMEM);
  raise_smem_attr((const void*)k_chol_diag<float, 64>, (int)DiagLayout<float, 64>::bytes);
  raise_smem_attr((const void*)k_chol_trsm<float, 64>, (int)TrsmLayout<float, 64>::bytes);
  // room for three stages wherever solve_stages may choose them
  auto stages = [&](size_t three) { return three <= (size_t)optin ? 3 : 2; };
  const int f64 = stages(solve_cta_bytes<float, 64>(3, max_np)) * SolveLayout<float, 64>::stage_bytes +
                  sizeof(float) * max_np;
  const int f32 = stages(solve_cta_bytes<float, 32>(3, max_np)) * SolveLayout<float, 32>::stage_bytes +
                  sizeof(float) * max_np;
  const int d32 = stages(solve_cta_bytes<double, 32>(3, max_np)) * SolveLayout<double, 32>::stage_bytes +
                  sizeof(double) * max_np;
  raise_smem_attr((const void*)k_tri_solve<float, 64, double, 8>, f64);
  raise_smem_attr((const void*)k_tri_solve<float, 32, double, 8>, f32);
  raise_smem_attr((const void*)k_tri_solve<double, 32, double, 8>, d32);
  raise_smem_attr((const void*)k_tri_solve<float, 64, double, 4>, f64);
  raise_smem_attr((const void*)k_tri_solve<float, 32, double, 4>, f32);
  raise_smem_attr((const void*)k_tri_solve<double, 32, double, 4>, d32);
  raise_smem_attr((const void*)k_tri_solve<float, 64, double, 2>, f64);
  raise_smem_attr((const void*)k_tri_solve<float, 32, double, 2>, f32);
  raise_smem_attr((const void*)k_tri_solve<double, 32, double, 2>, d32);
}

void launch_count_failures(const int* fail_flags, int l, DevState* st, cudaStream_t stream) {
  k_count_failures<<<1, 256, 0, stream>>>(fail_flags, l, st);
}

template void launch_factor<float>(const DevProblem&, const double*, const FactorBuffers&, const CholPlan&,
                                   cudaStream_t);
template void launch_factor<double>(const DevProblem&, const double*, const FactorBuffers&, const CholPlan&,
                                    cudaStream_t);
template void launch_solve<float>(const DevProblem&, const double*, const double*, const FactorBuffers&,
                                  const CholPlan&, int, double*, float*, cudaStream_t);
template void launch_solve<double>(const DevProblem&, const double*, const double*, const FactorBuffers&,
                                   const CholPlan&, int, double*, float*, cudaStream_t);

}  // namespace stba
