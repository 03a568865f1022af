// Device side of a new cluster assignment (Sec. 4.1-4.2): the observations are re-ordered by (point,
// cluster, camera), the virtual points (distinct (point, cluster) pairs) are numbered, and the per-camera
// observation lists of the camera pass are rebuilt.  The (point, camera) order fixed at create is the base:
// inside a point run the new order is the stable sort of the base by cluster, so a virtual point is a run
// of equal clusters and its observations stay ordered by camera.  Every step is deterministic.
#include <climits>

#include <cuda_runtime.h>

#include "stba_device.cuh"
#include "stba_internal.cuh"

namespace stba {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// cluster of the camera of every base observation
__global__ void k_base_keys(int q, const int* __restrict__ base_cam, const int* __restrict__ cam_cluster,
                            int* __restrict__ key) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o < q) key[o] = cam_cluster[base_cam[o]];
}

// New position of every base observation: its rank in the stable order by cluster inside its point run.
// Also marks the first observation of every virtual point and carries the per-observation data over.
template <typename real>
__global__ void k_reorder(ReorderArgs A, const int* __restrict__ key, const real* __restrict__ res_old,
                          real* __restrict__ res_new) {
  const int bo = blockIdx.x * blockDim.x + threadIdx.x;
  if (bo >= A.q) return;
  const int i = A.obs_pt[bo];
  const int b = A.pt_off[i], e = A.pt_off[i + 1];
  const int kb = key[bo];
  int rank = 0, same = 0;
  bool first = true;
  for (int o = b; o < e; ++o) {
    const int ko = key[o];
    rank += (ko < kb) || (ko == kb && o < bo);
    first = first && !(ko == kb && o < bo);
    same += ko == kb;
  }
  const int np = b + rank;
  A.inv_new[bo] = np;
  A.nsing[bo] = same == 1 ? (np | INT_MIN) : np;
  A.obs_base[np] = bo;
  A.obs_cam[np] = A.base_cam[bo];
  A.obs_perm[np] = A.base_src[bo];
  A.start[np] = first ? 1 : 0;
  if (A.obs_uv) reinterpret_cast<double2*>(A.obs_uv)[np] = reinterpret_cast<const double2*>(A.base_uv)[bo];
  if (A.obs_uvf) reinterpret_cast<float2*>(A.obs_uvf)[np] = reinterpret_cast<const float2*>(A.base_uvf)[bo];
  if (A.obs_uvdf) A.obs_uvdf[np] = A.base_uvdf[bo];
  if (res_old) {   // residuals at the current x, stored in the order of the previous assignment
    const int op = A.inv_old[bo];
    res_new[2 * (size_t)np] = res_old[2 * (size_t)op];
    res_new[2 * (size_t)np + 1] = res_old[2 * (size_t)op + 1];
  }
}

// per tile of SCAN_TILE observations: the number of virtual-point starts
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(int q, const int* __restrict__ start,
                                                             int* __restrict__ tile_sum) {
  __shared__ int ws[SCAN_THREADS / 32];
  const int base = blockIdx.x * SCAN_TILE;
  int s = 0;
#pragma unroll
  for (int t = 0; t < SCAN_ITEMS; ++t) {
    const int o = base + t * SCAN_THREADS + threadIdx.x;
    s += o < q ? start[o] : 0;
  }
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(FULL_MASK, s, d);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < SCAN_THREADS / 32; ++w) t += ws[w];
    tile_sum[blockIdx.x] = t;
  }
}

// exclusive scan of the tile sums (one CTA, sequential chunks of 1024); the total goes to counts[0]
__global__ void __launch_bounds__(1024) k_scan_partials(int ntiles, int* __restrict__ tile_sum,
                                                        long long* __restrict__ counts) {
  __shared__ int ws[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c0 = 0; c0 < ntiles; c0 += 1024) {
    const int i = c0 + threadIdx.x;
    const int v = i < ntiles ? tile_sum[i] : 0;
    int x = v;
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(FULL_MASK, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
      int z = ws[lane];
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(FULL_MASK, z, d);
        if (lane >= d) z += y;
      }
      ws[lane] = z;
    }
    __syncthreads();
    const int incl = x + (w > 0 ? ws[w - 1] : 0) + carry;
    if (i < ntiles) tile_sum[i] = incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) counts[0] = carry;
}

// virtual-point numbers: obs_vp, vp_off, vp_point, pt_vp_off
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(ReorderArgs A, const int* __restrict__ tile_off) {
  __shared__ int ws[SCAN_THREADS / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;   // contiguous items per thread
  int v[SCAN_ITEMS], s = 0;
#pragma unroll
  for (int t = 0; t < SCAN_ITEMS; ++t) {
    v[t] = base + t < A.q ? A.start[base + t] : 0;
    s += v[t];
  }
  int x = s;
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(FULL_MASK, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  int woff = 0;
  for (int u = 0; u < w; ++u) woff += ws[u];
  int run = tile_off[blockIdx.x] + woff + x - s;   // starts before this thread's first item
#pragma unroll
  for (int t = 0; t < SCAN_ITEMS; ++t) {
    const int o = base + t;
    if (o >= A.q) break;
    run += v[t];
    const int vp = run - 1;
    A.obs_vp[o] = vp;
    if (v[t]) {
      A.vp_off[vp] = o;
      const int i = A.obs_pt[o];
      A.vp_point[vp] = i;
      if (A.pt_off[i] == o) A.pt_vp_off[i] = vp;
    }
  }
}

// closing entries vp_off[nv] = q, pt_vp_off[n] = nv, and the number of camera-pair instances
__global__ void __launch_bounds__(256) k_vp_close(ReorderArgs A, long long* __restrict__ counts) {
  const long long nv = counts[0];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    A.vp_off[nv] = A.q;
    A.pt_vp_off[A.n] = (int)nv;
  }
  long long pairs = 0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
    const long long len = (v + 1 < nv ? A.vp_off[v + 1] : A.q) - A.vp_off[v];
    pairs += len * (len - 1) / 2;
  }
  for (int d = 16; d > 0; d >>= 1) pairs += __shfl_xor_sync(FULL_MASK, pairs, d);
  if ((threadIdx.x & 31) == 0 && pairs) atomicAdd(reinterpret_cast<unsigned long long*>(counts + 1),
                                                  (unsigned long long)pairs);
}

// Camera lists: the observations of every camera (new positions), those of single-observation virtual
// points first, each group in base order -- a stable partition of every camera's run of cam_base.  Whether
// an observation is alone in its virtual point (no other observation of its point in its cluster) comes
// from k_reorder, packed with its new position.
__global__ void k_cam_flag(ReorderArgs A, int* __restrict__ flag) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= A.q) return;
  const int x = A.nsing[A.cam_base[e]];   // one gather: the new position and whether it is alone
  A.eo[e] = x & INT_MAX;                  // for k_cam_place
  flag[e] = x < 0 ? 1 : 0;
}

// excl[e] = number of flags before e (tile offsets from k_scan_partials); excl[q] = total
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_excl(int q, const int* __restrict__ flag,
                                                            const int* __restrict__ tile_off,
                                                            const long long* __restrict__ total,
                                                            int* __restrict__ excl) {
  __shared__ int ws[SCAN_THREADS / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
  int v[SCAN_ITEMS], s = 0;
#pragma unroll
  for (int t = 0; t < SCAN_ITEMS; ++t) {
    v[t] = base + t < q ? flag[base + t] : 0;
    s += v[t];
  }
  int x = s;
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(FULL_MASK, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  int woff = 0;
  for (int u = 0; u < w; ++u) woff += ws[u];
  int run = tile_off[blockIdx.x] + woff + x - s;
#pragma unroll
  for (int t = 0; t < SCAN_ITEMS; ++t) {
    if (base + t >= q) break;
    excl[base + t] = run;
    run += v[t];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) excl[q] = (int)total[0];
}

__global__ void k_cam_place(ReorderArgs A, const int* __restrict__ flag, const int* __restrict__ excl) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= A.q) return;
  const int j = A.ecam[e];
  const int b = A.cam_off[j], cnt = A.cam_off[j + 1] - b;
  const int before = excl[e] - excl[b];               // singles of camera j before e
  const int nsingle = excl[b + cnt] - excl[b];
  const int idx = flag[e] ? before : nsingle + (e - b - before);
  const int o = A.eo[e];
  A.cam_obs[b + idx] = o;
  const size_t sl = 32 * (size_t)A.cam_warp_off[j] + idx;
  A.slots[sl] = o;
  A.slot_pv[sl] = make_int2(A.ept[e], flag[e] ? (A.obs_vp[o] | INT_MIN) : A.obs_vp[o]);
  if (A.slot_uvf) A.slot_uvf[sl] = A.euvf[e];
  if (A.slot_uvd) A.slot_uvd[sl] = A.euvd[e];
}

// chunks of the camera graph whose two cameras share a cluster
// a chunk is listed when its two cameras share a cluster that this process owns (every cluster unless sharded)
__global__ void k_chunk_flag(int nchunks, const int4* __restrict__ chunks, const int* __restrict__ cam_cluster,
                             const int* __restrict__ owned, int* __restrict__ flag) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nchunks) return;
  const int4 ch = chunks[c];
  const int k = cam_cluster[ch.x];
  flag[c] = (k == cam_cluster[ch.y] && owned[k]) ? 1 : 0;
}

__global__ void k_chunk_list(int nchunks, const int* __restrict__ flag, const int* __restrict__ excl,
                             int* __restrict__ active) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nchunks && flag[c]) active[excl[c]] = c;
}

// zeroes the per reals of the nv virtual points, nv read from the device counter
__global__ void __launch_bounds__(256) k_zero_vp(float4* __restrict__ p, const long long* __restrict__ counts,
                                                 int real_bytes, int per) {
  const long long n16 = (per * counts[0] * real_bytes + 15) / 16;   // the buffer holds per q reals, 16-byte padded
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n16; i += (long long)gridDim.x * blockDim.x)
    p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

}  // namespace

void launch_list_chunks(const PairChunks& B, const int* cam_cluster, const int* owned, long long* nactive,
                        cudaStream_t stream) {
  const int n = B.nchunks;
  if (n <= 0) return;
  const int g = (n + 255) / 256, ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  k_chunk_flag<<<g, 256, 0, stream>>>(n, B.chunks, cam_cluster, owned, B.flag);
  k_scan_tiles<<<ntiles, SCAN_THREADS, 0, stream>>>(n, B.flag, B.tile_sum);
  k_scan_partials<<<1, 1024, 0, stream>>>(ntiles, B.tile_sum, nactive);
  k_scan_excl<<<ntiles, SCAN_THREADS, 0, stream>>>(n, B.flag, B.tile_sum, nactive, B.excl);
  k_chunk_list<<<g, 256, 0, stream>>>(n, B.flag, B.excl, const_cast<int*>(B.active));
}

void launch_zero_vp(void* vp_acc, const long long* counts, int real_bytes, cudaStream_t stream) {
  k_zero_vp<<<2 * RED_BLOCKS, 256, 0, stream>>>(reinterpret_cast<float4*>(vp_acc), counts, real_bytes, 9);
}

void launch_zero_vp3(void* p, const long long* counts, int real_bytes, cudaStream_t stream) {
  k_zero_vp<<<2 * RED_BLOCKS, 256, 0, stream>>>(reinterpret_cast<float4*>(p), counts, real_bytes, 3);
}

template <typename real>
void launch_reorder(const ReorderArgs& A, int* key, int* tile_sum, long long* counts, const real* res_old,
                    real* res_new, cudaStream_t stream) {
  const int g = (A.q + 255) / 256;
  k_base_keys<<<g, 256, 0, stream>>>(A.q, A.base_cam, A.cam_cluster, key);
  k_reorder<real><<<g, 256, 0, stream>>>(A, key, res_old, res_new);
  const int ntiles = (A.q + SCAN_TILE - 1) / SCAN_TILE;
  k_scan_tiles<<<ntiles, SCAN_THREADS, 0, stream>>>(A.q, A.start, tile_sum);
  cudaMemsetAsync(counts, 0, 3 * sizeof(long long), stream);
  k_scan_partials<<<1, 1024, 0, stream>>>(ntiles, tile_sum, counts);
  k_scan_apply<<<ntiles, SCAN_THREADS, 0, stream>>>(A, tile_sum);
  k_vp_close<<<RED_BLOCKS, 256, 0, stream>>>(A, counts);
  // camera lists: flags, their exclusive scan (reusing the tile scan), placement
  int* flag = key;                 // the keys are no longer needed
  int* excl = A.start + A.q + 1;   // second half of the start buffer
  k_cam_flag<<<g, 256, 0, stream>>>(A, flag);
  k_scan_tiles<<<ntiles, SCAN_THREADS, 0, stream>>>(A.q, flag, tile_sum);
  k_scan_partials<<<1, 1024, 0, stream>>>(ntiles, tile_sum, counts + 2);
  k_scan_excl<<<ntiles, SCAN_THREADS, 0, stream>>>(A.q, flag, tile_sum, counts + 2, excl);
  k_cam_place<<<g, 256, 0, stream>>>(A, flag, excl);
}

template void launch_reorder<float>(const ReorderArgs&, int*, int*, long long*, const float*, float*, cudaStream_t);
template void launch_reorder<double>(const ReorderArgs&, int*, int*, long long*, const double*, double*,
                                     cudaStream_t);

}  // namespace stba
