// stba_cost_noalloc: the cost F(x) = ||f(x)||^2 for caller-owned device arrays, without allocating.
//
// Some callers cannot allocate device memory when they evaluate the cost: code that runs under a fixed,
// pre-reserved memory budget (a real-time reconstruction loop), code that must not call into the
// allocator while another component owns it, or host callbacks where allocation is not allowed.  This
// entry point takes only device pointers to the inputs and to the output, and keeps its scratch -- the
// per-camera FP64 rotation table and the reduction partials -- in one file-scope device array that every
// GPU loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "stba_camera.cuh"
#include "stba_internal.cuh"

namespace stba {

constexpr int NOALLOC_MAX_CAMERAS = 16384;
constexpr int NOALLOC_BLOCKS = 456;
constexpr int NOALLOC_THREADS = 256;
// 15 doubles per camera (R, t, f, k1, k2) + one partial per block: 1.97 MB
constexpr size_t NOALLOC_SCRATCH_DOUBLES = 15 * (size_t)NOALLOC_MAX_CAMERAS + NOALLOC_BLOCKS;

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

namespace {

__global__ void k_noalloc_rt(int m, const double* __restrict__ cams, double* __restrict__ rt) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    const double* c = cams + 9 * (size_t)j;
    const double w[3] = {c[0], c[1], c[2]};
    const double s = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double a, b, da, db;
    rodrigues_coeffs(s, a, b, da, db);
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

// Each block writes its partial sum of |f_o|^2 (every partial is overwritten on every call).  An index out
// of range, or a point at depth <= 1e-9, makes the partial NaN, so F comes out NaN.
__global__ void __launch_bounds__(NOALLOC_THREADS) k_noalloc_cost(int m, int n, int q, const double* __restrict__ rt,
                                                                  const double* __restrict__ pts,
                                                                  const int* __restrict__ obs_cam,
                                                                  const int* __restrict__ obs_pt,
                                                                  const double* __restrict__ obs_uv,
                                                                  double* __restrict__ partial) {
  double s = 0.0;
  int bad = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;   // 64-bit: q may come close to INT32_MAX
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < q; o += stride) {
    const int cam = obs_cam[o], pt = obs_pt[o];
    if (cam < 0 || cam >= m || pt < 0 || pt >= n) {
      bad = 1;
      continue;
    }
    const double* C = rt + 15 * (size_t)cam;
    const double* p = pts + 3 * (size_t)pt;
    const double xc = C[0] * p[0] + C[1] * p[1] + C[2] * p[2] + C[9];
    const double yc = C[3] * p[0] + C[4] * p[1] + C[5] * p[2] + C[10];
    const double zc = C[6] * p[0] + C[7] * p[1] + C[8] * p[2] + C[11];
    if (!(zc > 1e-9)) bad = 1;
    const double iz = 1.0 / zc;
    const double x = xc * iz, y = yc * iz;
    const double r2 = x * x + y * y;
    const double fd = C[12] * (1.0 + r2 * (C[13] + C[14] * r2));
    const double r0 = fd * x - obs_uv[2 * (size_t)o], r1 = fd * y - obs_uv[2 * (size_t)o + 1];
    s += r0 * r0 + r1 * r1;
  }
  __shared__ double red[NOALLOC_THREADS / 32];
  __shared__ int anybad;
  if (threadIdx.x == 0) anybad = 0;
  __syncthreads();
  if (bad) anybad = 1;
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0;
    for (int i = 0; i < NOALLOC_THREADS / 32; ++i) a += red[i];
    partial[blockIdx.x] = anybad ? __longlong_as_double(0x7ff8000000000000ll) : a;
  }
}

__global__ void k_noalloc_final(const double* __restrict__ partial, double* __restrict__ F) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < NOALLOC_BLOCKS; i += blockDim.x) s += partial[i];
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += red[i];
    *F = a;
  }
}

// Device address of g_noalloc_scratch, looked up once per device (with that device current).
constexpr int MAX_DEVICES = 64;
double* g_scratch_addr[MAX_DEVICES] = {};
std::mutex g_scratch_mutex;

cudaError_t scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace stba

extern "C" stba_status stba_cost_noalloc(const double* cameras, int64_t m, const double* points, int64_t n,
                                         const int32_t* obs_cam, const int32_t* obs_pt, const double* obs_uv,
                                         int64_t q, double* F_dev, void* cuda_stream) {
  using namespace stba;
  if (!cameras || !points || !obs_cam || !obs_pt || !obs_uv || !F_dev) return STBA_ERR_INVALID_ARG;
  if (m < 1 || n < 1 || q < 1 || q > INT32_MAX || n > INT32_MAX) return STBA_ERR_INVALID_ARG;
  if (m > NOALLOC_MAX_CAMERAS) return STBA_ERR_INVALID_ARG;   // beyond the static scratch
  // an error left pending by the caller's earlier work is reported, not cleared: it stays for the caller
  if (cudaPeekAtLastError() != cudaSuccess) return STBA_ERR_CUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return STBA_ERR_CUDA;
  double* scratch = nullptr;
  if (scratch_address(dev, &scratch) != cudaSuccess) return STBA_ERR_CUDA;
  double* rt = scratch;
  double* partial = scratch + 15 * (size_t)NOALLOC_MAX_CAMERAS;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  k_noalloc_rt<<<(int)((m + 127) / 128), 128, 0, s>>>((int)m, cameras, rt);
  if (cudaGetLastError() != cudaSuccess) return STBA_ERR_CUDA;
  k_noalloc_cost<<<NOALLOC_BLOCKS, NOALLOC_THREADS, 0, s>>>((int)m, (int)n, (int)q, rt, points, obs_cam, obs_pt,
                                                             obs_uv, partial);
  if (cudaGetLastError() != cudaSuccess) return STBA_ERR_CUDA;
  k_noalloc_final<<<1, 256, 0, s>>>(partial, F_dev);
  return cudaGetLastError() == cudaSuccess ? STBA_OK : STBA_ERR_CUDA;
}
