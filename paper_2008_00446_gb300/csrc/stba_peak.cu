// stba_measure_peaks: measured arithmetic peaks of this GPU, the denominators of the factorisation's
// roofline (the paper has no counterpart; it is measurement infrastructure).
//
//   FP32 SIMT: every thread runs 16 independent FMA chains (fmaf with run-time operands, so nothing folds);
//              4 CTAs of 256 threads per SM.  2 flops per FMA.
//   TF32 tensor: one CTA per SM issues back-to-back tcgen05.mma kind::tf32 of M = 128, N = 256, K = 8 into one
//              TMEM accumulator (operands are zero-filled shared memory; the rate does not depend on values).
//              2 M N K flops per MMA.  This is the dense TF32 rate; a 3xTF32 product delivers a third of it.
// Each kernel runs once untimed and then `reps` times between CUDA events on the caller's stream.
#include <cuda_runtime.h>

#include "stba_internal.cuh"
#include "stba_tc.cuh"

namespace stba {
namespace {

constexpr int PEAK_CHAINS = 16;

__global__ void __launch_bounds__(256) k_peak_fma(float* sink, int iters, float a, float b) {
  float x[PEAK_CHAINS];
#pragma unroll
  for (int i = 0; i < PEAK_CHAINS; ++i) x[i] = threadIdx.x * 1e-3f + (float)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < PEAK_CHAINS; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < PEAK_CHAINS; ++i) s += x[i];
  if (s == 1234567.f) sink[blockIdx.x] = s;   // keeps the chains alive; never true for these operands
}

constexpr int PEAK_N = 256;
constexpr size_t PEAK_SMEM = sizeof(uint32_t) * (128 * 32 + PEAK_N * 32);   // A 128 x 32, B 256 x 32: 48 KB

__global__ void __launch_bounds__(128) k_peak_tf32(int n_mma, int* err) {
  extern __shared__ __align__(128) uint32_t psm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t taddr_s;
  for (int i = threadIdx.x; i < 128 * 32 + PEAK_N * 32; i += blockDim.x) psm[i] = 0u;
  tc::fence_async_smem();
  if (threadIdx.x == 0) tc::mbar_init(&mbar, 1);
  if ((threadIdx.x >> 5) == 0) tc::tmem_alloc(&taddr_s, PEAK_N);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = taddr_s;
  if (threadIdx.x == 0) {
    constexpr uint32_t idesc = tc::idesc_tf32(128, PEAK_N);
    const uint32_t a0 = tc::smem_u32(psm), b0 = tc::smem_u32(psm + 128 * 32);
    for (int i = 0; i < n_mma; ++i) {
      const uint32_t ks = (uint32_t)(i & 3) * 256;   // four K steps of the 32-wide operands
      tc::mma_tf32(tmem, tc::smem_desc(a0 + ks, 128, 1024), tc::smem_desc(b0 + ks, 128, 1024), idesc, i > 0);
    }
    tc::mma_commit(&mbar);
  }
  if (!tc::mbar_wait_bounded(&mbar, 0, 1 << 26) && threadIdx.x == 0) atomicExch(err, 1);
  tc::fence_before_sync();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(tmem, PEAK_N);
}

}  // namespace
}  // namespace stba

extern "C" stba_status stba_measure_peaks(void* cuda_stream, int32_t reps, double* fp32_tflops, double* tf32_tflops) {
  using namespace stba;
  if (reps < 1 || (!fp32_tflops && !tf32_tflops)) return STBA_ERR_INVALID_ARG;
  if (cudaPeekAtLastError() != cudaSuccess) return STBA_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int sms = num_sms();
  float* sink = nullptr;
  int* err = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  stba_status st = STBA_OK;
  auto check = [&](cudaError_t e) {
    if (e != cudaSuccess && st == STBA_OK) st = STBA_ERR_CUDA;
    return e == cudaSuccess;
  };
  if (!check(cudaMalloc(&sink, sizeof(float) * 4 * sms)) || !check(cudaMalloc(&err, sizeof(int))) ||
      !check(cudaEventCreate(&e0)) || !check(cudaEventCreate(&e1))) {
    cudaFree(sink);
    cudaFree(err);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return STBA_ERR_CUDA;
  }
  check(cudaMemsetAsync(err, 0, sizeof(int), s));
  if (fp32_tflops) {
    const int iters = 1 << 16, grid = 4 * sms;
    k_peak_fma<<<grid, 256, 0, s>>>(sink, iters, 0.999f, 1e-4f);
    check(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r) k_peak_fma<<<grid, 256, 0, s>>>(sink, iters, 0.999f, 1e-4f);
    check(cudaEventRecord(e1, s));
    float ms = 0.f;
    if (check(cudaEventSynchronize(e1)) && check(cudaEventElapsedTime(&ms, e0, e1)))
      *fp32_tflops = 2.0 * PEAK_CHAINS * (double)iters * grid * 256 * reps / (ms * 1e-3) / 1e12;
  }
  if (tf32_tflops && st == STBA_OK) {
    const int n_mma = 4096;
    check(cudaFuncSetAttribute(k_peak_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PEAK_SMEM));
    k_peak_tf32<<<sms, 128, PEAK_SMEM, s>>>(n_mma, err);
    check(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r) k_peak_tf32<<<sms, 128, PEAK_SMEM, s>>>(n_mma, err);
    check(cudaEventRecord(e1, s));
    float ms = 0.f;
    int herr = 0;
    if (check(cudaEventSynchronize(e1)) && check(cudaEventElapsedTime(&ms, e0, e1)) &&
        check(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost))) {
      if (herr) st = STBA_ERR_TIMEOUT;
      *tf32_tflops = 2.0 * 128 * PEAK_N * 8 * (double)n_mma * sms * reps / (ms * 1e-3) / 1e12;
    }
  }
  check(cudaGetLastError());
  cudaFree(sink);
  cudaFree(err);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}
