// Arithmetic-rate probe: the measured peak of the FP64 and FP32 fused
// multiply-add pipes of this GPU, the denominators of the roofline of the
// ALU-bound chain kernels.  A measurement helper; the paper has no
// counterpart.
#include <cuda_runtime.h>
#include <math.h>

#include "../../include/mcfmm.h"

namespace {

constexpr int kChains = 8;     // independent FMA chains per thread
constexpr int kThreads = 256;  // 8 warps per CTA
constexpr int kCtasPerSm = 2;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_rate(T* out, long long iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
#pragma unroll 4
  for (long long i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += x[k];
  out[blockIdx.x * kThreads + threadIdx.x] = s;
}

template <typename T>
int time_rate(T* d_out, int blocks, long long iters, double* seconds) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return MC_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return MC_ERR_CUDA;
  }
  // a, b keep every chain bounded (fixed point b / (1 - a))
  const T a = (T)0.9999, b = (T)1e-4;
  int rc = MC_OK;
  cudaEventRecord(e0, 0);
  k_fma_rate<T><<<blocks, kThreads>>>(d_out, iters, a, b);
  cudaEventRecord(e1, 0);
  if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
    rc = MC_ERR_CUDA;
  } else {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *seconds = ms * 1e-3;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

template <typename T>
int fma_rate(double target_s, double* flops_out) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MC_ERR_CUDA;
  const int blocks = sms * kCtasPerSm;
  T* d_out = nullptr;
  if (cudaMalloc(&d_out, sizeof(T) * (size_t)blocks * kThreads) != cudaSuccess) return MC_ERR_NOMEM;
  // grow the loop until one launch lasts target_s, then keep the best of 3
  long long iters = 1024;
  double sec = 0.0;
  int rc = time_rate<T>(d_out, blocks, iters, &sec);
  while (rc == MC_OK && sec < 0.25 * target_s && iters < (1LL << 40)) {
    iters *= 4;
    rc = time_rate<T>(d_out, blocks, iters, &sec);
  }
  double best = 0.0;
  for (int r = 0; rc == MC_OK && r < 3; r++) {
    rc = time_rate<T>(d_out, blocks, iters, &sec);
    const double f = 2.0 * kChains * (double)iters * blocks * kThreads / sec;
    if (f > best) best = f;
  }
  cudaFree(d_out);
  if (rc == MC_OK) *flops_out = best;
  return rc;
}

}  // namespace

extern "C" int mc_probe_fma_rate(int fp64, double target_seconds, double* flops_out) {
  if (!flops_out || !(target_seconds > 0.0) || !(target_seconds <= 10.0)) return MC_ERR_ARG;
  return fp64 ? fma_rate<double>(target_seconds, flops_out)
              : fma_rate<float>(target_seconds, flops_out);
}
