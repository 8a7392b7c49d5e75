// ALU throughput probe (instrumentation, not part of the method): the rate at which
// this GPU retires independent fused multiply-adds in FP64 or FP32, the denominator
// of the roofline of the ALU-bound flux, SAT and relaxation kernels.
//
// Every thread runs kChains independent chains acc_k <- acc_k * a + b for `iters`
// rounds (a close to 1, b small, so the values stay normal and finite), enough
// warps per SM to hide the FMA latency, and stores the sum of its chains so the
// work cannot be removed.  One launch warms the clocks and caches; the timed
// launches are bracketed by CUDA events on the given stream.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../include/es.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T a, T b, int iters, T* __restrict__ out) {
  T acc[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc[k] = T(threadIdx.x + k) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) acc[k] = fma(acc[k], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += acc[k];
  out[blockIdx.x * (long long)blockDim.x + threadIdx.x] = s;
}

template <typename T>
int run(int blocks, int iters, int reps, cudaStream_t st, double* tflops) {
  T* out = nullptr;
  const size_t n = size_t(blocks) * kThreads;
  if (cudaMalloc(&out, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return ES_ERR_NOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = ES_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = ES_ERR_CUDA;
  const T a = T(0.999999), b = T(1e-7);
  if (rc == ES_OK) {
    k_fma_chains<T><<<blocks, kThreads, 0, st>>>(a, b, iters, out);  // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps; ++r) k_fma_chains<T><<<blocks, kThreads, 0, st>>>(a, b, iters, out);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = ES_ERR_CUDA;
  }
  if (rc == ES_OK) {
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * double(n) * kChains * 16.0 * iters * reps;
    *tflops = flops / (double(ms) * 1e-3) / 1e12;
  } else {
    cudaGetLastError();
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}

}  // namespace

extern "C" int es_fma_peak(int fp64, double* tflops, void* stream) {
  if (!tflops) return ES_ERR_INVALID;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return ES_ERR_CUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // 8 blocks of 256 threads per SM: 64 warps, full occupancy at <= 32 registers per
  // thread; FP64 rounds are ~64x slower per instruction, so fewer of them
  const int blocks = sms * 8;
  return fp64 ? run<double>(blocks, 256, 5, st, tflops) : run<float>(blocks, 8192, 5, st, tflops);
}
