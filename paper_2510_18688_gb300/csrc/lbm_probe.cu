// lbm_probe.cu -- lbm_probe_fma_rate: the fused multiply-add throughput of
// the current GPU, measured with independent dependent-chain FMAs.  It is
// the arithmetic ceiling the FP64 step is compared against: on this part the
// FP64 pipe, not HBM, bounds the double-precision step.
#include <cstdio>

#include <cuda_runtime.h>

#include "../../include/lbm.h"

namespace {

constexpr int kChains = 8;    // independent FMA chains per thread
constexpr int kUnroll = 16;   // FMAs per chain per loop trip
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_rate_kernel(T* __restrict__ out, int iters, T a,
                                                            T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) x[c] = T(threadIdx.x + c) * T(1e-3);
  for (int k = 0; k < iters; k++) {
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
#pragma unroll
      for (int c = 0; c < kChains; c++) x[c] = fma(x[c], a, b);
    }
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; c++) s += x[c];
  out[blockIdx.x * kThreads + threadIdx.x] = s;
}

template <typename T>
int run(int iters, double* flops_per_s, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return LBM_ERR_CUDA;
  const int blocks = sms * 8;
  T* out = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(T));
  if (e != cudaSuccess) return LBM_ERR_OOM;
  int st = LBM_OK;
  if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess) st = LBM_ERR_CUDA;
  float best = 0.f;
  // one warm-up launch, then the best of three
  for (int rep = 0; rep < 4 && st == LBM_OK; rep++) {
    cudaEventRecord(t0, s);
    fma_rate_kernel<T><<<blocks, kThreads, 0, s>>>(out, iters, T(0.999999), T(1e-7));
    cudaEventRecord(t1, s);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(t1) != cudaSuccess) {
      st = LBM_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (st == LBM_OK) {
    const double fmas = (double)blocks * kThreads * kChains * kUnroll * (double)iters;
    *flops_per_s = 2.0 * fmas / (best * 1e-3);
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaFree(out);
  return st;
}

}  // namespace

extern "C" int lbm_probe_fma_rate(int precision, double* flops_per_s, void* stream) {
  if (!flops_per_s) return LBM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == LBM_FP64) return run<double>(256, flops_per_s, s);
  if (precision == LBM_FP32) return run<float>(16384, flops_per_s, s);
  return LBM_ERR_ARG;
}
