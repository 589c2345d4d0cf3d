// FP32 FMA-rate probe: the ALU roofline's denominator, measured.
//
// Every thread runs kChains independent FMA chains x <- x * a + b, so that
// each warp scheduler always has independent FMAs to issue; the grid holds
// eight 256-thread blocks per SM.  a, b and the start values are runtime
// arguments (nothing folds at compile time) and each chain's result feeds a
// conditional store that never happens for finite inputs, so no chain is
// removed as dead code.
#include <cuda_runtime.h>

#include "sg.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) ffma_rate_kernel(float* sink, int iters, float a,
                                                             float b, float x0) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = x0 + (float)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == -1.f) sink[blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" sg_status sg_measure_fp32_fma_rate(void* stream, int32_t iters, int32_t repeats,
                                              float* tflops) {
  if (!tflops || iters < 1 || repeats < 1) return SG_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return SG_ERR_CUDA;
  const int blocks = 8 * sms;
  float* sink = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaMalloc(&sink, sizeof(float) * blocks * kThreads);
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  float best_ms = 0.f;
  for (int r = 0; r <= repeats && e == cudaSuccess; ++r) {   // run 0 is a warm-up
    e = cudaEventRecord(t0, s);
    if (e == cudaSuccess) {
      ffma_rate_kernel<<<blocks, kThreads, 0, s>>>(sink, iters, 0.9999999f, 1e-7f, 0.5f);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(t1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (e == cudaSuccess && r > 0 && (best_ms == 0.f || ms < best_ms)) best_ms = ms;
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess || !(best_ms > 0.f)) return SG_ERR_CUDA;
  const double flops = 2.0 * kChains * kUnroll * (double)iters * blocks * kThreads;
  *tflops = (float)(flops / (best_ms * 1e-3) / 1e12);
  return SG_OK;
}
