// FP32 CUDA-core peak of the device this runs on, measured (a measurement
// hook with no counterpart in the paper): the roofline denominator of the
// library's ALU-bound kernels (the fused t-FFT + Stolt row kernels).
//
// Every thread runs kChains independent chains of fused multiply-adds
// x <- x a + b (a just below 1, so the chains stay finite and normal), far
// more chains per SM than the FMA latency needs; the grid fills every SM
// with 2048 resident threads.  The result is kept alive by a conditional
// store to a file-scope device variable that never executes for these
// inputs.  flops = 2 x FMAs; the best of `reps` timed launches is reported.
#include <cuda_runtime.h>

#include "internal.h"

namespace ashrt {
namespace {

constexpr int kChains = 8, kUnroll = 16, kPeakThreads = 256, kPeakBlocksPerSm = 8;

__device__ float g_peak_sink;

__global__ void __launch_bounds__(kPeakThreads) k_ffma(int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = 1e-3f * (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == -1.0f) g_peak_sink = s;   // chains are positive: never taken
}

}  // namespace
}  // namespace ashrt

using namespace ashrt;

extern "C" ashrt_status ashrt_fp32_peak(int iters, int reps, double* tflops, int* sm_count,
                                        void* stream) {
  if (iters < 1 || reps < 1 || !tflops) {
    set_error("ashrt_fp32_peak: need iters >= 1, reps >= 1 and tflops");
    return ASHRT_EINVAL;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    set_error("ashrt_fp32_peak: %s", cudaGetErrorString(e));
    return ASHRT_ECUDA;
  }
  if (sm_count) *sm_count = sms;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int blocks = sms * kPeakBlocksPerSm;
  const double flops = 2.0 * kChains * kUnroll * (double)iters * blocks * kPeakThreads;
  double best = 0.0;
  // one untimed launch first (module load, clocks ramping up)
  for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, s);
    if (e != cudaSuccess) break;
    k_ffma<<<blocks, kPeakThreads, 0, s>>>(iters, 0.99999994f, 1e-6f);
    count_launches(1);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && ms > 0.f) {
      const double t = flops / (ms * 1e-3) / 1e12;
      if (t > best) best = t;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    set_error("ashrt_fp32_peak: %s", cudaGetErrorString(e));
    return ASHRT_ECUDA;
  }
  *tflops = best;
  return ASHRT_OK;
}
