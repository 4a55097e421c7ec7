// Deblending quality on the device (ch. 4, Eqs ch4_Qpd and ch4_Qr):
//   Q = 10 log10( ||d_o||^2 / ||d_o - d_t||^2 )
// per gather, with d_o the unblended gather and d_t the pseudo-deblended
// (Q_PD) or deblended (Q_R) one; the improvement of a solve is Q_R - Q_PD.
// Both squared norms are accumulated in FP64: each thread sums its elements
// in FP64 (the float differences are exact in double), a CTA reduces with
// warp shuffles, and one FP64 atomic per CTA and norm adds into the
// caller's per-gather sums.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "internal.h"

namespace ashrt {
namespace {

constexpr int kQThreads = 256;

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// grid (blocks per gather, batch); sums[2 g] += sum d_o^2, sums[2 g + 1] += sum (d_o - d_t)^2
__global__ void __launch_bounds__(kQThreads) k_quality(const float* __restrict__ d_o,
                                                       const float* __restrict__ d_t, long long n,
                                                       double* __restrict__ sums) {
  const int g = blockIdx.y;
  const float* o = d_o + (long long)g * n;
  const float* t = d_t + (long long)g * n;
  double so = 0.0, se = 0.0;
  for (long long i = blockIdx.x * (long long)kQThreads + threadIdx.x; i < n;
       i += (long long)gridDim.x * kQThreads) {
    const double a = (double)__ldg(o + i);
    const double e = a - (double)__ldg(t + i);
    so = fma(a, a, so);
    se = fma(e, e, se);
  }
  so = warp_sum(so);
  se = warp_sum(se);
  __shared__ double red[2][kQThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][w] = so;
    red[1][w] = se;
  }
  __syncthreads();
  if (w == 0) {
    so = lane < kQThreads / 32 ? red[0][lane] : 0.0;
    se = lane < kQThreads / 32 ? red[1][lane] : 0.0;
    so = warp_sum(so);
    se = warp_sum(se);
    if (lane == 0) {
      atomicAdd(sums + 2 * g, so);
      atomicAdd(sums + 2 * g + 1, se);
    }
  }
}

}  // namespace
}  // namespace ashrt

using namespace ashrt;

extern "C" ashrt_status ashrt_quality_db(const float* d_orig_dev, const float* d_test_dev,
                                         int batch, long long n_per_gather, double* sums_dev,
                                         double* q_db, void* stream) {
  if (!d_orig_dev || !d_test_dev || !sums_dev || batch < 1 || batch > 65535 || n_per_gather < 1) {
    set_error("ashrt_quality_db: need both gathers, sums_dev, 1 <= batch <= 65535 and "
              "n_per_gather >= 1");
    return ASHRT_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(sums_dev, 0, sizeof(double) * 2 * (size_t)batch, s);
  if (e != cudaSuccess) {
    set_error("ashrt_quality_db: %s", cudaGetErrorString(e));
    return ASHRT_ECUDA;
  }
  // about four CTAs per SM over the whole batch, at least one per gather
  long long per = (152LL * 4 + batch - 1) / batch;
  const long long need = (n_per_gather + kQThreads * 8 - 1) / (kQThreads * 8);
  if (per > need) per = need;
  if (per < 1) per = 1;
  k_quality<<<dim3((unsigned)per, (unsigned)batch), kQThreads, 0, s>>>(d_orig_dev, d_test_dev,
                                                                       n_per_gather, sums_dev);
  count_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("ashrt_quality_db launch: %s", cudaGetErrorString(e));
    return ASHRT_ECUDA;
  }
  if (!q_db) return ASHRT_OK;
  std::vector<double> h(2 * (size_t)batch);
  e = cudaMemcpyAsync(h.data(), sums_dev, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error("ashrt_quality_db: %s", cudaGetErrorString(e));
    return ASHRT_ECUDA;
  }
  for (int g = 0; g < batch; ++g) {
    const double so = h[2 * (size_t)g], se = h[2 * (size_t)g + 1];
    // an exact reconstruction of a non-zero gather is +inf dB; an all-zero gather has no Q
    q_db[g] = se > 0.0 ? 10.0 * std::log10(so / se) : (so > 0.0 ? HUGE_VAL : NAN);
  }
  return ASHRT_OK;
}
