// Blending, pseudo-deblending and gather sorting (ch. 2, Eqs ch2_blending and
// pseudodeblending_equ): the acquisition model around the deblending solve.
//
//   blending        b[r, t'] = sum_i D[i, r, t' - tau_i]   (0 <= t' - tau_i < nt)
//   pseudo-deblend  D~[i, r, t] = b[r, tau_i + t]          (0 <= tau_i + t < nb, else 0)
//   sorting         [n0][n1][nt] -> [n1][n0][nt]           (shot <-> receiver gathers)
//
// D is the cube of common-shot gathers [ns][nr][nt], b one continuous record
// per receiver [nr][nb], tau_i the firing sample of shot i (whole samples; a
// device array).  Pseudo-deblending is the exact transpose of blending.
// Blending is written as a gather (each record sample sums the shots whose
// window covers it, in shot order), so it needs no atomics and its result
// does not depend on scheduling; the other two are copies.  All three are
// memory-bound streams with coalesced rows along t.
#include <cuda_runtime.h>

#include "internal.h"

namespace ashrt {
namespace {

constexpr int kBThreads = 256;
constexpr int kBMaxShots = 8192;

// grid (blocks over t', nr); the firing samples are staged in shared memory.
__global__ void k_blend(const float* __restrict__ D, int ns, int nr, int nt,
                        const int* __restrict__ fire, float* __restrict__ b, int nb) {
  extern __shared__ int sf[];
  for (int i = threadIdx.x; i < ns; i += blockDim.x) sf[i] = fire[i];
  __syncthreads();
  const int r = blockIdx.y;
  for (int tp = blockIdx.x * blockDim.x + threadIdx.x; tp < nb; tp += gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int i = 0; i < ns; ++i) {
      const long long t = (long long)tp - sf[i];
      if (t >= 0 && t < nt) acc += __ldg(D + ((long long)i * nr + r) * nt + t);
    }
    b[(long long)r * nb + tp] = acc;
  }
}

// grid (blocks over t, nr, ns)
__global__ void k_pseudo_deblend(const float* __restrict__ b, int nr, int nb,
                                 const int* __restrict__ fire, int nt, float* __restrict__ D) {
  const int r = blockIdx.y, i = blockIdx.z;
  const long long f = fire[i];
  float* row = D + ((long long)i * nr + r) * nt;
  const float* rec = b + (long long)r * nb;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    const long long tp = f + t;
    row[t] = (tp >= 0 && tp < nb) ? __ldg(rec + tp) : 0.f;
  }
}

// grid (blocks over t, n1, n0): dst[j][i][:] = src[i][j][:]
__global__ void k_sort(const float* __restrict__ src, int n0, int n1, int nt,
                       float* __restrict__ dst) {
  const int j = blockIdx.y, i = blockIdx.z;
  const float* s = src + ((long long)i * n1 + j) * nt;
  float* d = dst + ((long long)j * n0 + i) * nt;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x)
    d[t] = __ldg(s + t);
}

int t_blocks(long long n) {
  long long b = (n + kBThreads - 1) / kBThreads;
  return (int)(b < 1 ? 1 : (b > 64 ? 64 : b));
}

ashrt_status launched(const char* name) {
  count_launches(1);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("%s: launch failed: %s", name, cudaGetErrorString(e));
    return ASHRT_ECUDA;
  }
  return ASHRT_OK;
}

}  // namespace
}  // namespace ashrt

using namespace ashrt;

extern "C" ashrt_status ashrt_blend(const float* shots_dev, int ns, int nr, int nt,
                                    const int* fire_dev, float* record_dev, int nb, void* stream) {
  if (!shots_dev || !fire_dev || !record_dev || ns < 1 || ns > kBMaxShots || nr < 1 ||
      nr > 65535 || nt < 1 || nb < 1) {
    set_error("ashrt_blend: need arrays, 1 <= ns <= %d, 1 <= nr <= 65535, nt >= 1, nb >= 1",
              kBMaxShots);
    return ASHRT_EINVAL;
  }
  k_blend<<<dim3(t_blocks(nb), nr), kBThreads, ns * sizeof(int), (cudaStream_t)stream>>>(
      shots_dev, ns, nr, nt, fire_dev, record_dev, nb);
  return launched("ashrt_blend");
}

extern "C" ashrt_status ashrt_pseudo_deblend(const float* record_dev, int nr, int nb,
                                             const int* fire_dev, int ns, int nt,
                                             float* shots_dev, void* stream) {
  if (!record_dev || !fire_dev || !shots_dev || ns < 1 || ns > 65535 || nr < 1 || nr > 65535 ||
      nt < 1 || nb < 1) {
    set_error("ashrt_pseudo_deblend: need arrays, 1 <= ns, nr <= 65535, nt >= 1, nb >= 1");
    return ASHRT_EINVAL;
  }
  k_pseudo_deblend<<<dim3(t_blocks(nt), nr, ns), kBThreads, 0, (cudaStream_t)stream>>>(
      record_dev, nr, nb, fire_dev, nt, shots_dev);
  return launched("ashrt_pseudo_deblend");
}

extern "C" ashrt_status ashrt_sort_gathers(const float* src_dev, int n0, int n1, int nt,
                                           float* dst_dev, void* stream) {
  if (!src_dev || !dst_dev || src_dev == dst_dev || n0 < 1 || n0 > 65535 || n1 < 1 ||
      n1 > 65535 || nt < 1) {
    set_error("ashrt_sort_gathers: need distinct arrays, 1 <= n0, n1 <= 65535, nt >= 1");
    return ASHRT_EINVAL;
  }
  k_sort<<<dim3(t_blocks(nt), n1, n0), kBThreads, 0, (cudaStream_t)stream>>>(src_dev, n0, n1,
                                                                              nt, dst_dev);
  return launched("ashrt_sort_gathers");
}
