// Time-domain ASHRT / AASHRT by hyperbolic summation: the thesis's classical
// form of the operator pair (ch. 3 Table ch3_table_Radon_operators, ASHRT row;
// ch. 6 Eq. ch6_AASHRT_adjoint) and the comparison system of its ch. 5 speed
// study, run here on the same GPU as the Stolt form.
//
// Adjoint (gather form):
//   m(tau, v_i, x_a, tau0_j) = sum_{x_r} d(s, x_r),
//   s = tau0_j / dt + sqrt(tau^2 + h^2) samples,  h = (x_r - x_a) / (v_i dt),
// with d read at the fractional sample s by linear interpolation (samples
// floor(s) and floor(s) + 1, each dropped when it lies at or past nt).  The
// forward is its exact transpose: every model sample is spread onto the same
// two data samples with the same weights.  Apex positions are the trace
// positions (x_a == x_r == x), as in the Stolt form.
//
// GPU layout.  Adjoint: one CTA per (gather, panel, block of A apexes); its
// 256 threads own the time samples tau = tid + 256 k, keep A x TPT running
// sums in registers, and stream the gather's traces through a double-buffered
// shared row (each trace read once per CTA).  Forward: one CTA per (gather,
// block of R output traces) accumulates its R traces in shared memory with
// shared-memory atomic adds while streaming every model row once (the
// accumulation order, and so the last bits of the forward, depend on the
// scheduling).  The traveltime is evaluated in FP32: for offsets up to a few
// hundred samples its rounding moves s by about 1e-4 samples at most.
// Neither call allocates; the per-panel constants travel in the kernel
// parameters.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace ashrt {
namespace {

constexpr int kTdThreads = 256;
constexpr int kTdMaxPanels = 256;

struct TdArgs {
  const float* in = nullptr;
  float* out = nullptr;
  int nt = 0, nx = 0, P = 0;
  float t0s[kTdMaxPanels];   // tau0_j / dt of panel p = j nv + i
  float cv[kTdMaxPanels];    // dx / (v_i dt): offset in samples per trace of x_r - x_a
};

// Fractional sample s of time sample tau on the hyperbola of offset hs
// (samples); i0 = floor(s), f = s - i0.
__device__ __forceinline__ void td_path(float t0s, float hs2, int tau, int& i0, float& f) {
  const float ft = (float)tau;
  const float s = t0s + sqrtf(fmaf(ft, ft, hs2));
  const float fl = floorf(s);
  i0 = (int)fl;
  f = s - fl;
}

// TPT time samples per thread (nt <= 256 TPT); A = 32 / TPT apexes per CTA.
template <int TPT>
__global__ void __launch_bounds__(kTdThreads) td_adjoint_kernel(TdArgs a) {
  constexpr int T = kTdThreads, A = 32 / TPT;
  extern __shared__ float tr[];                 // [2][nt]: current and next trace
  const int tid = threadIdx.x, b = blockIdx.z, p = blockIdx.y, a0 = blockIdx.x * A;
  const int nt = a.nt, nx = a.nx;
  const float* d = a.in + (long long)b * nx * nt;
  const float t0s = a.t0s[p], cv = a.cv[p];
  float acc[A][TPT];
#pragma unroll
  for (int i = 0; i < A; ++i)
#pragma unroll
    for (int k = 0; k < TPT; ++k) acc[i][k] = 0.f;
  float nxt[TPT];
#pragma unroll
  for (int k = 0; k < TPT; ++k) {
    const int tau = tid + T * k;
    nxt[k] = tau < nt ? __ldg(d + tau) : 0.f;
  }
  for (int r = 0; r < nx; ++r) {
    float* cur = tr + (r & 1) * nt;
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
      const int tau = tid + T * k;
      if (tau < nt) cur[tau] = nxt[k];
    }
    __syncthreads();
    if (r + 1 < nx) {
#pragma unroll
      for (int k = 0; k < TPT; ++k) {
        const int tau = tid + T * k;
        nxt[k] = tau < nt ? __ldg(d + (long long)(r + 1) * nt + tau) : 0.f;
      }
    }
#pragma unroll
    for (int i = 0; i < A; ++i) {
      const float hs = (float)(r - (a0 + i)) * cv;
      const float hs2 = hs * hs;
#pragma unroll
      for (int k = 0; k < TPT; ++k) {
        const int tau = tid + T * k;
        if (tau < nt) {
          int i0;
          float f;
          td_path(t0s, hs2, tau, i0, f);
          float v = 0.f;
          if (i0 < nt) v = (1.f - f) * cur[i0];
          if (i0 + 1 < nt) v = fmaf(f, cur[i0 + 1], v);
          acc[i][k] += v;
        }
      }
    }
  }
  float* m = a.out + ((long long)b * a.P + p) * nx * nt;
#pragma unroll
  for (int i = 0; i < A; ++i) {
    const int ai = a0 + i;
    if (ai >= nx) break;
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
      const int tau = tid + T * k;
      if (tau < nt) m[(long long)ai * nt + tau] = acc[i][k];
    }
  }
}

template <int TPT>
__host__ __device__ constexpr int td_traces_per_cta() {
  return TPT <= 4 ? 8 : 32 / TPT;
}

// Forward: R output traces per CTA, accumulated in shared memory.
template <int TPT>
__global__ void __launch_bounds__(kTdThreads) td_forward_kernel(TdArgs a) {
  constexpr int T = kTdThreads, R = td_traces_per_cta<TPT>();
  extern __shared__ float acc[];                // [R][nt]
  const int tid = threadIdx.x, b = blockIdx.y, r0 = blockIdx.x * R;
  const int nt = a.nt, nx = a.nx;
  for (int i = tid; i < R * nt; i += T) acc[i] = 0.f;
  __syncthreads();
  const float* m = a.in + (long long)b * a.P * nx * nt;
  const int rows = a.P * nx;                    // model rows (panel, apex)
  float nxt[TPT];
#pragma unroll
  for (int k = 0; k < TPT; ++k) {
    const int tau = tid + T * k;
    nxt[k] = tau < nt ? __ldg(m + tau) : 0.f;
  }
  for (int row = 0; row < rows; ++row) {
    float mv[TPT];
#pragma unroll
    for (int k = 0; k < TPT; ++k) mv[k] = nxt[k];
    if (row + 1 < rows) {
#pragma unroll
      for (int k = 0; k < TPT; ++k) {
        const int tau = tid + T * k;
        nxt[k] = tau < nt ? __ldg(m + (long long)(row + 1) * nt + tau) : 0.f;
      }
    }
    const int p = row / nx, ap = row - p * nx;
    const float t0s = a.t0s[p], cv = a.cv[p];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int r = r0 + i;
      if (r >= nx) break;
      const float hs = (float)(r - ap) * cv;
      const float hs2 = hs * hs;
      float* out = acc + i * nt;
#pragma unroll
      for (int k = 0; k < TPT; ++k) {
        const int tau = tid + T * k;
        if (tau < nt) {
          int i0;
          float f;
          td_path(t0s, hs2, tau, i0, f);
          if (i0 < nt) atomicAdd(out + i0, (1.f - f) * mv[k]);
          if (i0 + 1 < nt) atomicAdd(out + i0 + 1, f * mv[k]);
        }
      }
    }
  }
  __syncthreads();
  float* d = a.out + (long long)b * nx * nt;
  for (int i = 0; i < R; ++i) {
    const int r = r0 + i;
    if (r >= nx) break;
    for (int t = tid; t < nt; t += T) d[(long long)r * nt + t] = acc[i * nt + t];
  }
}

template <int TPT>
cudaError_t launch_td(bool adjoint, const TdArgs& a, int batch, cudaStream_t s) {
  if (adjoint) {
    constexpr int A = 32 / TPT;
    dim3 grid((a.nx + A - 1) / A, a.P, batch);
    td_adjoint_kernel<TPT><<<grid, kTdThreads, 2 * a.nt * sizeof(float), s>>>(a);
  } else {
    constexpr int R = td_traces_per_cta<TPT>();
    dim3 grid((a.nx + R - 1) / R, batch);
    td_forward_kernel<TPT><<<grid, kTdThreads, R * a.nt * sizeof(float), s>>>(a);
  }
  return cudaGetLastError();
}

ashrt_status td_call(const char* name, bool adjoint, int nt, int nx, double dt, double dx,
                     const float* velocities, int nv, const float* t0_shifts, int nt0,
                     const float* in, float* out, int batch, void* stream) {
  if (!in || !out || !velocities || nv < 1 || nt < 2 || nt > 4096 || nx < 1 || batch < 1 ||
      !(dt > 0.0) || !(dx > 0.0) || !std::isfinite(dt) || !std::isfinite(dx)) {
    set_error("%s: need in/out pointers, velocities, nv > 0, 2 <= nt <= 4096, nx > 0, "
              "batch > 0, dt > 0, dx > 0", name);
    return ASHRT_EINVAL;
  }
  if (nt0 < 1 || (!t0_shifts && nt0 != 1) || (long long)nv * nt0 > kTdMaxPanels) {
    set_error("%s: need nt0 >= 1 (1 when t0_shifts is NULL) and nv * nt0 <= %d", name,
              kTdMaxPanels);
    return ASHRT_EINVAL;
  }
  TdArgs a;
  a.in = in;
  a.out = out;
  a.nt = nt;
  a.nx = nx;
  a.P = nv * nt0;
  for (int i = 0; i < nv; ++i) {
    const double v = (double)velocities[i];
    if (!(v > 0.0) || !std::isfinite(v)) {
      set_error("%s: velocity %d must be positive and finite", name, i);
      return ASHRT_EINVAL;
    }
  }
  for (int j = 0; j < nt0; ++j) {
    const double t0 = t0_shifts ? (double)t0_shifts[j] : 0.0;
    if (!(t0 >= 0.0) || !std::isfinite(t0)) {
      set_error("%s: asymptote shift %d must be >= 0 and finite", name, j);
      return ASHRT_EINVAL;
    }
    for (int i = 0; i < nv; ++i) {
      a.t0s[j * nv + i] = (float)(t0 / dt);
      a.cv[j * nv + i] = (float)(dx / ((double)velocities[i] * dt));
    }
  }
  int tpt = 1;
  while (tpt * kTdThreads < nt) tpt *= 2;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  switch (tpt) {
    case 1: e = launch_td<1>(adjoint, a, batch, s); break;
    case 2: e = launch_td<2>(adjoint, a, batch, s); break;
    case 4: e = launch_td<4>(adjoint, a, batch, s); break;
    case 8: e = launch_td<8>(adjoint, a, batch, s); break;
    default: e = launch_td<16>(adjoint, a, batch, s); break;
  }
  count_launches(1);
  if (e != cudaSuccess) {
    set_error("%s: launch failed: %s", name, cudaGetErrorString(e));
    return ASHRT_ECUDA;
  }
  return ASHRT_OK;
}

}  // namespace
}  // namespace ashrt

using namespace ashrt;

extern "C" ashrt_status ashrt_td_forward(int nt, int nx, double dt, double dx,
                                         const float* velocities, int nv, const float* t0_shifts,
                                         int nt0, const float* m_dev, float* d_dev, int batch,
                                         void* stream) {
  return td_call("ashrt_td_forward", false, nt, nx, dt, dx, velocities, nv, t0_shifts, nt0, m_dev,
                 d_dev, batch, stream);
}

extern "C" ashrt_status ashrt_td_adjoint(int nt, int nx, double dt, double dx,
                                         const float* velocities, int nv, const float* t0_shifts,
                                         int nt0, const float* d_dev, float* m_dev, int batch,
                                         void* stream) {
  return td_call("ashrt_td_adjoint", true, nt, nx, dt, dx, velocities, nv, t0_shifts, nt0, d_dev,
                 m_dev, batch, stream);
}
