// Traces at irregular positions (ch. 6: for non-uniformly sampled x the F
// operator is replaced by a discrete Fourier transform evaluated at the
// trace positions; ch. 5, ch. 6 cost discussion).
//
// The model keeps its regular apex grid x_a = j dx (the Stolt map needs it),
// so only the data side of the operator pair changes: the trace-axis
// synthesis of the forward, which the regular plan does with a c2r FFT from
// the half spectrum Y[l][t] (l = 0 .. Nx/2), becomes
//   d[j][t] = sum_l c_l Re( E[j][l] Y[l][t] ),   E[j][l] = exp(+2 pi i l x_j / (Nx dx)),
// with c_0 = c_{Nx/2} = 1 and c_l = 2 otherwise (the half spectrum of a real
// field; the Nyquist row enters as cos(pi x_j / dx)), and the adjoint's
// trace-axis analysis becomes its transpose
//   Yhat[l][t] = sum_j conj(E[j][l]) d[j][t].
// At x_j = j dx both reduce to the regular transforms.  The tables are built
// on the host in FP64 (c_l folded into the synthesis table).
//
// Both are dense complex contractions per gather, M x N x K = nr x nt x Lh
// and Lh x nt x nr, done here as FP32 tiled kernels on the CUDA cores: a
// 64 x 64 output tile per CTA, K staged through shared memory in chunks of
// 16, 4 x 4 outputs per thread.  The IRLS weights and the trace mask are
// fused into the synthesis epilogue (with the per-gather squared norm of the
// output for the CG scalars) and into the analysis operand load.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "internal.h"

namespace ashrt {
namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16, kThr = 256;

__device__ __forceinline__ double warp_sum_dbl(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// d[g][j][t] = (sum_l Re(Es[j][l] Y[g][l][t])) * ew[g][j][t] * tmask[g][j];
// dot[g] += sum d^2.  grid (ceil(nt/64), ceil(nr/64), batch).
__global__ void __launch_bounds__(kThr) k_irr_synth(const float2* __restrict__ Es,
                                                    const float2* __restrict__ Y,
                                                    float* __restrict__ d, int nr, int nt, int Lh,
                                                    int ld, long long y_batch,
                                                    const float* __restrict__ ew,
                                                    const float* __restrict__ tmask,
                                                    double* __restrict__ dot) {
  __shared__ float2 As[kBK][kBM];   // As[l][j]
  __shared__ float2 Bs[kBK][kBN];   // Bs[l][t]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int t0 = blockIdx.x * kBN, j0 = blockIdx.y * kBM, g = blockIdx.z;
  const float2* Yg = Y + (long long)g * y_batch;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[i][q] = 0.f;
  for (int k0 = 0; k0 < Lh; k0 += kBK) {
    // A chunk: 64 j x 16 l complex; thread loads 4 (one j, 4 consecutive l)
    {
      const int jj = tid >> 2, kk = (tid & 3) * 4;
      const int j = j0 + jj;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int l = k0 + kk + u;
        As[kk + u][jj] = (j < nr && l < Lh) ? __ldg(Es + (long long)j * Lh + l)
                                            : make_float2(0.f, 0.f);
      }
    }
    // B chunk: 16 l x 64 t complex; thread loads 4 consecutive t of one l
    {
      const int kk = tid >> 4, tt = (tid & 15) * 4;
      const int l = k0 + kk;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int t = t0 + tt + u;
        Bs[kk][tt + u] = (l < Lh && t < nt) ? __ldg(Yg + (long long)l * ld + t)
                                            : make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kBK; ++k) {
      float2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty * 4 + i];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Bs[k][tx * 4 + q];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = fmaf(a[i].x, b[q].x, fmaf(-a[i].y, b[q].y, acc[i][q]));
    }
    __syncthreads();
  }
  float part = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int j = j0 + ty * 4 + i;
    if (j >= nr) continue;
    const float tm = tmask ? __ldg(tmask + (long long)g * nr + j) : 1.f;
    const long long row = ((long long)g * nr + j) * nt;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int t = t0 + tx * 4 + q;
      if (t >= nt) continue;
      float v = acc[i][q] * tm;
      if (ew) v *= __ldg(ew + row + t);
      d[row + t] = v;
      part = fmaf(v, v, part);
    }
  }
  if (dot) {
    __shared__ double red[kThr / 32];
    double p = warp_sum_dbl((double)part);
    if ((tid & 31) == 0) red[tid >> 5] = p;
    __syncthreads();
    if (tid < 32) {
      p = tid < kThr / 32 ? red[tid] : 0.0;
      p = warp_sum_dbl(p);
      if (tid == 0 && p != 0.0) atomicAdd(dot + g, p);
    }
  }
}

// Yhat[g][l][t] = sum_j Ea[l][j] (d[g][j][t] * ew[g][j][t] * tmask[g][j]),
// Ea = conj(E)^T.  grid (ceil(nt/64), ceil(Lh/64), batch).
__global__ void __launch_bounds__(kThr) k_irr_analysis(const float2* __restrict__ Ea,
                                                       const float* __restrict__ d,
                                                       float2* __restrict__ Yh, int nr, int nt,
                                                       int Lh, int ld, long long y_batch,
                                                       const float* __restrict__ ew,
                                                       const float* __restrict__ tmask) {
  __shared__ float2 As[kBK][kBM];   // As[j][l]
  __shared__ float Bs[kBK][kBN];    // Bs[j][t]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int t0 = blockIdx.x * kBN, l0 = blockIdx.y * kBM, g = blockIdx.z;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[i][q] = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < nr; k0 += kBK) {
    {
      const int ll = tid >> 2, kk = (tid & 3) * 4;
      const int l = l0 + ll;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = k0 + kk + u;
        As[kk + u][ll] = (l < Lh && j < nr) ? __ldg(Ea + (long long)l * nr + j)
                                            : make_float2(0.f, 0.f);
      }
    }
    {
      const int kk = tid >> 4, tt = (tid & 15) * 4;
      const int j = k0 + kk;
      const float tm = (j < nr && tmask) ? __ldg(tmask + (long long)g * nr + j) : 1.f;
      const long long row = ((long long)g * nr + j) * nt;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int t = t0 + tt + u;
        float v = 0.f;
        if (j < nr && t < nt) {
          v = __ldg(d + row + t) * tm;
          if (ew) v *= __ldg(ew + row + t);
        }
        Bs[kk][tt + u] = v;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kBK; ++k) {
      float2 a[4];
      float b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty * 4 + i];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Bs[k][tx * 4 + q];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[i][q].x = fmaf(a[i].x, b[q], acc[i][q].x);
          acc[i][q].y = fmaf(a[i].y, b[q], acc[i][q].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int l = l0 + ty * 4 + i;
    if (l >= Lh) continue;
    float2* out = Yh + (long long)g * y_batch + (long long)l * ld;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int t = t0 + tx * 4 + q;
      if (t < nt) out[t] = acc[i][q];
    }
  }
}

// r -= alpha q on the data side (the CGLS update the regular adjoint fuses
// into its trace-axis transform), per gather alpha = coef[g].z.
__global__ void k_irr_cg_r(float* __restrict__ r, const float* __restrict__ q, long long n,
                           const float4* __restrict__ coef) {
  const int g = blockIdx.y;
  const float a = coef[g].z;
  const long long off = (long long)g * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    r[off + i] = fmaf(-a, q[off + i], r[off + i]);
}

}  // namespace

bool build_irregular_tables(const double* x, int nr, int Nx, double dx, float2* Es, float2* Ea) {
  const int Lh = Nx / 2 + 1;
  for (int j = 0; j < nr; ++j) {
    if (!std::isfinite(x[j])) return false;
    for (int l = 0; l < Lh; ++l) {
      double re, im;
      if (l == Nx / 2) {
        re = std::cos(M_PI * x[j] / dx);
        im = 0.0;
      } else {
        // reduce the phase l x / (Nx dx) modulo 1 before scaling by 2 pi
        double ph = (double)l * x[j] / ((double)Nx * dx);
        ph -= std::floor(ph);
        re = std::cos(2.0 * M_PI * ph);
        im = std::sin(2.0 * M_PI * ph);
      }
      const double c = (l == 0 || l == Nx / 2) ? 1.0 : 2.0;
      Es[(size_t)j * Lh + l] = make_float2((float)(c * re), (float)(c * im));
      Ea[(size_t)l * nr + j] = make_float2((float)re, (float)(-im));
    }
  }
  return true;
}

cudaError_t launch_irr_synth(const float2* Es, const float2* Y, float* d, int nr, int nt, int Lh,
                             int ld, long long y_batch, const float* ew, const float* tmask,
                             double* dot, int batch, cudaStream_t s) {
  dim3 grid((nt + kBN - 1) / kBN, (nr + kBM - 1) / kBM, batch);
  k_irr_synth<<<grid, kThr, 0, s>>>(Es, Y, d, nr, nt, Lh, ld, y_batch, ew, tmask, dot);
  return cudaGetLastError();
}

cudaError_t launch_irr_analysis(const float2* Ea, const float* d, float2* Yh, int nr, int nt,
                                int Lh, int ld, long long y_batch, const float* ew,
                                const float* tmask, int batch, cudaStream_t s) {
  dim3 grid((nt + kBN - 1) / kBN, (Lh + kBM - 1) / kBM, batch);
  k_irr_analysis<<<grid, kThr, 0, s>>>(Ea, d, Yh, nr, nt, Lh, ld, y_batch, ew, tmask);
  return cudaGetLastError();
}

cudaError_t launch_irr_cg_r(float* r, const float* q, long long n, const float4* coef, int batch,
                            cudaStream_t s) {
  long long gx = (n + 256 * 8 - 1) / (256 * 8);
  if (gx > 1024) gx = 1024;
  k_irr_cg_r<<<dim3((unsigned)(gx < 1 ? 1 : gx), batch), 256, 0, s>>>(r, q, n, coef);
  return cudaGetLastError();
}

}  // namespace ashrt
