// Trace-axis (x) transforms of the Stolt ASHRT: the F_x part of the 2-D
// Fourier transforms F of ch. 5 Eqs ch5_forward_operator / ch5_adj_operator.
//
//   r2c: a real [nx][nt] panel, zero-padded to Nx traces, -> its half spectrum
//        in k_x, [Lh = Nx/2 + 1][nt] complex (analysis, exp(-i k_x x)).
//   c2r: a Hermitian half spectrum [Lh][nt] -> the real panel, synthesis
//        exp(+i k_x x), unnormalised, cropped to nx traces.
//
// One CTA transforms 2*C consecutive time columns of one panel: columns
// t0 + c and t0 + C + c are packed as the real and imaginary parts of one
// complex sequence, transformed together, and separated with the Hermitian
// symmetry of real signals.  The length-Nx transforms run as Stockham passes
// over a shared [Nx][C] tile; the first pass is fed straight from global
// memory and (c2r) the last pass stores straight to global memory.  The
// per-element weights of the IRLS operator (W_m^-1 on the model side,
// W_r and the sampling mask on the data side) are fused into those loads and
// stores, and the c2r kernel can also accumulate the FP64 sum of squares of
// what it stores (the CGLS norms) per gather.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace ashrt {

namespace {

constexpr int kCols = 8;   // complex columns per CTA (16 real time samples)

template <int DIR, int N, int C, int R>
__device__ __forceinline__ void col_pass(float2* sm, int Ns, const float2* __restrict__ tw,
                                         int off, int tid) {
  constexpr int T = N * C / 16, NB = 16 / R, JS = T / C;
  const int col = tid % C, j0 = tid / C;
  float2 v[16];
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int jb = j0 + JS * q;
#pragma unroll
    for (int r = 0; r < R; ++r) v[q * R + r] = sm[(jb + r * (N / R)) * C + col];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int jb = j0 + JS * q;
    const int k = jb & (Ns - 1);
    if (Ns > 1) twiddle_r<R>(&v[q * R], base_twiddle<DIR>(tw, off, k));
    dft_r<DIR, R>(&v[q * R]);
    const int base = (jb - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) sm[(base + r * Ns) * C + col] = v[q * R + r];
  }
  __syncthreads();
}

template <int DIR, int LOGN, int C, int Q0, int Q1>
__device__ __forceinline__ void col_pass_range(float2* sm, const float2* __restrict__ tw, int tid) {
  using S = Sched<LOGN>;
  if constexpr (Q0 < Q1) {
    col_pass<DIR, S::N, C, S::radix(Q0)>(sm, S::ns(Q0), tw, S::tw_off(Q0), tid);
    col_pass_range<DIR, LOGN, C, Q0 + 1, Q1>(sm, tw, tid);
  }
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Adds the CTA-wide sum of `part` to *dst (one atomic per CTA).
__device__ __forceinline__ void block_accumulate(double part, double* dst) {
  __shared__ double red[32];
  part = warp_sum(part);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = part;
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    double x = lane < nw ? red[lane] : 0.0;
    x = warp_sum(x);
    if (lane == 0) atomicAdd(dst, x);
  }
}

template <int LOGN>
__global__ void __launch_bounds__((1 << LOGN) * kCols / 16)
xfft_r2c_kernel(XfftArgs a) {
  constexpr int N = 1 << LOGN, C = kCols, T = N * C / 16, JS = T / C;
  using S = Sched<LOGN>;
  extern __shared__ float2 sm[];   // [N][C]
  const int tid = threadIdx.x, col = tid % C, j0 = tid / C;
  const long long slab = blockIdx.x;
  const int t0 = blockIdx.y * 2 * C;
  const int ta = t0 + col, tb = t0 + C + col;
  const bool oka = ta < a.nt, okb = tb < a.nt;
  const float* in = a.in_real + slab * a.slab_real;
  const float* ew = a.ew ? a.ew + slab * a.slab_real : nullptr;
  const float* tm = a.tmask ? a.tmask + (slab / a.slabs_per_gather) * a.nx : nullptr;

  // first pass (radix 8, Ns = 1): inputs at rows jb + r N/8; rows >= nx are the zero padding
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int jb = j0 + JS * q;
    float2 v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int row = jb + r * (N / 8);
      float xa = 0.f, xb = 0.f;
      if (row < a.nx) {
        const long long o = (long long)row * a.nt;
        float wa = 1.f, wb = 1.f;
        if (ew) { wa = oka ? __ldg(ew + o + ta) : 0.f; wb = okb ? __ldg(ew + o + tb) : 0.f; }
        const float g = tm ? __ldg(tm + row) : 1.f;
        xa = oka ? __ldg(in + o + ta) * wa * g : 0.f;
        xb = okb ? __ldg(in + o + tb) * wb * g : 0.f;
      }
      v[r] = make_float2(xa, xb);
    }
    dft8<-1>(v);
#pragma unroll
    for (int r = 0; r < 8; ++r) sm[(jb * 8 + r) * C + col] = v[r];
  }
  __syncthreads();
  col_pass_range<-1, LOGN, C, 1, S::NPASS>(sm, a.tw, tid);

  // separate the two packed real columns: A = (Z_l + conj Z_{N-l}) / 2,
  // B = (Z_l - conj Z_{N-l}) / (2i), for 0 <= l <= N/2
  float2* out = a.out_cplx + slab * a.slab_cplx;
  for (int f = tid; f < (N / 2 + 1) * C; f += T) {
    const int l = f / C, c = f % C;
    const float2 zl = sm[l * C + c];
    const float2 zm = sm[((N - l) & (N - 1)) * C + c];
    const float2 A = make_float2(0.5f * (zl.x + zm.x), 0.5f * (zl.y - zm.y));
    const float2 B = make_float2(0.5f * (zl.y + zm.y), -0.5f * (zl.x - zm.x));
    if (t0 + c < a.nt) out[(long long)l * a.ld + t0 + c] = A;
    if (t0 + C + c < a.nt) out[(long long)l * a.ld + t0 + C + c] = B;
  }
}

// Hermitian extension of a stored half spectrum: row l of the full length-N
// spectrum; rows 0 and N/2 keep their real parts only (real signal).
template <int N>
__device__ __forceinline__ float2 herm_load(const float2* __restrict__ base, int ld, int row, int t,
                                            bool ok) {
  if (!ok) return make_float2(0.f, 0.f);
  if (row == 0 || row == N / 2) {
    float2 y = __ldg(base + (long long)row * ld + t);
    return make_float2(y.x, 0.f);
  }
  if (row < N / 2) return __ldg(base + (long long)row * ld + t);
  float2 y = __ldg(base + (long long)(N - row) * ld + t);
  return make_float2(y.x, -y.y);
}

template <int LOGN>
__global__ void __launch_bounds__((1 << LOGN) * kCols / 16)
xfft_c2r_kernel(XfftArgs a) {
  constexpr int N = 1 << LOGN, C = kCols, T = N * C / 16, JS = T / C;
  using S = Sched<LOGN>;
  extern __shared__ float2 sm[];   // [N][C]
  const int tid = threadIdx.x, col = tid % C, j0 = tid / C;
  const long long slab = blockIdx.x;
  const int t0 = blockIdx.y * 2 * C;
  const int ta = t0 + col, tb = t0 + C + col;
  const bool oka = ta < a.nt, okb = tb < a.nt;
  const float2* in = a.in_cplx + slab * a.slab_cplx;

  // first pass: Z = A + i B with A, B the Hermitian-extended spectra of the two columns
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int jb = j0 + JS * q;
    float2 v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int row = jb + r * (N / 8);
      const float2 A = herm_load<N>(in, a.ld, row, ta, oka);
      const float2 B = herm_load<N>(in, a.ld, row, tb, okb);
      v[r] = make_float2(A.x - B.y, A.y + B.x);
    }
    dft8<+1>(v);
#pragma unroll
    for (int r = 0; r < 8; ++r) sm[(jb * 8 + r) * C + col] = v[r];
  }
  __syncthreads();
  col_pass_range<+1, LOGN, C, 1, S::NPASS - 1>(sm, a.tw, tid);

  // last pass straight to global: output r of butterfly jb is trace jb + r Ns
  constexpr int Q = S::NPASS - 1, R = S::radix(Q), NB = 16 / R, Ns = S::ns(Q);
  float2 v[16];
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int jb = j0 + JS * q;
#pragma unroll
    for (int r = 0; r < R; ++r) v[q * R + r] = sm[(jb + r * (N / R)) * C + col];
  }
  float* out = a.out_real + slab * a.slab_real;
  const float* ew = a.ew ? a.ew + slab * a.slab_real : nullptr;
  const float* tm = a.tmask ? a.tmask + (slab / a.slabs_per_gather) * a.nx : nullptr;
  float ss = 0.f;
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int jb = j0 + JS * q;
    if (Ns > 1) twiddle_r<R>(&v[q * R], base_twiddle<+1>(a.tw, S::tw_off(Q), jb));
    dft_r<+1, R>(&v[q * R]);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int row = jb + r * Ns;
      if (row < a.nx) {
        const long long o = (long long)row * a.nt;
        const float g = tm ? __ldg(tm + row) : 1.f;
        if (oka) {
          const float x = v[q * R + r].x * g * (ew ? __ldg(ew + o + ta) : 1.f);
          out[o + ta] = x;
          ss = fmaf(x, x, ss);
        }
        if (okb) {
          const float x = v[q * R + r].y * g * (ew ? __ldg(ew + o + tb) : 1.f);
          out[o + tb] = x;
          ss = fmaf(x, x, ss);
        }
      }
    }
  }
  if (a.dot) block_accumulate((double)ss, a.dot + slab / a.slabs_per_gather);
}

template <int LOGN>
cudaError_t launch_r2c_t(const XfftArgs& a, cudaStream_t s) {
  constexpr int N = 1 << LOGN, T = N * kCols / 16;
  const size_t smem = (size_t)N * kCols * sizeof(float2);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(xfft_r2c_kernel<LOGN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid(a.slabs, (a.nt + 2 * kCols - 1) / (2 * kCols));
  xfft_r2c_kernel<LOGN><<<grid, T, smem, s>>>(a);
  return cudaGetLastError();
}

template <int LOGN>
cudaError_t launch_c2r_t(const XfftArgs& a, cudaStream_t s) {
  constexpr int N = 1 << LOGN, T = N * kCols / 16;
  const size_t smem = (size_t)N * kCols * sizeof(float2);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(xfft_c2r_kernel<LOGN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid(a.slabs, (a.nt + 2 * kCols - 1) / (2 * kCols));
  xfft_c2r_kernel<LOGN><<<grid, T, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

int xfft_log2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

cudaError_t launch_xfft_r2c(const XfftArgs& a, cudaStream_t s) {
  switch (xfft_log2(a.Nx)) {
    case 4: return launch_r2c_t<4>(a, s);
    case 5: return launch_r2c_t<5>(a, s);
    case 6: return launch_r2c_t<6>(a, s);
    case 7: return launch_r2c_t<7>(a, s);
    case 8: return launch_r2c_t<8>(a, s);
    case 9: return launch_r2c_t<9>(a, s);
    case 10: return launch_r2c_t<10>(a, s);
    case 11: return launch_r2c_t<11>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_xfft_c2r(const XfftArgs& a, cudaStream_t s) {
  switch (xfft_log2(a.Nx)) {
    case 4: return launch_c2r_t<4>(a, s);
    case 5: return launch_c2r_t<5>(a, s);
    case 6: return launch_c2r_t<6>(a, s);
    case 7: return launch_c2r_t<7>(a, s);
    case 8: return launch_c2r_t<8>(a, s);
    case 9: return launch_c2r_t<9>(a, s);
    case 10: return launch_c2r_t<10>(a, s);
    case 11: return launch_c2r_t<11>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ashrt
