// Learned warm start: a 4-level U-Net (the same architecture as the FP64
// reference of the tests) with hand-written forward and backward kernels.
// BF16 storage for weights and activations, FP32 accumulation, FP32 master
// weights and gradients, Adam.  It maps a pseudo-deblended gather to an
// initial Radon model (P channels) and initial IRLS residual weights
// (log W_r, one channel) for the warm-started robust solve.
//
// Layouts: activations NHWC (image rows = traces x, columns = time t, so a
// gather [nx][nt] is an nx x nt image) with a per-tensor pixel stride and
// channel offset, so skip connections are written straight into the channel
// slice of the concatenation buffer they feed.  Convolution weights are kept
// in FP32 "OIHW" order (the reference's order) and converted every step to a
// BF16 [tap][ci][co] copy (forward) and a flipped, transposed [tap][co][ci]
// copy (gradient with respect to the input).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace {

using bf16 = __nv_bfloat16;

constexpr int kPix = 128;   // pixels (along a row) per CTA
constexpr int kCh = 16;     // input / output channel tile

template <typename T>
__device__ __forceinline__ float ld_f(const T* p, long long i);
template <>
__device__ __forceinline__ float ld_f<float>(const float* p, long long i) { return p[i]; }

template <typename T>
__device__ __forceinline__ void st_f(T* p, long long i, float v);
template <>
__device__ __forceinline__ void st_f<float>(float* p, long long i, float v) { p[i] = v; }
template <>
__device__ __forceinline__ void st_f<bf16>(bf16* p, long long i, float v) { p[i] = __float2bfloat16(v); }

struct Tensor {        // a channel slice of an NHWC buffer
  void* p = nullptr;
  int ps = 0;          // channels allocated per pixel
  int off = 0;         // first channel of the slice
};

struct ConvArgs {
  Tensor in;           // input: fp32 gradients (the CUDA-core fallback of the backward)
  Tensor mask;         // bf16 activation: multiply input by (mask > 0), or p == nullptr
  const bf16* w;       // [K*K][Cin][Cout]
  const float* bias;   // [Cout] or nullptr
  Tensor out;
  int N, H, W, Cin, Cout, relu;
};

// y[p, co] = bias[co] + sum_{tap, ci} x[p + tap, ci] * w[tap][ci][co], "same"
// zero padding, optional ReLU.  CTA: 128 consecutive pixels of one image row
// x 16 output channels; input channels in tiles of 16 staged in shared
// memory (3 rows x 130 pixels with the halo) together with the weight tile.
template <int K, typename TI, typename TO>
__global__ void __launch_bounds__(kPix) k_conv(ConvArgs a) {
  constexpr int R = K / 2, PW = kPix + 2 * R;
  __shared__ float xs[K][kCh][PW + 1];
  __shared__ __align__(16) float ws[K * K][kCh][kCh];
  const int tid = threadIdx.x;
  const int xt = (a.W + kPix - 1) / kPix;
  const int row = blockIdx.x / xt;               // n * H + y
  const int x0 = (blockIdx.x % xt) * kPix;
  const int n = row / a.H, y = row % a.H;
  const int co0 = blockIdx.y * kCh;
  const TI* in = (const TI*)a.in.p;
  const bf16* mk = (const bf16*)a.mask.p;
  float acc[kCh];
#pragma unroll
  for (int c = 0; c < kCh; ++c) acc[c] = 0.f;

  for (int ci0 = 0; ci0 < a.Cin; ci0 += kCh) {
    for (int e = tid; e < K * PW * kCh; e += kPix) {
      const int c = e % kCh, px = (e / kCh) % PW, r = e / (kCh * PW);
      const int yy = y + r - R, xx = x0 + px - R, ci = ci0 + c;
      float v = 0.f;
      if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W && ci < a.Cin) {
        const long long pix = ((long long)n * a.H + yy) * a.W + xx;
        v = ld_f(in, pix * a.in.ps + a.in.off + ci);
        if (mk && __bfloat162float(mk[pix * a.mask.ps + a.mask.off + ci]) <= 0.f) v = 0.f;
      }
      xs[r][c][px] = v;
    }
    for (int e = tid; e < K * K * kCh * kCh; e += kPix) {
      const int co = e % kCh, ci = (e / kCh) % kCh, tap = e / (kCh * kCh);
      float v = 0.f;
      if (ci0 + ci < a.Cin && co0 + co < a.Cout)
        v = __bfloat162float(a.w[((long long)tap * a.Cin + ci0 + ci) * a.Cout + co0 + co]);
      ws[tap][ci][co] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int ci = 0; ci < kCh; ++ci) {
#pragma unroll
      for (int tap = 0; tap < K * K; ++tap) {
        const float v = xs[tap / K][ci][tid + tap % K];
        const float4* wp = (const float4*)&ws[tap][ci][0];
#pragma unroll
        for (int q = 0; q < kCh / 4; ++q) {
          const float4 w4 = wp[q];
          acc[4 * q + 0] = fmaf(v, w4.x, acc[4 * q + 0]);
          acc[4 * q + 1] = fmaf(v, w4.y, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(v, w4.z, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(v, w4.w, acc[4 * q + 3]);
        }
      }
    }
    __syncthreads();
  }
  const int xx = x0 + tid;
  if (xx >= a.W) return;
  const long long pix = ((long long)n * a.H + y) * a.W + xx;
  TO* out = (TO*)a.out.p;
#pragma unroll
  for (int c = 0; c < kCh; ++c) {
    const int co = co0 + c;
    if (co >= a.Cout) break;
    float v = acc[c] + (a.bias ? a.bias[co] : 0.f);
    if (a.relu) v = fmaxf(v, 0.f);
    st_f(out, pix * a.out.ps + a.out.off + co, v);
  }
}

struct WgradArgs {
  Tensor in;          // bf16 layer input
  Tensor g;           // fp32 gradient of the layer output
  Tensor mask;        // bf16 layer output (ReLU mask) or p == nullptr
  float* gw;          // [Cout][Cin][K][K] fp32 (the master weights' layout), accumulated
  float* gb;          // [Cout] fp32, accumulated
  int N, H, W, Cin, Cout;
  int rows_per;       // image rows (over all N*H) one CTA reduces before its atomics
};

// gw[co][ci][tap] += sum_p x[p + tap, ci] g_eff[p, co]; gb[co] += sum_p g_eff[p, co]
// with g_eff = g (mask > 0).  CTA: a 128-pixel column strip of rows_per image
// rows x 16 input x 16 output channels; thread (ci, co) accumulates all K*K
// taps over the strip, then one atomic each.
template <int K>
__global__ void __launch_bounds__(256) k_wgrad(WgradArgs a) {
  constexpr int R = K / 2, PW = kPix + 2 * R;
  __shared__ float xs[K][kCh][PW + 1];
  __shared__ float gs[kCh][kPix + 1];
  const int tid = threadIdx.x;
  const int xt = (a.W + kPix - 1) / kPix;
  const int x0 = (blockIdx.x % xt) * kPix;
  const int row0 = (blockIdx.x / xt) * a.rows_per;
  const int row1 = min(row0 + a.rows_per, a.N * a.H);
  const int ci0 = blockIdx.y * kCh, co0 = blockIdx.z * kCh;
  const bf16* in = (const bf16*)a.in.p;
  const float* g = (const float*)a.g.p;
  const bf16* mk = (const bf16*)a.mask.p;
  const int ci = tid / kCh, co = tid % kCh;
  float acc[K * K];
#pragma unroll
  for (int t = 0; t < K * K; ++t) acc[t] = 0.f;
  float gsum = 0.f;
  for (int row = row0; row < row1; ++row) {
    const int n = row / a.H, y = row % a.H;
    for (int e = tid; e < K * PW * kCh; e += 256) {
      const int c = e % kCh, px = (e / kCh) % PW, r = e / (kCh * PW);
      const int yy = y + r - R, xx = x0 + px - R, cc = ci0 + c;
      float v = 0.f;
      if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W && cc < a.Cin)
        v = __bfloat162float(in[(((long long)n * a.H + yy) * a.W + xx) * a.in.ps + a.in.off + cc]);
      xs[r][c][px] = v;
    }
    for (int e = tid; e < kPix * kCh; e += 256) {
      const int c = e % kCh, px = e / kCh;
      const int xx = x0 + px, cc = co0 + c;
      float v = 0.f;
      if (xx < a.W && cc < a.Cout) {
        const long long pix = ((long long)n * a.H + y) * a.W + xx;
        v = g[pix * a.g.ps + a.g.off + cc];
        if (mk && __bfloat162float(mk[pix * a.mask.ps + a.mask.off + cc]) <= 0.f) v = 0.f;
      }
      gs[c][px] = v;
    }
    __syncthreads();
    for (int px = 0; px < kPix; ++px) {
      const float gv = gs[co][px];
      gsum += gv;
#pragma unroll
      for (int t = 0; t < K * K; ++t) acc[t] = fmaf(xs[t / K][ci][px + t % K], gv, acc[t]);
    }
    __syncthreads();
  }
  if (ci0 + ci < a.Cin && co0 + co < a.Cout) {
#pragma unroll
    for (int t = 0; t < K * K; ++t)
      atomicAdd(&a.gw[((long long)(co0 + co) * a.Cin + ci0 + ci) * (K * K) + t], acc[t]);
  }
  if (ci == 0 && blockIdx.y == 0 && co0 + co < a.Cout) atomicAdd(&a.gb[co0 + co], gsum);
}

// 2x2 average pooling (forward, bf16) and its transpose (accumulated, fp32).
__global__ void k_pool(Tensor in, Tensor out, int N, int H, int W, int C) {
  const int Ho = H / 2, Wo = W / 2;
  const long long total = (long long)N * Ho * Wo * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long p = i / C;
    const int xo = (int)(p % Wo), yo = (int)((p / Wo) % Ho), n = (int)(p / ((long long)Wo * Ho));
    float s = 0.f;
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const long long q = ((long long)n * H + 2 * yo + dy) * W + 2 * xo + dx;
        s += __bfloat162float(((const bf16*)in.p)[q * in.ps + in.off + c]);
      }
    ((bf16*)out.p)[p * out.ps + out.off + c] = __float2bfloat16(0.25f * s);
  }
}

__global__ void k_pool_bwd_acc(Tensor gout, Tensor gin, int N, int H, int W, int C) {
  const long long total = (long long)N * H * W * C;   // H, W: full-resolution sizes
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long p = i / C;
    const int x = (int)(p % W), y = (int)((p / W) % H), n = (int)(p / ((long long)W * H));
    const long long q = ((long long)n * (H / 2) + y / 2) * (W / 2) + x / 2;
    ((float*)gin.p)[p * gin.ps + gin.off + c] += 0.25f * ((const float*)gout.p)[q * gout.ps + gout.off + c];
  }
}

// nearest 2x upsampling (forward, bf16; 8 channels = 16 bytes per thread, C,
// strides and offsets multiples of 8) and its transpose (fp32, written)
__global__ void k_up(Tensor in, Tensor out, int N, int H, int W, int C) {   // H, W: output sizes
  const int C8 = C / 8;
  const long long total = (long long)N * H * W * C8;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C8) * 8;
    const long long p = i / C8;
    const int x = (int)(p % W);
    const long long ny = p / W;                 // n * H + y
    const int y = (int)(ny % H);
    const long long n = ny / H;
    const long long q = (n * (H / 2) + y / 2) * (W / 2) + x / 2;
    *(uint4*)((bf16*)out.p + p * out.ps + out.off + c) =
        *(const uint4*)((const bf16*)in.p + q * in.ps + in.off + c);
  }
}

__global__ void k_up_bwd(Tensor gout, Tensor gin, int N, int H, int W, int C) {   // H, W: input (low-res) sizes
  const long long total = (long long)N * H * W * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long p = i / C;
    const int x = (int)(p % W), y = (int)((p / W) % H), n = (int)(p / ((long long)W * H));
    float s = 0.f;
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const long long q = ((long long)n * (2 * H) + 2 * y + dy) * (2 * W) + 2 * x + dx;
        s += ((const float*)gout.p)[q * gout.ps + gout.off + c];
      }
    ((float*)gin.p)[p * gin.ps + gin.off + c] = s;
  }
}

// gathers [N][nx][nt] -> bf16 image [N][nx][nt][1] scaled by 1/rms[n]
__global__ void k_pack_in(const float* d, const float* rms, bf16* x, long long per, int N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per * N;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = __float2bfloat16(d[i] / rms[i / per]);
}

// sum of squares of every gather, many CTAs per gather (FP64 partials, one
// atomic per CTA), then rms = sqrt(sum / per)
__global__ void k_sumsq(const float* d, long long per, double* acc) {
  const int n = blockIdx.y;
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = d[n * per + i];
    s += v * v;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(acc + n, red[0]);
}

__global__ void k_rms_fin(const double* acc, long long per, float* rms, int N) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < N) rms[n] = (float)fmax(sqrt(acc[n] / (double)per), 1e-30);
}

// First layer (one input channel -> 16): one thread per pixel, the 3x3
// neighbourhood from the BF16 image, weights [9][16] from shared memory,
// 16 BF16 outputs written as two 16-byte vectors (out.ps, out.off multiples of 8).
__global__ void k_conv_first(const bf16* x, const bf16* w, const float* bias, Tensor out, int N,
                             int H, int W, int relu) {
  __shared__ float ws[9][16];
  __shared__ float bs[16];
  if (threadIdx.x < 144) ws[threadIdx.x / 16][threadIdx.x % 16] = __bfloat162float(w[threadIdx.x]);
  if (threadIdx.x < 16) bs[threadIdx.x] = bias[threadIdx.x];
  __syncthreads();
  const long long total = (long long)N * H * W;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    const int xx = (int)(p % W);
    const long long ny = p / W;
    const int y = (int)(ny % H);
    const long long n = ny / H;
    float acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = bs[c];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int yy = y + t / 3 - 1, xc = xx + t % 3 - 1;
      const float v = (yy >= 0 && yy < H && xc >= 0 && xc < W)
                          ? __bfloat162float(x[(n * H + yy) * W + xc]) : 0.f;
#pragma unroll
      for (int c = 0; c < 16; ++c) acc[c] = fmaf(v, ws[t][c], acc[c]);
    }
    __align__(16) bf16 o[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16(relu ? fmaxf(acc[c], 0.f) : acc[c]);
    bf16* dst = (bf16*)out.p + p * out.ps + out.off;
    *(uint4*)dst = *(const uint4*)o;
    *(uint4*)(dst + 8) = *(const uint4*)(o + 8);
  }
}

// The input of an input-gradient convolution on the tensor cores: the FP32
// gradient of a layer's output, masked by the layer's ReLU (act > 0), rounded
// to BF16 into a dense [pixels][C] buffer; 8 channels per thread (C, strides
// and offsets multiples of 8).
__global__ void k_gz_bf16(Tensor g, Tensor act, bf16* out, long long npix, int C) {
  const int C8 = C / 8;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npix * C8;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / C8;
    const int c = (int)(i % C8) * 8;
    const float4* gp = (const float4*)((const float*)g.p + p * g.ps + g.off + c);
    const float4 g0 = gp[0], g1 = gp[1];
    float v[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
    if (act.p) {
      __align__(16) bf16 m[8];
      *(uint4*)m = *(const uint4*)((const bf16*)act.p + p * act.ps + act.off + c);
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (__bfloat162float(m[j]) <= 0.f) v[j] = 0.f;
    }
    __align__(16) bf16 o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) o[j] = __float2bfloat16(v[j]);
    *(uint4*)(out + p * C + c) = *(const uint4*)o;
  }
}

// NHWC head output [N][P][cout] -> planar [N][cout][P] (P = pixels): one
// thread per pixel reads its C contiguous values; the planar stores of a warp
// are contiguous
__global__ void k_unpack_out(const float* y, float* out, long long P, int C, int N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P * N;
       i += (long long)gridDim.x * blockDim.x) {
    const long long n = i / P, p = i % P;
    for (int c = 0; c < C; ++c) out[(n * C + c) * P + p] = y[i * C + c];
  }
}

// loss = sum_c lam_c mean_p (y - t)^2 with y NHWC [N][P][C], t planar [N][C][P]
__global__ void k_mse(const float* y, const float* t, const float* lam, float* gy, long long P,
                      int C, int N, double* loss) {
  const double inv = 1.0 / ((double)P * N);
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P * C * N;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long p = (i / C) % P, n = i / (P * C);
    const float l = lam ? lam[c] : 1.f;
    const float e = y[i] - t[(n * C + c) * P + p];
    s += (double)l * e * e;
    gy[i] = (float)(2.0 * inv) * l * e;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] * inv);
}

// Adam on the flat FP32 master parameters
__global__ void k_adam(float* w, const float* g, float* m, float* v, long long n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// FP32 OIHW master -> BF16 [tap][ci][co] (forward, CUDA cores), flipped
// [tap'][co][ci] (input gradient, CUDA cores), [tap][co][ci] (forward, tensor
// cores) and flipped [tap'][ci][co] (input gradient, tensor cores)
__global__ void k_wconv(const float* w, bf16* wf, bf16* wt, bf16* wn, bf16* wtn, int co_n, int ci_n,
                        int K) {
  const int total = co_n * ci_n * K * K;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int kx = i % K, ky = (i / K) % K, ci = (i / (K * K)) % ci_n, co = i / (K * K * ci_n);
    const int tap = ky * K + kx, tapf = (K * K - 1) - tap;
    const bf16 b = __float2bfloat16(w[i]);
    wf[((long long)tap * ci_n + ci) * co_n + co] = b;
    wt[((long long)tapf * co_n + co) * ci_n + ci] = b;
    wn[((long long)tap * co_n + co) * ci_n + ci] = b;
    wtn[((long long)tapf * ci_n + ci) * co_n + co] = b;
  }
}

// ---------------------------------------------------------------------------
// Tensor-core forward convolution (mma.sync m16n8k16, BF16 operands, FP32
// accumulation) for layers whose input channels are a multiple of 16: an
// implicit GEMM with M = pixels, N = output channels, K = taps x input
// channels.  CTA: 128 consecutive pixels of one image row x NB*16 output
// channels, 8 warps of 16 pixels each.  Per chunk of KC input channels the
// three input rows (130 pixels with the halo) and the weights of all taps are
// staged in shared memory (rows padded by 8 elements against bank conflicts)
// and consumed by ldmatrix fragments; bias, ReLU and the BF16 (or FP32)
// store are fused into the epilogue.
__device__ __forceinline__ void ldsm_x4(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3,
                                        const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"((unsigned)__cvta_generic_to_shared(p)));
}

__device__ __forceinline__ void mma_bf16(float* c, uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

struct MmaConvArgs {
  Tensor in;             // bf16 NHWC slice, ps and off multiples of 8
  const bf16* w;         // [K*K][Cout][Cin]
  const float* bias;     // [Cout]
  Tensor out;            // bf16 or fp32 NHWC slice
  int N, H, W, Cin, Cout, relu;
};

template <int K, int KC, int NB, typename TO>
__global__ void __launch_bounds__(256, 2) k_conv_mma(MmaConvArgs a) {
  constexpr int R = K / 2, PW = 128 + 2 * R, LDA = KC + 8, NT = NB * 16, TAPS = K * K;
  extern __shared__ __align__(16) unsigned char smc[];
  bf16* xs = (bf16*)smc;                              // [K rows][PW px][LDA]
  bf16* ws = xs + K * PW * LDA;                       // [TAPS][NT co][LDA]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int xt = (a.W + 127) / 128;
  const int row = blockIdx.x / xt;
  const int x0 = (blockIdx.x % xt) * 128;
  const int n = row / a.H, y = row % a.H;
  const int co0 = blockIdx.y * NT;
  const bf16* in = (const bf16*)a.in.p;
  float acc[2 * NB][4];
#pragma unroll
  for (int j = 0; j < 2 * NB; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;

  for (int ci0 = 0; ci0 < a.Cin; ci0 += KC) {
    // stage the input rows: 16-byte vectors of 8 channels
    constexpr int VPX = KC / 8;
    for (int e = tid; e < K * PW * VPX; e += 256) {
      const int v = e % VPX, px = (e / VPX) % PW, r = e / (VPX * PW);
      const int yy = y + r - R, xx = x0 + px - R;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W)
        val = *(const uint4*)(in + (((long long)n * a.H + yy) * a.W + xx) * a.in.ps + a.in.off +
                              ci0 + 8 * v);
      *(uint4*)(xs + (r * PW + px) * LDA + 8 * v) = val;
    }
    for (int e = tid; e < TAPS * NT * VPX; e += 256) {
      const int v = e % VPX, c = (e / VPX) % NT, tap = e / (VPX * NT);
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (co0 + c < a.Cout)
        val = *(const uint4*)(a.w + ((long long)tap * a.Cout + co0 + c) * a.Cin + ci0 + 8 * v);
      *(uint4*)(ws + (tap * NT + c) * LDA + 8 * v) = val;
    }
    __syncthreads();
#pragma unroll
    for (int tap = 0; tap < TAPS; ++tap) {
      const int dy = tap / K, dx = tap % K;
#pragma unroll
      for (int kk = 0; kk < KC; kk += 16) {
        uint32_t a0, a1, a2, a3;
        // A: rows = the warp's 16 pixels (shifted by dx), k = channels kk..kk+15
        const int ar = lane & 15, ak = kk + ((lane >> 4) << 3);
        ldsm_x4(a0, a1, a2, a3, xs + (dy * PW + warp * 16 + ar + dx) * LDA + ak);
#pragma unroll
        for (int nb = 0; nb < NB; ++nb) {
          // B: two n8 blocks of 16 output channels, k = channels kk..kk+15
          uint32_t b0, b1, b2, b3;
          const int bn = nb * 16 + (lane & 7) + ((lane >> 4) << 3), bk = kk + (((lane >> 3) & 1) << 3);
          ldsm_x4(b0, b1, b2, b3, ws + (tap * NT + bn) * LDA + bk);
          mma_bf16(acc[2 * nb], a0, a1, a2, a3, b0, b1);
          mma_bf16(acc[2 * nb + 1], a0, a1, a2, a3, b2, b3);
        }
      }
    }
    __syncthreads();
  }
  // epilogue: c0, c1 at (pixel g, channels 2t, 2t+1), c2, c3 at pixel g + 8
  const int g = lane >> 2, t = lane & 3;
  TO* out = (TO*)a.out.p;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int xx = x0 + warp * 16 + g + 8 * h;
    if (xx >= a.W) continue;
    const long long pix = ((long long)n * a.H + y) * a.W + xx;
#pragma unroll
    for (int j = 0; j < 2 * NB; ++j) {
      const int co = co0 + 8 * j + 2 * t;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (co + u >= a.Cout) continue;
        float v = acc[j][2 * h + u] + a.bias[co + u];
        if (a.relu) v = fmaxf(v, 0.f);
        st_f(out, pix * a.out.ps + a.out.off + co + u, v);
      }
    }
  }
}

// Outputs back in input units: model panels (channels < C-1) scale with the
// data, residual weights max(|r|, eps)^((p-2)/2) with its power, so the last
// channel (log W_r in normalised units) becomes exp(y) * rms^wr_pow.
__global__ void k_rescale_out(float* y, const float* rms, long long P, int C, int N, float wr_pow) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P * C * N;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)((i / P) % C);
    const float r = rms[i / (P * C)];
    y[i] = (c < C - 1) ? y[i] * r : expf(y[i]) * powf(r, wr_pow);
  }
}

// Training targets in normalised units from a solve's model m [N][C-1][P] and
// final residual weights wr [N][P]: t = m / rms, log(wr) - wr_pow log(rms).
__global__ void k_targets(const float* m, const float* wr, const float* rms, float* t,
                          long long P, int C, int N, float wr_pow) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P * C * N;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i % P;
    const int c = (int)((i / P) % C);
    const long long n = i / (P * C);
    const float r = rms[n];
    t[i] = (c < C - 1) ? m[(n * (C - 1) + c) * P + p] / r
                       : logf(fmaxf(wr[n * P + p], 1e-30f)) - wr_pow * logf(r);
  }
}

// The warm start in input units: m0 [N][C-1][P] and wr0 [N][P] from the
// planar head output [N][C][P].
__global__ void k_predict_out(const float* y, const float* rms, float* m0, float* wr0,
                              long long P, int C, int N, float wr_pow) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P * N;
       i += (long long)gridDim.x * blockDim.x) {
    const long long n = i / P, p = i % P;
    const float r = rms[n];
    const float* yn = y + n * C * P + p;
    if (m0)
      for (int c = 0; c < C - 1; ++c) m0[(n * (C - 1) + c) * P + p] = yn[(long long)c * P] * r;
    if (wr0) wr0[n * P + p] = expf(yn[(long long)(C - 1) * P]) * powf(r, wr_pow);
  }
}

// -------------------------------------------------------------------------
struct Layer {
  int ci, co, k;
  long long w_off, b_off;   // into the flat parameter buffer
  bf16 *wf = nullptr, *wt = nullptr, *wn = nullptr, *wtn = nullptr;
};

int grid1d(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

}  // namespace

using namespace ashrt;

struct ashrt_unet {
  int H = 0, W = 0, cout = 0, maxb = 0;
  int ch[4] = {16, 48, 96, 192};
  std::vector<Layer> L;              // 15 layers, reference order
  long long nparam = 0;
  float *w = nullptr, *g = nullptr, *am = nullptr, *av = nullptr;   // master, grad, Adam
  long long adam_t = 0;
  // activations (bf16) and gradients (fp32)
  std::vector<void*> allocs;
  bf16 *x, *e1a, *cat1, *p1, *e2a, *cat2, *p2, *e3a, *cat3, *p3, *ba, *bb, *d3a, *d3b, *d2a, *d2b,
      *d1a, *d1b;
  float *y, *gy, *g1a, *gcat1, *gp1, *g2a, *gcat2, *gp2, *g3a, *gcat3, *gp3, *gba, *gbb, *gd3a,
      *gd3b, *gd2a, *gd2b, *gd1a, *gd1b;
  float *rms, *lam;
  double* rmsacc;
  bf16* gzb;   // BF16 masked output gradient of the layer being differentiated
  int* err;    // set by a tensor-core kernel whose bounded wait ran out
  double* loss;
  std::vector<float> lam_h;
};

namespace {

template <typename T>
cudaError_t dalloc(ashrt_unet* u, T** p, size_t n) {
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T) + 16);
  if (e == cudaSuccess) u->allocs.push_back(*p);
  return e;
}

Tensor T_(void* p, int ps, int off = 0) {
  Tensor t;
  t.p = p;
  t.ps = ps;
  t.off = off;
  return t;
}

template <int K, typename TI, typename TO>
void conv(Tensor in, Tensor mask, const bf16* w, const float* bias, Tensor out, int N, int H,
          int W, int Cin, int Cout, int relu, cudaStream_t s) {
  ConvArgs a;
  a.in = in;
  a.mask = mask;
  a.w = w;
  a.bias = bias;
  a.out = out;
  a.N = N;
  a.H = H;
  a.W = W;
  a.Cin = Cin;
  a.Cout = Cout;
  a.relu = relu;
  dim3 grid((unsigned)((long long)N * H * ((W + kPix - 1) / kPix)), (Cout + kCh - 1) / kCh);
  k_conv<K, TI, TO><<<grid, kPix, 0, s>>>(a);
  count_launches(1);
}

// ---------------------------------------------------------------------------
// 5th-generation tensor-core (tcgen05) forward convolution.  M = 128 pixels of
// one image row (one TMEM lane each), N = the layer's output channels rounded
// up to 16 (one tile, <= 256 FP32 TMEM columns), K = 16 input channels per
// MMA, one MMA per tap, accumulated in TMEM over taps and channel chunks.
// Per 16-channel chunk the CTA stages, in the canonical K-major no-swizzle
// layout of 8-row x 16-byte core matrices,
//   A: [dy][2 channel octets][130 pixels][8 channels]  (a tap's A operand
//      starts dx pixels in: rows 16 B apart, next 8 pixels at +128 B = SBO,
//      next channel octet at +130 x 16 B = LBO)
//   B: [tap][2 octets][NT channels][8 input channels]  (SBO 128 B, LBO NT x 16 B)
// with cp.async into one of two stages, so that the copies of the next chunk
// overlap the MMAs of the current one; one thread issues the taps' MMAs and
// commits them to the stage's mbarrier, which is waited on (bounded) before
// that stage is refilled.  The epilogue reads the accumulators with tcgen05.ld
// (warps w and w + 4: lanes 32 (w mod 4)..+31, alternate column groups) and
// fuses bias, ReLU and the store.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);   // version 1, no swizzle
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Waits for the barrier phase; false after about a second.
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity) {
  for (int i = 0; i < (1 << 22); ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (i > 64) __nanosleep(256);
  }
  return false;
}

struct TcConvArgs {
  Tensor in;             // bf16 NHWC slice, ps and off multiples of 8
  const bf16* w;         // [K*K][Cout][Cin]
  const float* bias;     // [Cout]
  Tensor out;            // bf16 or fp32 NHWC slice
  int N, H, W, Cin, Cout, relu;
  int* err;              // set to 1 if the MMA completion wait ran out
  int planar = 0;        // 1: out.p is planar [N][Cout][H*W] (ps, off unused)
};

__device__ __forceinline__ void cp16(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(dst)), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}

template <int K, int NT, int RR, typename TO>
__global__ void __launch_bounds__(256) k_conv_tc(TcConvArgs a) {
  constexpr int R = K / 2, PW = 128 + 2 * R, TAPS = K * K, T = 256, ROWS = RR + 2 * R;
  constexpr int DS = (NT + 31) / 32 * 32;        // TMEM columns per output row
  constexpr int NCOL = RR * DS <= 32 ? 32 : RR * DS <= 64 ? 64 : RR * DS <= 128 ? 128 : 256;
  static_assert(RR * DS <= 256, "TMEM tile");
  constexpr uint32_t A_PLANE = PW * 16, B_PLANE = NT * 16;       // bytes per channel octet
  constexpr uint32_t A_BYTES = ROWS * 2 * A_PLANE, B_BYTES = TAPS * 2 * B_PLANE;
  constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);        // F32 += BF16 x BF16, M 128
  extern __shared__ __align__(128) unsigned char smt[];
  // two stages of [A | B]; then two mbarriers (one per stage) and the TMEM slot
  uint64_t* bar = (uint64_t*)(smt + 2 * (A_BYTES + B_BYTES));
  uint32_t* tslot = (uint32_t*)(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int xt = (a.W + 127) / 128, yt = (a.H + RR - 1) / RR;
  const int x0 = (blockIdx.x % xt) * 128;
  const int rb = blockIdx.x / xt;                 // n * yt + row block
  const int n = rb / yt, y0 = (rb % yt) * RR;
  const int co0 = blockIdx.y * NT;                // output-channel tile
  const bf16* in = (const bf16*)a.in.p;
  const int nch = a.Cin / 16;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_addr(tslot)),
                 "r"((uint32_t)NCOL));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(bar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(bar + 1)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;

  // asynchronous copies of channel chunk c into stage st (zero-filled outside the image)
  auto stage = [&](int c, int st) {
    unsigned char* As = smt + st * (A_BYTES + B_BYTES);
    unsigned char* Bs = As + A_BYTES;
    const int ci0 = c * 16;
    for (int e = tid; e < ROWS * PW * 2; e += T) {
      const int o = e % 2, px = (e / 2) % PW, r = e / (2 * PW);
      const int yy = y0 + r - R, xx = x0 + px - R;
      const bool ok = yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
      const bf16* src = ok ? in + (((long long)n * a.H + yy) * a.W + xx) * a.in.ps + a.in.off +
                                 ci0 + 8 * o
                           : in;
      cp16(As + (r * 2 + o) * A_PLANE + px * 16, src, ok);
    }
    for (int e = tid; e < TAPS * NT * 2; e += T) {
      const int o = e % 2, c = (e / 2) % NT, tap = e / (2 * NT);
      const bool ok = co0 + c < a.Cout;
      const bf16* src = ok ? a.w + ((long long)tap * a.Cout + co0 + c) * a.Cin + ci0 + 8 * o : a.w;
      cp16(Bs + (tap * 2 + o) * B_PLANE + c * 16, src, ok);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };

  uint32_t uses[2] = {0u, 0u};   // completed MMA batches per stage (barrier parity)
  bool failed = false;
  stage(0, 0);
  for (int c = 0; c < nch; ++c) {
    const int st = c & 1;
    if (c + 1 < nch) {
      // stage c+1 goes into the buffers of chunk c-1: wait for its MMAs first
      if (c >= 1) {
        const bool ok = tc_wait(bar + (st ^ 1), uses[st ^ 1] & 1u);
        uses[st ^ 1] += 1u;
        if (__syncthreads_or(!ok)) {
          failed = true;
          break;
        }
      }
      stage(c + 1, st ^ 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const unsigned char* As = smt + st * (A_BYTES + B_BYTES);
      const unsigned char* Bs = As + A_BYTES;
#pragma unroll
      for (int r = 0; r < RR; ++r) {
#pragma unroll
        for (int tap = 0; tap < TAPS; ++tap) {
          const int dy = tap / K, dx = tap % K;
          const uint64_t ad =
              umma_desc(smem_addr(As + (r + dy) * 2 * A_PLANE + dx * 16), A_PLANE, 128);
          const uint64_t bd = umma_desc(smem_addr(Bs + tap * 2 * B_PLANE), B_PLANE, 128);
          const uint32_t acc = (c > 0 || tap > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                  tmem + (uint32_t)(r * DS)),
              "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              smem_addr(bar + st))
          : "memory");
    }
  }
  if (!failed) {
    // the last batch's completion implies all earlier ones (same issuing thread)
    const int st = (nch - 1) & 1;
    const bool ok = tc_wait(bar + st, uses[st] & 1u);
    if (__syncthreads_or(!ok)) failed = true;
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

  if (!failed) {
    // epilogue: thread = pixel (TMEM lane of its warp quarter); warps w and
    // w + 4 share lanes and split the (row, 16-column) groups
    const int lane_base = (warp & 3) * 32;
    const int xx = x0 + lane_base + (tid & 31);
    TO* out = (TO*)a.out.p;
    constexpr int G = NT / 16;
    for (int gi = warp >> 2; gi < RR * G; gi += 2) {
      const int r = gi / G, c0 = (gi % G) * 16;
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
          "%11, %12, %13, %14, %15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(r * DS + c0)));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      const int y = y0 + r;
      if (xx < a.W && y < a.H) {
        const long long pix = ((long long)n * a.H + y) * a.W + xx;
        const int cb = co0 + c0;                    // first output channel of the group
        float f[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          f[j] = __uint_as_float(v[j]) + ((a.bias && cb + j < a.Cout) ? a.bias[cb + j] : 0.f);
          if (a.relu) f[j] = fmaxf(f[j], 0.f);
        }
        const bool whole = cb + 16 <= a.Cout;
        if (a.planar) {
          // planar output [N][Cout][H*W]: the stores of a warp are contiguous
          const long long P = (long long)a.H * a.W, p = (long long)y * a.W + xx;
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (cb + j < a.Cout) st_f(out, ((long long)n * a.Cout + cb + j) * P + p, f[j]);
        } else if (sizeof(TO) == 2 && whole && ((a.out.ps | a.out.off) & 7) == 0) {
          __align__(16) bf16 o[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) o[j] = __float2bfloat16(f[j]);
          bf16* dst = (bf16*)out + pix * a.out.ps + a.out.off + cb;
          *(uint4*)dst = *(const uint4*)o;
          *(uint4*)(dst + 8) = *(const uint4*)(o + 8);
        } else if (sizeof(TO) == 4 && whole && ((a.out.ps | a.out.off) & 3) == 0) {
          float4* dst = (float4*)((float*)out + pix * a.out.ps + a.out.off + cb);
#pragma unroll
          for (int q = 0; q < 4; ++q) dst[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (cb + j < a.Cout) st_f(out, pix * a.out.ps + a.out.off + cb + j, f[j]);
        }
      }
    }
  } else if (tid == 0 && a.err) {
    atomicExch(a.err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"((uint32_t)NCOL));
  }
}

template <int K, int NT, int RR, typename TO>
void conv_tc_v(const TcConvArgs& a, cudaStream_t s) {
  constexpr int R = K / 2, PW = 128 + 2 * R, ROWS = RR + 2 * R, DS = (NT + 31) / 32 * 32;
  constexpr int NCOL = RR * DS <= 32 ? 32 : RR * DS <= 64 ? 64 : RR * DS <= 128 ? 128 : 256;
  // at most 512 / NCOL CTAs per SM may hold TMEM at once: request enough
  // shared memory that no more are resident (228 KB per SM, 1 KB reserved
  // per CTA), so that no CTA waits in tcgen05.alloc
  const size_t need = 2 * ((size_t)ROWS * 2 * PW * 16 + (size_t)K * K * 2 * NT * 16) + 32;
  const size_t floor_b = 233472 / (512 / NCOL + 1);
  const size_t smem = std::max(need, floor_b);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_conv_tc<K, NT, RR, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr = true;
  }
  dim3 grid((unsigned)((long long)a.N * ((a.H + RR - 1) / RR) * ((a.W + 127) / 128)),
            (unsigned)((a.Cout + NT - 1) / NT));
  k_conv_tc<K, NT, RR, TO><<<grid, 256, smem, s>>>(a);
  count_launches(1);
}

// tcgen05 forward convolution for the layer sizes of the network; false if the
// output-channel tile is not one of the compiled ones (the caller then uses
// the mma.sync kernel)
template <int K, typename TO>
bool conv_tc(Tensor in, const bf16* w, const float* bias, Tensor out, int N, int H, int W,
             int Cin, int Cout, int relu, int* err, cudaStream_t s, int planar = 0) {
  if (Cin % 16 != 0 || in.ps % 8 != 0 || in.off % 8 != 0) return false;
  TcConvArgs a;
  a.planar = planar;
  a.in = in;
  a.w = w;
  a.bias = bias;
  a.out = out;
  a.N = N;
  a.H = H;
  a.W = W;
  a.Cin = Cin;
  a.Cout = Cout;
  a.relu = relu;
  a.err = err;
  const int nt = (Cout + 15) / 16 * 16;
  if constexpr (K == 3) {
    // output rows per CTA: the staged input rows serve RR outputs (TMEM:
    // RR x NT <= 256); wider outputs are split into NT-channel tiles
    switch (nt) {
      case 16: conv_tc_v<3, 16, 4, TO>(a, s); return true;
      case 48: case 144: conv_tc_v<3, 48, 4, TO>(a, s); return true;
      case 64: conv_tc_v<3, 64, 4, TO>(a, s); return true;
      case 96: case 288: conv_tc_v<3, 96, 2, TO>(a, s); return true;
      case 192: conv_tc_v<3, 192, 1, TO>(a, s); return true;
      default: return false;
    }
  } else {
    switch (nt) {
      case 16: conv_tc_v<1, 16, 1, TO>(a, s); return true;
      case 32: conv_tc_v<1, 32, 1, TO>(a, s); return true;
      case 48: conv_tc_v<1, 48, 1, TO>(a, s); return true;
      default: return false;
    }
  }
}

template <int K, int KC, int NB, typename TO>
void conv_mma_v(const MmaConvArgs& a, cudaStream_t s) {
  constexpr int R = K / 2, PW = 128 + 2 * R, LDA = KC + 8;
  const size_t smem = (size_t)(K * PW * LDA + K * K * NB * 16 * LDA) * sizeof(bf16);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_conv_mma<K, KC, NB, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr = true;
  }
  dim3 grid((unsigned)((long long)a.N * a.H * ((a.W + 127) / 128)), (a.Cout + NB * 16 - 1) / (NB * 16));
  k_conv_mma<K, KC, NB, TO><<<grid, 256, smem, s>>>(a);
  count_launches(1);
}

// Tensor-core forward convolution (input channels a multiple of 16, channel
// strides and offsets multiples of 8): picks the channel chunk and the
// output-channel tile from the layer's sizes.
template <int K, typename TO>
void conv_mma(Tensor in, const bf16* w, const float* bias, Tensor out, int N, int H, int W,
              int Cin, int Cout, int relu, cudaStream_t s, int* err = nullptr) {
  if (conv_tc<K, TO>(in, w, bias, out, N, H, W, Cin, Cout, relu, err, s)) return;
  MmaConvArgs a;
  a.in = in;
  a.w = w;
  a.bias = bias;
  a.out = out;
  a.N = N;
  a.H = H;
  a.W = W;
  a.Cin = Cin;
  a.Cout = Cout;
  a.relu = relu;
  const bool kc32 = Cin % 32 == 0;
  const int nb = Cout % 64 == 0 ? 4 : Cout % 48 == 0 ? 3 : Cout % 32 == 0 ? 2 : Cout <= 16 ? 1
               : std::min(4, (Cout + 15) / 16);
  if (kc32) {
    switch (nb) {
      case 1: conv_mma_v<K, 32, 1, TO>(a, s); break;
      case 2: conv_mma_v<K, 32, 2, TO>(a, s); break;
      case 3: conv_mma_v<K, 32, 3, TO>(a, s); break;
      default: conv_mma_v<K, 32, 4, TO>(a, s); break;
    }
  } else {
    switch (nb) {
      case 1: conv_mma_v<K, 16, 1, TO>(a, s); break;
      case 2: conv_mma_v<K, 16, 2, TO>(a, s); break;
      case 3: conv_mma_v<K, 16, 3, TO>(a, s); break;
      default: conv_mma_v<K, 16, 4, TO>(a, s); break;
    }
  }
}

template <int K>
void wgrad(Tensor in, Tensor g, Tensor mask, float* gw, float* gb, int N, int H, int W, int Cin,
           int Cout, cudaStream_t s) {
  WgradArgs a;
  a.in = in;
  a.g = g;
  a.mask = mask;
  a.gw = gw;
  a.gb = gb;
  a.N = N;
  a.H = H;
  a.W = W;
  a.Cin = Cin;
  a.Cout = Cout;
  const int xt = (W + kPix - 1) / kPix;
  const long long ch_tiles = (long long)((Cin + kCh - 1) / kCh) * ((Cout + kCh - 1) / kCh);
  const long long want_strips = (152LL * 8 + ch_tiles - 1) / ch_tiles;   // ~8 CTAs per SM
  const long long rows = (long long)N * H;
  long long strips_per_col = (want_strips + xt - 1) / xt;
  if (strips_per_col > rows) strips_per_col = rows;
  if (strips_per_col < 1) strips_per_col = 1;
  a.rows_per = (int)((rows + strips_per_col - 1) / strips_per_col);
  const long long nstrip = (rows + a.rows_per - 1) / a.rows_per;
  dim3 grid((unsigned)(nstrip * xt), (Cin + kCh - 1) / kCh, (Cout + kCh - 1) / kCh);
  k_wgrad<K><<<grid, 256, 0, s>>>(a);
  count_launches(1);
}

// rms[g] of the n input gathers x [n][per]
void compute_rms(ashrt_unet* u, const float* x, long long per, int n, cudaStream_t s) {
  cudaMemsetAsync(u->rmsacc, 0, sizeof(double) * n, s);
  k_sumsq<<<dim3(64, n), 256, 0, s>>>(x, per, u->rmsacc);
  k_rms_fin<<<(n + 127) / 128, 128, 0, s>>>(u->rmsacc, per, u->rms, n);
  count_launches(2);
}

// Forward pass on `n` images already packed in u->x; writes u->y (NHWC fp32).
// head_planar: write the head's output there as planar [n][cout][H*W]
// (inference) instead of NHWC into u->y (training).
void net_forward(ashrt_unet* u, int n, cudaStream_t s, float* head_planar = nullptr) {
  const int H = u->H, W = u->W, c0 = u->ch[0], c1 = u->ch[1], c2 = u->ch[2], c3 = u->ch[3];
  const Tensor none = T_(nullptr, 0);
  auto& L = u->L;
  auto B = [&](int i) { return u->w + L[i].b_off; };
  auto grid = [&](long long cnt) { return grid1d(cnt); };
  // encoder
  k_conv_first<<<grid((long long)n * H * W), 256, 0, s>>>(u->x, L[0].wf, B(0), T_(u->e1a, c0), n,
                                                          H, W, 1);
  conv_mma<3, bf16>(T_(u->e1a, c0), L[1].wn, B(1), T_(u->cat1, c1 + c0, c1), n, H, W, c0, c0, 1, s, u->err);
  k_pool<<<grid((long long)n * H * W / 4 * c0), 256, 0, s>>>(T_(u->cat1, c1 + c0, c1), T_(u->p1, c0), n, H, W, c0);
  conv_mma<3, bf16>(T_(u->p1, c0), L[2].wn, B(2), T_(u->e2a, c1), n, H / 2, W / 2, c0, c1, 1, s, u->err);
  conv_mma<3, bf16>(T_(u->e2a, c1), L[3].wn, B(3), T_(u->cat2, c2 + c1, c2), n, H / 2, W / 2, c1, c1, 1, s, u->err);
  k_pool<<<grid((long long)n * H * W / 16 * c1), 256, 0, s>>>(T_(u->cat2, c2 + c1, c2), T_(u->p2, c1), n, H / 2, W / 2, c1);
  conv_mma<3, bf16>(T_(u->p2, c1), L[4].wn, B(4), T_(u->e3a, c2), n, H / 4, W / 4, c1, c2, 1, s, u->err);
  conv_mma<3, bf16>(T_(u->e3a, c2), L[5].wn, B(5), T_(u->cat3, c3 + c2, c3), n, H / 4, W / 4, c2, c2, 1, s, u->err);
  k_pool<<<grid((long long)n * H * W / 64 * c2), 256, 0, s>>>(T_(u->cat3, c3 + c2, c3), T_(u->p3, c2), n, H / 4, W / 4, c2);
  conv_mma<3, bf16>(T_(u->p3, c2), L[6].wn, B(6), T_(u->ba, c3), n, H / 8, W / 8, c2, c3, 1, s, u->err);
  conv_mma<3, bf16>(T_(u->ba, c3), L[7].wn, B(7), T_(u->bb, c3), n, H / 8, W / 8, c3, c3, 1, s, u->err);
  // decoder
  k_up<<<grid((long long)n * H * W / 16 * c3 / 8), 256, 0, s>>>(T_(u->bb, c3), T_(u->cat3, c3 + c2, 0), n, H / 4, W / 4, c3);
  conv_mma<3, bf16>(T_(u->cat3, c3 + c2), L[8].wn, B(8), T_(u->d3a, c2), n, H / 4, W / 4, c3 + c2, c2, 1, s, u->err);
  conv_mma<3, bf16>(T_(u->d3a, c2), L[9].wn, B(9), T_(u->d3b, c2), n, H / 4, W / 4, c2, c2, 1, s, u->err);
  k_up<<<grid((long long)n * H * W / 4 * c2 / 8), 256, 0, s>>>(T_(u->d3b, c2), T_(u->cat2, c2 + c1, 0), n, H / 2, W / 2, c2);
  conv_mma<3, bf16>(T_(u->cat2, c2 + c1), L[10].wn, B(10), T_(u->d2a, c1), n, H / 2, W / 2, c2 + c1, c1, 1, s, u->err);
  conv_mma<3, bf16>(T_(u->d2a, c1), L[11].wn, B(11), T_(u->d2b, c1), n, H / 2, W / 2, c1, c1, 1, s, u->err);
  k_up<<<grid((long long)n * H * W * c1 / 8), 256, 0, s>>>(T_(u->d2b, c1), T_(u->cat1, c1 + c0, 0), n, H, W, c1);
  conv_mma<3, bf16>(T_(u->cat1, c1 + c0), L[12].wn, B(12), T_(u->d1a, c0), n, H, W, c1 + c0, c0, 1, s, u->err);
  conv_mma<3, bf16>(T_(u->d1a, c0), L[13].wn, B(13), T_(u->d1b, c0), n, H, W, c0, c0, 1, s, u->err);
  if (!head_planar || !conv_tc<1, float>(T_(u->d1b, c0), L[14].wn, B(14), T_(head_planar, 1), n, H,
                                         W, c0, u->cout, 0, u->err, s, 1)) {
    conv_mma<1, float>(T_(u->d1b, c0), L[14].wn, B(14), T_(u->y, u->cout), n, H, W, c0, u->cout,
                       0, s);
    if (head_planar) {
      k_unpack_out<<<grid1d((long long)H * W * n), 256, 0, s>>>(u->y, head_planar,
                                                               (long long)H * W, u->cout, n);
      count_launches(1);
    }
  }
  count_launches(7);   // pools, upsamplings, first layer
}

// Weight and bias gradients of a 3x3 layer on the tensor cores (mma.sync
// m16n8k16, BF16 operands, FP32 accumulation): for every tap, an implicit GEMM
// gw[co][ci] += sum_p gz[p][co] x[p + tap][ci] over the pixels p, M = output
// channels, N = input channels, K = pixels.  A CTA owns 16 MT output x 32 input
// channels and all nine taps and reduces a 128-pixel column strip of rows_per
// image rows: per row it stages the BF16 masked output gradient [128][16 MT]
// and the three input rows [3][130][32] in their NHWC order and reads both
// operands with ldmatrix.trans; the FP32 partial sums leave with one atomic
// each.  CTAs of the first input-channel tile also sum the bias gradient.
struct WgMmaArgs {
  Tensor in;            // bf16 layer input slice (ps, off multiples of 8)
  const bf16* gz;       // bf16 masked output gradient, dense [pixels][Cout]
  float* gw;            // [Cout][Cin][3][3] fp32, accumulated
  float* gb;            // [Cout] fp32, accumulated
  int N, H, W, Cin, Cout, rows_per;
};

__device__ __forceinline__ void ldsm_x4_t(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3,
                                          const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"((unsigned)__cvta_generic_to_shared(p)));
}

__device__ __forceinline__ void ldsm_x2_t(uint32_t& r0, uint32_t& r1, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];\n"
               : "=r"(r0), "=r"(r1)
               : "r"((unsigned)__cvta_generic_to_shared(p)));
}

template <int MT>
__global__ void __launch_bounds__(256) k_wgrad_mma(WgMmaArgs a) {
  constexpr int CO_T = 16 * MT, CI_T = 32, LDX = CI_T + 8, LDG = CO_T + 8, PW = 130;
  constexpr int TILES = 9 * MT * 4, PER = (TILES + 7) / 8;
  __shared__ __align__(16) bf16 xs[3 * PW * LDX];
  __shared__ __align__(16) bf16 gs[128 * LDG];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int xt = (a.W + 127) / 128;
  const int x0 = (blockIdx.x % xt) * 128;
  const int row0 = (blockIdx.x / xt) * a.rows_per;
  const int row1 = min(row0 + a.rows_per, a.N * a.H);
  const int ci0 = blockIdx.y * CI_T, co0 = blockIdx.z * CO_T;
  const bf16* in = (const bf16*)a.in.p;
  float acc[PER][4];
#pragma unroll
  for (int j = 0; j < PER; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  float bsum = 0.f;

  for (int row = row0; row < row1; ++row) {
    const int n = row / a.H, y = row % a.H;
    for (int e = tid; e < 3 * PW * 4; e += 256) {
      const int q = e % 4, px = (e / 4) % PW, r = e / (4 * PW);
      const int yy = y + r - 1, xx = x0 + px - 1, c = ci0 + 8 * q;
      const bool ok = yy >= 0 && yy < a.H && xx >= 0 && xx < a.W && c < a.Cin;
      const bf16* src = ok ? in + (((long long)n * a.H + yy) * a.W + xx) * a.in.ps + a.in.off + c : in;
      cp16(xs + (r * PW + px) * LDX + 8 * q, src, ok);
    }
    for (int e = tid; e < 128 * (CO_T / 8); e += 256) {
      const int q = e % (CO_T / 8), px = e / (CO_T / 8);
      const int xx = x0 + px, c = co0 + 8 * q;
      const bool ok = xx < a.W && c < a.Cout;
      const bf16* src = ok ? a.gz + (((long long)n * a.H + y) * a.W + xx) * a.Cout + c : a.gz;
      cp16(gs + px * LDG + 8 * q, src, ok);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    if (blockIdx.y == 0 && tid < CO_T)
      for (int px = 0; px < 128; ++px) bsum += __bfloat162float(gs[px * LDG + tid]);
#pragma unroll 2
    for (int kb = 0; kb < 128; kb += 16) {
      uint32_t af[MT][4];
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        const int kr = kb + (lane & 7) + ((lane >> 4) << 3), mc = mt * 16 + (((lane >> 3) & 1) << 3);
        ldsm_x4_t(af[mt][0], af[mt][1], af[mt][2], af[mt][3], gs + kr * LDG + mc);
      }
#pragma unroll
      for (int j = 0; j < PER; ++j) {
        const int id = warp + 8 * j;
        if (id < TILES) {
          const int tap = id / (4 * MT), mt = (id / 4) % MT, nt = id % 4;
          const int dy = tap / 3, dx = tap % 3;
          const int kr = kb + dx + (lane & 7) + (((lane >> 3) & 1) << 3);
          uint32_t b0, b1;
          ldsm_x2_t(b0, b1, xs + (dy * PW + kr) * LDX + nt * 8);
          // select the A fragment with conditionals (a register array indexed
          // by a runtime value would live in local memory)
          const bool m1 = MT > 1 && mt == 1;
          mma_bf16(acc[j], m1 ? af[MT - 1][0] : af[0][0], m1 ? af[MT - 1][1] : af[0][1],
                   m1 ? af[MT - 1][2] : af[0][2], m1 ? af[MT - 1][3] : af[0][3], b0, b1);
        }
      }
    }
    __syncthreads();
  }
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int id = warp + 8 * j;
    if (id >= TILES) continue;
    const int tap = id / (4 * MT), mt = (id / 4) % MT, nt = id % 4;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int co = co0 + mt * 16 + g + 8 * h;
      if (co >= a.Cout) continue;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int ci = ci0 + nt * 8 + 2 * t + u;
        if (ci < a.Cin) atomicAdd(&a.gw[((long long)co * a.Cin + ci) * 9 + tap], acc[j][2 * h + u]);
      }
    }
  }
  if (blockIdx.y == 0 && tid < CO_T && co0 + tid < a.Cout) atomicAdd(&a.gb[co0 + tid], bsum);
}

template <int MT>
void wgrad_mma_v(const WgMmaArgs& a0, cudaStream_t s) {
  WgMmaArgs a = a0;
  const int xt = (a.W + 127) / 128;
  const long long ch_tiles = (long long)((a.Cin + 31) / 32) * ((a.Cout + 16 * MT - 1) / (16 * MT));
  const long long want = (152LL * 8 + ch_tiles - 1) / ch_tiles;
  const long long rows = (long long)a.N * a.H;
  long long per_col = (want + xt - 1) / xt;
  per_col = std::max(1LL, std::min(per_col, rows));
  a.rows_per = (int)((rows + per_col - 1) / per_col);
  const long long nstrip = (rows + a.rows_per - 1) / a.rows_per;
  dim3 grid((unsigned)(nstrip * xt), (a.Cin + 31) / 32, (a.Cout + 16 * MT - 1) / (16 * MT));
  k_wgrad_mma<MT><<<grid, 256, 0, s>>>(a);
  count_launches(1);
}

// Backward of 3x3 layer l (input `in`, output gradient g masked by its ReLU
// output act): weight and bias gradients and, if out.p, the input gradient.
// On the tensor cores the masked gradient is rounded to BF16 once and serves
// both products; otherwise the CUDA-core kernels work on the FP32 gradient.
void layer_backward(ashrt_unet* u, Tensor in, Tensor g, Tensor act, const Layer& l, float* gw,
                    float* gb, Tensor out, int n, int H, int W, int Cin, int Cout, cudaStream_t s) {
  const long long npix = (long long)n * H * W;
  const bool tc = Cin % 16 == 0 && Cout % 16 == 0 && ((in.ps | in.off) & 7) == 0 &&
                  ((g.ps | g.off) & 7) == 0 && ((act.ps | act.off) & 7) == 0;
  if (!tc) {
    wgrad<3>(in, g, act, gw, gb, n, H, W, Cin, Cout, s);
    if (out.p) conv<3, float, float>(g, act, l.wt, nullptr, out, n, H, W, Cout, Cin, 0, s);
    return;
  }
  k_gz_bf16<<<grid1d(npix * Cout / 8), 256, 0, s>>>(g, act, u->gzb, npix, Cout);
  count_launches(1);
  WgMmaArgs a;
  a.in = in;
  a.gz = u->gzb;
  a.gw = gw;
  a.gb = gb;
  a.N = n;
  a.H = H;
  a.W = W;
  a.Cin = Cin;
  a.Cout = Cout;
  if (Cout <= 16) wgrad_mma_v<1>(a, s);
  else wgrad_mma_v<2>(a, s);
  if (out.p && !conv_tc<3, float>(T_(u->gzb, Cout), l.wtn, nullptr, out, n, H, W, Cout, Cin, 0,
                                  u->err, s))
    conv<3, float, float>(g, act, l.wt, nullptr, out, n, H, W, Cout, Cin, 0, s);
}

// Backward pass from u->gy (NHWC fp32); accumulates parameter gradients in u->g.
void net_backward(ashrt_unet* u, int n, cudaStream_t s) {
  const int H = u->H, W = u->W, c0 = u->ch[0], c1 = u->ch[1], c2 = u->ch[2], c3 = u->ch[3];
  const Tensor none = T_(nullptr, 0);
  auto& L = u->L;
  auto GW = [&](int i) { return u->g + L[i].w_off; };
  auto GB = [&](int i) { return u->g + L[i].b_off; };
  auto grid = [&](long long cnt) { return grid1d(cnt); };
  // Each conv layer i maps (input tensor in_i) -> (output act_i); given the
  // gradient G of its output (masked by act_i > 0 when it has a ReLU):
  //   wgrad(in_i, G, mask act_i) and, unless it is the first layer,
  //   G_in = conv(G masked, flipped weights).
  // head (no ReLU)
  wgrad<1>(T_(u->d1b, c0), T_(u->gy, u->cout), none, GW(14), GB(14), n, H, W, c0, u->cout, s);
  conv<1, float, float>(T_(u->gy, u->cout), none, L[14].wt, nullptr, T_(u->gd1b, c0), n, H, W, u->cout, c0, 0, s);
  // dec1
  layer_backward(u, T_(u->d1a, c0), T_(u->gd1b, c0), T_(u->d1b, c0), L[13], GW(13), GB(13), T_(u->gd1a, c0), n, H, W, c0, c0, s);
  layer_backward(u, T_(u->cat1, c1 + c0), T_(u->gd1a, c0), T_(u->d1a, c0), L[12], GW(12), GB(12), T_(u->gcat1, c1 + c0), n, H, W, c1 + c0, c0, s);
  k_up_bwd<<<grid((long long)n * H * W / 4 * c1), 256, 0, s>>>(T_(u->gcat1, c1 + c0, 0), T_(u->gd2b, c1), n, H / 2, W / 2, c1);
  // dec2
  layer_backward(u, T_(u->d2a, c1), T_(u->gd2b, c1), T_(u->d2b, c1), L[11], GW(11), GB(11), T_(u->gd2a, c1), n, H / 2, W / 2, c1, c1, s);
  layer_backward(u, T_(u->cat2, c2 + c1), T_(u->gd2a, c1), T_(u->d2a, c1), L[10], GW(10), GB(10), T_(u->gcat2, c2 + c1), n, H / 2, W / 2, c2 + c1, c1, s);
  k_up_bwd<<<grid((long long)n * H * W / 16 * c2), 256, 0, s>>>(T_(u->gcat2, c2 + c1, 0), T_(u->gd3b, c2), n, H / 4, W / 4, c2);
  // dec3
  layer_backward(u, T_(u->d3a, c2), T_(u->gd3b, c2), T_(u->d3b, c2), L[9], GW(9), GB(9), T_(u->gd3a, c2), n, H / 4, W / 4, c2, c2, s);
  layer_backward(u, T_(u->cat3, c3 + c2), T_(u->gd3a, c2), T_(u->d3a, c2), L[8], GW(8), GB(8), T_(u->gcat3, c3 + c2), n, H / 4, W / 4, c3 + c2, c2, s);
  k_up_bwd<<<grid((long long)n * H * W / 64 * c3), 256, 0, s>>>(T_(u->gcat3, c3 + c2, 0), T_(u->gbb, c3), n, H / 8, W / 8, c3);
  // bottleneck
  layer_backward(u, T_(u->ba, c3), T_(u->gbb, c3), T_(u->bb, c3), L[7], GW(7), GB(7), T_(u->gba, c3), n, H / 8, W / 8, c3, c3, s);
  layer_backward(u, T_(u->p3, c2), T_(u->gba, c3), T_(u->ba, c3), L[6], GW(6), GB(6), T_(u->gp3, c2), n, H / 8, W / 8, c2, c3, s);
  k_pool_bwd_acc<<<grid((long long)n * H * W / 16 * c2), 256, 0, s>>>(T_(u->gp3, c2), T_(u->gcat3, c3 + c2, c3), n, H / 4, W / 4, c2);
  // enc3 (its output s3 lives in cat3[c3:], gradient in gcat3[c3:])
  layer_backward(u, T_(u->e3a, c2), T_(u->gcat3, c3 + c2, c3), T_(u->cat3, c3 + c2, c3), L[5], GW(5), GB(5), T_(u->g3a, c2), n, H / 4, W / 4, c2, c2, s);
  layer_backward(u, T_(u->p2, c1), T_(u->g3a, c2), T_(u->e3a, c2), L[4], GW(4), GB(4), T_(u->gp2, c1), n, H / 4, W / 4, c1, c2, s);
  k_pool_bwd_acc<<<grid((long long)n * H * W / 4 * c1), 256, 0, s>>>(T_(u->gp2, c1), T_(u->gcat2, c2 + c1, c2), n, H / 2, W / 2, c1);
  // enc2
  layer_backward(u, T_(u->e2a, c1), T_(u->gcat2, c2 + c1, c2), T_(u->cat2, c2 + c1, c2), L[3], GW(3), GB(3), T_(u->g2a, c1), n, H / 2, W / 2, c1, c1, s);
  layer_backward(u, T_(u->p1, c0), T_(u->g2a, c1), T_(u->e2a, c1), L[2], GW(2), GB(2), T_(u->gp1, c0), n, H / 2, W / 2, c0, c1, s);
  k_pool_bwd_acc<<<grid((long long)n * H * W * c0), 256, 0, s>>>(T_(u->gp1, c0), T_(u->gcat1, c1 + c0, c1), n, H, W, c0);
  // enc1
  layer_backward(u, T_(u->e1a, c0), T_(u->gcat1, c1 + c0, c1), T_(u->cat1, c1 + c0, c1), L[1], GW(1), GB(1), T_(u->g1a, c0), n, H, W, c0, c0, s);
  layer_backward(u, T_(u->x, 1), T_(u->g1a, c0), T_(u->e1a, c0), L[0], GW(0), GB(0), none, n, H, W, 1, c0, s);
  count_launches(6);
}

cudaError_t refresh_bf16_weights(ashrt_unet* u, cudaStream_t s) {
  for (auto& l : u->L) {
    const int total = l.co * l.ci * l.k * l.k;
    k_wconv<<<(total + 255) / 256, 256, 0, s>>>(u->w + l.w_off, l.wf, l.wt, l.wn, l.wtn, l.co,
                                                l.ci, l.k);
    count_launches(1);
  }
  return cudaGetLastError();
}

}  // namespace

extern "C" {

ashrt_status ashrt_unet_create(ashrt_unet** out, int H, int W, int out_channels, int max_batch,
                               const float* init_params, long long n_init) {
  if (!out || H < 8 || W < 8 || H % 8 || W % 8 || out_channels < 1 || max_batch < 1) {
    set_error("ashrt_unet_create: need H, W multiples of 8 (>= 8), out_channels >= 1, max_batch >= 1");
    return ASHRT_EINVAL;
  }
  *out = nullptr;
  ashrt_unet* u = new ashrt_unet();
  u->H = H;
  u->W = W;
  u->cout = out_channels;
  u->maxb = max_batch;
  const int c0 = u->ch[0], c1 = u->ch[1], c2 = u->ch[2], c3 = u->ch[3];
  const int spec[15][3] = {{1, c0, 3},       {c0, c0, 3},      {c0, c1, 3}, {c1, c1, 3},
                           {c1, c2, 3},      {c2, c2, 3},      {c2, c3, 3}, {c3, c3, 3},
                           {c3 + c2, c2, 3}, {c2, c2, 3},      {c2 + c1, c1, 3}, {c1, c1, 3},
                           {c1 + c0, c0, 3}, {c0, c0, 3},      {c0, out_channels, 1}};
  long long off = 0;
  for (auto& sp : spec) {
    Layer l;
    l.ci = sp[0];
    l.co = sp[1];
    l.k = sp[2];
    l.w_off = off;
    off += (long long)l.co * l.ci * l.k * l.k;
    l.b_off = off;
    off += l.co;
    u->L.push_back(l);
  }
  u->nparam = off;
  const long long P0 = (long long)max_batch * H * W;
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, size_t n) {
    if (e == cudaSuccess) e = dalloc(u, p, n);
  };
  A(&u->w, off);
  A(&u->g, off);
  A(&u->am, off);
  A(&u->av, off);
  for (auto& l : u->L) {
    A(&l.wf, (size_t)l.co * l.ci * l.k * l.k);
    A(&l.wt, (size_t)l.co * l.ci * l.k * l.k);
    A(&l.wn, (size_t)l.co * l.ci * l.k * l.k);
    A(&l.wtn, (size_t)l.co * l.ci * l.k * l.k);
  }
  A(&u->x, P0);
  A(&u->e1a, P0 * c0);
  A(&u->cat1, P0 * (c1 + c0));
  A(&u->p1, P0 / 4 * c0);
  A(&u->e2a, P0 / 4 * c1);
  A(&u->cat2, P0 / 4 * (c2 + c1));
  A(&u->p2, P0 / 16 * c1);
  A(&u->e3a, P0 / 16 * c2);
  A(&u->cat3, P0 / 16 * (c3 + c2));
  A(&u->p3, P0 / 64 * c2);
  A(&u->ba, P0 / 64 * c3);
  A(&u->bb, P0 / 64 * c3);
  A(&u->d3a, P0 / 16 * c2);
  A(&u->d3b, P0 / 16 * c2);
  A(&u->d2a, P0 / 4 * c1);
  A(&u->d2b, P0 / 4 * c1);
  A(&u->d1a, P0 * c0);
  A(&u->d1b, P0 * c0);
  A(&u->y, P0 * out_channels);
  A(&u->gy, P0 * out_channels);
  A(&u->g1a, P0 * c0);
  A(&u->gcat1, P0 * (c1 + c0));
  A(&u->gp1, P0 / 4 * c0);
  A(&u->g2a, P0 / 4 * c1);
  A(&u->gcat2, P0 / 4 * (c2 + c1));
  A(&u->gp2, P0 / 16 * c1);
  A(&u->g3a, P0 / 16 * c2);
  A(&u->gcat3, P0 / 16 * (c3 + c2));
  A(&u->gp3, P0 / 64 * c2);
  A(&u->gba, P0 / 64 * c3);
  A(&u->gbb, P0 / 64 * c3);
  A(&u->gd3a, P0 / 16 * c2);
  A(&u->gd3b, P0 / 16 * c2);
  A(&u->gd2a, P0 / 4 * c1);
  A(&u->gd2b, P0 / 4 * c1);
  A(&u->gd1a, P0 * c0);
  A(&u->gd1b, P0 * c0);
  A(&u->rms, max_batch);
  A(&u->rmsacc, max_batch);
  A(&u->gzb, P0 * c0);
  A(&u->err, 1);
  A(&u->lam, out_channels);
  A(&u->loss, 1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("ashrt_unet_create: cudaMalloc failed: %s", cudaGetErrorString(e));
    for (void* p : u->allocs) cudaFree(p);
    delete u;
    return ASHRT_ENOMEM;
  }
  // parameters: given, or He-normal from a fixed-seed generator (host, Box-Muller)
  std::vector<float> h(off, 0.f);
  if (init_params) {
    if (n_init != off) {
      set_error("ashrt_unet_create: %lld initial parameters given, the network has %lld", n_init, off);
      for (void* p : u->allocs) cudaFree(p);
      delete u;
      return ASHRT_EINVAL;
    }
    for (long long i = 0; i < off; ++i) h[i] = init_params[i];
  } else {
    uint64_t st = 0x9e3779b97f4a7c15ull;
    auto uni = [&]() {
      st ^= st << 13;
      st ^= st >> 7;
      st ^= st << 17;
      return ((st >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    for (auto& l : u->L) {
      const double sd = std::sqrt(2.0 / (l.ci * l.k * l.k));
      for (long long i = 0; i < (long long)l.co * l.ci * l.k * l.k; ++i) {
        const double a = uni(), b = uni();
        h[l.w_off + i] = (float)(sd * std::sqrt(-2.0 * std::log(a)) * std::cos(6.283185307179586 * b));
      }
    }
  }
  e = cudaMemcpy(u->w, h.data(), off * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(u->am, 0, off * 4);
  if (e == cudaSuccess) e = cudaMemset(u->err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(u->av, 0, off * 4);
  if (e == cudaSuccess) e = cudaMemset(u->g, 0, off * 4);
  if (e == cudaSuccess) e = refresh_bf16_weights(u, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    set_error("ashrt_unet_create: init failed: %s", cudaGetErrorString(e));
    for (void* p : u->allocs) cudaFree(p);
    delete u;
    return ASHRT_ECUDA;
  }
  u->lam_h.assign(out_channels, 1.f);
  cudaMemcpy(u->lam, u->lam_h.data(), out_channels * 4, cudaMemcpyHostToDevice);
  *out = u;
  return ASHRT_OK;
}

void ashrt_unet_destroy(ashrt_unet* u) {
  if (!u) return;
  cudaDeviceSynchronize();
  for (void* p : u->allocs) cudaFree(p);
  delete u;
}

long long ashrt_unet_param_count(const ashrt_unet* u) { return u ? u->nparam : 0; }

ashrt_status ashrt_unet_get(const ashrt_unet* u, float* params, float* grads, long long n) {
  if (!u || n != u->nparam) {
    set_error("ashrt_unet_get: NULL network or wrong count");
    return ASHRT_EINVAL;
  }
  cudaError_t e = cudaDeviceSynchronize();
  int err = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&err, u->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && err) {
    cudaMemset(u->err, 0, sizeof(int));
    set_error("ashrt_unet_get: a tensor-core kernel's bounded wait ran out in an earlier call");
    return ASHRT_ETIMEOUT;
  }
  if (e == cudaSuccess && params) e = cudaMemcpy(params, u->w, n * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && grads) e = cudaMemcpy(grads, u->g, n * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    set_error("ashrt_unet_get: %s", cudaGetErrorString(e));
    return ASHRT_ECUDA;
  }
  return ASHRT_OK;
}

// x: [n][H][W] fp32 inputs (gathers [nx][nt]); y: [n][cout][H][W] fp32 outputs.
// Inputs are scaled by their RMS; with `rescale` the outputs are returned in
// input units for an IRLS misfit power p: channels < cout-1 multiplied by the
// RMS (model panels), the last channel as exp(y) * RMS^((p-2)/2) (residual
// weights).
ashrt_status ashrt_unet_forward(ashrt_unet* u, const float* x, float* y, int n, int rescale,
                                float p, void* stream) {
  if (!u || !x || !y || n < 1 || n > u->maxb) {
    set_error("ashrt_unet_forward: NULL argument or n outside [1, max_batch]");
    return ASHRT_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const long long per = (long long)u->H * u->W;
  compute_rms(u, x, per, n, s);
  k_pack_in<<<grid1d(per * n), 256, 0, s>>>(x, u->rms, u->x, per, n);
  count_launches(1);
  net_forward(u, n, s, y);
  if (rescale) {
    k_rescale_out<<<grid1d(per * u->cout * n), 256, 0, s>>>(y, u->rms, per, u->cout, n,
                                                           0.5f * (p - 2.f));
    count_launches(1);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("ashrt_unet_forward: %s", cudaGetErrorString(e));
    return ASHRT_ECUDA;
  }
  return ASHRT_OK;
}

// One training step on n pairs: x [n][H][W], target [n][cout][H][W] (targets
// in the network's normalised units), per-channel loss weights (host, cout
// values, or NULL = 1).  Adam with the given learning rate; returns the loss.
ashrt_status ashrt_unet_train_step(ashrt_unet* u, const float* x, const float* target, int n,
                                   const float* channel_weight, float lr, double* loss_out,
                                   void* stream) {
  if (!u || !x || !target || n < 1 || n > u->maxb) {
    set_error("ashrt_unet_train_step: NULL argument or n outside [1, max_batch]");
    return ASHRT_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const long long per = (long long)u->H * u->W;
  if (channel_weight) {
    bool same = true;
    for (int c = 0; c < u->cout; ++c) same = same && (u->lam_h[c] == channel_weight[c]);
    if (!same) {
      u->lam_h.assign(channel_weight, channel_weight + u->cout);
      cudaMemcpyAsync(u->lam, u->lam_h.data(), u->cout * 4, cudaMemcpyHostToDevice, s);
    }
  }
  cudaMemsetAsync(u->loss, 0, sizeof(double), s);
  cudaMemsetAsync(u->g, 0, u->nparam * 4, s);
  compute_rms(u, x, per, n, s);
  k_pack_in<<<grid1d(per * n), 256, 0, s>>>(x, u->rms, u->x, per, n);
  count_launches(1);
  net_forward(u, n, s);
  k_mse<<<grid1d(per * u->cout * n), 256, 0, s>>>(u->y, target, u->lam, u->gy, per, u->cout, n,
                                                  u->loss);
  count_launches(1);
  net_backward(u, n, s);
  if (lr > 0.f) {
    u->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)u->adam_t);
    const float c2 = 1.f - std::pow(b2, (float)u->adam_t);
    k_adam<<<grid1d(u->nparam), 256, 0, s>>>(u->w, u->g, u->am, u->av, u->nparam, lr, b1, b2,
                                            1e-8f, c1, c2);
    count_launches(1);
    refresh_bf16_weights(u, s);
  }
  cudaError_t e = cudaGetLastError();
  int err = 0;
  if (e == cudaSuccess && loss_out) {
    e = cudaMemcpyAsync(loss_out, u->loss, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, u->err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) {
    set_error("ashrt_unet_train_step: %s", cudaGetErrorString(e));
    return ASHRT_ECUDA;
  }
  if (err) {
    cudaMemsetAsync(u->err, 0, sizeof(int), s);
    set_error("ashrt_unet_train_step: a tensor-core kernel's bounded wait ran out");
    return ASHRT_ETIMEOUT;
  }
  return ASHRT_OK;
}

ashrt_status ashrt_unet_targets(ashrt_unet* u, const float* x, const float* m, const float* wr,
                                float* t, int n, float p, void* stream) {
  if (!u || !x || !m || !wr || !t || n < 1 || n > u->maxb) {
    set_error("ashrt_unet_targets: NULL argument or n outside [1, max_batch]");
    return ASHRT_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const long long per = (long long)u->H * u->W;
  compute_rms(u, x, per, n, s);
  k_targets<<<grid1d(per * u->cout * n), 256, 0, s>>>(m, wr, u->rms, t, per, u->cout, n,
                                                      0.5f * (p - 2.f));
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("ashrt_unet_targets: %s", cudaGetErrorString(e));
    return ASHRT_ECUDA;
  }
  return ASHRT_OK;
}

ashrt_status ashrt_unet_predict(ashrt_unet* u, const float* x, float* m0, float* wr0, int n,
                                float p, void* stream) {
  if (!u || !x || (!m0 && !wr0) || n < 1 || n > u->maxb) {
    set_error("ashrt_unet_predict: NULL argument or n outside [1, max_batch]");
    return ASHRT_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const long long per = (long long)u->H * u->W;
  compute_rms(u, x, per, n, s);
  k_pack_in<<<grid1d(per * n), 256, 0, s>>>(x, u->rms, u->x, per, n);
  count_launches(1);
  net_forward(u, n, s, u->y);
  k_predict_out<<<grid1d(per * n), 256, 0, s>>>(u->y, u->rms, m0, wr0, per, u->cout,
                                                          n, 0.5f * (p - 2.f));
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("ashrt_unet_predict: %s", cudaGetErrorString(e));
    return ASHRT_ECUDA;
  }
  return ASHRT_OK;
}

}  // extern "C"

