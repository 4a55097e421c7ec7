// Fused time-axis FFT + Stolt map + velocity/asymptote sum (forward) or
// spray (adjoint), one CTA per (gather pair, k_x) row.
//
// Forward, ch. 5 Eq. ch5_forward_operator / ch. 6 Eq. ch6_forward_operator,
// for the row of wavenumber index l of gather b:
//   for every panel p = (tau0_j, v_i):  load the x-transformed model row
//     X_p(l, tau) (nt samples), zero-pad to Nt, FFT along tau -> M_p(w_tau),
//     map w <- w_tau by the dispersion relation w_tau = sgn(w) sqrt(w^2 - (v k_x)^2)
//     (ch. 5) with linear interpolation, and accumulate
//     D(w) += exp(-i w tau0_j) V_p(w)   (T and the sums S / A)
//   D *= W(w) (wavelet C, band limit, 1/(Nt Nx)); inverse FFT along t; keep nt.
// Adjoint (ch. 5 Eq. ch5_adj_operator / ch. 6 Eq. ch6_adj_operator): the
// exact transpose: FFT the data row once, weight by W, and for each panel
// scatter every mapped bin to its two interpolation taps (transposed linear
// weights, conjugate phase), inverse FFT, keep nt samples.
//
// One CTA handles one k_x row of a PAIR of gathers, the two rows interleaved
// element by element (16-byte shared accesses; twiddles and Stolt taps
// computed once for both).  The panel spectrum, the map and the accumulation
// never leave the SM: the accumulator D lives in registers (each thread owns
// bins k = tid + T s), the spectrum of the current panel in one shared row,
// and the next panel's rows are staged with cp.async while the current one
// is transformed.
//
// The Stolt taps come from a table built on the host in FP64 (one word per
// (v, l, |k|): floor(u) and the 20-bit fraction of u = sqrt(k^2 - a^2), or
// "unmapped" when k^2 <= a^2), staged into shared memory with the panel, so
// the GPU and the FP64 oracle agree on cone membership and on the taps to
// 5e-7 in the interpolation weight.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace ashrt {

namespace {

struct Tap {
  int i0, i1;
  float w0, w1;
  bool valid;
};

// Interpolation taps of output bin k (natural index in [0, N)) from the tap
// word of |k|.  For w > 0 the taps are floor(u), floor(u)+1; for w < 0 the
// mirrored -floor(|u|), -floor(|u|)-1, which is the same linear interpolation
// at u = -|u| (odd extension keeps real output).  A tap on the w-Nyquist bin
// carries weight 0.
template <int N>
__device__ __forceinline__ Tap tap_decode(int k, unsigned w) {
  Tap t;
  t.valid = (k != N / 2) && (w != kTapInvalid);
  const int k0 = (int)(w >> 20);
  const float f = (float)(w & 0xfffffu) * (1.0f / 1048576.0f);
  if (k < N / 2) {
    t.i0 = k0;
    t.i1 = k0 + 1;
  } else {
    t.i0 = (N - k0) & (N - 1);
    t.i1 = (N - k0 - 1) & (N - 1);
  }
  t.w0 = 1.f - f;
  t.w1 = (t.i1 == N / 2) ? 0.f : f;
  return t;
}

template <int N>
__device__ __forceinline__ int kabs_of(int k) {
  return k <= N / 2 ? k : N - k;
}

// 16-byte asynchronous global -> shared copies (Ampere-style cp.async; no
// waits beyond cp.async.wait_group, which the hardware completes).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// Stage the rows of gathers A and B (B may be absent) of one panel: ld
// complex values each (ld is a multiple of 4, rows are 32-byte aligned).
__device__ __forceinline__ void stage_rows(float2* stage, const float2* rowA, const float2* rowB,
                                           int ld, int tid, int T) {
  const int chunks = ld >> 1;   // 16-byte chunks of two complex values
  for (int c = tid; c < chunks; c += T) cp_async16(stage + 2 * c, rowA + 2 * c);
  if (rowB)
    for (int c = tid; c < chunks; c += T) cp_async16(stage + ld + 2 * c, rowB + 2 * c);
}

// Stage one tap row (taps_ld words, a multiple of 4; 16-byte aligned).
__device__ __forceinline__ void stage_taps(unsigned* dst, const unsigned* src, int taps_ld, int tid,
                                           int T) {
  for (int c = tid; c < (taps_ld >> 2); c += T) cp_async16(dst + 4 * c, src + 4 * c);
}

template <int N>
__device__ __forceinline__ void load_pair(float4* v, const float2* __restrict__ rowA,
                                          const float2* __restrict__ rowB, int nt, int tid) {
  constexpr int T = N / 8;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = tid + r * T;
    const float2 za = i < nt ? __ldg(rowA + i) : make_float2(0.f, 0.f);
    const float2 zb = (rowB && i < nt) ? __ldg(rowB + i) : make_float2(0.f, 0.f);
    v[r] = pack2(za, zb);
  }
}

// Forward rows.  CTA = (k_x row l, pair of gathers b0, b0+1): the two rows
// are interleaved element by element, so every shared access is 16 bytes and
// the twiddles and Stolt taps are computed once for both gathers.
template <int LOGN, bool SHIFT, int MINB>
__global__ void __launch_bounds__((1 << LOGN) / 8, MINB)
stolt_fwd_rows(RowArgs a) {
  constexpr int N = 1 << LOGN, T = N / 8;
  using S = Sched<LOGN>;
  extern __shared__ float4 smem4[];
  float4* buf = smem4;                         // N interleaved (A, B) complex values
  float2* stage = (float2*)(smem4 + N);        // next panel: row A [ld], row B [ld]
  unsigned* stap0 = (unsigned*)(stage + 2 * a.ld);   // tap rows, double-buffered by panel
  unsigned* stap1 = stap0 + a.taps_ld;
  const int tid = threadIdx.x, l = blockIdx.x, b0 = 2 * blockIdx.y;
  const bool hasB = b0 + 1 < a.batch;
  const float2* xA = a.X + (long long)b0 * a.x_batch + (long long)l * a.ld;
  const float2* xB = hasB ? xA + a.x_batch : nullptr;

  float4 acc[8];
  float2 ph[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    acc[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    ph[s] = make_float2(1.f, 0.f);
  }
  const unsigned* trow = a.taps + (long long)l * a.taps_ld;   // velocity iv: + iv * Lh * taps_ld
  const long long tstep = (long long)a.Lh * a.taps_ld;
  stage_rows(stage, xA, xB, a.ld, tid, T);
  stage_taps(stap0, trow, a.taps_ld, tid, T);
  cp_async_commit();

  int iv = 0, jt = 0;
  for (int p = 0; p < a.P; ++p) {
    unsigned* stap = (p & 1) ? stap1 : stap0;
    cp_async_wait_all();
    __syncthreads();
    float4 v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = tid + r * T;
      const float2 za = i < a.nt ? stage[i] : make_float2(0.f, 0.f);
      const float2 zb = (hasB && i < a.nt) ? stage[a.ld + i] : make_float2(0.f, 0.f);
      v[r] = pack2(za, zb);
    }
    __syncthreads();
    if (p + 1 < a.P) {
      const long long o = (long long)(p + 1) * a.x_panel;
      const int ivn = iv + 1 == a.nv ? 0 : iv + 1;
      stage_rows(stage, xA + o, hasB ? xB + o : nullptr, a.ld, tid, T);
      stage_taps((p & 1) ? stap0 : stap1, trow + ivn * tstep, a.taps_ld, tid, T);
      cp_async_commit();
    }
    if (SHIFT && iv == 0) {
#pragma unroll
      for (int s = 0; s < 8; ++s) ph[s] = __ldg(a.phase + (long long)jt * N + tid + T * s);
    }
    row_first_pass<-1, N>(buf, v, tid);
    row_pass_range<-1, LOGN, 1, S::NPASS>(buf, a.tw, tid);

#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int k = tid + T * s;
      const Tap t = tap_decode<N>(k, stap[kabs_of<N>(k)]);
      if (t.valid) {
        float4 vk = cscale(buf[swz4(t.i0)], t.w0);
        vk = cfma(t.w1, buf[swz4(t.i1)], vk);
        if (SHIFT) vk = cmul(vk, ph[s]);
        acc[s] = cadd(acc[s], vk);
      }
    }
    if (++iv == a.nv) {
      iv = 0;
      ++jt;
    }
    __syncthreads();
  }
#pragma unroll
  for (int s = 0; s < 8; ++s) acc[s] = cscale(acc[s], __ldg(a.wt + tid + T * s));
  // own bins are exactly the first-pass inputs of the inverse transform
  row_first_pass<+1, N>(buf, acc, tid);
  row_pass_range<+1, LOGN, 1, S::NPASS - 1>(buf, a.tw, tid);
  float2* yA = a.Yw + (long long)b0 * a.y_batch + (long long)l * a.ld;
  row_last_pass_global<+1, LOGN>(buf, a.tw, tid, yA, hasB ? yA + a.y_batch : nullptr, a.nt);
}

// Adjoint rows: the exact transpose, in gather form.  The data rows of the
// gather pair are transformed once and kept in shared memory (weighted by W).
// For every panel, thread t computes the output bins j = t + T s of the
// w_tau spectrum.  With J = |j|, bin j receives (1 - f) D(k) from every
// source k on its side of the spectrum with floor(u(|k|)) = J and f D(k) from
// every source with floor(u(|k|)) = J - 1 (bin 0 takes the primary taps of
// both sides).  floor(u) is non-decreasing in |k|, so those sources are one
// run of |k| starting at the first |k| with floor(u) >= J - 1: located from
// the inverse |k| = sqrt(J^2 + a^2) and corrected on the staged tap row.
// Every bin is written once, by its owner: no atomics, no clearing pass, and
// the strided ownership spreads the bins outside the cone over all warps.
template <int LOGN, bool SHIFT, int MINB>
__global__ void __launch_bounds__((1 << LOGN) / 8, MINB)
stolt_adj_rows(RowArgs a) {
  constexpr int N = 1 << LOGN, T = N / 8, H = N / 2;
  using S = Sched<LOGN>;
  extern __shared__ float4 smem4[];
  float4* buf = smem4;                          // per-panel w_tau spectrum, then its inverse FFT
  float4* dsp = smem4 + N;                      // data spectrum x W (both gathers)
  unsigned* stap = (unsigned*)(smem4 + 2 * N);  // tap row of the current panel
  const int tid = threadIdx.x, l = blockIdx.x, b0 = 2 * blockIdx.y;
  const bool hasB = b0 + 1 < a.batch;
  const float2* yA = a.Y + (long long)b0 * a.y_batch + (long long)l * a.ld;
  const unsigned* trow = a.taps + (long long)l * a.taps_ld;
  const long long tstep = (long long)a.Lh * a.taps_ld;
  stage_taps(stap, trow, a.taps_ld, tid, T);
  cp_async_commit();

  float4 v[8];
  load_pair<N>(v, yA, hasB ? yA + a.y_batch : nullptr, a.nt, tid);
  row_first_pass<-1, N>(buf, v, tid);
  row_pass_range<-1, LOGN, 1, S::NPASS>(buf, a.tw, tid);
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int k = tid + T * s;
    dsp[swz4(k)] = cscale(buf[swz4(k)], __ldg(a.wt + k));
  }

  float2* xA = a.Xw + (long long)b0 * a.x_batch + (long long)l * a.ld;
  float2* xB = hasB ? xA + a.x_batch : nullptr;
  int iv = 0, jt = 0;
  for (int p = 0; p < a.P; ++p) {
    cp_async_wait_all();
    __syncthreads();
    const int km = __ldg(a.kmin + iv * a.Lh + l);
    const float2 ac = __ldg(a.acone + iv * a.Lh + l);
    const float af = ac.x + ac.y;
    const float2* phj = SHIFT ? a.phase + (long long)jt * N : nullptr;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int j = tid + T * s;
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      if (j != H && km < H) {
        const bool pos = j < H;
        const int J = pos ? j : N - j;
        // first |k| >= km with floor(u(|k|)) >= J - 1
        int k = km;
        if (J > 1) {
          const float x = (float)(J - 1);
          k = (int)ceilf(sqrtf(fmaf(x, x, af * af)));
          k = min(max(k, km), H);
          while (k > km && (int)(stap[k - 1] >> 20) >= J - 1) --k;
          while (k < H && (int)(stap[k] >> 20) < J - 1) ++k;
        }
        for (; k < H; ++k) {
          const unsigned w = stap[k];
          const int b = (int)(w >> 20);
          if (b > J) break;
          const float f = (float)(w & 0xfffffu) * (1.0f / 1048576.0f);
          const int kn = pos ? k : N - k;
          float4 d = dsp[swz4(kn)];
          if (SHIFT) d = cmul(d, cconj(__ldg(phj + kn)));
          if (b == J) {
            if (J == 0) {                       // bin 0: primary taps of +k and -k
              float4 dm = dsp[swz4(N - k)];
              if (SHIFT) dm = cmul(dm, cconj(__ldg(phj + (N - k))));
              d = cadd(d, dm);
            }
            acc = cfma(1.f - f, d, acc);
          } else {                              // b == J - 1: secondary tap
            acc = cfma(f, d, acc);
          }
        }
      }
      buf[swz4(j)] = acc;
    }
    __syncthreads();
    if (p + 1 < a.P) {
      const int ivn = iv + 1 == a.nv ? 0 : iv + 1;
      stage_taps(stap, trow + ivn * tstep, a.taps_ld, tid, T);
      cp_async_commit();
    }
    row_pass_range<+1, LOGN, 0, S::NPASS - 1>(buf, a.tw, tid);
    const long long o = (long long)p * a.x_panel;
    row_last_pass_global<+1, LOGN>(buf, a.tw, tid, xA + o, hasB ? xB + o : nullptr, a.nt);
    if (++iv == a.nv) {
      iv = 0;
      ++jt;
    }
  }
}

template <typename K>
cudaError_t set_smem(K kern, size_t bytes, bool& done) {
  if (done || bytes <= 48 * 1024) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e == cudaSuccess) done = true;
  return e;
}

// Resident CTAs per SM the row kernels are compiled for: up to Nt = 2048 the
// register cap of 3 CTAs (80 registers) measured 1.4x (forward) and 1.9x
// (adjoint) faster than the uncapped build; Nt = 4096 CTAs have 512 threads.
template <int LOGN>
__host__ __device__ constexpr int rows_minb() { return LOGN <= 11 ? 3 : 1; }

// Largest dynamic shared memory a launch of the LOGN kernels may request
// (ld <= Nt, taps row <= Nt/2 + 4 words): the attribute is set once to it.
template <int LOGN>
size_t smem_cap(bool fwd) {
  constexpr int N = 1 << LOGN;
  const size_t taps = (size_t)(N / 2 + 4) * sizeof(unsigned);
  return fwd ? (size_t)N * sizeof(float4) + (size_t)2 * N * sizeof(float2) + 2 * taps
             : (size_t)2 * N * sizeof(float4) + taps;
}

template <int LOGN, bool SHIFT, int MINB>
cudaError_t launch_fwd_v(const RowArgs& a, cudaStream_t s) {
  constexpr int N = 1 << LOGN;
  static bool attr = false;
  const size_t smem = (size_t)N * sizeof(float4) + (size_t)2 * a.ld * sizeof(float2) +
                      (size_t)2 * a.taps_ld * sizeof(unsigned);
  cudaError_t e = set_smem(stolt_fwd_rows<LOGN, SHIFT, MINB>, smem_cap<LOGN>(true), attr);
  if (e != cudaSuccess) return e;
  stolt_fwd_rows<LOGN, SHIFT, MINB><<<dim3(a.Lh, (a.batch + 1) / 2), N / 8, smem, s>>>(a);
  return cudaGetLastError();
}

template <int LOGN, bool SHIFT, int MINB>
cudaError_t launch_adj_v(const RowArgs& a, cudaStream_t s) {
  constexpr int N = 1 << LOGN;
  static bool attr = false;
  const size_t smem = (size_t)2 * N * sizeof(float4) + (size_t)a.taps_ld * sizeof(unsigned);
  cudaError_t e = set_smem(stolt_adj_rows<LOGN, SHIFT, MINB>, smem_cap<LOGN>(false), attr);
  if (e != cudaSuccess) return e;
  stolt_adj_rows<LOGN, SHIFT, MINB><<<dim3(a.Lh, (a.batch + 1) / 2), N / 8, smem, s>>>(a);
  return cudaGetLastError();
}

template <int LOGN>
cudaError_t launch_fwd_t(const RowArgs& a, cudaStream_t s) {
  constexpr int M = rows_minb<LOGN>();
  return a.phase ? launch_fwd_v<LOGN, true, M>(a, s) : launch_fwd_v<LOGN, false, M>(a, s);
}

template <int LOGN>
cudaError_t launch_adj_t(const RowArgs& a, cudaStream_t s) {
  constexpr int M = rows_minb<LOGN>();
  return a.phase ? launch_adj_v<LOGN, true, M>(a, s) : launch_adj_v<LOGN, false, M>(a, s);
}

int row_log2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

}  // namespace

cudaError_t launch_stolt_fwd_rows(const RowArgs& a, cudaStream_t s) {
  switch (row_log2(a.Nt)) {
    case 6: return launch_fwd_t<6>(a, s);
    case 7: return launch_fwd_t<7>(a, s);
    case 8: return launch_fwd_t<8>(a, s);
    case 9: return launch_fwd_t<9>(a, s);
    case 10: return launch_fwd_t<10>(a, s);
    case 11: return launch_fwd_t<11>(a, s);
    case 12: return launch_fwd_t<12>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_stolt_adj_rows(const RowArgs& a, cudaStream_t s) {
  switch (row_log2(a.Nt)) {
    case 6: return launch_adj_t<6>(a, s);
    case 7: return launch_adj_t<7>(a, s);
    case 8: return launch_adj_t<8>(a, s);
    case 9: return launch_adj_t<9>(a, s);
    case 10: return launch_adj_t<10>(a, s);
    case 11: return launch_adj_t<11>(a, s);
    case 12: return launch_adj_t<12>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ashrt
