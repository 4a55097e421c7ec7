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

#include "stolt_common.cuh"

namespace ashrt {

namespace {

// Forward rows.  CTA = (k_x row l, pair of gathers b0, b0+1): the two rows
// are interleaved element by element, so every shared access is 16 bytes and
// the twiddles and Stolt taps are computed once for both gathers.
// HALF: nt <= Nt / 2, so inputs tid + r Nt/8 with r >= 4 are zero padding.
template <int LOGN, bool SHIFT, int MINB, bool HALF>
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
      if (HALF && r >= 4) {
        v[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        continue;
      }
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
    row_first_pass<-1, N, float4, HALF>(buf, v, tid);
    row_pass_range<-1, LOGN, 1, S::NPASS, float4, true>(buf, a.tw, tid);   // natural order, unswizzled

#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int k = tid + T * s;
      const bool pos = s < 4;                      // k < N/2 exactly for the first half of s
      const Tap t = tap_decode_side<N>(k, stap[pos ? k : N - k], pos);
      if (t.valid) {
        float4 vk = cscale(buf[t.i0], t.w0);
        vk = cfma(t.w1, buf[t.i1], vk);
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
  row_last_pass_global<+1, LOGN, float4, HALF>(buf, a.tw, tid, yA,
                                               hasB ? yA + a.y_batch : nullptr, a.nt);
}


template <int LOGN, bool SHIFT, int MINB, bool HALF>
cudaError_t launch_fwd_vh(const RowArgs& a, cudaStream_t s) {
  constexpr int N = 1 << LOGN;
  static bool attr = false;
  const size_t smem = (size_t)N * sizeof(float4) + (size_t)2 * a.ld * sizeof(float2) +
                      (size_t)2 * a.taps_ld * sizeof(unsigned);
  cudaError_t e = set_smem(stolt_fwd_rows<LOGN, SHIFT, MINB, HALF>, smem_cap<LOGN>(true), attr);
  if (e != cudaSuccess) return e;
  stolt_fwd_rows<LOGN, SHIFT, MINB, HALF><<<dim3(a.Lh, (a.batch + 1) / 2), N / 8, smem, s>>>(a);
  return cudaGetLastError();
}

template <int LOGN, bool SHIFT, int MINB>
cudaError_t launch_fwd_v(const RowArgs& a, cudaStream_t s) {
  return 2 * a.nt <= a.Nt ? launch_fwd_vh<LOGN, SHIFT, MINB, true>(a, s)
                          : launch_fwd_vh<LOGN, SHIFT, MINB, false>(a, s);
}

// Register-cap variant: resident CTAs per SM the kernel is compiled for
// (a.minb = 1: no cap; 2 or 3: caps for Nt <= 2048; Nt = 4096 CTAs have 512
// threads and always use 1).  Chosen by the autotuner, default 3.
template <int LOGN, bool SHIFT>
cudaError_t launch_fwd_s(const RowArgs& a, cudaStream_t s) {
  if constexpr (LOGN >= 9 && LOGN <= 11) {
    if (a.minb == 3) return launch_fwd_v<LOGN, SHIFT, 3>(a, s);
    if (a.minb == 2) return launch_fwd_v<LOGN, SHIFT, 2>(a, s);
    return launch_fwd_v<LOGN, SHIFT, 1>(a, s);
  } else if constexpr (LOGN < 9) {
    return launch_fwd_v<LOGN, SHIFT, 3>(a, s);
  } else {
    return launch_fwd_v<LOGN, SHIFT, 1>(a, s);
  }
}

template <int LOGN>
cudaError_t launch_fwd_t(const RowArgs& a, cudaStream_t s) {
  return a.phase ? launch_fwd_s<LOGN, true>(a, s) : launch_fwd_s<LOGN, false>(a, s);
}

}  // namespace

// Variants (a.minb): 1..3 radix-8 with that register cap; 4, 5 and 8 use the
// radix-16 pair forward (stolt_r16.cu), 9 its tensor-memory-accumulator form
// (Nt = 2048; the register form elsewhere), 6 and 7 the single-gather radix-16
// forward (stolt_r16s.cu) where their twiddles exist, else cap 3.
cudaError_t launch_stolt_fwd_rows(const RowArgs& a, cudaStream_t s) {
  if ((a.minb == 6 || a.minb == 7) && a.tw16) return launch_stolt_fwd_rows16s(a, s);
  if (a.minb == 9 && a.tw16) return launch_stolt_fwd_rows16_tm(a, s);
  if (a.minb >= 4 && a.tw16) return launch_stolt_fwd_rows16(a, s);
  RowArgs b = a;
  if (b.minb > 3) b.minb = 3;
  switch (row_log2(b.Nt)) {
    case 6: return launch_fwd_t<6>(b, s);
    case 7: return launch_fwd_t<7>(b, s);
    case 8: return launch_fwd_t<8>(b, s);
    case 9: return launch_fwd_t<9>(b, s);
    case 10: return launch_fwd_t<10>(b, s);
    case 11: return launch_fwd_t<11>(b, s);
    case 12: return launch_fwd_t<12>(b, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ashrt
