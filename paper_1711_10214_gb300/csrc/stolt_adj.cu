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

// Adjoint rows: the exact transpose, in gather form.  The data rows of the
// gather pair are transformed once and kept in shared memory (weighted by W).
// For every panel, thread t computes the output bins j = t + T s of the
// w_tau spectrum.  Bin j receives (1 - f) D(k) from the source k on its side
// of the spectrum whose tap floor index is |j| (primary) and f D(k) from the
// one whose floor index is |j| - 1 (secondary); floor(u) is strictly
// increasing in |k|, so there is at most one of each, and a host-built
// source table (one 8-byte entry per |j|: both sources' index and fraction,
// taken from the tap words; see build_adj_table) staged per panel gives them
// directly.  Every output bin is written once, by its owner: no atomics, no
// clearing pass, no search, and the strided ownership spreads the bins
// outside the cone over all warps.
template <int LOGN, bool SHIFT, int MINB, bool HALF>
__global__ void __launch_bounds__((1 << LOGN) / 8, MINB)
stolt_adj_rows(RowArgs a) {
  constexpr int N = 1 << LOGN, T = N / 8, H = N / 2;
  using S = Sched<LOGN>;
  extern __shared__ float4 smem4[];
  float4* buf = smem4;                          // per-panel w_tau spectrum, then its inverse FFT
  float4* dsp = smem4 + N;                      // data spectrum x W (both gathers)
  uint2* stab = (uint2*)(smem4 + 2 * N);        // source-table row of the current panel
  const int tid = threadIdx.x, l = blockIdx.x, b0 = 2 * blockIdx.y;
  const bool hasB = b0 + 1 < a.batch;
  const float2* yA = a.Y + (long long)b0 * a.y_batch + (long long)l * a.ld;
  const uint2* arow = a.atab + (long long)l * a.atab_ld;
  const long long astep = (long long)a.Lh * a.atab_ld;
  stage_tab(stab, arow, a.atab_ld, tid, T);
  cp_async_commit();

  float4 v[8];
  load_pair<N>(v, yA, hasB ? yA + a.y_batch : nullptr, a.nt, tid);
  row_first_pass<-1, N>(buf, v, tid);
  row_pass_range<-1, LOGN, 1, S::NPASS, float4, true>(buf, a.tw, tid);
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int k = tid + T * s;
    dsp[k] = cscale(buf[k], __ldg(a.wt + k));   // natural order, unswizzled
  }

  float2* xA = a.Xw + (long long)b0 * a.x_batch + (long long)l * a.ld;
  float2* xB = hasB ? xA + a.x_batch : nullptr;
  int iv = 0, jt = 0;
  int km = __ldg(a.kmin + l);                   // cone start of the panel's (velocity, k_x)
  for (int p = 0; p < a.P; ++p) {
    cp_async_wait_all();
    __syncthreads();
    const bool mapped = km < H;
    // the next panel's, loaded a panel ahead of its use
    if (p + 1 < a.P) km = __ldg(a.kmin + (iv + 1 == a.nv ? 0 : iv + 1) * a.Lh + l);
    const float2* phj = SHIFT ? a.phase + (long long)jt * N : nullptr;
    // the bins this thread gathers, j = tid + T s, are exactly the inputs of
    // its first inverse-FFT butterfly: they stay in registers
    float4 accs[8];
#pragma unroll
    for (int s = 0; s < 8; ++s)
      accs[s] = mapped ? adj_gather_bin<N, 0, SHIFT>(dsp, stab, tid + T * s, phj, s < 4)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid == 0 && mapped) accs[0] = adj_gather_bin0_mirror<N, 0, SHIFT>(dsp, stab, phj, accs[0]);
    // first pass from the registers (its barrier also ends every thread's
    // reads of the source-table row, which is then restaged)
    row_first_pass<+1, N>(buf, accs, tid);
    if (p + 1 < a.P) {
      const int ivn = iv + 1 == a.nv ? 0 : iv + 1;
      stage_tab(stab, arow + ivn * astep, a.atab_ld, tid, T);
      cp_async_commit();
    }
    row_pass_range<+1, LOGN, 1, S::NPASS - 1>(buf, a.tw, tid);
    const long long o = (long long)p * a.x_panel;
    row_last_pass_global<+1, LOGN, float4, HALF>(buf, a.tw, tid, xA + o, hasB ? xB + o : nullptr,
                                                 a.nt);
    if (++iv == a.nv) {
      iv = 0;
      ++jt;
    }
  }
}


template <int LOGN, bool SHIFT, int MINB, bool HALF>
cudaError_t launch_adj_vh(const RowArgs& a, cudaStream_t s) {
  constexpr int N = 1 << LOGN;
  static bool attr = false;
  const size_t smem = (size_t)2 * N * sizeof(float4) + (size_t)a.atab_ld * sizeof(uint2);
  cudaError_t e = set_smem(stolt_adj_rows<LOGN, SHIFT, MINB, HALF>, smem_cap<LOGN>(false), attr);
  if (e != cudaSuccess) return e;
  stolt_adj_rows<LOGN, SHIFT, MINB, HALF><<<dim3(a.Lh, (a.batch + 1) / 2), N / 8, smem, s>>>(a);
  return cudaGetLastError();
}

// HALF: nt <= Nt / 2, so each panel's inverse transform keeps only its
// lower half and the last pass forms only those outputs.
template <int LOGN, bool SHIFT, int MINB>
cudaError_t launch_adj_v(const RowArgs& a, cudaStream_t s) {
  return 2 * a.nt <= a.Nt ? launch_adj_vh<LOGN, SHIFT, MINB, true>(a, s)
                          : launch_adj_vh<LOGN, SHIFT, MINB, false>(a, s);
}

// Register-cap variant: resident CTAs per SM the kernel is compiled for
// (a.minb = 1: no cap; 2 or 3: caps for Nt <= 2048; Nt = 4096 CTAs have 512
// threads and always use 1).  Chosen by the autotuner, default 3.
template <int LOGN, bool SHIFT>
cudaError_t launch_adj_s(const RowArgs& a, cudaStream_t s) {
  if constexpr (LOGN >= 9 && LOGN <= 11) {
    if (a.minb == 3) return launch_adj_v<LOGN, SHIFT, 3>(a, s);
    if (a.minb == 2) return launch_adj_v<LOGN, SHIFT, 2>(a, s);
    return launch_adj_v<LOGN, SHIFT, 1>(a, s);
  } else if constexpr (LOGN < 9) {
    return launch_adj_v<LOGN, SHIFT, 3>(a, s);
  } else {
    return launch_adj_v<LOGN, SHIFT, 1>(a, s);
  }
}

template <int LOGN>
cudaError_t launch_adj_t(const RowArgs& a, cudaStream_t s) {
  return a.phase ? launch_adj_s<LOGN, true>(a, s) : launch_adj_s<LOGN, false>(a, s);
}

}  // namespace

// Variants (a.minb): 1..3 radix-8 with that register cap; 4 and 7 radix-8
// cap 3 (the forward alone is radix-16); 5 and 9 the radix-16 pair adjoint
// (stolt_r16.cu), 6 and 8 the single-gather radix-16 adjoint (stolt_r16s.cu)
// where their twiddles exist, else cap 3.
cudaError_t launch_stolt_adj_rows(const RowArgs& a, cudaStream_t s) {
  if ((a.minb == 6 || a.minb == 8) && a.tw16) return launch_stolt_adj_rows16s(a, s);
  if ((a.minb == 5 || a.minb == 9) && a.tw16) return launch_stolt_adj_rows16(a, s);
  RowArgs b = a;
  if (b.minb > 3) b.minb = 3;
  switch (row_log2(b.Nt)) {
    case 6: return launch_adj_t<6>(b, s);
    case 7: return launch_adj_t<7>(b, s);
    case 8: return launch_adj_t<8>(b, s);
    case 9: return launch_adj_t<9>(b, s);
    case 10: return launch_adj_t<10>(b, s);
    case 11: return launch_adj_t<11>(b, s);
    case 12: return launch_adj_t<12>(b, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ashrt
