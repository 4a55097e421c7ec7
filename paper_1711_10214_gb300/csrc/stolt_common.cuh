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
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace ashrt {

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

// tap_decode for a bin whose side of the spectrum the caller knows: pos means
// k < N/2; otherwise k >= N/2 (the w-Nyquist bin k = N/2 is unmapped).  The
// row kernels' bins k = tid + T s lie on the positive side exactly for the
// first half of the slots s, so after unrolling `pos` is a constant and the
// side selection and the table index fold away.
template <int N>
__device__ __forceinline__ Tap tap_decode_side(int k, unsigned w, bool pos) {
  Tap t;
  t.valid = (pos || k != N / 2) && (w != kTapInvalid);
  const int k0 = (int)(w >> 20);
  const float f = (float)(w & 0xfffffu) * (1.0f / 1048576.0f);
  if (pos) {
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

// Stage one adjoint source-table row (n entries, n even; 16-byte aligned).
__device__ __forceinline__ void stage_tab(uint2* dst, const uint2* src, int n, int tid, int T) {
  for (int c = tid; c < (n >> 1); c += T) cp_async16(dst + 2 * c, src + 2 * c);
}

// Swizzle of a shared float4 row: XOR the 16-byte bank group (low 3 bits)
// with bits SW..SW+2 of the index (SW = 3: swz4 of common.cuh); SW = 0: no
// swizzle (a row written in natural order by consecutive lanes).
template <int SW>
__device__ __forceinline__ int swz_g(int i) {
  if constexpr (SW == 0) return i;
  else return i ^ ((i >> SW) & 7);
}

// One output bin j of the transposed Stolt map, gather form: the secondary
// source kB - 1 (weight f(kB - 1)) and the primary source kB (weight
// 1 - f(kB)) of |j| from the staged source-table row (see build_adj_table),
// on j's side of the spectrum; the w-Nyquist bin takes nothing.  dsp holds
// the weighted data spectrum; with SHIFT each source is multiplied by the
// conjugate asymptote phase of its own bin.
// pos: j < N/2 when the caller knows the side (see tap_decode_side), else
// j >= N/2.
template <int N, int SW, bool SHIFT>
__device__ __forceinline__ float4 adj_gather_bin(const float4* dsp, const uint2* stab, int j,
                                                 const float2* __restrict__ phj, bool pos) {
  constexpr int H = N / 2;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (!pos && j == H) return acc;
  const uint2 e = stab[pos ? j : N - j];
  const int kB = (int)(e.x >> 20);
  if (e.y & (1u << 21)) {
    const int kn = pos ? kB - 1 : N - kB + 1;
    float4 d = dsp[swz_g<SW>(kn)];
    if (SHIFT) d = cmul(d, cconj(__ldg(phj + kn)));
    acc = cscale(d, (float)(e.y & 0xfffffu) * (1.0f / 1048576.0f));
  }
  if (e.y & (1u << 20)) {
    const int kn = pos ? kB : N - kB;
    float4 d = dsp[swz_g<SW>(kn)];
    if (SHIFT) d = cmul(d, cconj(__ldg(phj + kn)));
    acc = cfma(1.f - (float)(e.x & 0xfffffu) * (1.0f / 1048576.0f), d, acc);
  }
  return acc;
}

// Bin 0 also takes the primary tap of -kB (w = 0 lies on both sides).
template <int N, int SW, bool SHIFT>
__device__ __forceinline__ float4 adj_gather_bin0_mirror(const float4* dsp, const uint2* stab,
                                                         const float2* __restrict__ phj, float4 acc) {
  const uint2 e = stab[0];
  if (e.y & (1u << 20)) {
    const int kn = N - (int)(e.x >> 20);
    float4 d = dsp[swz_g<SW>(kn)];
    if (SHIFT) d = cmul(d, cconj(__ldg(phj + kn)));
    acc = cfma(1.f - (float)(e.x & 0xfffffu) * (1.0f / 1048576.0f), d, acc);
  }
  return acc;
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

template <typename K>
inline cudaError_t set_smem(K kern, size_t bytes, bool& done) {
  if (done || bytes <= 48 * 1024) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e == cudaSuccess) done = true;
  return e;
}

// Shared bytes of the adjoint's source-table row (atab_row_len entries)
inline constexpr size_t adj_tab_bytes(int N) { return (size_t)(((N / 2 + 1) + 1) & ~1) * 8; }

// Largest dynamic shared memory a launch of the LOGN kernels may request
// (ld <= Nt, taps row <= Nt/2 + 4 words, source-table row Nt/2 + 2
// entries): the attribute is set once to it.
template <int LOGN>
inline size_t smem_cap(bool fwd) {
  constexpr int N = 1 << LOGN;
  const size_t taps = (size_t)(N / 2 + 4) * sizeof(unsigned);
  return fwd ? (size_t)N * sizeof(float4) + (size_t)2 * N * sizeof(float2) + 2 * taps
             : (size_t)2 * N * sizeof(float4) + adj_tab_bytes(N);
}

inline int row_log2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

}  // namespace ashrt
