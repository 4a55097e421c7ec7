// Radix-16 Stockham building blocks for the t-FFT of the row kernels, for
// one complex row per element (E = float2) or two interleaved rows (E =
// float4).  A length-2^LOGN transform takes radix-16 passes while four or
// more factors of two remain, then one radix 2, 4 or 8 pass (see common.cuh
// for the Stockham index rules); each thread holds 16 values, so a CTA has
// N/16 threads.
//
// Shared rows are swizzled per 128-byte bank row: float4 rows (eight
// elements per bank row) with i ^ ((i >> 4) & 7), float2 rows (sixteen per
// bank row) with i ^ ((i >> 4) & 15).  The first pass writes 16 consecutive
// outputs per thread, i.e. a stride of 16 elements across the lanes, which
// both swizzles spread over all bank groups.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace ashrt {

constexpr float kCos8 = 0.92387953251128676f;   // cos(pi / 8)
constexpr float kSin8 = 0.38268343236508977f;   // sin(pi / 8)

// a * (c + DIR i s)
template <int DIR>
__device__ __forceinline__ float2 crot(float2 a, float c, float s) {
  const float sd = DIR < 0 ? -s : s;
  return make_float2(fmaf(a.x, c, -a.y * sd), fmaf(a.x, sd, a.y * c));
}
template <int DIR>
__device__ __forceinline__ float4 crot(float4 a, float c, float s) {
  const float sd = DIR < 0 ? -s : s;
  return make_float4(fmaf(a.x, c, -a.y * sd), fmaf(a.x, sd, a.y * c), fmaf(a.z, c, -a.w * sd),
                     fmaf(a.z, sd, a.w * c));
}

// Length-16 DFT as 4 x 4: input n = 4 n1 + n2, output k = k1 + 4 k2,
//   X[k1 + 4 k2] = sum_n2 W4^(n2 k2) W16^(n2 k1) sum_n1 W4^(n1 k1) x[4 n1 + n2],
// W_m = exp(DIR 2 pi i / m).
template <int DIR, typename E>
__device__ __forceinline__ void dft16(E* v) {
  E y[16];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    E a0 = v[n2], a1 = v[n2 + 4], a2 = v[n2 + 8], a3 = v[n2 + 12];
    dft4<DIR>(a0, a1, a2, a3);
    y[4 * n2] = a0;
    y[4 * n2 + 1] = a1;
    y[4 * n2 + 2] = a2;
    y[4 * n2 + 3] = a3;
  }
  // y[4 n2 + k1] *= W16^(n2 k1)
  y[5] = crot<DIR>(y[5], kCos8, kSin8);     // W16^1
  y[6] = mul_eighth<DIR>(y[6]);             // W16^2
  y[7] = crot<DIR>(y[7], kSin8, kCos8);     // W16^3
  y[9] = mul_eighth<DIR>(y[9]);             // W16^2
  y[10] = mul_quarter<DIR>(y[10]);          // W16^4
  y[11] = mul_3eighth<DIR>(y[11]);          // W16^6
  y[13] = crot<DIR>(y[13], kSin8, kCos8);   // W16^3
  y[14] = mul_3eighth<DIR>(y[14]);          // W16^6
  y[15] = crot<DIR>(y[15], -kCos8, -kSin8); // W16^9 = -W16^1
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    E b0 = y[k1], b1 = y[4 + k1], b2 = y[8 + k1], b3 = y[12 + k1];
    dft4<DIR>(b0, b1, b2, b3);
    v[k1] = b0;
    v[k1 + 4] = b1;
    v[k1 + 8] = b2;
    v[k1 + 12] = b3;
  }
}

// dft16 of inputs v[0..7] with v[8..15] = 0 (a zero-padded half): the first
// stage's length-4 transforms have two zero inputs.
template <int DIR, typename E>
__device__ __forceinline__ void dft16_half(E* v) {
  E y[16];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    E a0 = v[n2], a1 = v[n2 + 4], a2, a3;
    dft4_half<DIR>(a0, a1, a2, a3);
    y[4 * n2] = a0;
    y[4 * n2 + 1] = a1;
    y[4 * n2 + 2] = a2;
    y[4 * n2 + 3] = a3;
  }
  y[5] = crot<DIR>(y[5], kCos8, kSin8);
  y[6] = mul_eighth<DIR>(y[6]);
  y[7] = crot<DIR>(y[7], kSin8, kCos8);
  y[9] = mul_eighth<DIR>(y[9]);
  y[10] = mul_quarter<DIR>(y[10]);
  y[11] = mul_3eighth<DIR>(y[11]);
  y[13] = crot<DIR>(y[13], kSin8, kCos8);
  y[14] = mul_3eighth<DIR>(y[14]);
  y[15] = crot<DIR>(y[15], -kCos8, -kSin8);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    E b0 = y[k1], b1 = y[4 + k1], b2 = y[8 + k1], b3 = y[12 + k1];
    dft4<DIR>(b0, b1, b2, b3);
    v[k1] = b0;
    v[k1 + 4] = b1;
    v[k1 + 8] = b2;
    v[k1 + 12] = b3;
  }
}

template <int DIR, int R, typename E>
__device__ __forceinline__ void dft16_r(E* v) {
  if constexpr (R == 16) dft16<DIR>(v);
  else dft_r<DIR, R>(v);
}

// v[r] *= w^r, r = 1..R-1: powers by products of at most four factors,
// each used for r and r + 8 as soon as it is formed (few live registers).
template <int R, typename E>
__device__ __forceinline__ void twiddle16_r(E* v, float2 w) {
  if constexpr (R == 16) {
    const float2 w2 = cmul(w, w), w4 = cmul(w2, w2), w8 = cmul(w4, w4);
    const float2 w3 = cmul(w2, w);
    v[8] = cmul(v[8], w8);
    v[1] = cmul(v[1], w);
    v[9] = cmul(v[9], cmul(w8, w));
    v[2] = cmul(v[2], w2);
    v[10] = cmul(v[10], cmul(w8, w2));
    v[3] = cmul(v[3], w3);
    v[11] = cmul(v[11], cmul(w8, w3));
    v[4] = cmul(v[4], w4);
    v[12] = cmul(v[12], cmul(w8, w4));
    const float2 w5 = cmul(w4, w);
    v[5] = cmul(v[5], w5);
    v[13] = cmul(v[13], cmul(w8, w5));
    const float2 w6 = cmul(w4, w2);
    v[6] = cmul(v[6], w6);
    v[14] = cmul(v[14], cmul(w8, w6));
    const float2 w7 = cmul(w4, w3);
    v[7] = cmul(v[7], w7);
    v[15] = cmul(v[15], cmul(w8, w7));
  } else {
    twiddle_r<R>(v, w);
  }
}

// The powers w^1 .. w^(R-1) (p[r], p[0] unused) formed by exactly the
// products twiddle16_r (R = 16) and twiddle_r (R = 8) form, so that applying
// them with twiddle_apply gives the same values bit for bit.
template <int R>
__device__ __forceinline__ void twiddle_powers(float2 w, float2* p) {
  static_assert(R == 8 || R == 16, "radix 8 or 16");
  const float2 w2 = cmul(w, w), w4 = cmul(w2, w2), w3 = cmul(w2, w);
  p[1] = w;
  p[2] = w2;
  p[3] = w3;
  p[4] = w4;
  p[5] = cmul(w4, w);
  p[6] = cmul(w4, w2);
  p[7] = cmul(w4, w3);
  if constexpr (R == 16) {
    const float2 w8 = cmul(w4, w4);
    p[8] = w8;
#pragma unroll
    for (int r = 1; r < 8; ++r) p[8 + r] = cmul(w8, p[r]);
  }
}
template <int R, typename E>
__device__ __forceinline__ void twiddle_apply(E* v, const float2* p) {
#pragma unroll
  for (int r = 1; r < R; ++r) v[r] = cmul(v[r], p[r]);
}

// Radix schedule of a length 2^LOGN transform: radix 16 while four or more
// factors of two remain, then one radix 2, 4 or 8 pass.
template <int LOGN>
struct Sched16 {
  static constexpr int N = 1 << LOGN;
  static constexpr int N16 = LOGN / 4;
  static constexpr int RL = 1 << (LOGN % 4);
  static constexpr int NPASS = N16 + (RL > 1 ? 1 : 0);
  __host__ __device__ static constexpr int radix(int q) { return q < N16 ? 16 : RL; }
  __host__ __device__ static constexpr int ns(int q) {
    int s = 1;
    for (int i = 0; i < q; ++i) s *= radix(i);
    return s;
  }
  __host__ __device__ static constexpr int tw_off(int q) {
    int o = 0;
    for (int i = 0; i < q; ++i) o += ns(i);
    return o;
  }
};

template <typename E>
__device__ __forceinline__ int swz16(int i) {
  if constexpr (sizeof(E) == 16) return i ^ ((i >> 4) & 7);
  else return i ^ ((i >> 4) & 15);
}
// swz16(i + c) = swz16(i) + c when c is a multiple of 128 (float4) or 256
// (float2) and i has no bits at or above c's lowest set bit: the XOR term
// reads bits 4..6 (4..7) only.
template <typename E>
__host__ __device__ constexpr bool swz16_shift_free(int c) {
  return c % (sizeof(E) == 16 ? 128 : 256) == 0;
}

// One in-place Stockham pass, T = N/16 threads, each with 16 / R butterflies
// of radix R; PLAIN_OUT as in row_pass (common.cuh).  PW: the twiddle powers
// of the thread's butterflies are given, butterfly q's power r at pw[q R + r]
// (see twiddle_powers), instead of formed from tw.
template <int DIR, int N, int R, typename E, bool PLAIN_OUT = false, bool PW = false,
          bool WAIT_CP1 = false>
__device__ __forceinline__ void r16_pass(E* buf, int Ns, const float2* __restrict__ tw, int off,
                                         int tid, const float2* pw = nullptr) {
  constexpr int T = N / 16, NB = 16 / R;
  constexpr bool rd_lin = swz16_shift_free<E>(N / R);   // jb < N/R
  E v[16];
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int jb = tid + T * q;
    const int jbs = swz16<E>(jb);
#pragma unroll
    for (int r = 0; r < R; ++r)
      v[q * R + r] = buf[rd_lin ? jbs + r * (N / R) : swz16<E>(jb + r * (N / R))];
  }
  __syncthreads();
  // base = (jb - k) R + k has zero bits from Ns up to Ns R, where r Ns lands
  const bool wr_lin = swz16_shift_free<E>(Ns);
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int jb = tid + T * q;
    const int k = jb & (Ns - 1);
    if constexpr (PW) twiddle_apply<R>(&v[q * R], pw + q * R);
    else if (Ns > 1) twiddle16_r<R>(&v[q * R], base_twiddle<DIR>(tw, off, k));
    dft16_r<DIR, R>(&v[q * R]);
    const int base = (jb - k) * R + k;
    const int bases = PLAIN_OUT ? base : swz16<E>(base);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int o = base + r * Ns;
      buf[PLAIN_OUT ? o : (wr_lin ? bases + r * Ns : swz16<E>(o))] = v[q * R + r];
    }
  }
  // WAIT_CP1: the thread's cp.async groups but the newest complete before the
  // barrier, so the copies they staged are visible after it
  if constexpr (WAIT_CP1) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
  __syncthreads();
}

// LAST_PLAIN: pass Q1 - 1 is the transform's last and leaves its
// natural-order output unswizzled.
template <int DIR, int LOGN, int Q0, int Q1, typename E, bool LAST_PLAIN = false>
__device__ __forceinline__ void r16_pass_range(E* buf, const float2* __restrict__ tw, int tid) {
  using S = Sched16<LOGN>;
  if constexpr (Q0 < Q1) {
    constexpr bool plain = LAST_PLAIN && Q0 + 1 == Q1 && Q1 == S::NPASS;
    r16_pass<DIR, S::N, S::radix(Q0), E, plain>(buf, S::ns(Q0), tw, S::tw_off(Q0), tid);
    r16_pass_range<DIR, LOGN, Q0 + 1, Q1, E, LAST_PLAIN>(buf, tw, tid);
  }
}

// First pass (radix 16, Ns = 1) from registers v[r] = x[tid + r N/16];
// HALF: v[8..15] are zero (a row zero-padded to twice its length).
template <int DIR, typename E, bool HALF = false>
__device__ __forceinline__ void r16_first_pass(E* buf, E* v, int tid) {
  if constexpr (HALF) dft16_half<DIR>(v);
  else dft16<DIR>(v);
#pragma unroll
  for (int r = 0; r < 16; ++r) buf[swz16<E>(tid * 16 + r)] = v[r];
  __syncthreads();
}

// Last pass read from shared memory and stored to the global rows outA / outB
// (outB may be null; unused for float2), keeping outputs with index < n_keep.
// Ns = N/R > jb, so output r of butterfly jb is element jb + r Ns.  KEEP_LOW:
// n_keep <= N/2, so outputs r >= R/2 (elements >= N/2) are not formed.  PW
// as in r16_pass.
template <int DIR, int LOGN, typename E, bool KEEP_LOW = false, bool PW = false>
__device__ __forceinline__ void r16_last_pass_global(const E* buf, const float2* __restrict__ tw,
                                                     int tid, float2* __restrict__ outA,
                                                     float2* __restrict__ outB, int n_keep,
                                                     const float2* pw = nullptr) {
  using S = Sched16<LOGN>;
  constexpr int Q = S::NPASS - 1, R = S::radix(Q), N = S::N, T = N / 16, NB = 16 / R;
  constexpr int Ns = S::ns(Q);
  constexpr bool rd_lin = swz16_shift_free<E>(N / R);   // jb < N/R
  E v[16];
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int jb = tid + T * q;
    const int jbs = swz16<E>(jb);
#pragma unroll
    for (int r = 0; r < R; ++r)
      v[q * R + r] = buf[rd_lin ? jbs + r * (N / R) : swz16<E>(jb + r * (N / R))];
  }
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int jb = tid + T * q;
    if constexpr (PW) twiddle_apply<R>(&v[q * R], pw + q * R);
    else twiddle16_r<R>(&v[q * R], base_twiddle<DIR>(tw, S::tw_off(Q), jb));
    dft16_r<DIR, R>(&v[q * R]);
#pragma unroll
    for (int r = 0; r < (KEEP_LOW ? R / 2 : R); ++r) {
      const int idx = jb + r * Ns;
      if (idx < n_keep) store_out(outA, outB, idx, v[q * R + r]);
    }
  }
}

}  // namespace ashrt
