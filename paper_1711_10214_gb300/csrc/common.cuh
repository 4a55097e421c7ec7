// Device building blocks shared by the ASHRT kernels: complex arithmetic,
// radix-2/4/8 DFT butterflies, and one Stockham (self-sorting) FFT pass.
//
// FFT convention (reading of ch. 5 Eqs ch5_Stolt_adj1 / ch5_Stolt_forward):
// DIR = -1 is the analysis transform sum x exp(-2 pi i k j / N), DIR = +1 the
// unnormalised synthesis sum X exp(+2 pi i k j / N).
//
// Stockham pass with radix R over a length-N sequence, after the previous
// passes have built sub-transforms of length Ns: butterfly jb in [0, N/R)
// reads its R inputs at jb + r N/R, multiplies input r by w^r with
// w = exp(DIR 2 pi i k / (Ns R)), k = jb mod Ns, applies the radix-R DFT and
// writes output r at (jb - k) R + k + r Ns.  After the last pass the result is
// in natural order.  Passes use radix 8 while three or more factors of two
// remain, then one radix-2 or radix-4 pass.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ashrt {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cfma(float s, float2 a, float2 acc) {
  return make_float2(fmaf(s, a.x, acc.x), fmaf(s, a.y, acc.y));
}
// a * exp(DIR i pi / 2) = a * (DIR i)
template <int DIR>
__device__ __forceinline__ float2 mul_quarter(float2 a) {
  return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}
// a * exp(DIR i pi / 4)
template <int DIR>
__device__ __forceinline__ float2 mul_eighth(float2 a) {
  const float c = 0.70710678118654752f;
  return DIR < 0 ? make_float2((a.x + a.y) * c, (a.y - a.x) * c)
                 : make_float2((a.x - a.y) * c, (a.x + a.y) * c);
}
// a * exp(DIR 3 i pi / 4)
template <int DIR>
__device__ __forceinline__ float2 mul_3eighth(float2 a) {
  const float c = 0.70710678118654752f;
  return DIR < 0 ? make_float2((a.y - a.x) * c, -(a.x + a.y) * c)
                 : make_float2(-(a.x + a.y) * c, (a.x - a.y) * c);
}

// Two interleaved complex numbers (gather A in .x/.y, gather B in .z/.w): the
// same operations applied to both halves, so one 16-byte shared-memory access
// serves two rows and one twiddle serves both.
__device__ __forceinline__ float2 lo2(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi2(float4 a) { return make_float2(a.z, a.w); }
__device__ __forceinline__ float4 pack2(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
__device__ __forceinline__ float4 cadd(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float4 csub(float4 a, float4 b) {
  return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
__device__ __forceinline__ float4 cmul(float4 a, float2 w) {
  return make_float4(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x),
                     fmaf(a.z, w.x, -a.w * w.y), fmaf(a.z, w.y, a.w * w.x));
}
__device__ __forceinline__ float4 cscale(float4 a, float s) {
  return make_float4(a.x * s, a.y * s, a.z * s, a.w * s);
}
__device__ __forceinline__ float4 cfma(float s, float4 a, float4 acc) {
  return make_float4(fmaf(s, a.x, acc.x), fmaf(s, a.y, acc.y), fmaf(s, a.z, acc.z),
                     fmaf(s, a.w, acc.w));
}
template <int DIR>
__device__ __forceinline__ float4 mul_quarter(float4 a) {
  return DIR < 0 ? make_float4(a.y, -a.x, a.w, -a.z) : make_float4(-a.y, a.x, -a.w, a.z);
}
template <int DIR>
__device__ __forceinline__ float4 mul_eighth(float4 a) {
  return pack2(mul_eighth<DIR>(lo2(a)), mul_eighth<DIR>(hi2(a)));
}
template <int DIR>
__device__ __forceinline__ float4 mul_3eighth(float4 a) {
  return pack2(mul_3eighth<DIR>(lo2(a)), mul_3eighth<DIR>(hi2(a)));
}

template <int DIR, typename E>
__device__ __forceinline__ void dft2(E* v) {
  E a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <int DIR, typename E>
__device__ __forceinline__ void dft4(E& v0, E& v1, E& v2, E& v3) {
  E t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3);
  E t3 = mul_quarter<DIR>(csub(v1, v3));
  v0 = cadd(t0, t2);
  v2 = csub(t0, t2);
  v1 = cadd(t1, t3);
  v3 = csub(t1, t3);
}

template <int DIR, typename E>
__device__ __forceinline__ void dft8(E* v) {
  // even / odd split: X_q = E_q + w^q O_q, X_{q+4} = E_q - w^q O_q, w = exp(DIR i pi/4)
  E e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  E o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<DIR>(e0, e1, e2, e3);
  dft4<DIR>(o0, o1, o2, o3);
  o1 = mul_eighth<DIR>(o1);
  o2 = mul_quarter<DIR>(o2);
  o3 = mul_3eighth<DIR>(o3);
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

// dft4 of (v0, v1, 0, 0): the upper half of the inputs is zero.
template <int DIR, typename E>
__device__ __forceinline__ void dft4_half(E& v0, E& v1, E& v2, E& v3) {
  const E a = v0, q = mul_quarter<DIR>(v1);
  v0 = cadd(a, v1);
  v2 = csub(a, v1);
  v1 = cadd(a, q);
  v3 = csub(a, q);
}

// dft8 of inputs v[0..3] with v[4..7] = 0 (a zero-padded half).
template <int DIR, typename E>
__device__ __forceinline__ void dft8_half(E* v) {
  E e0 = v[0], e1 = v[2], e2, e3;
  E o0 = v[1], o1 = v[3], o2, o3;
  dft4_half<DIR>(e0, e1, e2, e3);
  dft4_half<DIR>(o0, o1, o2, o3);
  o1 = mul_eighth<DIR>(o1);
  o2 = mul_quarter<DIR>(o2);
  o3 = mul_3eighth<DIR>(o3);
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

template <int DIR, int R, typename E>
__device__ __forceinline__ void dft_r(E* v) {
  if constexpr (R == 2) dft2<DIR>(v);
  else if constexpr (R == 4) dft4<DIR>(v[0], v[1], v[2], v[3]);
  else dft8<DIR>(v);
}

// v[r] *= w^r, r = 1..R-1 (w already carries the direction).
template <int R, typename E>
__device__ __forceinline__ void twiddle_r(E* v, float2 w) {
  if constexpr (R == 2) {
    v[1] = cmul(v[1], w);
  } else if constexpr (R == 4) {
    float2 w2 = cmul(w, w);
    v[1] = cmul(v[1], w);
    v[2] = cmul(v[2], w2);
    v[3] = cmul(v[3], cmul(w2, w));
  } else {
    float2 w2 = cmul(w, w), w4 = cmul(w2, w2);
    float2 w3 = cmul(w2, w);
    v[1] = cmul(v[1], w);
    v[2] = cmul(v[2], w2);
    v[3] = cmul(v[3], w3);
    v[4] = cmul(v[4], w4);
    v[5] = cmul(v[5], cmul(w4, w));
    v[6] = cmul(v[6], cmul(w4, w2));
    v[7] = cmul(v[7], cmul(w4, w3));
  }
}

// 16-byte asynchronous global -> shared copies (Ampere-style cp.async; no
// waits beyond cp.async.wait_group, which the hardware completes).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// Radix schedule of a length 2^LOGN transform.
template <int LOGN>
struct Sched {
  static constexpr int N = 1 << LOGN;
  static constexpr int N8 = LOGN / 3;                    // radix-8 passes
  static constexpr int RL = 1 << (LOGN % 3);             // last radix (1 = none)
  static constexpr int NPASS = N8 + (RL > 1 ? 1 : 0);
  __host__ __device__ static constexpr int radix(int q) { return q < N8 ? 8 : RL; }
  __host__ __device__ static constexpr int ns(int q) {   // product of earlier radices
    int s = 1;
    for (int i = 0; i < q; ++i) s *= radix(i);
    return s;
  }
  // offset of pass q's base-twiddle table inside the per-length table
  __host__ __device__ static constexpr int tw_off(int q) {
    int o = 0;
    for (int i = 0; i < q; ++i) o += ns(i);
    return o;
  }
  static constexpr int TW_LEN = tw_off(NPASS);
};

// Shared-memory swizzles for one length-N row: XOR the column bits of a
// 128-byte bank row with the next bits of the index, which spreads the
// strided Stockham writes over all banks.  float2 rows: 16 elements per bank
// row; float4 rows (two interleaved complex rows): 8.  Bijections on [0, N).
__device__ __forceinline__ int swz(int i) { return i ^ ((i >> 4) & 15); }
__device__ __forceinline__ int swz4(int i) { return i ^ ((i >> 3) & 7); }
template <typename E>
__device__ __forceinline__ int swz_e(int i) {
  if constexpr (sizeof(E) == 16) return swz4(i);
  else return swz(i);
}
// The swizzle XORs bits [SB, SB + 3) (float4) or [SB, SB + 4) (float2) into the
// low bits, SB the log2 of the elements per bank row.  Adding a multiple of
// 2^(2 SB) (float4: 64, float2: 256) to an index whose bits at and above that
// power are zero changes neither those bits nor the XOR term, so
// swz(i + c) = swz(i) + c: a pass whose element strides are such multiples
// swizzles one base index per butterfly and reaches the others at constant
// offsets.
template <typename E>
__host__ __device__ constexpr bool swz_e_shift_free(int c) {
  return c % (sizeof(E) == 16 ? 64 : 256) == 0;
}

// Base twiddle of pass q: exp(DIR 2 pi i k / (Ns R)) read from the per-length
// table (stored for DIR = -1; conjugated for the synthesis direction).
template <int DIR>
__device__ __forceinline__ float2 base_twiddle(const float2* __restrict__ tw, int off, int k) {
  float2 w = __ldg(tw + off + k);
  if (DIR > 0) w.y = -w.y;
  return w;
}

// ---------------------------------------------------------------------------
// One in-place Stockham pass on a single shared row of N float2, executed by
// T = N/8 threads (each handles 8 values: one radix-8, two radix-4 or four
// radix-2 butterflies).  Reads everything, barrier, writes, barrier.
// PLAIN_OUT writes the (natural-order) outputs without the swizzle: meant for
// the last pass, whose butterfly jb < Ns writes elements jb + r Ns, i.e.
// consecutive elements across the lanes.
template <int DIR, int N, int R, typename E, bool PLAIN_OUT = false>
__device__ __forceinline__ void row_pass(E* buf, int Ns, const float2* __restrict__ tw,
                                         int tw_off, int tid) {
  constexpr int T = N / 8;
  constexpr int NB = 8 / R;
  constexpr bool rd_lin = swz_e_shift_free<E>(N / R);   // jb < N/R
  E v[8];
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int jb = tid + T * q;
    const int jbs = swz_e<E>(jb);
#pragma unroll
    for (int r = 0; r < R; ++r)
      v[q * R + r] = buf[rd_lin ? jbs + r * (N / R) : swz_e<E>(jb + r * (N / R))];
  }
  __syncthreads();
  // base = (jb - k) R + k has zero bits from Ns up to Ns R, where r Ns lands
  const bool wr_lin = swz_e_shift_free<E>(Ns);
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int jb = tid + T * q;
    const int k = jb & (Ns - 1);
    if (Ns > 1) twiddle_r<R>(&v[q * R], base_twiddle<DIR>(tw, tw_off, k));
    dft_r<DIR, R>(&v[q * R]);
    const int base = (jb - k) * R + k;
    const int bases = PLAIN_OUT ? base : swz_e<E>(base);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int o = base + r * Ns;
      buf[PLAIN_OUT ? o : (wr_lin ? bases + r * Ns : swz_e<E>(o))] = v[q * R + r];
    }
  }
  __syncthreads();
}

// Passes Q0 <= q < Q1 of a length-2^LOGN transform, in place in shared memory;
// LAST_PLAIN: pass Q1 - 1 is the transform's last and leaves its natural-order
// output unswizzled.
template <int DIR, int LOGN, int Q0, int Q1, typename E, bool LAST_PLAIN = false>
__device__ __forceinline__ void row_pass_range(E* buf, const float2* __restrict__ tw,
                                               int tid) {
  using S = Sched<LOGN>;
  if constexpr (Q0 < Q1) {
    constexpr int R = S::radix(Q0);
    constexpr bool plain = LAST_PLAIN && Q0 + 1 == Q1 && Q1 == S::NPASS;
    row_pass<DIR, S::N, R, E, plain>(buf, S::ns(Q0), tw, S::tw_off(Q0), tid);
    row_pass_range<DIR, LOGN, Q0 + 1, Q1, E, LAST_PLAIN>(buf, tw, tid);
  }
}

// Last pass of a length-2^LOGN transform, read from shared memory and written
// to global rows, keeping outputs with index < n_keep (the crop back to nt).
// In the last pass Ns = N/R > jb, so output r of butterfly jb lands at
// jb + r Ns: consecutive threads store consecutive addresses.  For float4
// elements the two interleaved rows go to outA and outB (outB may be null).
__device__ __forceinline__ void store_out(float2* outA, float2* outB, int idx, float2 v) {
  outA[idx] = v;
}
__device__ __forceinline__ void store_out(float2* outA, float2* outB, int idx, float4 v) {
  outA[idx] = lo2(v);
  if (outB) outB[idx] = hi2(v);
}

// KEEP_LOW: n_keep <= N/2, so outputs r >= R/2 (elements >= N/2) are not formed.
template <int DIR, int LOGN, typename E, bool KEEP_LOW = false>
__device__ __forceinline__ void row_last_pass_global(E* buf, const float2* __restrict__ tw,
                                                     int tid, float2* __restrict__ outA,
                                                     float2* __restrict__ outB, int n_keep) {
  using S = Sched<LOGN>;
  constexpr int Q = S::NPASS - 1;
  constexpr int R = S::radix(Q);
  constexpr int N = S::N, T = N / 8, NB = 8 / R, Ns = S::ns(Q);
  constexpr bool rd_lin = swz_e_shift_free<E>(N / R);   // jb < N/R
  E v[8];
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int jb = tid + T * q;
    const int jbs = swz_e<E>(jb);
#pragma unroll
    for (int r = 0; r < R; ++r)
      v[q * R + r] = buf[rd_lin ? jbs + r * (N / R) : swz_e<E>(jb + r * (N / R))];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int jb = tid + T * q;
    if (Ns > 1) twiddle_r<R>(&v[q * R], base_twiddle<DIR>(tw, S::tw_off(Q), jb));
    dft_r<DIR, R>(&v[q * R]);
#pragma unroll
    for (int r = 0; r < (KEEP_LOW ? R / 2 : R); ++r) {
      const int idx = jb + r * Ns;
      if (idx < n_keep) store_out(outA, outB, idx, v[q * R + r]);
    }
  }
}

// First pass (radix 8, Ns = 1, no twiddles) from registers v[r] = x[tid + r N/8];
// HALF: v[4..7] are zero (a row zero-padded to twice its length).
template <int DIR, int N, typename E, bool HALF = false>
__device__ __forceinline__ void row_first_pass(E* buf, E* v, int tid) {
  if constexpr (HALF) dft8_half<DIR>(v);
  else dft8<DIR>(v);
#pragma unroll
  for (int r = 0; r < 8; ++r) buf[swz_e<E>(tid * 8 + r)] = v[r];
  __syncthreads();
}

}  // namespace ashrt
