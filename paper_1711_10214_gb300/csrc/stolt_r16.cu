// Radix-16 variant of the fused t-FFT + Stolt map row kernels (forward and
// adjoint of ch. 5 Eqs ch5_forward_operator / ch5_adj_operator, ch. 6 Eqs
// ch6_forward_operator / ch6_adj_operator), for Nt = 1024, 2048 and 4096.
//
// The operator, the tables (Stolt taps, adjoint sources, spectral weight, phase)
// and the CTA work split (one k_x row of a pair of gathers, the two rows
// interleaved as float4) are those of stolt_fwd.cu / stolt_adj.cu.  What
// changes is the transform: each thread holds 16 values instead of 8, so a
// length-Nt transform takes three Stockham passes (16 x 16 x {4, 8, 16})
// instead of four (8 x 8 x 8 x {2, 4}) and each element crosses shared memory
// two times fewer per transform.  The kernels are bound by shared-memory
// wavefronts, so this is the quantity that matters; the price is Nt/16
// threads per CTA with twice the registers each (the cap allows 168).
//
// Shared rows use the swizzle i ^ ((i >> 4) & 7) (float4 elements, eight per
// 128-byte bank row): the first pass writes 16 consecutive outputs per
// thread, i.e. a stride of 16 elements across the lanes, which this swizzle
// spreads over all eight 16-byte bank groups of every quarter warp.
#include <cuda_runtime.h>

#include "stolt_common.cuh"

namespace ashrt {

namespace {

constexpr float kCos8 = 0.92387953251128676f;   // cos(pi / 8)
constexpr float kSin8 = 0.38268343236508977f;   // sin(pi / 8)

// a * (c + DIR i s), both interleaved values
template <int DIR>
__device__ __forceinline__ float4 crot(float4 a, float c, float s) {
  const float sd = DIR < 0 ? -s : s;
  return make_float4(fmaf(a.x, c, -a.y * sd), fmaf(a.x, sd, a.y * c), fmaf(a.z, c, -a.w * sd),
                     fmaf(a.z, sd, a.w * c));
}

// Length-16 DFT as 4 x 4: input n = 4 n1 + n2, output k = k1 + 4 k2,
//   X[k1 + 4 k2] = sum_n2 W4^(n2 k2) W16^(n2 k1) sum_n1 W4^(n1 k1) x[4 n1 + n2],
// W_m = exp(DIR 2 pi i / m).
template <int DIR>
__device__ __forceinline__ void dft16(float4* v) {
  float4 y[16];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    float4 a0 = v[n2], a1 = v[n2 + 4], a2 = v[n2 + 8], a3 = v[n2 + 12];
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
    float4 b0 = y[k1], b1 = y[4 + k1], b2 = y[8 + k1], b3 = y[12 + k1];
    dft4<DIR>(b0, b1, b2, b3);
    v[k1] = b0;
    v[k1 + 4] = b1;
    v[k1 + 8] = b2;
    v[k1 + 12] = b3;
  }
}

template <int DIR, int R>
__device__ __forceinline__ void dft16_r(float4* v) {
  if constexpr (R == 16) dft16<DIR>(v);
  else dft_r<DIR, R>(v);
}

// v[r] *= w^r, r = 1..R-1: powers by products of at most four factors,
// each used for r and r + 8 as soon as it is formed (few live registers).
template <int R>
__device__ __forceinline__ void twiddle16_r(float4* v, float2 w) {
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

__device__ __forceinline__ int swz16(int i) { return swz_g<4>(i); }

// One in-place Stockham pass (see common.cuh for the index rules), T = N/16
// threads, each with 16 / R butterflies of radix R.
template <int DIR, int N, int R>
__device__ __forceinline__ void r16_pass(float4* buf, int Ns, const float2* __restrict__ tw, int off,
                                         int tid) {
  constexpr int T = N / 16, NB = 16 / R;
  float4 v[16];
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int jb = tid + T * q;
#pragma unroll
    for (int r = 0; r < R; ++r) v[q * R + r] = buf[swz16(jb + r * (N / R))];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int jb = tid + T * q;
    const int k = jb & (Ns - 1);
    if (Ns > 1) twiddle16_r<R>(&v[q * R], base_twiddle<DIR>(tw, off, k));
    dft16_r<DIR, R>(&v[q * R]);
    const int base = (jb - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) buf[swz16(base + r * Ns)] = v[q * R + r];
  }
  __syncthreads();
}

template <int DIR, int LOGN, int Q0, int Q1>
__device__ __forceinline__ void r16_pass_range(float4* buf, const float2* __restrict__ tw, int tid) {
  using S = Sched16<LOGN>;
  if constexpr (Q0 < Q1) {
    r16_pass<DIR, S::N, S::radix(Q0)>(buf, S::ns(Q0), tw, S::tw_off(Q0), tid);
    r16_pass_range<DIR, LOGN, Q0 + 1, Q1>(buf, tw, tid);
  }
}

// First pass (radix 16, Ns = 1) from registers v[r] = x[tid + r N/16].
template <int DIR>
__device__ __forceinline__ void r16_first_pass(float4* buf, float4* v, int tid) {
  dft16<DIR>(v);
#pragma unroll
  for (int r = 0; r < 16; ++r) buf[swz16(tid * 16 + r)] = v[r];
  __syncthreads();
}

// Last pass read from shared memory and stored to the global rows outA / outB
// (outB may be null), keeping outputs with index < n_keep.  Ns = N/R > jb, so
// output r of butterfly jb is element jb + r Ns.
template <int DIR, int LOGN>
__device__ __forceinline__ void r16_last_pass_global(const float4* buf, const float2* __restrict__ tw,
                                                     int tid, float2* __restrict__ outA,
                                                     float2* __restrict__ outB, int n_keep) {
  using S = Sched16<LOGN>;
  constexpr int Q = S::NPASS - 1, R = S::radix(Q), N = S::N, T = N / 16, NB = 16 / R;
  constexpr int Ns = S::ns(Q);
  float4 v[16];
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int jb = tid + T * q;
#pragma unroll
    for (int r = 0; r < R; ++r) v[q * R + r] = buf[swz16(jb + r * (N / R))];
  }
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int jb = tid + T * q;
    twiddle16_r<R>(&v[q * R], base_twiddle<DIR>(tw, S::tw_off(Q), jb));
    dft16_r<DIR, R>(&v[q * R]);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int idx = jb + r * Ns;
      if (idx < n_keep) {
        outA[idx] = lo2(v[q * R + r]);
        if (outB) outB[idx] = hi2(v[q * R + r]);
      }
    }
  }
}

// Resident CTAs per SM each length is compiled for (register cap 65536 /
// (threads x CTAs)): Nt 1024 -> 64 threads x 6, 2048 -> 128 x 3, 4096 -> 256 x 1
// (the last is bound by shared memory to one CTA anyway).
template <int LOGN>
constexpr int r16_minb() {
  return LOGN == 10 ? 6 : (LOGN == 11 ? 3 : 1);
}

// Forward rows: as stolt_fwd_rows, with 16 bins per thread.
template <int LOGN, bool SHIFT>
__global__ void __launch_bounds__((1 << LOGN) / 16, r16_minb<LOGN>())
stolt_fwd_rows16(RowArgs a) {
  constexpr int N = 1 << LOGN, T = N / 16;
  using S = Sched16<LOGN>;
  extern __shared__ float4 smem4[];
  float4* buf = smem4;                          // N interleaved (A, B) values
  float2* stage = (float2*)(smem4 + N);         // next panel: row A [ld], row B [ld]
  unsigned* stap0 = (unsigned*)(stage + 2 * a.ld);
  unsigned* stap1 = stap0 + a.taps_ld;
  const int tid = threadIdx.x, l = blockIdx.x, b0 = 2 * blockIdx.y;
  const bool hasB = b0 + 1 < a.batch;
  const float2* xA = a.X + (long long)b0 * a.x_batch + (long long)l * a.ld;
  const float2* xB = hasB ? xA + a.x_batch : nullptr;

  float4 acc[16];
#pragma unroll
  for (int s = 0; s < 16; ++s) acc[s] = make_float4(0.f, 0.f, 0.f, 0.f);
  const unsigned* trow = a.taps + (long long)l * a.taps_ld;
  const long long tstep = (long long)a.Lh * a.taps_ld;
  stage_rows(stage, xA, xB, a.ld, tid, T);
  stage_taps(stap0, trow, a.taps_ld, tid, T);
  cp_async_commit();

  int iv = 0, jt = 0;
  for (int p = 0; p < a.P; ++p) {
    const unsigned* stap = (p & 1) ? stap1 : stap0;
    cp_async_wait_all();
    __syncthreads();
    float4 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
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
    r16_first_pass<-1>(buf, v, tid);
    r16_pass_range<-1, LOGN, 1, S::NPASS>(buf, a.tw16, tid);

#pragma unroll
    for (int s = 0; s < 16; ++s) {
      const int k = tid + T * s;
      const Tap t = tap_decode<N>(k, stap[kabs_of<N>(k)]);
      if (t.valid) {
        float4 vk = cscale(buf[swz16(t.i0)], t.w0);
        vk = cfma(t.w1, buf[swz16(t.i1)], vk);
        if (SHIFT) vk = cmul(vk, __ldg(a.phase + (long long)jt * N + k));
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
  for (int s = 0; s < 16; ++s) acc[s] = cscale(acc[s], __ldg(a.wt + tid + T * s));
  r16_first_pass<+1>(buf, acc, tid);
  r16_pass_range<+1, LOGN, 1, S::NPASS - 1>(buf, a.tw16, tid);
  float2* yA = a.Yw + (long long)b0 * a.y_batch + (long long)l * a.ld;
  r16_last_pass_global<+1, LOGN>(buf, a.tw16, tid, yA, hasB ? yA + a.y_batch : nullptr, a.nt);
}

// Adjoint rows: as stolt_adj_rows (gather form of the transposed map over the
// source table), with 16 output bins per thread.
template <int LOGN, bool SHIFT>
__global__ void __launch_bounds__((1 << LOGN) / 16, r16_minb<LOGN>())
stolt_adj_rows16(RowArgs a) {
  constexpr int N = 1 << LOGN, T = N / 16, H = N / 2;
  using S = Sched16<LOGN>;
  extern __shared__ float4 smem4[];
  float4* buf = smem4;                          // per-panel w_tau spectrum, then its inverse FFT
  float4* dsp = smem4 + N;                      // data spectrum x W (both gathers)
  uint2* stab = (uint2*)(smem4 + 2 * N);        // source-table row of the current panel
  const int tid = threadIdx.x, l = blockIdx.x, b0 = 2 * blockIdx.y;
  const bool hasB = b0 + 1 < a.batch;
  const float2* yA = a.Y + (long long)b0 * a.y_batch + (long long)l * a.ld;
  const float2* yB = hasB ? yA + a.y_batch : nullptr;
  const uint2* arow = a.atab + (long long)l * a.atab_ld;
  const long long astep = (long long)a.Lh * a.atab_ld;
  stage_tab(stab, arow, a.atab_ld, tid, T);
  cp_async_commit();

  {
    float4 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int i = tid + r * T;
      const float2 za = i < a.nt ? __ldg(yA + i) : make_float2(0.f, 0.f);
      const float2 zb = (yB && i < a.nt) ? __ldg(yB + i) : make_float2(0.f, 0.f);
      v[r] = pack2(za, zb);
    }
    r16_first_pass<-1>(buf, v, tid);
  }
  r16_pass_range<-1, LOGN, 1, S::NPASS>(buf, a.tw16, tid);
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    const int k = tid + T * s;
    dsp[swz16(k)] = cscale(buf[swz16(k)], __ldg(a.wt + k));
  }

  float2* xA = a.Xw + (long long)b0 * a.x_batch + (long long)l * a.ld;
  float2* xB = hasB ? xA + a.x_batch : nullptr;
  int iv = 0, jt = 0;
  for (int p = 0; p < a.P; ++p) {
    cp_async_wait_all();
    __syncthreads();
    const bool mapped = __ldg(a.kmin + iv * a.Lh + l) < H;
    const float2* phj = SHIFT ? a.phase + (long long)jt * N : nullptr;
    float4 accs[16];
#pragma unroll
    for (int s = 0; s < 16; ++s)
      accs[s] = mapped ? adj_gather_bin<N, 4, SHIFT>(dsp, stab, tid + T * s, phj)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid == 0 && mapped) accs[0] = adj_gather_bin0_mirror<N, 4, SHIFT>(dsp, stab, phj, accs[0]);
    // its barrier also ends every thread's reads of the source-table row
    r16_first_pass<+1>(buf, accs, tid);
    if (p + 1 < a.P) {
      const int ivn = iv + 1 == a.nv ? 0 : iv + 1;
      stage_tab(stab, arow + ivn * astep, a.atab_ld, tid, T);
      cp_async_commit();
    }
    r16_pass_range<+1, LOGN, 1, S::NPASS - 1>(buf, a.tw16, tid);
    const long long o = (long long)p * a.x_panel;
    r16_last_pass_global<+1, LOGN>(buf, a.tw16, tid, xA + o, xB ? xB + o : nullptr, a.nt);
    if (++iv == a.nv) {
      iv = 0;
      ++jt;
    }
  }
}

template <int LOGN, bool SHIFT>
cudaError_t launch_fwd16(const RowArgs& a, cudaStream_t s) {
  constexpr int N = 1 << LOGN;
  static bool attr = false;
  const size_t smem = (size_t)N * sizeof(float4) + (size_t)2 * a.ld * sizeof(float2) +
                      (size_t)2 * a.taps_ld * sizeof(unsigned);
  cudaError_t e = set_smem(stolt_fwd_rows16<LOGN, SHIFT>, smem_cap<LOGN>(true), attr);
  if (e != cudaSuccess) return e;
  stolt_fwd_rows16<LOGN, SHIFT><<<dim3(a.Lh, (a.batch + 1) / 2), N / 16, smem, s>>>(a);
  return cudaGetLastError();
}

template <int LOGN, bool SHIFT>
cudaError_t launch_adj16(const RowArgs& a, cudaStream_t s) {
  constexpr int N = 1 << LOGN;
  static bool attr = false;
  const size_t smem = (size_t)2 * N * sizeof(float4) + (size_t)a.atab_ld * sizeof(uint2);
  cudaError_t e = set_smem(stolt_adj_rows16<LOGN, SHIFT>, smem_cap<LOGN>(false), attr);
  if (e != cudaSuccess) return e;
  stolt_adj_rows16<LOGN, SHIFT><<<dim3(a.Lh, (a.batch + 1) / 2), N / 16, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool rows16_supported(int logNt) { return logNt >= 10 && logNt <= 12; }

cudaError_t launch_stolt_fwd_rows16(const RowArgs& a, cudaStream_t s) {
  if (!a.tw16) return cudaErrorInvalidValue;
  const bool sh = a.phase != nullptr;
  switch (row_log2(a.Nt)) {
    case 10: return sh ? launch_fwd16<10, true>(a, s) : launch_fwd16<10, false>(a, s);
    case 11: return sh ? launch_fwd16<11, true>(a, s) : launch_fwd16<11, false>(a, s);
    case 12: return sh ? launch_fwd16<12, true>(a, s) : launch_fwd16<12, false>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_stolt_adj_rows16(const RowArgs& a, cudaStream_t s) {
  if (!a.tw16) return cudaErrorInvalidValue;
  const bool sh = a.phase != nullptr;
  switch (row_log2(a.Nt)) {
    case 10: return sh ? launch_adj16<10, true>(a, s) : launch_adj16<10, false>(a, s);
    case 11: return sh ? launch_adj16<11, true>(a, s) : launch_adj16<11, false>(a, s);
    case 12: return sh ? launch_adj16<12, true>(a, s) : launch_adj16<12, false>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ashrt
