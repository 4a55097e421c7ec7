// Single-gather radix-16 row kernels: the fused t-FFT + Stolt map + sum
// (forward) and its exact transpose (adjoint) of ch. 5 Eqs
// ch5_forward_operator / ch5_adj_operator and ch. 6 Eqs ch6_forward_operator /
// ch6_adj_operator, for Nt = 1024, 2048 and 4096, one CTA per (gather, k_x
// row) with one complex row per element (float2).
//
// The operator, the tables and the transforms are those of stolt_r16.cu (three
// radix-16-first Stockham passes per transform).  What changes is the shape of
// the CTA: a single gather halves its shared memory (an Nt-long float2 row
// instead of two interleaved rows), so about twice as many CTAs are resident
// per SM to hide the latency of the dependent shared-memory passes, and the
// per-bin tables are not staged through shared memory: each thread loads the
// Stolt tap words (forward) or adjoint source-table entries of its own 16 bins
// straight from global memory, the adjoint one panel ahead.  Those tables
// depend on (velocity, k_x) only, and the grid runs the gathers of a row
// next to each other (blockIdx.x = gather), so they are served by L2.  Per
// bin and panel this leaves the transform's passes and the map's two
// interpolation reads as the shared-memory traffic.
#include <cuda_runtime.h>

#include "stolt_common.cuh"
#include "stolt_r16.cuh"

namespace ashrt {

namespace {

// Resident CTAs per SM each length is compiled for: the register cap is
// 65536 / (N/16 threads x CTAs).  The adjoint fits about 96 registers a
// thread; the forward, which holds its accumulator, the transform and the
// panel's tap words at once, needs about 128.
template <int LOGN>
constexpr int r16s_minb_adj() {
  return LOGN == 10 ? 10 : (LOGN == 11 ? 5 : 2);
}
template <int LOGN>
constexpr int r16s_minb_fwd() {
  return LOGN == 10 ? 8 : (LOGN == 11 ? 4 : 2);
}

// Stage one row of ld complex values (ld a multiple of 4, 32-byte aligned).
__device__ __forceinline__ void stage_row1(float2* stage, const float2* row, int ld, int tid,
                                           int T) {
  for (int c = tid; c < (ld >> 1); c += T) cp_async16(stage + 2 * c, row + 2 * c);
}

// One output bin j of the transposed map for a single gather, from its
// source-table entry e (see build_adj_table and adj_gather_bin in
// stolt_common.cuh, of which this is the float2, register-entry form).
template <int N, bool SHIFT>
__device__ __forceinline__ float2 adj_gather1(const float2* dsp, uint2 e, int j,
                                              const float2* __restrict__ phj) {
  constexpr int H = N / 2;
  float2 acc = make_float2(0.f, 0.f);
  if (j == H) return acc;
  const bool pos = j < H;
  const int kB = (int)(e.x >> 20);
  if (e.y & (1u << 21)) {
    const int kn = pos ? kB - 1 : N - kB + 1;
    float2 d = dsp[kn];
    if (SHIFT) d = cmul(d, cconj(__ldg(phj + kn)));
    acc = cscale(d, (float)(e.y & 0xfffffu) * (1.0f / 1048576.0f));
  }
  if (e.y & (1u << 20)) {
    const int kn = pos ? kB : N - kB;
    float2 d = dsp[kn];
    if (SHIFT) d = cmul(d, cconj(__ldg(phj + kn)));
    acc = cfma(1.f - (float)(e.x & 0xfffffu) * (1.0f / 1048576.0f), d, acc);
  }
  return acc;
}

// Forward rows, one gather: for every panel, stage the x-transformed model
// row, FFT it along tau, and accumulate the interpolated bins of the Stolt
// map (taps from the tap word of |k|) times the asymptote phase in registers;
// finally weight by W(w) / (Nt Nx), inverse FFT, keep nt samples.
template <int LOGN, bool SHIFT, bool HALF>
__global__ void __launch_bounds__((1 << LOGN) / 16, r16s_minb_fwd<LOGN>())
stolt_fwd_rows16s(RowArgs a) {
  constexpr int N = 1 << LOGN, T = N / 16;
  using S = Sched16<LOGN>;
  extern __shared__ float2 sm2[];
  float2* buf = sm2;              // the N-bin spectrum of the current panel
  float2* stage = sm2 + N;        // the next panel's row [ld]
  const int tid = threadIdx.x, b = blockIdx.x, l = blockIdx.y;
  const float2* xr = a.X + (long long)b * a.x_batch + (long long)l * a.ld;

  float2 acc[16];
#pragma unroll
  for (int s = 0; s < 16; ++s) acc[s] = make_float2(0.f, 0.f);
  const unsigned* trow = a.taps + (long long)l * a.taps_ld;
  const long long tstep = (long long)a.Lh * a.taps_ld;
  stage_row1(stage, xr, a.ld, tid, T);
  cp_async_commit();

  int iv = 0, jt = 0;
  for (int p = 0; p < a.P; ++p) {
    // this panel's tap words, consumed after the transform
    unsigned tw[16];
    const unsigned* tr = trow + iv * tstep;
#pragma unroll
    for (int s = 0; s < 16; ++s) tw[s] = __ldg(tr + kabs_of<N>(tid + T * s));
    cp_async_wait_all();
    __syncthreads();
    float2 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int i = tid + r * T;
      v[r] = (!(HALF && r >= 8) && i < a.nt) ? stage[i] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (p + 1 < a.P) {
      stage_row1(stage, xr + (long long)(p + 1) * a.x_panel, a.ld, tid, T);
      cp_async_commit();
    }
    r16_first_pass<-1, float2, HALF>(buf, v, tid);
    r16_pass_range<-1, LOGN, 1, S::NPASS, float2, true>(buf, a.tw16, tid);   // natural, unswizzled
#pragma unroll
    for (int s = 0; s < 16; ++s) {
      const int k = tid + T * s;
      const Tap t = tap_decode_side<N>(k, tw[s], s < 8);
      if (t.valid) {
        float2 vk = cscale(buf[t.i0], t.w0);
        vk = cfma(t.w1, buf[t.i1], vk);
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
  // own bins are exactly the first-pass inputs of the inverse transform
  r16_first_pass<+1>(buf, acc, tid);
  r16_pass_range<+1, LOGN, 1, S::NPASS - 1>(buf, a.tw16, tid);
  r16_last_pass_global<+1, LOGN>(buf, a.tw16, tid,
                                 a.Yw + (long long)b * a.y_batch + (long long)l * a.ld, nullptr,
                                 a.nt);
}

// Adjoint rows, one gather: FFT the data row once and weight it by W(w); for
// every panel gather each output bin j = tid + T s from its at most two
// sources (source-table entry of |j|, loaded one panel ahead), inverse FFT,
// keep nt samples.  A (velocity, k_x) row entirely outside the cone gives a
// zero panel row without a transform.
template <int LOGN, bool SHIFT>
__global__ void __launch_bounds__((1 << LOGN) / 16, r16s_minb_adj<LOGN>())
stolt_adj_rows16s(RowArgs a) {
  constexpr int N = 1 << LOGN, T = N / 16, H = N / 2;
  using S = Sched16<LOGN>;
  extern __shared__ float2 sm2[];
  float2* buf = sm2;              // per-panel w_tau spectrum, then its inverse FFT
  float2* dsp = sm2 + N;          // data spectrum x W
  const int tid = threadIdx.x, b = blockIdx.x, l = blockIdx.y;
  const float2* yr = a.Y + (long long)b * a.y_batch + (long long)l * a.ld;
  const uint2* arow = a.atab + (long long)l * a.atab_ld;
  const long long astep = (long long)a.Lh * a.atab_ld;

  uint2 ent[16];
#pragma unroll
  for (int s = 0; s < 16; ++s) ent[s] = __ldg(arow + kabs_of<N>(tid + T * s));
  {
    float2 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int i = tid + r * T;
      v[r] = i < a.nt ? __ldg(yr + i) : make_float2(0.f, 0.f);
    }
    r16_first_pass<-1>(buf, v, tid);
  }
  r16_pass_range<-1, LOGN, 1, S::NPASS, float2, true>(buf, a.tw16, tid);
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    const int k = tid + T * s;
    dsp[k] = cscale(buf[k], __ldg(a.wt + k));   // natural order, unswizzled
  }

  float2* xr = a.Xw + (long long)b * a.x_batch + (long long)l * a.ld;
  int iv = 0, jt = 0;
  int km = __ldg(a.kmin + l);                   // cone start of the panel's (velocity, k_x)
  for (int p = 0; p < a.P; ++p) {
    // dsp complete (first panel); the previous panel's reads of buf done
    __syncthreads();
    const long long o = (long long)p * a.x_panel;
    const int ivn = iv + 1 == a.nv ? 0 : iv + 1;
    const bool more = p + 1 < a.P;
    const bool unmapped = km >= H;
    if (more) km = __ldg(a.kmin + ivn * a.Lh + l);   // the next panel's, a panel ahead
    if (unmapped) {
      // no bin of this (velocity, k_x) row is mapped: the panel row is zero
      for (int i = tid; i < a.nt; i += T) xr[o + i] = make_float2(0.f, 0.f);
      if (more) {
#pragma unroll
        for (int s = 0; s < 16; ++s) ent[s] = __ldg(arow + ivn * astep + kabs_of<N>(tid + T * s));
      }
    } else {
      const float2* phj = SHIFT ? a.phase + (long long)jt * N : nullptr;
      float2 accs[16];
#pragma unroll
      for (int s = 0; s < 16; ++s) accs[s] = adj_gather1<N, SHIFT>(dsp, ent[s], tid + T * s, phj);
      if (tid == 0 && (ent[0].y & (1u << 20))) {
        // bin 0 also takes the primary tap of -kB (w = 0 lies on both sides)
        const int kn = N - (int)(ent[0].x >> 20);
        float2 d = dsp[kn];
        if (SHIFT) d = cmul(d, cconj(__ldg(phj + kn)));
        accs[0] = cfma(1.f - (float)(ent[0].x & 0xfffffu) * (1.0f / 1048576.0f), d, accs[0]);
      }
      if (more) {
#pragma unroll
        for (int s = 0; s < 16; ++s) ent[s] = __ldg(arow + ivn * astep + kabs_of<N>(tid + T * s));
      }
      r16_first_pass<+1>(buf, accs, tid);
      r16_pass_range<+1, LOGN, 1, S::NPASS - 1>(buf, a.tw16, tid);
      r16_last_pass_global<+1, LOGN>(buf, a.tw16, tid, xr + o, nullptr, a.nt);
    }
    iv = ivn;
    if (iv == 0) ++jt;
  }
}

template <int LOGN, bool SHIFT, bool HALF>
cudaError_t launch_fwd16s_h(const RowArgs& a, cudaStream_t s) {
  constexpr int N = 1 << LOGN;
  static bool attr = false;
  const size_t smem = (size_t)(N + a.ld) * sizeof(float2);
  cudaError_t e = set_smem(stolt_fwd_rows16s<LOGN, SHIFT, HALF>, (size_t)2 * N * sizeof(float2),
                           attr);
  if (e != cudaSuccess) return e;
  stolt_fwd_rows16s<LOGN, SHIFT, HALF><<<dim3(a.batch, a.Lh), N / 16, smem, s>>>(a);
  return cudaGetLastError();
}

template <int LOGN, bool SHIFT>
cudaError_t launch_fwd16s(const RowArgs& a, cudaStream_t s) {
  return 2 * a.nt <= a.Nt ? launch_fwd16s_h<LOGN, SHIFT, true>(a, s)
                          : launch_fwd16s_h<LOGN, SHIFT, false>(a, s);
}

template <int LOGN, bool SHIFT>
cudaError_t launch_adj16s(const RowArgs& a, cudaStream_t s) {
  constexpr int N = 1 << LOGN;
  static bool attr = false;
  const size_t smem = (size_t)2 * N * sizeof(float2);
  cudaError_t e = set_smem(stolt_adj_rows16s<LOGN, SHIFT>, smem, attr);
  if (e != cudaSuccess) return e;
  stolt_adj_rows16s<LOGN, SHIFT><<<dim3(a.batch, a.Lh), N / 16, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_stolt_fwd_rows16s(const RowArgs& a, cudaStream_t s) {
  if (!a.tw16 || a.ld > a.Nt) return cudaErrorInvalidValue;
  const bool sh = a.phase != nullptr;
  switch (row_log2(a.Nt)) {
    case 10: return sh ? launch_fwd16s<10, true>(a, s) : launch_fwd16s<10, false>(a, s);
    case 11: return sh ? launch_fwd16s<11, true>(a, s) : launch_fwd16s<11, false>(a, s);
    case 12: return sh ? launch_fwd16s<12, true>(a, s) : launch_fwd16s<12, false>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_stolt_adj_rows16s(const RowArgs& a, cudaStream_t s) {
  if (!a.tw16) return cudaErrorInvalidValue;
  const bool sh = a.phase != nullptr;
  switch (row_log2(a.Nt)) {
    case 10: return sh ? launch_adj16s<10, true>(a, s) : launch_adj16s<10, false>(a, s);
    case 11: return sh ? launch_adj16s<11, true>(a, s) : launch_adj16s<11, false>(a, s);
    case 12: return sh ? launch_adj16s<12, true>(a, s) : launch_adj16s<12, false>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ashrt
