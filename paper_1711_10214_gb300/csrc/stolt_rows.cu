// Fused time-axis FFT + Stolt map + velocity/asymptote sum (forward) or
// spray (adjoint), one CTA per (gather, k_x) row.
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
// The panel spectrum, the map and the accumulation never leave the SM: the
// accumulator D lives in registers (each thread owns bins k = tid + T s), the
// spectrum of the current panel in one shared row, and the next panel's row
// is prefetched into registers while the current one is transformed.
//
// Cone membership (k^2 > a^2, strict; never the w-Nyquist bin) comes from
// the host's FP64 table kmin[v][l], so the GPU and the FP64 oracle agree on
// every bin; the fractional index u = sqrt((|k| - a)(|k| + a)) is evaluated
// in FP32 with a carried as a (hi, lo) pair of floats.
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

// Interpolation taps of output bin k (natural index in [0, N)) of one
// (velocity, k_x) row.  For w > 0 the taps are floor(u), floor(u)+1; for
// w < 0 the mirrored -floor(|u|), -floor(|u|)-1, which is the same linear
// interpolation at u = -|u| (odd extension keeps real output).  A tap on the
// w-Nyquist bin carries weight 0.
template <int N>
__device__ __forceinline__ Tap stolt_tap(int k, int kmin, float2 ac) {
  Tap t;
  const int kk = k <= N / 2 ? k : k - N;
  const int kabs = kk < 0 ? -kk : kk;
  t.valid = (k != N / 2) && (kabs >= kmin);
  const float fk = (float)kabs;
  const float d1 = (fk - ac.x) - ac.y;
  const float s1 = (fk + ac.x) + ac.y;
  const float ua = sqrtf(fmaxf(d1 * s1, 0.f));
  const int k0 = (int)ua;
  const float f = ua - (float)k0;
  if (kk > 0) {
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
__device__ __forceinline__ void load_row(float2* v, const float2* __restrict__ row, int nt, int tid) {
  constexpr int T = N / 8;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = tid + r * T;
    v[r] = i < nt ? __ldg(row + i) : make_float2(0.f, 0.f);
  }
}

template <int LOGN, bool SHIFT>
__global__ void __launch_bounds__((1 << LOGN) / 8)
stolt_fwd_rows(RowArgs a) {
  constexpr int N = 1 << LOGN, T = N / 8;
  using S = Sched<LOGN>;
  __shared__ float2 buf[N];
  const int tid = threadIdx.x, l = blockIdx.x, b = blockIdx.y;
  const float2* xrow = a.X + (long long)b * a.x_batch + (long long)l * a.ld;

  float2 acc[8], accj[8], pf[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) acc[s] = accj[s] = make_float2(0.f, 0.f);
  load_row<N>(pf, xrow, a.nt, tid);

  int iv = 0, jt = 0;
  for (int p = 0; p < a.P; ++p) {
    float2 v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = pf[r];
    if (p + 1 < a.P) load_row<N>(pf, xrow + (long long)(p + 1) * a.x_panel, a.nt, tid);
    row_first_pass<-1, N>(buf, v, tid);
    row_pass_range<-1, LOGN, 1, S::NPASS>(buf, a.tw, tid);

    const int km = __ldg(a.kmin + iv * a.Lh + l);
    const float2 ac = __ldg(a.acone + iv * a.Lh + l);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int k = tid + T * s;
      const Tap t = stolt_tap<N>(k, km, ac);
      if (t.valid) {
        float2 vk = cscale(buf[swz(t.i0)], t.w0);
        vk = cfma(t.w1, buf[swz(t.i1)], vk);
        if (SHIFT) accj[s] = cadd(accj[s], vk);
        else acc[s] = cadd(acc[s], vk);
      }
    }
    if (++iv == a.nv) {
      if (SHIFT) {
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          const int k = tid + T * s;
          acc[s] = cadd(acc[s], cmul(__ldg(a.phase + (long long)jt * N + k), accj[s]));
          accj[s] = make_float2(0.f, 0.f);
        }
      }
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
  float2* yrow = a.Yw + (long long)b * a.y_batch + (long long)l * a.ld;
  row_last_pass_global<+1, LOGN>(buf, a.tw, tid, yrow, a.nt);
}

template <int LOGN, bool SHIFT>
__global__ void __launch_bounds__((1 << LOGN) / 8)
stolt_adj_rows(RowArgs a) {
  constexpr int N = 1 << LOGN, T = N / 8;
  using S = Sched<LOGN>;
  __shared__ float2 buf[N];
  const int tid = threadIdx.x, l = blockIdx.x, b = blockIdx.y;
  const float2* yrow = a.Y + (long long)b * a.y_batch + (long long)l * a.ld;

  float2 v[8];
  load_row<N>(v, yrow, a.nt, tid);
  row_first_pass<-1, N>(buf, v, tid);
  row_pass_range<-1, LOGN, 1, S::NPASS>(buf, a.tw, tid);
  float2 ds[8], dj[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int k = tid + T * s;
    ds[s] = cscale(buf[swz(k)], __ldg(a.wt + k));
    dj[s] = ds[s];
  }
  __syncthreads();

  float2* xrow = a.Xw + (long long)b * a.x_batch + (long long)l * a.ld;
  int iv = 0, jt = 0;
  for (int p = 0; p < a.P; ++p) {
    if (SHIFT && iv == 0) {
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int k = tid + T * s;
        dj[s] = cmul(ds[s], cconj(__ldg(a.phase + (long long)jt * N + k)));
      }
    }
#pragma unroll
    for (int s = 0; s < 8; ++s) buf[swz(tid + T * s)] = make_float2(0.f, 0.f);
    __syncthreads();
    const int km = __ldg(a.kmin + iv * a.Lh + l);
    const float2 ac = __ldg(a.acone + iv * a.Lh + l);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const Tap t = stolt_tap<N>(tid + T * s, km, ac);
      if (t.valid) {
        float2* p0 = &buf[swz(t.i0)];
        atomicAdd(&p0->x, t.w0 * dj[s].x);
        atomicAdd(&p0->y, t.w0 * dj[s].y);
        if (t.w1 != 0.f) {
          float2* p1 = &buf[swz(t.i1)];
          atomicAdd(&p1->x, t.w1 * dj[s].x);
          atomicAdd(&p1->y, t.w1 * dj[s].y);
        }
      }
    }
    __syncthreads();
    row_pass_range<+1, LOGN, 0, S::NPASS - 1>(buf, a.tw, tid);
    row_last_pass_global<+1, LOGN>(buf, a.tw, tid, xrow + (long long)p * a.x_panel, a.nt);
    if (++iv == a.nv) {
      iv = 0;
      ++jt;
    }
  }
}

template <int LOGN>
cudaError_t launch_fwd_t(const RowArgs& a, cudaStream_t s) {
  dim3 grid(a.Lh, a.batch);
  if (a.phase) stolt_fwd_rows<LOGN, true><<<grid, (1 << LOGN) / 8, 0, s>>>(a);
  else stolt_fwd_rows<LOGN, false><<<grid, (1 << LOGN) / 8, 0, s>>>(a);
  return cudaGetLastError();
}

template <int LOGN>
cudaError_t launch_adj_t(const RowArgs& a, cudaStream_t s) {
  dim3 grid(a.Lh, a.batch);
  if (a.phase) stolt_adj_rows<LOGN, true><<<grid, (1 << LOGN) / 8, 0, s>>>(a);
  else stolt_adj_rows<LOGN, false><<<grid, (1 << LOGN) / 8, 0, s>>>(a);
  return cudaGetLastError();
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
