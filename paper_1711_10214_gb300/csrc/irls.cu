// Robust l_p - l_q Radon deblending by IRLS with an inner CGLS (ch. 4):
//   J = ||d - L m||_p^p + mu ||m||_q^q                          (Eq. ch4_cost_fn)
//   [W]_ii = max(|x_i|, eps)^((p-2)/2)   (W_r, W_m definitions, read with |x_i|)
//   eps_r = b_r MAD(r) / 0.6745, MAD = Med(|r - Med(r)|)        (Eq. ch4_epcilon_r)
//   eps_m = b_m max|m| / 100
//   each outer iteration: CGLS on min ||W_r (L W_m^-1 u - d)||^2 + mu ||u||^2
//   with u = W_m m                                              (Eqs equ:10, equ:11)
//
// Everything runs on the device for all gathers of the batch at once.  Each
// gather has its own CG scalars (gamma, delta, alpha, beta), accumulated and
// kept in FP64 device memory and read by the vector kernels directly, so the
// CG loop has no host synchronisation.  The weighted operator
// A = W_r S C L W_m^-1 is the plain operator with W_m^-1 fused into the
// model-side loads/stores and W_r, S into the data-side ones; ||A p||^2 and
// ||A^T r||^2 are accumulated by the operator's last kernel.  Medians use a
// per-gather 4 x 8-bit radix select over the live samples.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "internal.h"
#include "ops.h"

namespace ashrt {

namespace {

// scalar slots, laid out scal[slot * B + g]
enum Slot {
  S_GAM0 = 0, S_GAM1 = 1,     // gamma = ||s||^2 (double-buffered by CG iteration parity)
  S_DEL0 = 2, S_DEL1 = 3,     // delta = ||A p||^2 + mu ||p||^2 (double-buffered)
  S_EPSR = 4, S_EPSM = 5,
  S_MIS = 6,                  // misfit of the current model
  S_ACTIVE = 7,               // 1 while the gather iterates, 0 once stopped on tol
  S_MED = 8, S_MAXR = 9, S_NLIVE = 10, S_MAXM = 11, S_BREAK = 12,
  S_HIST = 16                 // misfit history, 64 slots
};
constexpr int kSlots = S_HIST + 64;
static_assert(kSlots <= kScalStride, "scalar slots exceed the plan allocation");

constexpr int kThreads = 256;

__device__ __forceinline__ unsigned fkey(float x) {
  const unsigned u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__device__ __forceinline__ double warp_sum_d(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ void block_add(double part, double* dst) {
  __shared__ double red[32];
  part = warp_sum_d(part);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = part;
  __syncthreads();
  if (w == 0) {
    double x = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    x = warp_sum_d(x);
    if (lane == 0 && x != 0.0) atomicAdd(dst, x);
  }
}

// Kahan-compensated FP32 accumulator (per thread), combined in FP64.
struct Kahan {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// ---- elementwise kernels (grid: (blocks, B); each CTA strides inside one gather)
__global__ void k_nonfinite(const float* __restrict__ d, long long n, int* count) {
  int c = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    if (!isfinite(d[i])) ++c;
  if (c) atomicAdd(count, c);
}

__device__ __forceinline__ bool live_at(const float* tm, int g, int nx, long long i_in_gather, int nt) {
  return tm == nullptr || __ldg(tm + (long long)g * nx + i_in_gather / nt) != 0.f;
}

// r0 = S (d - y) on live samples (0 elsewhere); misfit sum |r0|^p, max|r0|, live count.
__global__ void k_resid(const float* __restrict__ d, const float* __restrict__ y,
                        const float* __restrict__ tm, float* __restrict__ r0, int nx, int nt,
                        float p, double* scal, int B) {
  const int g = blockIdx.y;
  const long long n = (long long)nx * nt, off = (long long)g * n;
  double mis = 0.0, cnt = 0.0;
  float mx = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const bool live = live_at(tm, g, nx, i, nt);
    const float rv = live ? d[off + i] - y[off + i] : 0.f;
    r0[off + i] = rv;
    if (live) {
      const float a = fabsf(rv);
      mis += (p == 1.f) ? (double)a : (p == 2.f) ? (double)a * a : (double)powf(a, p);
      mx = fmaxf(mx, a);
      cnt += 1.0;
    }
  }
  block_add(mis, scal + S_MIS * B + g);
  block_add(cnt, scal + S_NLIVE * B + g);
  // max |r0| as ordered bits (non-negative floats order like their bit patterns)
  __shared__ unsigned smx;
  if (threadIdx.x == 0) smx = 0u;
  __syncthreads();
  atomicMax(&smx, __float_as_uint(mx));
  __syncthreads();
  if (threadIdx.x == 0)
    atomicMax((unsigned long long*)(scal + S_MAXR * B + g), (unsigned long long)smx);
}

// ---- radix select of order statistics over the live samples of each gather.
// sel layout per gather (kSelStride words): [0,256) histogram, 256 prefix,
// 257 rank, 260 count of keys equal to the rank-k1 key at or after its rank,
// 261 smallest key above it.
constexpr int SEL_PREFIX = 256, SEL_RANK = 257, SEL_LE = 260, SEL_MINGT = 261;

// value transform: mode 0 -> x, mode 1 -> |x - med|
__device__ __forceinline__ float sel_value(float x, int mode, double med) {
  return mode == 0 ? x : fabsf(x - (float)med);
}

__global__ void k_sel_init(unsigned* sel, const double* scal, int B) {
  const int g = blockIdx.x;
  unsigned* s = sel + (long long)g * kSelStride;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) s[i] = 0u;
  if (threadIdx.x == 0) {
    const long long n = (long long)scal[S_NLIVE * B + g];
    s[SEL_PREFIX] = 0u;
    s[SEL_RANK] = n > 0 ? (unsigned)((n - 1) / 2) : 0u;
    s[SEL_MINGT] = 0xffffffffu;
  }
}

__global__ void k_sel_hist(const float* __restrict__ x, const float* __restrict__ tm, int nx, int nt,
                           unsigned* sel, const double* scal, int B, int shift, int mode) {
  __shared__ unsigned h[256];
  const int g = blockIdx.y;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  unsigned* s = sel + (long long)g * kSelStride;
  const unsigned prefix = s[SEL_PREFIX];
  const unsigned mask = shift >= 24 ? 0u : (0xffffffffu << (shift + 8));
  const double med = scal[S_MED * B + g];
  const long long n = (long long)nx * nt, off = (long long)g * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (!live_at(tm, g, nx, i, nt)) continue;
    const unsigned key = fkey(sel_value(x[off + i], mode, med));
    if ((key & mask) == prefix) atomicAdd(&h[(key >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&s[i], h[i]);
}

// One CTA (256 threads) per gather: pick the bucket holding the rank.
__global__ void k_sel_scan(unsigned* sel, int shift) {
  __shared__ unsigned h[256];
  __shared__ unsigned cum[256];
  const int g = blockIdx.x;
  unsigned* s = sel + (long long)g * kSelStride;
  const int t = threadIdx.x;
  h[t] = s[t];
  __syncthreads();
  if (t == 0) {
    unsigned c = 0;
    for (int i = 0; i < 256; ++i) {
      cum[i] = c;
      c += h[i];
    }
    const unsigned rank = s[SEL_RANK];
    int b = 255;
    for (int i = 0; i < 256; ++i)
      if (rank < cum[i] + h[i]) {
        b = i;
        break;
      }
    s[SEL_RANK] = rank - cum[b];
    s[SEL_PREFIX] |= ((unsigned)b << shift);
    if (shift == 0) s[SEL_LE] = h[b] - (rank - cum[b]);   // keys equal to k1-key at or after its rank
  }
  __syncthreads();
  s[t] = 0u;
}

// smallest key strictly above the selected one (needed when rank k2 = k1 + 1
// lies beyond the run of keys equal to the k1 key)
__global__ void k_sel_mingt(const float* __restrict__ x, const float* __restrict__ tm, int nx, int nt,
                            unsigned* sel, const double* scal, int B, int mode) {
  const int g = blockIdx.y;
  unsigned* s = sel + (long long)g * kSelStride;
  const unsigned k1 = s[SEL_PREFIX];
  const double med = scal[S_MED * B + g];
  const long long n = (long long)nx * nt, off = (long long)g * n;
  unsigned best = 0xffffffffu;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (!live_at(tm, g, nx, i, nt)) continue;
    const unsigned key = fkey(sel_value(x[off + i], mode, med));
    if (key > k1 && key < best) best = key;
  }
  for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0 && best != 0xffffffffu) atomicMin(&s[SEL_MINGT], best);
}

// median = (x_(k1) + x_(k2)) / 2 with k1 = (n-1)/2, k2 = n/2; mode 0 -> S_MED,
// mode 1 -> eps_r = b_r MAD / 0.6745 with the zero-MAD guard.
__global__ void k_sel_finish(unsigned* sel, double* scal, int B, int mode, double b_r,
                             double eps_fixed) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= B) return;
  unsigned* s = sel + (long long)g * kSelStride;
  const long long n = (long long)scal[S_NLIVE * B + g];
  double med = 0.0;
  if (n > 0) {
    const float v1 = fkey_inv(s[SEL_PREFIX]);
    float v2 = v1;
    if ((n % 2) == 0 && s[SEL_LE] < 2u) v2 = fkey_inv(s[SEL_MINGT]);
    med = 0.5 * ((double)v1 + (double)v2);
  }
  if (mode == 0) {
    scal[S_MED * B + g] = med;
  } else {
    double e = b_r * med / 0.6745;
    if (e == 0.0) {
      const unsigned long long mb = *(const unsigned long long*)(scal + S_MAXR * B + g);
      e = 1e-6 * (double)__uint_as_float((unsigned)mb);
    }
    if (e == 0.0) e = 1e-30;
    if (eps_fixed > 0.0) e = eps_fixed;
    scal[S_EPSR * B + g] = e;
  }
}

// W_r = max(|r0|, eps_r)^((p-2)/2)
__global__ void k_wr(const float* __restrict__ r0, float* __restrict__ wr, long long n, float p,
                     const double* scal, int B) {
  const int g = blockIdx.y;
  const long long off = (long long)g * n;
  const float e = (float)scal[S_EPSR * B + g];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float a = fmaxf(fabsf(r0[off + i]), e);
    wr[off + i] = (p == 2.f) ? 1.f : (p == 1.f) ? rsqrtf(a) : powf(a, 0.5f * (p - 2.f));
  }
}

__global__ void k_maxabs(const float* __restrict__ m, long long n, double* scal, int B) {
  const int g = blockIdx.y;
  const long long off = (long long)g * n;
  float mx = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    mx = fmaxf(mx, fabsf(m[off + i]));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0)
    atomicMax((unsigned long long*)(scal + S_MAXM * B + g), (unsigned long long)__float_as_uint(mx));
}

__global__ void k_epsm(double* scal, int B, double b_m, double eps_fixed) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= B) return;
  const unsigned long long mb = *(const unsigned long long*)(scal + S_MAXM * B + g);
  const double mx = (double)__uint_as_float((unsigned)mb);
  double e = b_m * mx / 100.0;
  if (eps_fixed > 0.0) e = eps_fixed;
  scal[S_EPSM * B + g] = e;   // 0 means m == 0: W_m = I
}

// W_m^-1 = max(|m|, eps_m)^((2-q)/2) (1 when eps_m == 0) and the CG start:
// u = W_m m (warm) or 0; or, when u is null (the fused CG path, which keeps
// m itself), m is set to the start W_m^-1 u0: 0 on absent apexes and, for a
// cold CG start, everywhere (gathers stopped on tol keep their model).
__global__ void k_wm(float* __restrict__ m, float* __restrict__ wminv, float* __restrict__ u,
                     long long n, float q, const double* scal, int B, int warm,
                     const float* __restrict__ amask, int nx, int nt) {
  const int g = blockIdx.y;
  const long long off = (long long)g * n;
  const float e = (float)scal[S_EPSM * B + g];
  const bool active = scal[S_ACTIVE * B + g] != 0.0;
  auto weight = [&](float mv) {
    float w = 1.f;
    if (e > 0.f) {
      const float a = fmaxf(fabsf(mv), e);
      w = (q == 2.f) ? 1.f : (q == 1.f) ? sqrtf(a) : powf(a, 0.5f * (2.f - q));
    }
    return w;
  };
  if (!amask && (n & 3) == 0) {
    // four elements per thread and iteration: enough loads in flight to
    // stream the model at the memory's rate (the vectors are 16-byte aligned:
    // n is a multiple of 4 and the buffers are)
    float4* m4 = (float4*)(m + off);
    float4* w4 = (float4*)(wminv + off);
    float4* u4 = u ? (float4*)(u + off) : nullptr;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n / 4;
         i += (long long)gridDim.x * blockDim.x) {
      const float4 mv = m4[i];
      const float4 w = make_float4(weight(mv.x), weight(mv.y), weight(mv.z), weight(mv.w));
      w4[i] = w;
      if (u4) {
        u4[i] = make_float4(warm ? mv.x / w.x : 0.f, warm ? mv.y / w.y : 0.f,
                            warm ? mv.z / w.z : 0.f, warm ? mv.w / w.w : 0.f);
      } else if (active) {
        if (!warm) m4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    return;
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float mv = m[off + i];
    float w = weight(mv);
    if (amask && __ldg(amask + (long long)g * nx + (i / nt) % nx) == 0.f) w = 0.f;
    wminv[off + i] = w;
    if (u) u[off + i] = (warm && w != 0.f) ? mv / w : 0.f;
    else if (active && (!warm || w == 0.f)) m[off + i] = 0.f;
  }
}

// CGLS start: r = W_r S (d - y) when warm (A u0 = W_r S L m = W_r S y), else W_r S d
__global__ void k_cg_init_r(const float* __restrict__ d, const float* __restrict__ y,
                            const float* __restrict__ wr, const float* __restrict__ tm,
                            float* __restrict__ r, int nx, int nt, int use_y) {
  const int g = blockIdx.y;
  const long long n = (long long)nx * nt, off = (long long)g * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const bool live = live_at(tm, g, nx, i, nt);
    const float dv = d[off + i] - (use_y ? y[off + i] : 0.f);
    r[off + i] = live ? wr[off + i] * dv : 0.f;
  }
}

// s -= mu u and gamma += ||s||^2 (only used when mu > 0)
__global__ void k_smu(float* __restrict__ s, const float* __restrict__ u, long long n, float mu,
                      double* gam, int B) {
  const int g = blockIdx.y;
  const long long off = (long long)g * n;
  Kahan acc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float v = s[off + i] - mu * u[off + i];
    s[off + i] = v;
    acc.add(v * v);
  }
  block_add(acc.value(), gam + g);
}

__device__ __forceinline__ double cg_alpha(const double* scal, int B, int g, int it) {
  const double gam = scal[(S_GAM0 + (it & 1)) * B + g];
  const double del = scal[(S_DEL0 + (it & 1)) * B + g];
  if (scal[S_ACTIVE * B + g] == 0.0 || !(del > 0.0) || !(gam > 0.0)) return 0.0;
  return gam / del;
}

// u += alpha p (model), r -= alpha q (data)
__global__ void k_upd_ur(float* __restrict__ u, const float* __restrict__ p, long long nm,
                         float* __restrict__ r, const float* __restrict__ q, long long nd,
                         const double* scal, int B, int it) {
  const int g = blockIdx.y;
  const float a = (float)cg_alpha(scal, B, g, it);
  if (a == 0.f) return;
  const long long om = (long long)g * nm, od = (long long)g * nd;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nm;
       i += (long long)gridDim.x * blockDim.x)
    u[om + i] = fmaf(a, p[om + i], u[om + i]);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nd;
       i += (long long)gridDim.x * blockDim.x)
    r[od + i] = fmaf(-a, q[od + i], r[od + i]);
}

// p = s + beta p, beta = gamma_{it+1} / gamma_it; optionally delta_{it+1} = mu ||p||^2
__global__ void k_upd_p(float* __restrict__ p, const float* __restrict__ s, long long nm,
                        double* scal, int B, int it, float mu) {
  const int g = blockIdx.y;
  const double gcur = scal[(S_GAM0 + (it & 1)) * B + g];
  const double gnext = scal[(S_GAM0 + ((it + 1) & 1)) * B + g];
  const bool act = scal[S_ACTIVE * B + g] != 0.0 && gcur > 0.0;
  const float beta = act ? (float)(gnext / gcur) : 0.f;
  const long long om = (long long)g * nm;
  Kahan acc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nm;
       i += (long long)gridDim.x * blockDim.x) {
    const float v = act ? fmaf(beta, p[om + i], s[om + i]) : p[om + i];
    p[om + i] = v;
    if (mu > 0.f) acc.add(v * v);
  }
  if (mu > 0.f) block_add((double)mu * acc.value(), scal + (S_DEL0 + ((it + 1) & 1)) * B + g);
}

// Coefficients of the CGLS updates fused into the transforms (mu = 0 path).
// Forward of iteration it: p_it = s_it + beta p_{it-1} (p_0 = s_0), and the
// deferred u += alpha_{it-1} p_{it-1}; a stopped gather keeps p and u.
__global__ void k_cg_coef_fwd(const double* scal, int B, int it, float4* coef) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= B) return;
  if (it == 0) {
    coef[g] = make_float4(1.f, 0.f, 0.f, 0.f);
    return;
  }
  const float4 prev = coef[g];
  const double gprev = scal[(S_GAM0 + ((it - 1) & 1)) * B + g];
  const double gcur = scal[(S_GAM0 + (it & 1)) * B + g];
  const bool act = scal[S_ACTIVE * B + g] != 0.0 && gprev > 0.0;
  const float alpha = (float)cg_alpha(scal, B, g, it - 1);
  // the model takes its updates two at a time, on odd iterations:
  // alpha_{it-1} p~_{it-1} + alpha_{it-2} p~_{it-2}; an even iteration only
  // keeps its alpha_{it-1} (in .w, where the next one finds it)
  const float az = (it & 1) ? alpha : 0.f;
  const float aw = (it & 1) ? (it >= 3 ? prev.w : 0.f) : alpha;
  coef[g] = act ? make_float4(1.f, (float)(gcur / gprev), az, aw)
                : make_float4(0.f, 1.f, az, aw);
}

// Adjoint of iteration it: r -= alpha_it q_it.
__global__ void k_cg_coef_adj(const double* scal, int B, int it, float4* coef) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= B) return;
  coef[g] = make_float4(0.f, 0.f, (float)cg_alpha(scal, B, g, it), 0.f);
}

// The model updates still deferred after the last CGLS iteration it:
// u += alpha_it p, and after an even it also the one kept from it - 1,
// alpha_{it-1} pprev (alpha_{it-1} in the forward coefficients' .w).
__global__ void k_upd_u2(float* __restrict__ u, const float* __restrict__ p,
                         const float* __restrict__ pprev, long long nm, const double* scal, int B,
                         int it, const float4* __restrict__ coef) {
  const int g = blockIdx.y;
  const float a = (float)cg_alpha(scal, B, g, it);
  const float a2 = (it & 1) ? 0.f : coef[g].w;
  if (a == 0.f && a2 == 0.f) return;
  const long long om = (long long)g * nm;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nm;
       i += (long long)gridDim.x * blockDim.x)
    u[om + i] = fmaf(a, p[om + i], fmaf(a2, pprev[om + i], u[om + i]));
}

// p = s at the start of CGLS; delta_0 = mu ||p||^2
__global__ void k_copy_p(float* __restrict__ p, const float* __restrict__ s, long long nm,
                         double* scal, int B, float mu) {
  const int g = blockIdx.y;
  const long long om = (long long)g * nm;
  Kahan acc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nm;
       i += (long long)gridDim.x * blockDim.x) {
    const float v = s[om + i];
    p[om + i] = v;
    if (mu > 0.f) acc.add(v * v);
  }
  if (mu > 0.f) block_add((double)mu * acc.value(), scal + S_DEL0 * B + g);
}

// m = W_m^-1 u for active gathers (stopped gathers keep their model)
__global__ void k_model(float* __restrict__ m, const float* __restrict__ wminv,
                        const float* __restrict__ u, long long nm, const double* scal, int B) {
  const int g = blockIdx.y;
  if (scal[S_ACTIVE * B + g] == 0.0) return;
  const long long om = (long long)g * nm;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nm;
       i += (long long)gridDim.x * blockDim.x)
    m[om + i] = wminv[om + i] * u[om + i];
}

// record J_k, apply the stopping rule, count the outer iteration
__global__ void k_outer_done(double* scal, int* flags, int* outer_cnt, int B, int k, double tol) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= B) return;
  if (scal[S_ACTIVE * B + g] == 0.0) return;
  const double J = scal[S_MIS * B + g];
  scal[(S_HIST + k) * B + g] = J;
  outer_cnt[g] = k + 1;
  if (tol > 0.0 && k > 0) {
    const double Jp = scal[(S_HIST + k - 1) * B + g];
    if (Jp > 0.0 && fabs(J - Jp) / Jp < tol) {
      scal[S_ACTIVE * B + g] = 0.0;
      flags[g] |= 1;
    }
  }
}

__global__ void k_set(double* x, double v, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

#define LAUNCH(kern, grid, block, ...)       \
  do {                                       \
    kern<<<(grid), (block), 0, s>>>(__VA_ARGS__); \
    count_launches(1);                       \
  } while (0)

int grid_for(long long n_per_gather, int B) {
  // about 8 CTAs per SM in total over all gathers, at least one per gather
  long long per = (152LL * 8 + B - 1) / B;
  long long need = (n_per_gather + kThreads * 4 - 1) / (kThreads * 4);
  long long gx = per < need ? per : need;
  return (int)(gx < 1 ? 1 : gx);
}

}  // namespace

// Order statistic machinery: median (mode 0) or eps_r from the MAD (mode 1)
static cudaError_t select_median(const ashrt_plan* P, const float* x, const float* tm, int B,
                                 int mode, double b_r, double eps_fixed, cudaStream_t s) {
  const int nx = P->nr, nt = P->nt;   // data traces
  dim3 grid(grid_for((long long)nx * nt, B), B);
  LAUNCH(k_sel_init, B, kThreads, P->sel, P->scal, B);
  for (int shift = 24; shift >= 0; shift -= 8) {
    LAUNCH(k_sel_hist, grid, kThreads, x, tm, nx, nt, P->sel, P->scal, B, shift, mode);
    LAUNCH(k_sel_scan, B, 256, P->sel, shift);
  }
  LAUNCH(k_sel_mingt, grid, kThreads, x, tm, nx, nt, P->sel, P->scal, B, mode);
  LAUNCH(k_sel_finish, (B + 127) / 128, 128, P->sel, P->scal, B, mode, b_r, eps_fixed);
  return cudaGetLastError();
}

}  // namespace ashrt

using namespace ashrt;

extern "C" {

void irls_default_opts(irls_opts* o) {
  if (!o) return;
  o->p = 1.0;
  o->q = 1.0;
  o->n_outer = 5;
  o->n_cg = 20;
  o->tol = 0.0;
  o->b_r = 1.345;
  o->b_m = 1.0;
  o->mu = 0.0;
  o->warm_start_cg = 1;
  o->eps_r_fixed = 0.0;
  o->eps_m_fixed = 0.0;
  o->trace_mask_dev = nullptr;
  o->apex_mask_dev = nullptr;
  o->use_graph = 0;
  o->m0_dev = nullptr;
  o->wr0_dev = nullptr;
  o->wr_out_dev = nullptr;
}

ashrt_status robust_irls_deblend(const ashrt_plan* P, const float* d, float* m, float* drec,
                                 int B, const irls_opts* opts, irls_report* rep, void* stream) {
  if (!P || !d || !m) {
    set_error("robust_irls_deblend: NULL plan or array");
    return ASHRT_EINVAL;
  }
  if (!P->with_solver) {
    set_error("robust_irls_deblend: plan was created without with_solver");
    return ASHRT_EINVAL;
  }
  if (B < 1 || B > P->max_batch) {
    set_error("robust_irls_deblend: batch %d outside [1, %d]", B, P->max_batch);
    return ASHRT_EINVAL;
  }
  irls_opts o;
  irls_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.p > 0.0 && o.p <= 2.0) || !(o.q > 0.0 && o.q <= 2.0) || o.n_outer < 1 ||
      o.n_outer > 64 || o.n_cg < 0 || !(o.mu >= 0.0) || !(o.tol >= 0.0)) {
    set_error("robust_irls_deblend: need 0<p,q<=2, 1<=n_outer<=64, n_cg>=0, mu>=0, tol>=0");
    return ASHRT_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const float* tm = o.trace_mask_dev;
  const float* am = o.apex_mask_dev;
  const bool fused = !(o.mu > 0);   // the mu = 0 CG with its updates fused into the transforms
  const long long nd = (long long)P->nr * P->nt;          // data samples per gather
  const long long nm = (long long)P->nx * P->nt * P->P;   // model samples per gather
  const int nx = P->nx, nr = P->nr, nt = P->nt;
  double* scal = P->scal;
  int* flags = P->flags;
  float* r0 = P->qv;   // the IRLS residual shares the CG q buffer (not live at the same time)

#define CK(x)                                                                      \
  do {                                                                             \
    cudaError_t e_ = (x);                                                          \
    if (e_ != cudaSuccess) {                                                       \
      set_error("robust_irls_deblend: %s (%s)", #x, cudaGetErrorString(e_));       \
      return ASHRT_ECUDA;                                                          \
    }                                                                              \
  } while (0)

  // flags layout: [0, B) status bits, [B, 2B) outer iterations done, [2B] scratch counter
  int* outer_cnt = flags + B;
  int* d_cnt = flags + 2 * B;
  // non-finite input check (one host synchronisation)
  CK(cudaMemsetAsync(d_cnt, 0, sizeof(int), s));
  LAUNCH(k_nonfinite, 152 * 4, kThreads, d, nd * B, d_cnt);
  CK(cudaGetLastError());
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, d_cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (bad) {
    set_error("robust_irls_deblend: %d non-finite values in d", bad);
    return ASHRT_ENAN;
  }

  int applies_f = 0, applies_a = 0;
  // Everything below is asynchronous on stream s (and capturable as a graph
  // when tol == 0: the tol rule synchronises once per outer iteration).
  auto enqueue = [&](cudaStream_t s) -> ashrt_status {
    CK(cudaMemsetAsync(scal, 0, sizeof(double) * kSlots * B, s));
    LAUNCH(k_set, (B + 127) / 128, 128, scal + S_ACTIVE * B, 1.0, B);
    CK(cudaMemsetAsync(flags, 0, sizeof(int) * B, s));
    CK(cudaMemsetAsync(outer_cnt, 0, sizeof(int) * B, s));

    const dim3 gm(grid_for(nm, B), B), gd(grid_for(nd, B), B);
    const float pf = (float)o.p, qf = (float)o.q, muf = (float)o.mu;

    for (int k = 0; k < o.n_outer; ++k) {
      const bool warm = (k > 0 || o.m0_dev) && o.warm_start_cg;
      if (k == 0 && !o.m0_dev) {
        // cold start: W_m^-1 = 1 (0 on absent apexes), u = 0 (m = 0); W_r = wr0 or 1
        if (fused) CK(cudaMemsetAsync(m, 0, sizeof(float) * nm * B, s));
        else CK(cudaMemsetAsync(P->u, 0, sizeof(float) * nm * B, s));
        LAUNCH(k_wm, gm, kThreads, m, P->wminv, fused ? nullptr : P->u, nm, qf, scal, B, 0, am,
               nx, nt);   // eps_m = 0 -> 1
        LAUNCH(k_set, (B + 127) / 128, 128, scal + S_EPSR * B, 1.0, B);
        if (o.wr0_dev) CK(cudaMemcpyAsync(P->wr, o.wr0_dev, sizeof(float) * nd * B,
                                          cudaMemcpyDeviceToDevice, s));
        else LAUNCH(k_wr, gd, kThreads, d, P->wr, nd, 2.f, scal, B);      // p=2 -> 1
      } else {
        if (k == 0) {
          // warm start: m = m0, its residual r0 = S(d - C L m0), then reweight as usual
          CK(cudaMemcpyAsync(m, o.m0_dev, sizeof(float) * nm * B, cudaMemcpyDeviceToDevice, s));
          CK(op_forward(P, m, P->y, nullptr, nullptr, nullptr, nullptr, B, s));
          ++applies_f;
          CK(cudaMemsetAsync(scal + S_MIS * B, 0, sizeof(double) * B, s));
          CK(cudaMemsetAsync(scal + S_NLIVE * B, 0, sizeof(double) * B, s));
          CK(cudaMemsetAsync(scal + S_MAXR * B, 0, sizeof(double) * B, s));
          LAUNCH(k_resid, gd, kThreads, d, P->y, tm, r0, nr, nt, pf, scal, B);
        }
        if (k == 0 && o.wr0_dev) {
          CK(cudaMemcpyAsync(P->wr, o.wr0_dev, sizeof(float) * nd * B, cudaMemcpyDeviceToDevice, s));
        } else {
          // r0 and the misfit were computed at the end of the previous outer iteration
          select_median(P, r0, tm, B, 0, o.b_r, o.eps_r_fixed, s);
          select_median(P, r0, tm, B, 1, o.b_r, o.eps_r_fixed, s);
          LAUNCH(k_wr, gd, kThreads, r0, P->wr, nd, pf, scal, B);
        }
        CK(cudaMemsetAsync(scal + S_MAXM * B, 0, sizeof(double) * B, s));
        LAUNCH(k_maxabs, gm, kThreads, m, nm, scal, B);
        LAUNCH(k_epsm, (B + 127) / 128, 128, scal, B, o.b_m, o.eps_m_fixed);
        LAUNCH(k_wm, gm, kThreads, m, P->wminv, fused ? nullptr : P->u, nm, qf, scal, B,
               warm ? 1 : 0, am, nx, nt);
      }
      CK(cudaGetLastError());
      // ---- CGLS on A = W_r S C L W_m^-1, b = W_r S d
      LAUNCH(k_cg_init_r, gd, kThreads, d, P->y, P->wr, tm, P->r, nr, nt, warm ? 1 : 0);
      CK(cudaMemsetAsync(scal + S_GAM0 * B, 0, sizeof(double) * 4 * B, s));
      CgFuse f0;
      f0.model_ew_sq = fused ? 1 : 0;     // s~ = W_m^-1 s
      CK(op_adjoint(P, P->r, P->sv, P->wminv, P->wr, tm, o.mu > 0 ? nullptr : scal + S_GAM0 * B, B,
                    s, &f0));
      ++applies_a;
      if (o.mu > 0) LAUNCH(k_smu, gm, kThreads, P->sv, P->u, nm, muf, scal + S_GAM0 * B, B);
      // The adjoint after the last iteration's update would only serve a
      // next direction: it is not run.
      if (o.mu > 0) {
        LAUNCH(k_copy_p, gm, kThreads, P->pv, P->sv, nm, scal, B, muf);
        for (int it = 0; it < o.n_cg; ++it) {
          // delta_it (+= ||A p||^2; the mu ||p||^2 part was added when p was formed)
          CK(op_forward(P, P->pv, P->qv, P->wminv, P->wr, tm, scal + (S_DEL0 + (it & 1)) * B, B, s));
          ++applies_f;
          LAUNCH(k_upd_ur, gm, kThreads, P->u, P->pv, nm, P->r, P->qv, nd, scal, B, it);
          if (it + 1 == o.n_cg) break;
          const int nxt = (it + 1) & 1;
          CK(cudaMemsetAsync(scal + (S_GAM0 + nxt) * B, 0, sizeof(double) * B, s));
          CK(cudaMemsetAsync(scal + (S_DEL0 + nxt) * B, 0, sizeof(double) * B, s));
          CK(op_adjoint(P, P->r, P->sv, P->wminv, P->wr, tm, nullptr, B, s));
          ++applies_a;
          LAUNCH(k_smu, gm, kThreads, P->sv, P->u, nm, muf, scal + (S_GAM0 + nxt) * B, B);
          LAUNCH(k_upd_p, gm, kThreads, P->pv, P->sv, nm, scal, B, it, muf);
          CK(cudaGetLastError());
        }
      } else {
        // mu = 0: the vector updates ride on the transforms' loads, and the
        // vectors are kept premultiplied by W_m^-1: p~ = W_m^-1 p, s~ = W_m^-1 s
        // and the model m = W_m^-1 u itself, so the forward's input p~ needs no
        // weight.  The forward of iteration it forms p~_it = s~_it + beta
        // p~_{it-1} and applies the deferred m += alpha_{it-1} p~_{it-1}; the
        // adjoint forms r -= alpha_it q_it and returns s~ = W_m^-2 L^T (..) with
        // gamma = ||W_m^-1 L^T (..)||^2.  The model takes its deferred updates
        // two at a time (odd iterations: alpha_{it-1} p~_{it-1} +
        // alpha_{it-2} p~_{it-2}), so p~ alternates between two buffers (the
        // unweighted path's u is free here): iteration it reads p~_{it-1} and
        // writes p~_it over p~_{it-2}, after reading it when it is odd.  What
        // is still deferred after the last iteration runs on its own.
        float4* cf_f = P->cg_coef;
        float4* cf_a = P->cg_coef + B;
        float* const pb[2] = {P->pv, P->u};     // p~_it in pb[it & 1]
        for (int it = 0; it < o.n_cg; ++it) {
          LAUNCH(k_cg_coef_fwd, (B + 127) / 128, 128, scal, B, it, cf_f);
          CgFuse ff;
          ff.mode = 1;
          ff.s = P->sv;
          ff.u = m;
          ff.pout = pb[it & 1];
          ff.p2_read = (it & 1) && it >= 3;
          ff.u_rw = it & 1;                     // even iterations leave the model alone
          ff.coef = cf_f;
          CK(op_forward(P, pb[(it + 1) & 1], P->qv, nullptr, P->wr, tm,
                        scal + (S_DEL0 + (it & 1)) * B, B, s, &ff));
          ++applies_f;
          if (it + 1 == o.n_cg) {
            LAUNCH(k_upd_u2, gm, kThreads, m, pb[it & 1], pb[(it + 1) & 1], nm, scal, B, it, cf_f);
            break;
          }
          LAUNCH(k_cg_coef_adj, (B + 127) / 128, 128, scal, B, it, cf_a);
          const int nxt = (it + 1) & 1;
          CK(cudaMemsetAsync(scal + (S_GAM0 + nxt) * B, 0, sizeof(double) * B, s));
          CK(cudaMemsetAsync(scal + (S_DEL0 + nxt) * B, 0, sizeof(double) * B, s));
          CgFuse fa;
          fa.mode = 2;
          fa.s = P->qv;
          fa.coef = cf_a;
          fa.model_ew_sq = 1;
          CK(op_adjoint(P, P->r, P->sv, P->wminv, P->wr, tm, scal + (S_GAM0 + nxt) * B, B, s, &fa));
          ++applies_a;
          CK(cudaGetLastError());
        }
      }
      // ---- m = W_m^-1 u (the fused path keeps m), y = C L m (no mask),
      //      residual and misfit J_k
      if (!fused) LAUNCH(k_model, gm, kThreads, m, P->wminv, P->u, nm, scal, B);
      CK(op_forward(P, m, P->y, nullptr, nullptr, nullptr, nullptr, B, s));
      ++applies_f;
      CK(cudaMemsetAsync(scal + S_MIS * B, 0, sizeof(double) * B, s));
      CK(cudaMemsetAsync(scal + S_NLIVE * B, 0, sizeof(double) * B, s));
      CK(cudaMemsetAsync(scal + S_MAXR * B, 0, sizeof(double) * B, s));
      LAUNCH(k_resid, gd, kThreads, d, P->y, tm, r0, nr, nt, pf, scal, B);
      LAUNCH(k_outer_done, (B + 127) / 128, 128, scal, flags, outer_cnt, B, k, o.tol);
      CK(cudaGetLastError());
      if (o.tol > 0.0) {
        std::vector<double> act(B);
        CK(cudaMemcpyAsync(act.data(), scal + S_ACTIVE * B, sizeof(double) * B,
                           cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        bool any = false;
        for (double a : act) any = any || a != 0.0;
        if (!any) break;
      }
    }
    if (drec) CK(cudaMemcpyAsync(drec, P->y, sizeof(float) * nd * B, cudaMemcpyDeviceToDevice, s));
    if (o.wr_out_dev) {
      // the weights the next outer iteration would take from the final residual
      select_median(P, r0, tm, B, 0, o.b_r, o.eps_r_fixed, s);
      select_median(P, r0, tm, B, 1, o.b_r, o.eps_r_fixed, s);
      LAUNCH(k_wr, gd, kThreads, r0, o.wr_out_dev, nd, pf, scal, B);
      CK(cudaGetLastError());
    }
    return ASHRT_OK;
  };

  ashrt_plan* Pm = const_cast<ashrt_plan*>(P);
  const bool graph = o.use_graph && o.tol <= 0.0;
  if (!graph) {
    ashrt_status st = enqueue(s);
    if (st != ASHRT_OK) return st;
  } else {
    GraphKey key;
    key.d = d; key.m = m; key.drec = drec; key.B = B; key.opts = o;
    if (!Pm->graph_exec || !(Pm->graph_key == key)) {
      if (Pm->graph_exec) {
        cudaGraphExecDestroy(Pm->graph_exec);
        Pm->graph_exec = nullptr;
      }
      if (!Pm->cap_stream) CK(cudaStreamCreateWithFlags(&Pm->cap_stream, cudaStreamNonBlocking));
      CK(cudaStreamBeginCapture(Pm->cap_stream, cudaStreamCaptureModeThreadLocal));
      prof_capture_begin();
      ashrt_status st = enqueue(Pm->cap_stream);
      const long long kernels = prof_capture_end();
      cudaGraph_t g = nullptr;
      cudaError_t ec = cudaStreamEndCapture(Pm->cap_stream, &g);
      if (st != ASHRT_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      CK(ec);
      ec = cudaGraphInstantiate(&Pm->graph_exec, g, 0);
      cudaGraphDestroy(g);
      CK(ec);
      Pm->graph_key = key;
      Pm->graph_kernels = kernels;
      Pm->graph_applies_f = applies_f;
      Pm->graph_applies_a = applies_a;
    }
    CK(cudaGraphLaunch(Pm->graph_exec, s));
    count_launches((int)Pm->graph_kernels);
    applies_f = Pm->graph_applies_f;
    applies_a = Pm->graph_applies_a;
  }

  std::vector<int> outer_cnt_h(B, 0);
  std::vector<double> hist((size_t)64 * B);
  std::vector<int> fl(B);
  CK(cudaMemcpyAsync(hist.data(), scal + S_HIST * B, sizeof(double) * 64 * B,
                     cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(fl.data(), flags, sizeof(int) * B, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(outer_cnt_h.data(), outer_cnt, sizeof(int) * B, cudaMemcpyDeviceToHost, s));
  int dev_err = 0;
  CK(cudaMemcpyAsync(&dev_err, P->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (dev_err) {
    cudaMemsetAsync(P->dev_err, 0, sizeof(int), s);
    set_error("robust_irls_deblend: a device-side wait for a tile copy ran out");
    return ASHRT_ETIMEOUT;
  }
#undef CK
  if (rep) {
    for (int g = 0; g < B; ++g) {
      rep[g].outer_done = outer_cnt_h[g];
      rep[g].applies_fwd = applies_f;
      rep[g].applies_adj = applies_a;
      rep[g].flags = fl[g];
      for (int k = 0; k < 64; ++k) rep[g].misfit[k] = k < outer_cnt_h[g] ? hist[(size_t)k * B + g] : 0.0;
    }
  }
  return ASHRT_OK;
}

}  // extern "C"
