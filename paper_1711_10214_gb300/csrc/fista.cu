// l2-l1 sparse inversion by FISTA for AASHRT interpolation (ch. 6, "Sparse
// inversion": Eq. cost_fn with p = 2, q = 1):
//   minimise J(m) = ||S (d - L m)||_2^2 + mu ||m||_1,
// S the trace-sampling operator, L the Stolt ASHRT/AASHRT forward of the plan.
// The step is 1 / Lf with Lf = 2 lambda_max(L^T S^T S L), lambda_max from
// Rayleigh's power method; the iteration is Beck and Teboulle's (2009):
//   x_k = soft(y_k - grad f(y_k) / Lf, mu / Lf),  grad f(y) = 2 L^T S^T (S L y - S d)
//   y_{k+1} = x_k + beta_k (x_k - x_{k-1}),  beta_k = (t_k - 1) / t_{k+1},
//   t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,  t_1 = 1,  x_0 = y_1 = 0.
// Every gather of the batch runs the same iteration count with its own
// lambda (FP64, device memory); the momentum sequence is the same for all
// and is computed on the host.  The operator applications are the plan's
// (ashrt_forward / ashrt_adjoint kernels); the vector work is three small
// elementwise kernels.  No host synchronisation until the end.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "internal.h"
#include "ops.h"

namespace ashrt {
namespace {

constexpr int kFThreads = 256;

__device__ __forceinline__ double f_warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ void f_block_add(double part, double* dst) {
  __shared__ double red[32];
  part = f_warp_sum(part);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = part;
  __syncthreads();
  if (w == 0) {
    double x = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    x = f_warp_sum(x);
    if (lane == 0) atomicAdd(dst, x);
  }
}

// grid (blocks, B): each CTA strides inside gather blockIdx.y of n elements.
__global__ void k_f_sumsq(const float* __restrict__ x, long long n, double* out) {
  const int g = blockIdx.y;
  const float* xg = x + (long long)g * n;
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = (double)xg[i];
    s += v * v;
  }
  f_block_add(s, out + g);
}

// dst = src / sqrt(sumsq[g]) (0 where sumsq[g] == 0); dst may be src.
__global__ void k_f_normalise(const float* src, float* dst, long long n, const double* sumsq) {
  const int g = blockIdx.y;
  const double ss = sumsq[g];
  const float sc = ss > 0.0 ? (float)(1.0 / sqrt(ss)) : 0.f;
  const long long off = (long long)g * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[off + i] = src[off + i] * sc;
}

__global__ void k_f_lambda(const double* sumsq, double* lam, int B) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < B) lam[g] = sqrt(sumsq[g]);
}

// q <- q - S d (S the per-trace weight, 1 without a mask)
__global__ void k_f_resid(float* __restrict__ q, const float* __restrict__ d,
                          const float* __restrict__ tm, int nx, int nt) {
  const int g = blockIdx.y;
  const long long n = (long long)nx * nt, off = (long long)g * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float sw = tm ? __ldg(tm + (long long)g * nx + i / nt) : 1.f;
    q[off + i] -= sw * d[off + i];
  }
}

// One FISTA update per gather g with lambda = lam[g] (Lf = 2 lambda):
//   x_new = soft(y - w / lambda, mu / (2 lambda)),  y <- x_new + beta (x_new - x),  x <- x_new,
// w = L^T S^T (S L y - S d) (half the gradient).  lambda <= 0: x = y = 0.
__global__ void k_f_step(float* __restrict__ y, const float* __restrict__ w, float* __restrict__ x,
                         const double* lam, double mu, float beta, long long n) {
  const int g = blockIdx.y;
  const double l = lam[g];
  const long long off = (long long)g * n;
  const bool ok = l > 0.0;
  const float inv = ok ? (float)(1.0 / l) : 0.f;
  const float thr = ok ? (float)(mu / (2.0 * l)) : 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (!ok) {
      x[off + i] = 0.f;
      y[off + i] = 0.f;
      continue;
    }
    const float z = fmaf(-inv, w[off + i], y[off + i]);
    const float xn = copysignf(fmaxf(fabsf(z) - thr, 0.f), z);
    const float xo = x[off + i];
    y[off + i] = fmaf(beta, xn - xo, xn);
    x[off + i] = xn;
  }
}

int f_grid(long long n_per_gather, int B) {
  long long per = (152LL * 8 + B - 1) / B;
  long long need = (n_per_gather + kFThreads * 4 - 1) / (kFThreads * 4);
  long long gx = per < need ? per : need;
  return (int)(gx < 1 ? 1 : gx);
}

}  // namespace
}  // namespace ashrt

using namespace ashrt;

extern "C" void fista_default_opts(fista_opts* o) {
  if (!o) return;
  o->mu = 0.0;
  o->n_iter = 50;
  o->n_power = 20;
}

extern "C" ashrt_status ashrt_fista(const ashrt_plan* P, const float* d, const float* tmask,
                                    const float* v0, float* m, float* drec, int B,
                                    const fista_opts* opts, double* lipschitz, void* stream) {
  if (!P || !d || !v0 || !m) {
    set_error("ashrt_fista: NULL plan or array");
    return ASHRT_EINVAL;
  }
  if (!P->with_solver) {
    set_error("ashrt_fista: plan was created without with_solver");
    return ASHRT_EINVAL;
  }
  if (B < 1 || B > P->max_batch) {
    set_error("ashrt_fista: batch %d outside [1, %d]", B, P->max_batch);
    return ASHRT_EINVAL;
  }
  fista_opts o;
  fista_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.mu >= 0.0) || !std::isfinite(o.mu) || o.n_iter < 1 || o.n_power < 1) {
    set_error("ashrt_fista: need mu >= 0 (finite), n_iter >= 1, n_power >= 1");
    return ASHRT_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const long long nm = (long long)model_elems(P), nd = (long long)data_elems(P);
  float* v = P->u;      // power-method vector
  float* w = P->sv;     // adjoint output (model-sized)
  float* y = P->pv;     // FISTA extrapolated point
  float* q = P->qv;     // data-sized: S L y - S d
  double* dot = P->scal;            // [B] ||w||^2
  double* lam = P->scal + B;        // [B] lambda_max estimate
  double* n0 = P->scal + 2 * B;     // [B] ||v0||^2
  const dim3 gm(f_grid(nm, B), B), gd(f_grid(nd, B), B);

#define FK(x)                                                                  \
  do {                                                                         \
    cudaError_t e_ = (x);                                                      \
    if (e_ != cudaSuccess) {                                                   \
      set_error("ashrt_fista: %s (%s)", #x, cudaGetErrorString(e_));           \
      return ASHRT_ECUDA;                                                      \
    }                                                                          \
  } while (0)
#define FLAUNCH(kern, grid, ...)                                               \
  do {                                                                         \
    kern<<<(grid), kFThreads, 0, s>>>(__VA_ARGS__);                            \
    count_launches(1);                                                         \
    FK(cudaGetLastError());                                                    \
  } while (0)

  FK(cudaMemsetAsync(P->scal, 0, sizeof(double) * 3 * B, s));
  // power method on L^T S^T S L from v0 / ||v0||
  FK(cudaMemcpyAsync(v, v0, sizeof(float) * nm * B, cudaMemcpyDeviceToDevice, s));
  FLAUNCH(k_f_sumsq, gm, v, nm, n0);
  FLAUNCH(k_f_normalise, gm, v, v, nm, n0);
  for (int it = 0; it < o.n_power; ++it) {
    FK(op_forward(P, v, q, nullptr, nullptr, tmask, nullptr, B, s));
    FK(cudaMemsetAsync(dot, 0, sizeof(double) * B, s));
    FK(op_adjoint(P, q, w, nullptr, nullptr, tmask, dot, B, s));
    FLAUNCH(k_f_normalise, gm, w, v, nm, dot);
  }
  FLAUNCH(k_f_lambda, dim3((B + kFThreads - 1) / kFThreads), dot, lam, B);

  // FISTA from x_0 = y_1 = 0
  FK(cudaMemsetAsync(m, 0, sizeof(float) * nm * B, s));
  FK(cudaMemsetAsync(y, 0, sizeof(float) * nm * B, s));
  double t = 1.0;
  for (int k = 0; k < o.n_iter; ++k) {
    const double t1 = (1.0 + std::sqrt(1.0 + 4.0 * t * t)) / 2.0;
    const float beta = (float)((t - 1.0) / t1);
    t = t1;
    FK(op_forward(P, y, q, nullptr, nullptr, tmask, nullptr, B, s));
    FLAUNCH(k_f_resid, gd, q, d, tmask, P->nr, P->nt);
    FK(op_adjoint(P, q, w, nullptr, nullptr, tmask, nullptr, B, s));
    FLAUNCH(k_f_step, gm, y, w, m, lam, o.mu, beta, nm);
  }
  if (drec) FK(op_forward(P, m, drec, nullptr, nullptr, nullptr, nullptr, B, s));

  std::vector<double> lam_h(B);
  FK(cudaMemcpyAsync(lam_h.data(), lam, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
  int dev_err = 0;
  FK(cudaMemcpyAsync(&dev_err, P->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  FK(cudaStreamSynchronize(s));
#undef FLAUNCH
#undef FK
  if (dev_err) {
    cudaMemsetAsync(P->dev_err, 0, sizeof(int), s);
    set_error("ashrt_fista: a device-side wait for a tile copy ran out");
    return ASHRT_ETIMEOUT;
  }
  if (lipschitz)
    for (int g = 0; g < B; ++g) lipschitz[g] = 2.0 * lam_h[g];
  return ASHRT_OK;
}
