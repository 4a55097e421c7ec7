// ashrt_forward_static: the forward Stolt ASHRT/AASHRT operator for callers
// that cannot allocate device memory.
//
// Who needs it: host applications that hand this library pre-allocated
// input/output buffers but own the rest of device memory (a framework whose
// caching allocator has reserved the GPU, a plug-in host with a fixed device
// budget), and latency-critical acquisition loops where a cudaMalloc would
// synchronise the device and stall the stream.  ashrt_plan_create allocates
// its tables and workspace with cudaMalloc, so those callers cannot use a plan.
//
// This entry point needs no plan: every table (twiddles, spectral weight,
// cone table, asymptote phases) and the operator workspace (the x-transformed
// model rows and the data spectrum) live in one file-scope __device__ array of
// kStaticScratchBytes, which every GPU that loads the library keeps for the
// life of the process.  The caller passes inputs and outputs only.  The kernels
// are ones ashrt_forward launches too (the row kernel in its radix-8 form).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "internal.h"

namespace ashrt {
namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;   // 16 MiB per device

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of the scratch array on the current device.  Looked up on
// every call (cudaGetSymbolAddress with the calling device current; cheap),
// so nothing is cached across devices or across a cudaDeviceReset.
ashrt_status static_scratch(unsigned char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || !p) {
    set_error("ashrt_forward_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    return ASHRT_ECUDA;
  }
  *out = (unsigned char*)p;
  return ASHRT_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int log2_ceil(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

}  // namespace
}  // namespace ashrt

using namespace ashrt;

extern "C" ashrt_status ashrt_forward_static(int nt, int nx, double dt, double dx,
                                             const float* velocities, int nv,
                                             const float* t0_shifts, int nt0,
                                             const ashrt_opts* opts, const float* m_dev,
                                             float* d_dev, const float* trace_mask_dev,
                                             int batch, void* stream) {
  ashrt_opts o;
  ashrt_default_opts(&o);
  if (opts) o = *opts;
  if (o.pad_t <= 0) o.pad_t = 2;
  if (o.pad_x <= 0) o.pad_x = 2;
  if (!m_dev || !d_dev || !velocities || nv <= 0 || nt < 2 || nx < 2 || !(dt > 0) ||
      !(dx > 0) || batch < 1) {
    set_error("ashrt_forward_static: need m_dev, d_dev, velocities, nv > 0, nt >= 2, nx >= 2, "
              "dt > 0, dx > 0, batch >= 1");
    return ASHRT_EINVAL;
  }
  if (!t0_shifts) {
    if (nt0 != 1 && nt0 != 0) {
      set_error("ashrt_forward_static: t0_shifts NULL requires nt0 = 1");
      return ASHRT_EINVAL;
    }
    nt0 = 1;
  } else if (nt0 <= 0) {
    set_error("ashrt_forward_static: nt0 must be positive");
    return ASHRT_EINVAL;
  }
  if (!(o.fmax_hz >= 0.f) || !(o.wavelet_peak_hz >= 0.f)) {
    set_error("ashrt_forward_static: fmax_hz and wavelet_peak_hz must be >= 0");
    return ASHRT_EINVAL;
  }
  for (int i = 0; i < nv; ++i)
    if (!(velocities[i] >= 0.f) || !std::isfinite(velocities[i])) {
      set_error("ashrt_forward_static: velocity %d is negative or not finite", i);
      return ASHRT_EINVAL;
    }
  int logNt = log2_ceil(o.pad_t * nt), logNx = log2_ceil(o.pad_x * nx);
  if (logNt < 6) logNt = 6;
  if (logNx < 4) logNx = 4;
  const int Nt = 1 << logNt, Nx = 1 << logNx, Lh = Nx / 2 + 1, ld = (nt + 3) & ~3;
  const int P = nv * nt0;
  if (Nt > 4096 || Nx > 2048) {
    set_error("ashrt_forward_static: padded sizes Nt=%d, Nx=%d exceed 4096 / 2048", Nt, Nx);
    return ASHRT_EINVAL;
  }

  // scratch layout, every piece 256-byte aligned
  const size_t tw_t_len = twiddle_table_len(logNt), tw_x_len = twiddle_table_len(logNx);
  size_t off = 0;
  const size_t o_twt = off;   off = align256(off + tw_t_len * sizeof(float2));
  const size_t o_twx = off;   off = align256(off + tw_x_len * sizeof(float2));
  const size_t o_wt = off;    off = align256(off + (size_t)Nt * sizeof(float));
  const size_t o_kmin = off;  off = align256(off + (size_t)nv * Lh * sizeof(int));
  const size_t o_acone = off; off = align256(off + (size_t)nv * Lh * sizeof(float2));
  const size_t o_taps = off;  off = align256(off + (size_t)nv * Lh * taps_row_len(Nt) * sizeof(unsigned));
  const size_t o_phase = off; off = align256(off + (size_t)nt0 * Nt * sizeof(float2));
  const size_t o_X = off;     off = align256(off + (size_t)batch * P * Lh * ld * sizeof(float2));
  const size_t o_Y = off;     off = align256(off + (size_t)batch * Lh * ld * sizeof(float2));
  if (off > kStaticScratchBytes) {
    set_error("ashrt_forward_static: this call needs %zu bytes of scratch but the static "
              "scratch holds %zu bytes (16 MiB); use a plan (ashrt_plan_create) or a smaller "
              "batch / panel count",
              off, kStaticScratchBytes);
    return ASHRT_EINVAL;
  }
  // The host tables below are uploaded from memory that is freed when this
  // call returns, which a captured graph would read at replay: refuse capture.
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t ce = cudaStreamIsCapturing(s, &cap);
  if (ce != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    set_error("ashrt_forward_static: not usable while a stream capture is active (%s)",
              ce != cudaSuccess ? cudaGetErrorString(ce) : "the stream is capturing");
    return ASHRT_EINVAL;
  }
  unsigned char* base = nullptr;
  ashrt_status st = static_scratch(&base);
  if (st != ASHRT_OK) return st;

  // host tables (the same builders ashrt_plan_create uses)
  std::vector<float2> twt(tw_t_len), twx(tw_x_len);
  build_twiddle_table(logNt, twt.data());
  build_twiddle_table(logNx, twx.data());
  std::vector<float> wt(Nt);
  for (int k = 0; k < Nt; ++k) {
    const int kk = k <= Nt / 2 ? k : k - Nt;
    const double f = std::fabs((double)kk) / (Nt * dt);
    double w = 1.0;
    if (o.wavelet_peak_hz > 0.f) {
      const double z = (f / o.wavelet_peak_hz) * (f / o.wavelet_peak_hz);
      w = z * std::exp(1.0 - z);
    }
    if (o.fmax_hz > 0.f && f > o.fmax_hz) w = 0.0;
    if (k == Nt / 2) w = 0.0;
    wt[k] = (float)(w / ((double)Nt * (double)Nx));
  }
  std::vector<int> kmin((size_t)nv * Lh);
  std::vector<float2> acone((size_t)nv * Lh);
  std::vector<unsigned> taps((size_t)nv * Lh * taps_row_len(Nt));
  build_tap_rows(velocities, nv, Nt, Nx, Lh, dt, dx, taps.data(), kmin.data(), acone.data());
  std::vector<float2> phase((size_t)nt0 * Nt);
  bool shift = false;
  for (int j = 0; j < nt0; ++j) {
    const double t0 = t0_shifts ? (double)t0_shifts[j] : 0.0;
    if (!std::isfinite(t0)) {
      set_error("ashrt_forward_static: t0 shift %d is not finite", j);
      return ASHRT_EINVAL;
    }
    if (t0 != 0.0) shift = true;
    for (int k = 0; k < Nt; ++k) {
      const int kk = k <= Nt / 2 ? k : k - Nt;
      const double ang = -2.0 * M_PI * (double)kk * t0 / ((double)Nt * dt);
      phase[(size_t)j * Nt + k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
  }

  auto put = [&](size_t o2, const void* src, size_t bytes) {
    return cudaMemcpyAsync(base + o2, src, bytes, cudaMemcpyHostToDevice, s);
  };
  cudaError_t e = put(o_twt, twt.data(), twt.size() * sizeof(float2));
  if (e == cudaSuccess) e = put(o_twx, twx.data(), twx.size() * sizeof(float2));
  if (e == cudaSuccess) e = put(o_wt, wt.data(), wt.size() * sizeof(float));
  if (e == cudaSuccess) e = put(o_kmin, kmin.data(), kmin.size() * sizeof(int));
  if (e == cudaSuccess) e = put(o_acone, acone.data(), acone.size() * sizeof(float2));
  if (e == cudaSuccess) e = put(o_taps, taps.data(), taps.size() * sizeof(unsigned));
  if (e == cudaSuccess && shift) e = put(o_phase, phase.data(), phase.size() * sizeof(float2));
  if (e != cudaSuccess) {
    set_error("ashrt_forward_static: table upload failed: %s", cudaGetErrorString(e));
    return ASHRT_ECUDA;
  }

  // every workspace element the kernels read is written earlier in this
  // call (rows read t < nt of X and Y only), so nothing needs clearing
  float2* X = (float2*)(base + o_X);
  float2* Y = (float2*)(base + o_Y);
  XfftArgs ax;
  ax.in_real = m_dev;
  ax.out_cplx = X;
  ax.nx = nx;
  ax.nt = nt;
  ax.ld = ld;
  ax.Lh = Lh;
  ax.Nx = Nx;
  ax.slab_real = (long long)nx * nt;
  ax.slab_cplx = (long long)Lh * ld;
  ax.slabs_per_gather = P;
  ax.slabs = batch * P;
  ax.tw = (const float2*)(base + o_twx);
  e = launch_xfft_r2c(ax, s);
  if (e == cudaSuccess) {
    RowArgs ra;
    ra.X = X;
    ra.Yw = Y;
    ra.nt = nt;
    ra.ld = ld;
    ra.Lh = Lh;
    ra.P = P;
    ra.nv = nv;
    ra.nt0 = nt0;
    ra.Nt = Nt;
    ra.x_panel = (long long)Lh * ld;
    ra.x_batch = ra.x_panel * P;
    ra.y_batch = ra.x_panel;
    ra.tw = (const float2*)(base + o_twt);
    ra.wt = (const float*)(base + o_wt);
    ra.kmin = (const int*)(base + o_kmin);
    ra.acone = (const float2*)(base + o_acone);
    ra.taps = (const unsigned*)(base + o_taps);
    ra.taps_ld = taps_row_len(Nt);
    ra.phase = shift ? (const float2*)(base + o_phase) : nullptr;
    ra.batch = batch;
    e = launch_stolt_fwd_rows(ra, s);
  }
  if (e == cudaSuccess) {
    XfftArgs ay = ax;
    ay.in_cplx = Y;
    ay.out_real = d_dev;
    ay.tmask = trace_mask_dev;
    ay.slabs_per_gather = 1;
    ay.slabs = batch;
    e = launch_xfft_c2r(ay, s);
  }
  if (e != cudaSuccess) {
    set_error("ashrt_forward_static: launch failed: %s", cudaGetErrorString(e));
    return ASHRT_ECUDA;
  }
  count_launches(3);
  return ASHRT_OK;
}
