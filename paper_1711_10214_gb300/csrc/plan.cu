// Plan creation (host tables in FP64), the operator pair ashrt_forward /
// ashrt_adjoint, and the ABI's error plumbing.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "ops.h"

namespace ashrt {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

static int ilog2_ceil(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

// Base twiddles exp(-2 pi i k / (Ns R)), k < Ns, for every pass of a
// length-2^logn Stockham schedule (radix 2^lr passes, then one smaller radix).
int twiddle_table_len(int logn, int lr) {
  int nf = logn / lr, rl = 1 << (logn % lr), np = nf + (rl > 1 ? 1 : 0);
  int len = 0, ns = 1;
  for (int q = 0; q < np; ++q) {
    len += ns;
    ns *= (q < nf ? (1 << lr) : rl);
  }
  return len;
}

void build_twiddle_table(int logn, float2* out, int lr) {
  int nf = logn / lr, rl = 1 << (logn % lr), np = nf + (rl > 1 ? 1 : 0);
  int off = 0, ns = 1;
  for (int q = 0; q < np; ++q) {
    const int R = q < nf ? (1 << lr) : rl;
    for (int k = 0; k < ns; ++k) {
      const double ang = -2.0 * M_PI * (double)k / (double)(ns * R);
      out[off + k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    off += ns;
    ns *= R;
  }
}

// Cone table and Stolt taps for every (velocity, l) row, in FP64: the same
// expressions as the FP64 reference, a = ((v*l)*Nt)*dt/(Nx*dx), mapped iff
// k*k > a*a, u = sqrt(k^2 - a^2).
void build_tap_rows(const float* velocities, int nv, int Nt, int Nx, int Lh, double dt, double dx,
                    unsigned* taps, int* kmin, float2* acone) {
  const int H = Nt / 2, ldt = taps_row_len(Nt);
  for (int i = 0; i < nv; ++i) {
    const double v = (double)velocities[i];
    for (int l = 0; l < Lh; ++l) {
      const double a = ((v * (double)l) * (double)Nt) * dt / ((double)Nx * dx);
      const double a2 = a * a;
      long long km = Nt;   // a >= Nt: nothing of this row is mapped
      if (a < (double)Nt) {
        km = (long long)std::floor(a);
        if (km < 0) km = 0;
        while ((double)(km * km) <= a2) ++km;
        while (km > 0 && (double)((km - 1) * (km - 1)) > a2) --km;
      }
      const size_t row = (size_t)i * Lh + l;
      kmin[row] = (int)std::min<long long>(km, Nt);
      const float hi = (float)a;
      acone[row] = make_float2(hi, (float)(a - (double)hi));
      unsigned* t = taps + row * ldt;
      for (int k = 0; k < ldt; ++k) {
        if (k >= H || (double)k * (double)k <= a2) {
          t[k] = kTapInvalid;
          continue;
        }
        const double u = std::sqrt((double)k * (double)k - a2);
        long long k0 = (long long)std::floor(u);
        long long q = std::llround((u - (double)k0) * 1048576.0);
        if (q >= 1048576) {
          ++k0;
          q = 0;
        }
        t[k] = ((unsigned)k0 << 20) | (unsigned)q;
      }
    }
  }
}

bool build_adj_table(const unsigned* taps, const int* kmin, int nv, int Lh, int Nt, uint2* atab) {
  const int H = Nt / 2, ldt = taps_row_len(Nt), lda = atab_row_len(Nt);
  std::vector<int> ks(H + 2);
  for (size_t row = 0; row < (size_t)nv * Lh; ++row) {
    uint2* r = atab + row * lda;
    for (int J = 0; J < lda; ++J) r[J] = make_uint2(0u, 0u);
    const int km = kmin[row];
    if (km >= H) continue;
    const unsigned* t = taps + row * ldt;
    int k = km;
    for (int J = 0; J <= H + 1; ++J) {
      while (k < H && (int)(t[k] >> 20) < J) ++k;
      ks[J] = k;
    }
    for (int J = 0; J <= H; ++J) {
      const int kB = ks[J], kC = ks[J + 1], kA = J > 0 ? ks[J - 1] : kB;
      if (kC - kB > 1 || kB - kA > 1) return false;
      unsigned x = (unsigned)kB << 20, y = 0u;
      if (kC - kB == 1) {
        x |= t[kB] & 0xfffffu;
        y |= 1u << 20;
      }
      if (kB - kA == 1) y |= (t[kB - 1] & 0xfffffu) | (1u << 21);
      r[J] = make_uint2(x, y);
    }
  }
  return true;
}

static ashrt_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return ASHRT_ECUDA;
}

#define ASHRT_CUDA(call, what)                         \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

static void free_plan_memory(ashrt_plan* p) {
  void* ptrs[] = {p->tw_t, p->tw_t16, p->tw_x, p->wt, p->kmin, p->acone, p->taps, p->atab,
                  p->phase, p->Es, p->Ea, p->X, p->Y, p->u, p->pv, p->sv, p->wminv, p->r, p->qv, p->wr, p->y,
                  p->scal, p->sel, p->flags, p->cg_coef, p->dev_err};
  for (void* q : ptrs)
    if (q) cudaFree(q);
}

template <typename T>
static ashrt_status dev_alloc(T** ptr, size_t count, size_t* total) {
  const size_t bytes = count * sizeof(T);
  cudaError_t e = cudaMalloc((void**)ptr, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    set_error("cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    return ASHRT_ENOMEM;
  }
  if (total) *total += bytes;
  return ASHRT_OK;
}

template <typename T>
static ashrt_status upload(T** ptr, const std::vector<T>& host, size_t* total) {
  ashrt_status st = dev_alloc(ptr, host.size(), total);
  if (st != ASHRT_OK) return st;
  cudaError_t e = cudaMemcpy(*ptr, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy (plan tables)");
  return ASHRT_OK;
}

size_t model_elems(const ashrt_plan* p) { return (size_t)p->P * p->nx * p->nt; }
size_t data_elems(const ashrt_plan* p) { return (size_t)p->nr * p->nt; }

// ---------------------------------------------------------------------------
// Operator application with the fused IRLS weights.
//   forward: d = tmask * ew_data * L(ew_model * m); dot[g] += ||d_g||^2
//   adjoint: m = ew_model * L^T(tmask * ew_data * d); dot[g] += ||m_g||^2
cudaError_t op_forward(const ashrt_plan* p, const float* m, float* d, const float* ew_model,
                       const float* ew_data, const float* tmask, double* dot, int batch,
                       cudaStream_t s, const CgFuse* cg) {
  XfftArgs ax;
  ax.in_real = m;
  ax.out_cplx = p->X;
  ax.nx = p->nx;
  ax.nt = p->nt;
  ax.ld = p->ld;
  ax.Lh = p->Lh;
  ax.Nx = p->Nx;
  ax.slab_real = (long long)p->nx * p->nt;
  ax.slab_cplx = (long long)p->Lh * p->ld;
  ax.ew = ew_model;
  ax.slabs_per_gather = p->P;
  ax.slabs = batch * p->P;
  ax.tw = p->tw_x;
  ax.cols = p->xfft_cols;
  ax.err = p->dev_err;
  if (cg && cg->mode == 1) {
    ax.cg_mode = 1;
    ax.cg_io = const_cast<float*>(m);
    ax.cg_s = cg->s;
    ax.cg_u = cg->u;
    ax.cg_pout = cg->pout;
    ax.cg_p2_read = cg->p2_read;
    ax.cg_u_rw = cg->u_rw;
    ax.cg_coef = cg->coef;
  }
  prof_begin(PROF_XR2C, s);
  cudaError_t e = launch_xfft_r2c(ax, s);
  prof_end(PROF_XR2C, s);
  if (e != cudaSuccess) return e;

  RowArgs ra;
  ra.X = p->X;
  ra.Yw = p->Y;
  ra.nt = p->nt;
  ra.ld = p->ld;
  ra.Lh = p->Lh;
  ra.P = p->P;
  ra.nv = p->nv;
  ra.nt0 = p->nt0;
  ra.Nt = p->Nt;
  ra.x_panel = (long long)p->Lh * p->ld;
  ra.x_batch = ra.x_panel * p->P;
  ra.y_batch = ra.x_panel;
  ra.tw = p->tw_t;
  ra.tw16 = p->tw_t16;
  ra.wt = p->wt;
  ra.kmin = p->kmin;
  ra.acone = p->acone;
  ra.taps = p->taps;
  ra.taps_ld = taps_row_len(p->Nt);
  ra.phase = p->shift ? p->phase : nullptr;
  ra.batch = batch;
  ra.minb = p->rows_minb;
  prof_begin(PROF_ROWS_FWD, s);
  e = launch_stolt_fwd_rows(ra, s);
  prof_end(PROF_ROWS_FWD, s);
  if (e != cudaSuccess) return e;

  prof_begin(PROF_XC2R_DATA, s);
  if (p->irregular) {
    e = launch_irr_synth(p->Es, p->Y, d, p->nr, p->nt, p->Lh, p->ld, ra.y_batch, ew_data, tmask,
                         dot, batch, s);
  } else {
    XfftArgs ay = ax;
    ay.in_cplx = p->Y;
    ay.out_real = d;
    ay.ew = ew_data;
    ay.tmask = tmask;
    ay.slabs_per_gather = 1;
    ay.slabs = batch;
    ay.dot = dot;
    e = launch_xfft_c2r(ay, s);
  }
  prof_end(PROF_XC2R_DATA, s);
  return e;
}

cudaError_t op_adjoint(const ashrt_plan* p, const float* d, float* m, const float* ew_model,
                       const float* ew_data, const float* tmask, double* dot, int batch,
                       cudaStream_t s, const CgFuse* cg) {
  XfftArgs ay;
  ay.in_real = d;
  ay.out_cplx = p->Y;
  ay.nx = p->nx;
  ay.nt = p->nt;
  ay.ld = p->ld;
  ay.Lh = p->Lh;
  ay.Nx = p->Nx;
  ay.slab_real = (long long)p->nx * p->nt;
  ay.slab_cplx = (long long)p->Lh * p->ld;
  ay.ew = ew_data;
  ay.tmask = tmask;
  ay.slabs_per_gather = 1;
  ay.slabs = batch;
  ay.tw = p->tw_x;
  ay.cols = p->xfft_cols;
  ay.err = p->dev_err;
  cudaError_t e = cudaSuccess;
  if (p->irregular) {
    // the CGLS update r -= alpha q runs on its own, then the analysis at the traces
    if (cg && cg->mode == 2) {
      e = launch_irr_cg_r(const_cast<float*>(d), cg->s, (long long)p->nr * p->nt, cg->coef,
                          batch, s);
      count_launches(1);
      if (e != cudaSuccess) return e;
    }
    prof_begin(PROF_XR2C_DATA, s);
    e = launch_irr_analysis(p->Ea, d, p->Y, p->nr, p->nt, p->Lh, p->ld,
                            (long long)p->Lh * p->ld, ew_data, tmask, batch, s);
    prof_end(PROF_XR2C_DATA, s);
  } else {
    if (cg && cg->mode == 2) {
      ay.cg_mode = 2;
      ay.cg_io = const_cast<float*>(d);
      ay.cg_s = cg->s;
      ay.cg_coef = cg->coef;
    }
    prof_begin(PROF_XR2C_DATA, s);
    e = launch_xfft_r2c(ay, s);
    prof_end(PROF_XR2C_DATA, s);
  }
  if (e != cudaSuccess) return e;

  RowArgs ra;
  ra.Y = p->Y;
  ra.Xw = p->X;
  ra.nt = p->nt;
  ra.ld = p->ld;
  ra.Lh = p->Lh;
  ra.P = p->P;
  ra.nv = p->nv;
  ra.nt0 = p->nt0;
  ra.Nt = p->Nt;
  ra.x_panel = (long long)p->Lh * p->ld;
  ra.x_batch = ra.x_panel * p->P;
  ra.y_batch = ra.x_panel;
  ra.tw = p->tw_t;
  ra.tw16 = p->tw_t16;
  ra.wt = p->wt;
  ra.kmin = p->kmin;
  ra.acone = p->acone;
  ra.taps = p->taps;
  ra.taps_ld = taps_row_len(p->Nt);
  ra.atab = p->atab;
  ra.atab_ld = atab_row_len(p->Nt);
  ra.phase = p->shift ? p->phase : nullptr;
  ra.batch = batch;
  ra.minb = p->rows_minb;
  prof_begin(PROF_ROWS_ADJ, s);
  e = launch_stolt_adj_rows(ra, s);
  prof_end(PROF_ROWS_ADJ, s);
  if (e != cudaSuccess) return e;

  XfftArgs ax = ay;
  ax.in_cplx = p->X;
  ax.out_real = m;
  ax.ew = ew_model;
  ax.tmask = nullptr;
  ax.slabs_per_gather = p->P;
  ax.slabs = batch * p->P;
  ax.dot = dot;
  ax.ew_sq = cg ? cg->model_ew_sq : 0;
  prof_begin(PROF_XC2R, s);
  e = launch_xfft_c2r(ax, s);
  prof_end(PROF_XC2R, s);
  return e;
}

}  // namespace ashrt

using namespace ashrt;

extern "C" {

void ashrt_default_opts(ashrt_opts* o) {
  if (!o) return;
  o->pad_t = 2;
  o->pad_x = 2;
  o->fmax_hz = 0.f;
  o->wavelet_peak_hz = 0.f;
  o->max_batch = 1;
  o->with_solver = 0;
}

const char* ashrt_last_error(void) { return g_err.c_str(); }

const char* ashrt_status_string(ashrt_status s) {
  switch (s) {
    case ASHRT_OK: return "ASHRT_OK";
    case ASHRT_EINVAL: return "ASHRT_EINVAL";
    case ASHRT_ENOMEM: return "ASHRT_ENOMEM";
    case ASHRT_ECUDA: return "ASHRT_ECUDA";
    case ASHRT_ENAN: return "ASHRT_ENAN";
    case ASHRT_ENOTCONV: return "ASHRT_ENOTCONV";
    case ASHRT_ETIMEOUT: return "ASHRT_ETIMEOUT";
    case ASHRT_EINTERNAL: return "ASHRT_EINTERNAL";
  }
  return "ASHRT_UNKNOWN";
}

}  // extern "C"

// Plan creation; xr (host, nr positions in metres) or NULL for traces at the
// apex positions j dx.
static ashrt_status plan_create_impl(ashrt_plan** out, int nt, int nx, double dt, double dx,
                                     const float* velocities, int nv, const float* apex_x,
                                     int napex, const float* t0_shifts, int nt0,
                                     const ashrt_opts* opts, const double* xr, int nr) {
  g_err.clear();
  if (!out) {
    set_error("plan_create: out is NULL");
    return ASHRT_EINVAL;
  }
  *out = nullptr;
  ashrt_opts o;
  ashrt_default_opts(&o);
  if (opts) o = *opts;
  if (o.pad_t <= 0) o.pad_t = 2;
  if (o.pad_x <= 0) o.pad_x = 2;
  if (o.max_batch <= 0) o.max_batch = 1;
  if (nt < 2 || nx < 2 || !(dt > 0) || !(dx > 0) || nv <= 0 || !velocities) {
    set_error("plan_create: need nt >= 2, nx >= 2, dt > 0, dx > 0, nv > 0 and velocities");
    return ASHRT_EINVAL;
  }
  for (int i = 0; i < nv; ++i)
    if (!(velocities[i] >= 0.f) || !std::isfinite(velocities[i])) {
      set_error("plan_create: velocity %d is negative or not finite", i);
      return ASHRT_EINVAL;
    }
  if (apex_x) {
    if (napex != nx) {
      set_error("plan_create: the Stolt operator needs one apex per trace (napex == nx)");
      return ASHRT_EINVAL;
    }
    for (int j = 0; j < nx; ++j)
      if (std::fabs((double)apex_x[j] - j * dx) > 1e-3 * dx) {
        set_error("plan_create: apex %d is not at trace position %g (x_a must equal x)", j, j * dx);
        return ASHRT_EINVAL;
      }
  }
  if (t0_shifts == nullptr) {
    if (nt0 != 1 && nt0 != 0) {
      set_error("plan_create: t0_shifts NULL requires nt0 = 1");
      return ASHRT_EINVAL;
    }
    nt0 = 1;
  } else if (nt0 <= 0) {
    set_error("plan_create: nt0 must be positive");
    return ASHRT_EINVAL;
  } else {
    for (int j = 0; j < nt0; ++j)
      if (!std::isfinite(t0_shifts[j])) {
        set_error("plan_create: t0 shift %d is not finite", j);
        return ASHRT_EINVAL;
      }
  }
  if (!(o.fmax_hz >= 0.f) || !(o.wavelet_peak_hz >= 0.f)) {
    set_error("plan_create: fmax_hz and wavelet_peak_hz must be >= 0");
    return ASHRT_EINVAL;
  }
  if (xr) {
    if (nr < 1 || o.max_batch > 65535) {
      set_error("plan_create_irregular: need nr >= 1 trace positions and max_batch <= 65535");
      return ASHRT_EINVAL;
    }
    for (int j = 0; j < nr; ++j)
      if (!std::isfinite(xr[j])) {
        set_error("plan_create_irregular: trace position %d is not finite", j);
        return ASHRT_EINVAL;
      }
  }

  ashrt_plan* p = new ashrt_plan();
  cudaGetDevice(&p->device);
  p->nt = nt;
  p->nx = nx;
  p->nv = nv;
  p->nt0 = nt0;
  p->P = nv * nt0;
  p->dt = dt;
  p->dx = dx;
  p->logNt = ilog2_ceil(o.pad_t * nt);
  p->logNx = ilog2_ceil(o.pad_x * nx);
  if (p->logNt < 6) p->logNt = 6;
  if (p->logNx < 4) p->logNx = 4;
  p->Nt = 1 << p->logNt;
  p->Nx = 1 << p->logNx;
  if (p->Nt > 4096 || p->Nx > 2048) {
    set_error("plan_create: padded sizes Nt=%d, Nx=%d exceed 4096 / 2048", p->Nt, p->Nx);
    delete p;
    return ASHRT_EINVAL;
  }
  p->Lh = p->Nx / 2 + 1;
  p->ld = (nt + 3) & ~3;
  p->irregular = xr != nullptr;
  p->nr = xr ? nr : nx;
  p->max_batch = o.max_batch;
  p->with_solver = o.with_solver;
  p->opts = o;

  const int Nt = p->Nt, Nx = p->Nx, Lh = p->Lh;
  // spectral weight W(w) / (Nt Nx): wavelet amplitude spectrum, band limit, no Nyquist
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
  // cone table and Stolt taps (FP64, host)
  std::vector<int> kmin((size_t)nv * Lh);
  std::vector<float2> acone((size_t)nv * Lh);
  std::vector<unsigned> taps((size_t)nv * Lh * taps_row_len(Nt));
  build_tap_rows(velocities, nv, Nt, Nx, Lh, dt, dx, taps.data(), kmin.data(), acone.data());
  std::vector<uint2> atab((size_t)nv * Lh * atab_row_len(Nt));
  if (!build_adj_table(taps.data(), kmin.data(), nv, Lh, Nt, atab.data())) {
    set_error("ashrt_plan_create: a bin of the transposed Stolt map has two sources of one kind");
    delete p;
    return ASHRT_EINTERNAL;
  }
  // asymptote shift T: exp(-i w tau0), w = 2 pi kk / (Nt dt)
  std::vector<float2> phase((size_t)nt0 * Nt);
  bool shift = false;
  for (int j = 0; j < nt0; ++j) {
    const double t0 = t0_shifts ? (double)t0_shifts[j] : 0.0;
    if (t0 != 0.0) shift = true;
    for (int k = 0; k < Nt; ++k) {
      const int kk = k <= Nt / 2 ? k : k - Nt;
      const double ang = -2.0 * M_PI * (double)kk * t0 / ((double)Nt * dt);
      phase[(size_t)j * Nt + k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
  }
  p->shift = shift;
  std::vector<float2> twt(twiddle_table_len(p->logNt)), twx(twiddle_table_len(p->logNx));
  build_twiddle_table(p->logNt, twt.data());
  build_twiddle_table(p->logNx, twx.data());

  size_t total = 0;
  ashrt_status st = ASHRT_OK;
  auto chk = [&](ashrt_status s2) {
    if (st == ASHRT_OK) st = s2;
  };
  chk(upload(&p->tw_t, twt, &total));
  chk(upload(&p->tw_x, twx, &total));
  if (rows16_supported(p->logNt)) {
    std::vector<float2> tw16(twiddle_table_len(p->logNt, 4));
    build_twiddle_table(p->logNt, tw16.data(), 4);
    chk(upload(&p->tw_t16, tw16, &total));
    // the fastest pair measured: at Nt = 2048 radix-16 both ways with the
    // forward's accumulator in tensor memory, elsewhere radix-16 forward and
    // radix-8 adjoint
    p->rows_minb = p->logNt == 11 ? 9 : 4;
  }
  chk(upload(&p->wt, wt, &total));
  chk(upload(&p->kmin, kmin, &total));
  chk(upload(&p->acone, acone, &total));
  chk(upload(&p->taps, taps, &total));
  chk(upload(&p->atab, atab, &total));
  chk(upload(&p->phase, phase, &total));
  if (p->irregular) {
    std::vector<float2> es((size_t)p->nr * Lh), ea((size_t)Lh * p->nr);
    build_irregular_tables(xr, p->nr, Nx, dx, es.data(), ea.data());
    chk(upload(&p->Es, es, &total));
    chk(upload(&p->Ea, ea, &total));
  }
  const size_t B = (size_t)p->max_batch;
  const size_t xpan = (size_t)Lh * p->ld;
  if (st == ASHRT_OK) chk(dev_alloc(&p->X, B * p->P * xpan, &total));
  if (st == ASHRT_OK) chk(dev_alloc(&p->Y, B * xpan, &total));
  if (st == ASHRT_OK) chk(dev_alloc(&p->dev_err, 1, &total));
  if (st == ASHRT_OK && cudaMemset(p->dev_err, 0, sizeof(int)) != cudaSuccess) st = ASHRT_ECUDA;
  if (st == ASHRT_OK && p->with_solver) {
    const size_t me = B * model_elems(p), de = B * data_elems(p);
    chk(dev_alloc(&p->u, me, &total));
    chk(dev_alloc(&p->pv, me, &total));
    chk(dev_alloc(&p->sv, me, &total));
    chk(dev_alloc(&p->wminv, me, &total));
    chk(dev_alloc(&p->r, de, &total));
    chk(dev_alloc(&p->qv, de, &total));
    chk(dev_alloc(&p->wr, de, &total));
    chk(dev_alloc(&p->y, de, &total));
    chk(dev_alloc(&p->scal, B * kScalStride, &total));
    chk(dev_alloc(&p->sel, B * kSelStride, &total));
    chk(dev_alloc(&p->flags, 2 * B + 1, &total));
    chk(dev_alloc(&p->cg_coef, 2 * B, &total));
  }
  if (st == ASHRT_OK) {
    // the padding columns of the spectra rows are never written: keep them zero
    cudaError_t e = cudaMemset(p->X, 0, B * p->P * xpan * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemset(p->Y, 0, B * xpan * sizeof(float2));
    // the CG's two direction buffers enter the first update times beta = 0:
    // they must hold finite values from the start
    if (e == cudaSuccess && p->with_solver) {
      const size_t me = B * model_elems(p);
      e = cudaMemset(p->pv, 0, me * sizeof(float));
      if (e == cudaSuccess) e = cudaMemset(p->u, 0, me * sizeof(float));
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = cuda_fail(e, "plan_create workspace init");
  }
  if (st != ASHRT_OK) {
    free_plan_memory(p);
    delete p;
    return st;
  }
  p->ws_bytes = total;
  *out = p;
  return ASHRT_OK;
}

extern "C" {

ashrt_status ashrt_plan_create(ashrt_plan** out, int nt, int nx, double dt, double dx,
                               const float* velocities, int nv, const float* apex_x, int napex,
                               const float* t0_shifts, int nt0, const ashrt_opts* opts) {
  return plan_create_impl(out, nt, nx, dt, dx, velocities, nv, apex_x, napex, t0_shifts, nt0,
                          opts, nullptr, 0);
}

ashrt_status ashrt_plan_create_irregular(ashrt_plan** out, int nt, int nx, double dt, double dx,
                                         const float* velocities, int nv,
                                         const float* t0_shifts, int nt0,
                                         const double* trace_x, int nr,
                                         const ashrt_opts* opts) {
  if (!trace_x) {
    g_err.clear();
    set_error("plan_create_irregular: trace_x is NULL");
    if (out) *out = nullptr;
    return ASHRT_EINVAL;
  }
  return plan_create_impl(out, nt, nx, dt, dx, velocities, nv, nullptr, 0, t0_shifts, nt0, opts,
                          trace_x, nr);
}

void ashrt_plan_destroy(ashrt_plan* p) {
  if (!p) return;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  free_plan_memory(p);
  cudaSetDevice(dev);
  delete p;
}

ashrt_status ashrt_plan_info(const ashrt_plan* p, int* Nt, int* Nx, int* n_panels, size_t* ws) {
  if (!p) {
    set_error("plan_info: plan is NULL");
    return ASHRT_EINVAL;
  }
  if (Nt) *Nt = p->Nt;
  if (Nx) *Nx = p->Nx;
  if (n_panels) *n_panels = p->P;
  if (ws) *ws = p->ws_bytes;
  return ASHRT_OK;
}

static ashrt_status check_call(const ashrt_plan* p, const void* a, const void* b, int batch,
                               const char* who) {
  g_err.clear();
  if (!p || !a || !b) {
    set_error("%s: NULL plan or array", who);
    return ASHRT_EINVAL;
  }
  if (batch < 1 || batch > p->max_batch) {
    set_error("%s: batch %d outside [1, max_batch = %d]", who, batch, p->max_batch);
    return ASHRT_EINVAL;
  }
  return ASHRT_OK;
}

ashrt_status ashrt_forward(const ashrt_plan* p, const float* m, float* d, const float* tmask,
                           int batch, void* stream) {
  ashrt_status st = check_call(p, m, d, batch, "ashrt_forward");
  if (st != ASHRT_OK) return st;
  cudaError_t e = op_forward(p, m, d, nullptr, nullptr, tmask, nullptr, batch,
                             (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "ashrt_forward launch");
  return ASHRT_OK;
}

ashrt_status ashrt_adjoint(const ashrt_plan* p, const float* d, float* m, const float* tmask,
                           int batch, void* stream) {
  ashrt_status st = check_call(p, d, m, batch, "ashrt_adjoint");
  if (st != ASHRT_OK) return st;
  cudaError_t e = op_adjoint(p, d, m, nullptr, nullptr, tmask, nullptr, batch,
                             (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "ashrt_adjoint launch");
  return ASHRT_OK;
}

}  // extern "C"
