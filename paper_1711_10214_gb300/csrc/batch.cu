// Batches of receiver gathers with uneven trace and sample counts.
//
// The Stolt operator of a gather with nx traces is the operator of a wider
// gather with the same padded width Nx (= next power of two >= pad_x nx)
// restricted to its first nx traces and apexes: the trace-axis transform pads
// with zeros to Nx either way, so for a model that is zero on the extra apexes
// the first nx output traces agree, and the adjoint of a data gather that is
// zero on the extra traces, cropped to nx apexes, agrees.  Inside the IRLS
// solve the extra traces are dead samples (trace mask 0: excluded from the
// residual, the median/MAD and the misfit) and the extra apexes are removed
// from the unknowns (apex mask 0: W_m^-1 = 0).  So gathers are grouped by Nx
// class, packed into a resident class batch of width nxc (the widest gather of
// the class) with zero padding, and solved together by one plan per class;
// the classes run concurrently on their own streams.  Gathers of different
// sample counts nt fall into different classes (a plan's time grid is its
// own).  Gather streams larger than the resident batch are processed chunk
// by chunk.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

#include "internal.h"

namespace {

// Copy `count` gathers [nx_g][nt] (packed at element offset off[g]) into
// slots [nxc][nt] of a class buffer, zero-padding traces nx_g..nxc-1.  Also
// writes the per-slot trace mask (1 for j < nx_g).  rows = traces per panel;
// panels > 1 handles the model layout [P][nx][nt].
__global__ void k_pack(const float* __restrict__ src, float* __restrict__ dst,
                       const long long* __restrict__ off, const int* __restrict__ nxg, int nxc,
                       int nt, int panels, float* __restrict__ mask) {
  const int slot = blockIdx.y;
  const int nx = nxg[slot];
  const long long per = (long long)panels * nxc * nt;
  const float* s = src ? src + off[slot] : nullptr;
  float* d = dst + (long long)slot * per;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i % nt);
    const long long r = i / nt;
    const int j = (int)(r % nxc);
    const int p = (int)(r / nxc);
    d[i] = (s && j < nx) ? s[((long long)p * nx + j) * nt + t] : 0.f;
  }
  if (mask && blockIdx.x == 0)
    for (int j = threadIdx.x; j < nxc; j += blockDim.x) mask[(long long)slot * nxc + j] = j < nx ? 1.f : 0.f;
}

// Inverse of k_pack: slots [panels][nxc][nt] -> packed [panels][nx_g][nt].
__global__ void k_unpack(const float* __restrict__ src, float* __restrict__ dst,
                         const long long* __restrict__ off, const int* __restrict__ nxg, int nxc,
                         int nt, int panels) {
  const int slot = blockIdx.y;
  const int nx = nxg[slot];
  const long long per = (long long)panels * nx * nt;
  const float* s = src + (long long)slot * panels * nxc * nt;
  float* d = dst + off[slot];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i % nt);
    const long long r = i / nt;
    const int j = (int)(r % nx);
    const int p = (int)(r / nx);
    d[i] = s[((long long)p * nxc + j) * nt + t];
  }
}

int next_pow2(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

}  // namespace

struct ashrt_batch {
  int ngather = 0, P = 0;
  std::vector<int> nx, nt;
  std::vector<long long> doff, moff;   // packed element offsets of each gather
  long long data_elems = 0, model_elems = 0;
  size_t ws_bytes = 0;
  struct Class {
    int nt = 0, Nx = 0, nxc = 0, mb = 0;
    std::vector<int> gathers;
    ashrt_plan* plan = nullptr;
    float *d = nullptr, *m = nullptr, *drec = nullptr, *tmask = nullptr;
    long long* doff_dev = nullptr;   // [n in class]: data offsets, chunk order
    long long* moff_dev = nullptr;
    int* nx_dev = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
  };
  std::vector<Class> cls;
  cudaEvent_t start = nullptr;
};

using namespace ashrt;

static void free_batch(ashrt_batch* b) {
  for (auto& c : b->cls) {
    if (c.plan) ashrt_plan_destroy(c.plan);
    void* ptrs[] = {c.d, c.m, c.drec, c.tmask, c.doff_dev, c.moff_dev, c.nx_dev};
    for (void* q : ptrs)
      if (q) cudaFree(q);
    if (c.st) cudaStreamDestroy(c.st);
    if (c.done) cudaEventDestroy(c.done);
  }
  if (b->start) cudaEventDestroy(b->start);
  delete b;
}

extern "C" {

ashrt_status ashrt_batch_create(ashrt_batch** out, int nt, const int* nx_per_gather, int ngather,
                                double dt, double dx, const float* velocities, int nv,
                                const float* t0_shifts, int nt0, const ashrt_opts* opts) {
  if (!out || !nx_per_gather || ngather < 1) {
    set_error("ashrt_batch_create: need out, nx_per_gather and ngather >= 1");
    return ASHRT_EINVAL;
  }
  std::vector<int> nts(ngather, nt);
  return ashrt_batch_create_uneven(out, nts.data(), nx_per_gather, ngather, dt, dx, velocities, nv,
                                   t0_shifts, nt0, opts);
}

ashrt_status ashrt_batch_create_uneven(ashrt_batch** out, const int* nt_per_gather,
                                       const int* nx_per_gather, int ngather, double dt, double dx,
                                       const float* velocities, int nv, const float* t0_shifts,
                                       int nt0, const ashrt_opts* opts) {
  if (!out || !nt_per_gather || !nx_per_gather || ngather < 1) {
    set_error("ashrt_batch_create: need out, nt_per_gather, nx_per_gather and ngather >= 1");
    return ASHRT_EINVAL;
  }
  *out = nullptr;
  ashrt_opts o;
  ashrt_default_opts(&o);
  if (opts) o = *opts;
  if (o.pad_x <= 0) o.pad_x = 2;
  if (o.max_batch <= 0) o.max_batch = 64;
  for (int g = 0; g < ngather; ++g)
    if (nx_per_gather[g] < 2 || nt_per_gather[g] < 2) {
      set_error("ashrt_batch_create: gather %d has %d traces of %d samples (need >= 2 each)", g,
                nx_per_gather[g], nt_per_gather[g]);
      return ASHRT_EINVAL;
    }
  ashrt_batch* b = new ashrt_batch();
  b->ngather = ngather;
  b->P = nv * (t0_shifts ? nt0 : 1);
  b->nx.assign(nx_per_gather, nx_per_gather + ngather);
  b->nt.assign(nt_per_gather, nt_per_gather + ngather);
  b->doff.resize(ngather);
  b->moff.resize(ngather);
  for (int g = 0; g < ngather; ++g) {
    b->doff[g] = b->data_elems;
    b->moff[g] = b->model_elems;
    b->data_elems += (long long)b->nx[g] * b->nt[g];
    b->model_elems += (long long)b->P * b->nx[g] * b->nt[g];
  }
  // classes: one per (nt, padded width Nx)
  std::map<std::pair<int, int>, std::vector<int>> by;
  for (int g = 0; g < ngather; ++g)
    by[std::make_pair(b->nt[g], next_pow2(o.pad_x * b->nx[g]))].push_back(g);
  ashrt_status st = ASHRT_OK;
  for (auto& kv : by) {
    ashrt_batch::Class c;
    c.nt = kv.first.first;
    c.Nx = kv.first.second;
    c.gathers = kv.second;
    for (int g : c.gathers) c.nxc = std::max(c.nxc, b->nx[g]);
    c.mb = std::min<int>((int)c.gathers.size(), o.max_batch);
    b->cls.push_back(c);
  }
  for (auto& c : b->cls) {
    ashrt_opts oc = o;
    oc.max_batch = c.mb;
    // pad_x chosen so that the class plan has exactly this class's Nx
    st = ashrt_plan_create(&c.plan, c.nt, c.nxc, dt, dx, velocities, nv, nullptr, 0, t0_shifts,
                           nt0, &oc);
    if (st != ASHRT_OK) break;
    int Nx = 0;
    ashrt_plan_info(c.plan, nullptr, &Nx, nullptr, &b->ws_bytes);
    if (Nx != c.Nx) {
      set_error("ashrt_batch_create: class Nx %d but plan Nx %d", c.Nx, Nx);
      st = ASHRT_EINTERNAL;
      break;
    }
    const size_t de = (size_t)c.mb * c.nxc * c.nt, me = de * b->P;
    const size_t n = c.gathers.size();
    cudaError_t e = cudaMalloc(&c.d, de * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c.drec, de * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c.m, me * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c.tmask, (size_t)c.mb * c.nxc * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c.doff_dev, n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&c.moff_dev, n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&c.nx_dev, n * 4);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("ashrt_batch_create: cudaMalloc failed: %s", cudaGetErrorString(e));
      st = ASHRT_ENOMEM;
      break;
    }
    b->ws_bytes += (2 * de + me + (size_t)c.mb * c.nxc) * 4 + n * 20;
    std::vector<long long> dof(n), mof(n);
    std::vector<int> nxs(n);
    for (size_t i = 0; i < n; ++i) {
      dof[i] = b->doff[c.gathers[i]];
      mof[i] = b->moff[c.gathers[i]];
      nxs[i] = b->nx[c.gathers[i]];
    }
    e = cudaMemcpy(c.doff_dev, dof.data(), n * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c.moff_dev, mof.data(), n * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c.nx_dev, nxs.data(), n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      set_error("ashrt_batch_create: %s", cudaGetErrorString(e));
      st = ASHRT_ECUDA;
      break;
    }
  }
  if (st == ASHRT_OK && cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming) != cudaSuccess) {
    set_error("ashrt_batch_create: cudaEventCreate failed");
    st = ASHRT_ECUDA;
  }
  if (st != ASHRT_OK) {
    free_batch(b);
    return st;
  }
  *out = b;
  return ASHRT_OK;
}

void ashrt_batch_destroy(ashrt_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  free_batch(b);
}

ashrt_status ashrt_batch_autotune(ashrt_batch* b, const char* cache_path) {
  if (!b) {
    set_error("ashrt_batch_autotune: NULL batch");
    return ASHRT_EINVAL;
  }
  for (auto& c : b->cls) {
    ashrt_status st = ashrt_plan_autotune(c.plan, c.mb, cache_path, nullptr, nullptr);
    if (st != ASHRT_OK) return st;
  }
  return ASHRT_OK;
}

ashrt_status ashrt_batch_info(const ashrt_batch* b, int* n_classes, long long* data_elems,
                              long long* model_elems, size_t* workspace_bytes) {
  if (!b) {
    set_error("ashrt_batch_info: NULL batch");
    return ASHRT_EINVAL;
  }
  if (n_classes) *n_classes = (int)b->cls.size();
  if (data_elems) *data_elems = b->data_elems;
  if (model_elems) *model_elems = b->model_elems;
  if (workspace_bytes) *workspace_bytes = b->ws_bytes;
  return ASHRT_OK;
}

}  // extern "C"

// Runs `work(class, first, count, stream)` for every resident chunk of every
// class; classes run concurrently on their own streams, joined to `stream`.
template <typename F>
static ashrt_status for_each_chunk(ashrt_batch* b, cudaStream_t stream, F work) {
  if (cudaEventRecord(b->start, stream) != cudaSuccess) {
    set_error("batch: cudaEventRecord failed");
    return ASHRT_ECUDA;
  }
  for (auto& c : b->cls) {
    if (cudaStreamWaitEvent(c.st, b->start, 0) != cudaSuccess) {
      set_error("batch: cudaStreamWaitEvent failed");
      return ASHRT_ECUDA;
    }
    for (size_t first = 0; first < c.gathers.size(); first += c.mb) {
      const int count = (int)std::min<size_t>(c.mb, c.gathers.size() - first);
      ashrt_status st = work(c, (int)first, count, c.st);
      if (st != ASHRT_OK) return st;
    }
    cudaEventRecord(c.done, c.st);
    cudaStreamWaitEvent(stream, c.done, 0);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("batch: %s", cudaGetErrorString(e));
    return ASHRT_ECUDA;
  }
  return ASHRT_OK;
}

static dim3 pack_grid(long long per_slot, int count) {
  long long gx = (per_slot + 256 * 8 - 1) / (256 * 8);
  if (gx > 1024) gx = 1024;
  return dim3((unsigned)std::max<long long>(gx, 1), count);
}

extern "C" {

ashrt_status ashrt_batch_forward(ashrt_batch* b, const float* m, float* d, void* stream) {
  if (!b || !m || !d) {
    set_error("ashrt_batch_forward: NULL argument");
    return ASHRT_EINVAL;
  }
  const int P = b->P;
  return for_each_chunk(b, (cudaStream_t)stream,
                        [&](ashrt_batch::Class& c, int first, int count, cudaStream_t s) {
    const int nt = c.nt;
    const long long per_m = (long long)P * c.nxc * nt, per_d = (long long)c.nxc * nt;
    k_pack<<<pack_grid(per_m, count), 256, 0, s>>>(m, c.m, c.moff_dev + first, c.nx_dev + first,
                                                    c.nxc, nt, P, c.tmask);
    count_launches(1);
    ashrt_status st = ashrt_forward(c.plan, c.m, c.d, nullptr, count, s);
    if (st != ASHRT_OK) return st;
    k_unpack<<<pack_grid(per_d, count), 256, 0, s>>>(c.d, d, c.doff_dev + first, c.nx_dev + first,
                                                      c.nxc, nt, 1);
    count_launches(1);
    return ASHRT_OK;
  });
}

ashrt_status ashrt_batch_adjoint(ashrt_batch* b, const float* d, float* m, void* stream) {
  if (!b || !m || !d) {
    set_error("ashrt_batch_adjoint: NULL argument");
    return ASHRT_EINVAL;
  }
  const int P = b->P;
  return for_each_chunk(b, (cudaStream_t)stream,
                        [&](ashrt_batch::Class& c, int first, int count, cudaStream_t s) {
    const int nt = c.nt;
    const long long per_m = (long long)P * c.nxc * nt, per_d = (long long)c.nxc * nt;
    k_pack<<<pack_grid(per_d, count), 256, 0, s>>>(d, c.d, c.doff_dev + first, c.nx_dev + first,
                                                    c.nxc, nt, 1, c.tmask);
    count_launches(1);
    ashrt_status st = ashrt_adjoint(c.plan, c.d, c.m, nullptr, count, s);
    if (st != ASHRT_OK) return st;
    k_unpack<<<pack_grid(per_m, count), 256, 0, s>>>(c.m, m, c.moff_dev + first, c.nx_dev + first,
                                                      c.nxc, nt, P);
    count_launches(1);
    return ASHRT_OK;
  });
}

ashrt_status ashrt_batch_deblend(ashrt_batch* b, const float* d, float* m, float* drec,
                                 const irls_opts* opts, irls_report* reports, void* stream) {
  if (!b || !d || !m) {
    set_error("ashrt_batch_deblend: NULL argument");
    return ASHRT_EINVAL;
  }
  irls_opts o;
  irls_default_opts(&o);
  if (opts) o = *opts;
  if (o.trace_mask_dev || o.apex_mask_dev) {
    set_error("ashrt_batch_deblend: per-call masks are set by the batch layer (pass NULL)");
    return ASHRT_EINVAL;
  }
  for (auto& c : b->cls)
    if (!c.plan->with_solver) {
      set_error("ashrt_batch_deblend: the batch was created without with_solver");
      return ASHRT_EINVAL;
    }
  const int P = b->P;
  std::vector<irls_report> rep;
  return for_each_chunk(b, (cudaStream_t)stream,
                        [&](ashrt_batch::Class& c, int first, int count, cudaStream_t s) {
    const int nt = c.nt;
    const long long per_m = (long long)P * c.nxc * nt, per_d = (long long)c.nxc * nt;
    k_pack<<<pack_grid(per_d, count), 256, 0, s>>>(d, c.d, c.doff_dev + first, c.nx_dev + first,
                                                    c.nxc, nt, 1, c.tmask);
    count_launches(1);
    irls_opts oc = o;
    oc.trace_mask_dev = c.tmask;   // padded traces are dead samples
    oc.apex_mask_dev = c.tmask;    // and padded apexes are not unknowns
    rep.assign(count, irls_report{});
    ashrt_status st = robust_irls_deblend(c.plan, c.d, c.m, c.drec, count, &oc, rep.data(), s);
    if (st != ASHRT_OK) return st;
    k_unpack<<<pack_grid(per_m, count), 256, 0, s>>>(c.m, m, c.moff_dev + first, c.nx_dev + first,
                                                      c.nxc, nt, P);
    count_launches(1);
    if (drec) {
      k_unpack<<<pack_grid(per_d, count), 256, 0, s>>>(c.drec, drec, c.doff_dev + first,
                                                        c.nx_dev + first, c.nxc, nt, 1);
      count_launches(1);
    }
    if (reports)
      for (int i = 0; i < count; ++i) reports[c.gathers[first + i]] = rep[i];
    return ASHRT_OK;
  });
}

}  // extern "C"
