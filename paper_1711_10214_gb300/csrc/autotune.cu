// Autotuner: picks the kernel variants of a plan (the row kernels' register
// cap, i.e. resident CTAs per SM, or their radix-16 form, and the trace-axis
// FFT column tile) by timing
// forward+adjoint operator pairs on the plan's own sizes, and keeps the choice
// in a JSON-lines cache keyed by device and problem shape.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "ops.h"

namespace {

__global__ void k_fill_hash(float* x, long long n, unsigned seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    unsigned h = (unsigned)i * 2654435761u ^ seed;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    x[i] = (float)(h & 0xffffu) * (1.f / 32768.f) - 1.f;
  }
}

std::string tune_key(const ashrt_plan* p, int batch) {
  cudaDeviceProp prop;
  char name[256] = "unknown";
  if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) snprintf(name, sizeof(name), "%s", prop.name);
  char buf[512];
  snprintf(buf, sizeof(buf), "%s|variants=9|nt=%d|nx=%d|Nt=%d|Nx=%d|P=%d|shift=%d|B=%d", name,
           p->nt, p->nx,
           p->Nt, p->Nx, p->P, p->shift ? 1 : 0, batch);
  return buf;
}

bool cache_lookup(const char* path, const std::string& key, int* minb, int* cols) {
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  const std::string needle = "\"key\": \"" + key + "\"";
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    if (!strstr(line, needle.c_str())) continue;
    const char* a = strstr(line, "\"rows_minb\": ");
    const char* b = strstr(line, "\"xfft_cols\": ");
    if (a && b && sscanf(a + 13, "%d", minb) == 1 && sscanf(b + 13, "%d", cols) == 1) found = true;
  }
  fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, int minb, int cols, double ms) {
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "{\"key\": \"%s\", \"rows_minb\": %d, \"xfft_cols\": %d, \"pair_ms\": %.4f}\n",
          key.c_str(), minb, cols, ms);
  fclose(f);
}

}  // namespace

using namespace ashrt;

extern "C" ashrt_status ashrt_plan_autotune(ashrt_plan* p, int batch, const char* cache_path,
                                            int* rows_minb, int* xfft_cols) {
  if (!p || batch < 1 || batch > p->max_batch) {
    set_error("ashrt_plan_autotune: NULL plan or batch outside [1, max_batch]");
    return ASHRT_EINVAL;
  }
  const std::string key = tune_key(p, batch);
  int minb = p->rows_minb, cols = p->xfft_cols;
  if (cache_lookup(cache_path, key, &minb, &cols)) {
    p->rows_minb = minb;
    p->xfft_cols = cols;
    if (rows_minb) *rows_minb = minb;
    if (xfft_cols) *xfft_cols = cols;
    return ASHRT_OK;
  }
  const size_t nd = (size_t)batch * data_elems(p), nm = (size_t)batch * model_elems(p);
  float *m = nullptr, *d = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&m, nm * 4);
  if (e == cudaSuccess) e = cudaMalloc(&d, nd * 4);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  auto cleanup = [&]() {
    if (m) cudaFree(m);
    if (d) cudaFree(d);
    if (s) cudaStreamDestroy(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("ashrt_plan_autotune: setup failed: %s", cudaGetErrorString(e));
    cleanup();
    return ASHRT_ENOMEM;
  }
  k_fill_hash<<<152 * 4, 256, 0, s>>>(m, (long long)nm, 17u);
  k_fill_hash<<<152 * 4, 256, 0, s>>>(d, (long long)nd, 91u);
  count_launches(2);

  auto time_pair = [&](double* ms) -> cudaError_t {
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {   // 1 warm-up + 3 timed
      if (rep == 1) cudaEventRecord(e0, s);
      err = op_forward(p, m, d, nullptr, nullptr, nullptr, nullptr, batch, s);
      if (err == cudaSuccess) err = op_adjoint(p, d, m, nullptr, nullptr, nullptr, nullptr, batch, s);
    }
    cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float t = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
    *ms = t / 3.0;
    return err;
  };

  // the plan's default variant is timed first and kept unless another one is
  // faster by more than 2% (timing noise does not flip the choice)
  const int def_minb = p->rows_minb;
  std::vector<int> minbs = {def_minb};
  std::vector<int> cand = {3};
  if (p->logNt >= 9 && p->logNt <= 11) cand = {3, 2, 1};
  if (rows16_supported(p->logNt) && p->tw_t16) {
    for (int v : {4, 5, 6, 7, 8}) cand.push_back(v);
    if (p->logNt == 11) cand.push_back(9);
  }
  for (int v : cand)
    if (v != def_minb) minbs.push_back(v);
  std::vector<int> colss = {16};
  if (p->logNx <= 9) colss = {16, 8};
  double best = 1e30;
  int best_minb = minbs[0], best_cols = colss[0];
  for (int mb : minbs) {
    p->rows_minb = mb;
    p->xfft_cols = best_cols;
    double ms = 0.0;
    e = time_pair(&ms);
    if (e != cudaSuccess) break;
    if (ms < (mb == def_minb ? best : 0.98 * best)) {
      best = ms;
      best_minb = mb;
    }
  }
  for (size_t i = 1; i < colss.size() && e == cudaSuccess; ++i) {
    p->rows_minb = best_minb;
    p->xfft_cols = colss[i];
    double ms = 0.0;
    e = time_pair(&ms);
    if (e == cudaSuccess && ms < 0.98 * best) {
      best = ms;
      best_cols = colss[i];
    }
  }
  cleanup();
  p->rows_minb = best_minb;
  p->xfft_cols = best_cols;
  if (e != cudaSuccess) {
    set_error("ashrt_plan_autotune: timing failed: %s", cudaGetErrorString(e));
    return ASHRT_ECUDA;
  }
  cache_store(cache_path, key, best_minb, best_cols, best);
  if (rows_minb) *rows_minb = best_minb;
  if (xfft_cols) *xfft_cols = best_cols;
  return ASHRT_OK;
}

extern "C" ashrt_status ashrt_plan_set_variant(ashrt_plan* p, int rows_minb, int xfft_cols) {
  if (!p || rows_minb < 1 || rows_minb > 9 || (xfft_cols != 8 && xfft_cols != 16)) {
    set_error("ashrt_plan_set_variant: need a plan, rows_minb in 1..9, xfft_cols 8 or 16");
    return ASHRT_EINVAL;
  }
  if (rows_minb >= 4 && !p->tw_t16) {
    set_error("ashrt_plan_set_variant: the radix-16 row kernels (4..9) need Nt = 1024, 2048 or "
              "4096");
    return ASHRT_EINVAL;
  }
  p->rows_minb = rows_minb;
  p->xfft_cols = xfft_cols;
  return ASHRT_OK;
}
