// Launch accounting and optional per-kernel-class timing with CUDA events,
// used by measurement tools (the bench) to time the library's own kernels on
// the stream they run on.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "internal.h"

namespace ashrt {

namespace {
std::atomic<long long> g_launches{0};
std::atomic<int> g_prof_on{0};
std::mutex g_mu;
struct Rec {
  int cls;
  cudaEvent_t a, b;
};
std::vector<Rec> g_open;       // pending records (events not yet read)
std::vector<cudaEvent_t> g_pool;
double g_ms[kProfClasses] = {0};
long long g_cnt[kProfClasses] = {0};
thread_local cudaEvent_t t_start = nullptr;
thread_local bool t_capturing = false;
thread_local long long t_captured = 0;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void count_launches(int n) {
  if (t_capturing) t_captured += n;
  else g_launches.fetch_add(n, std::memory_order_relaxed);
}

void prof_capture_begin() {
  t_capturing = true;
  t_captured = 0;
}

long long prof_capture_end() {
  t_capturing = false;
  return t_captured;
}

void prof_begin(int cls, cudaStream_t s) {
  (void)cls;
  count_launches(1);
  if (t_capturing || !g_prof_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  t_start = take_event();
  cudaEventRecord(t_start, s);
}

void prof_end(int cls, cudaStream_t s) {
  if (t_capturing || !g_prof_on.load(std::memory_order_relaxed) || !t_start) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t e = take_event();
  cudaEventRecord(e, s);
  g_open.push_back(Rec{cls, t_start, e});
  t_start = nullptr;
}

}  // namespace ashrt

using namespace ashrt;

extern "C" {

void ashrt_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_prof_on.store(on ? 1 : 0);
}

int ashrt_profile_read(double* ms, long long* launches, int n) {
  std::lock_guard<std::mutex> lk(g_mu);
  int status = 0;
  for (const Rec& r : g_open) {
    float t = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) {
      status = 1;
      cudaGetLastError();
    }
    g_ms[r.cls] += t;
    g_cnt[r.cls] += 1;
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_open.clear();
  for (int i = 0; i < n && i < kProfClasses; ++i) {
    if (ms) ms[i] = g_ms[i];
    if (launches) launches[i] = g_cnt[i];
    g_ms[i] = 0.0;
    g_cnt[i] = 0;
  }
  return status;
}

long long ashrt_kernel_launches(void) { return g_launches.load(); }

}  // extern "C"
