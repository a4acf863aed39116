// Launch counting and optional per-kernel-class CUDA-event timing.
//
// Every launcher in the library calls count_launch(); with profiling on,
// the driver brackets the launches of a kernel class with an event pair on
// the stream the kernels run on, so a caller can divide algorithmic work by
// measured device time without an external profiler.
#include <atomic>
#include <mutex>
#include <vector>

#include "kernels.cuh"

namespace rqk {

namespace {
std::atomic<long long> g_launches{0};
std::mutex g_mu;
bool g_on = false;
struct Pair {
  cudaEvent_t a, b;
};
std::vector<Pair> g_pool[kProfClasses];
size_t g_used[kProfClasses] = {};
}  // namespace

Tuning &tuning() {
  static thread_local Tuning t = {0, 0, 0, 0, 0};
  return t;
}

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

int prof_start(int cls, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on || cls < 0 || cls >= kProfClasses) return -1;
  auto &pool = g_pool[cls];
  if (g_used[cls] == pool.size()) {
    Pair p;
    if (cudaEventCreate(&p.a) != cudaSuccess) return -1;
    if (cudaEventCreate(&p.b) != cudaSuccess) return -1;
    pool.push_back(p);
  }
  const int idx = (int)g_used[cls]++;
  cudaEventRecord(pool[idx].a, st);
  return idx;
}

void prof_stop(int cls, int idx, cudaStream_t st) {
  if (idx < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEventRecord(g_pool[cls][idx].b, st);
}

}  // namespace rqk

using namespace rqk;

extern "C" {

long long rqlp_launch_count(void) { return launch_count(); }

int rqlp_profile_begin(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (int c = 0; c < kProfClasses; ++c) g_used[c] = 0;
  g_on = true;
  return RQLP_OK;
}

int rqlp_profile_end(double *ms, long long *count, int nclass) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = false;
  for (int c = 0; c < kProfClasses && c < nclass; ++c) {
    double tot = 0.0;
    for (size_t i = 0; i < g_used[c]; ++i) {
      if (cudaEventSynchronize(g_pool[c][i].b) != cudaSuccess) return RQLP_ERR_CUDA;
      float t = 0.f;
      if (cudaEventElapsedTime(&t, g_pool[c][i].a, g_pool[c][i].b) != cudaSuccess) return RQLP_ERR_CUDA;
      tot += t;
    }
    if (ms) ms[c] = tot;
    if (count) count[c] = (long long)g_used[c];
  }
  return RQLP_OK;
}

}  // extern "C"
