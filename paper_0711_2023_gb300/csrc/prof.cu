// Opt-in kernel timing: CUDA events recorded on the launching stream around the hot-path
// kernels, with each launch's algorithmic FLOPs and bytes, named counters of the iterative
// parts (values summed), plus a count of every kernel launch the library makes.  Used by the
// benchmark to report achieved rates against the roofline.
#include <atomic>
#include <mutex>
#include <string.h>
#include <vector>

#include "internal.h"

namespace tk {

std::atomic<long long> g_launch_count{0};

namespace {
struct Rec {
  const char* name;
  cudaEvent_t a, b;
  double flops, bytes;
};
bool g_on = false;
std::mutex g_mu;
std::vector<Rec> g_recs;

void clear_locked() {
  for (auto& r : g_recs) {
    if (!r.a) continue;  // a counter has no events
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_recs.clear();
}
}  // namespace

void count_launch() { g_launch_count.fetch_add(1, std::memory_order_relaxed); }

namespace {
thread_local long long t_syncs = 0;
}
int host_sync(cudaStream_t s) {
  ++t_syncs;
  TK_CUDA(cudaStreamSynchronize(s));
  return TUCKER_OK;
}
long long host_sync_count() { return t_syncs; }
long long launch_count() { return g_launch_count.load(std::memory_order_relaxed); }

ProfScope::ProfScope(const char* name, cudaStream_t s, double flops, double bytes)
    : name_(name), s_(s), flops_(flops), bytes_(bytes) {
  if (!g_on) return;
  if (cudaEventCreate(&a_) != cudaSuccess) return;
  if (cudaEventCreate(&b_) != cudaSuccess) {
    cudaEventDestroy(a_);
    return;
  }
  cudaEventRecord(a_, s_);
  active_ = true;
}

void prof_count(const char* name, double value) {
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.push_back(Rec{name, nullptr, nullptr, value, 0.0});
}

void ProfScope::end() {
  if (!active_) return;
  active_ = false;
  cudaEventRecord(b_, s_);
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.push_back(Rec{name_, a_, b_, flops_, bytes_});
}

}  // namespace tk

using namespace tk;

extern "C" {

void tucker_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaDeviceSynchronize();
  clear_locked();
  g_on = on != 0;
}

int tucker_profile_query(const char* name, int64_t* launches, double* total_ms, double* flops,
                         double* bytes) {
  if (!name) return TUCKER_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  int64_t n = 0;
  double ms = 0.0, f = 0.0, by = 0.0;
  for (auto& r : g_recs) {
    if (strcmp(r.name, name) != 0) continue;
    if (!r.a) {  // a counter: no timing, its value summed into *flops
      ++n;
      f += r.flops;
      continue;
    }
    if (cudaEventSynchronize(r.b) != cudaSuccess) return TUCKER_ECUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return TUCKER_ECUDA;
    ++n;
    ms += t;
    f += r.flops;
    by += r.bytes;
  }
  if (launches) *launches = n;
  if (total_ms) *total_ms = ms;
  if (flops) *flops = f;
  if (bytes) *bytes = by;
  return TUCKER_OK;
}

int64_t tucker_launch_count(void) { return g_launch_count.load(); }

}  // extern "C"
