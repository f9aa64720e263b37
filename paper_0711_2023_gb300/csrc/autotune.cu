// Autotuner for steps that have several equivalent kernels (same result up to the order of
// FP32 summation): on the first call for a shape class it times every variant once on the
// caller's stream, keeps the fastest for the rest of the process and runs it once more so the
// caller's outputs come from the kept variant.  Later calls (single-tensor or batched, on any
// stream) run the kept variant only, so results are reproducible within a process.  A mutex is
// held while a class is tuned, so concurrent first calls wait for one decision.
#include <atomic>
#include <mutex>
#include <vector>

#include "internal.h"

namespace tk {

namespace {

struct Decision {
  int family;
  int key[3];
  int variant;
  double ms[2];
};

std::mutex g_mu;
std::vector<Decision> g_decisions;
std::atomic<bool> g_enabled{true};

const Decision* find_locked(int family, int a, int b, int c) {
  for (const auto& d : g_decisions)
    if (d.family == family && d.key[0] == a && d.key[1] == b && d.key[2] == c) return &d;
  return nullptr;
}

}  // namespace

int autotune_run(int family, int a, int b, int c, const std::function<int(int)>& run,
                 cudaStream_t s) {
  std::unique_lock<std::mutex> lk(g_mu);
  const Decision* d = find_locked(family, a, b, c);
  if (d) {
    const int v = d->variant;
    lk.unlock();
    return run(v);
  }
  if (!g_enabled.load()) {
    lk.unlock();
    return run(0);
  }
  // Time both variants (each after one untimed run, so that first-touch costs are excluded).
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  TK_CUDA(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    TK_CUDA(ce);
  }
  double ms[2] = {0.0, 0.0};
  int st = TUCKER_OK;
  for (int v = 0; v < 2 && st == TUCKER_OK; ++v) {
    st = run(v);
    if (st != TUCKER_OK) break;
    cudaEventRecord(e0, s);
    st = run(v);
    cudaEventRecord(e1, s);
    if (st != TUCKER_OK) break;
    float t = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
      st = TUCKER_ECUDA;
    ms[v] = t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != TUCKER_OK) return st;
  const int best = ms[1] < ms[0] ? 1 : 0;
  g_decisions.push_back(Decision{family, {a, b, c}, best, {ms[best], ms[1 - best]}});
  return run(best);
}

}  // namespace tk

using namespace tk;

extern "C" {

void tucker_autotune_enable(int on) { g_enabled.store(on != 0); }

int tucker_autotune_count(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  return (int)g_decisions.size();
}

int tucker_autotune_decision(int32_t i, int32_t* family, int32_t key[3], int32_t* variant,
                             double* ms_chosen, double* ms_other) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (i < 0 || i >= (int32_t)g_decisions.size()) return TUCKER_EINVAL;
  const Decision& d = g_decisions[i];
  if (family) *family = d.family;
  if (key)
    for (int j = 0; j < 3; ++j) key[j] = d.key[j];
  if (variant) *variant = d.variant;
  if (ms_chosen) *ms_chosen = d.ms[0];
  if (ms_other) *ms_other = d.ms[1];
  return TUCKER_OK;
}

}  // extern "C"
