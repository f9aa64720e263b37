// Shared device/host helpers of the Tucker library (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "tucker.h"

namespace tk {

// ---- status plumbing ------------------------------------------------------------------------
#define TK_CUDA(call)                                                               \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      tk::set_last_cuda_error(e_, #call, __FILE__, __LINE__);                       \
      return e_ == cudaErrorMemoryAllocation ? TUCKER_ENOMEM : TUCKER_ECUDA;        \
    }                                                                               \
  } while (0)

#define TK_LAUNCH()                                                                 \
  do {                                                                              \
    tk::count_launch();                                                             \
    cudaError_t e_ = cudaGetLastError();                                            \
    if (e_ != cudaSuccess) {                                                        \
      tk::set_last_cuda_error(e_, "kernel launch", __FILE__, __LINE__);             \
      return TUCKER_ECUDA;                                                          \
    }                                                                               \
  } while (0)

#define TK_TRY(expr)                   \
  do {                                 \
    int s_ = (expr);                   \
    if (s_ != TUCKER_OK) return s_;    \
  } while (0)

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);
void set_error_detail(const char* msg);
void keep_pool_memory();  // once per device: freed work buffers stay in the stream pool
void count_launch();
// Stream synchronisation that the host waits on (counted per host thread), and the counters.
int host_sync(cudaStream_t s);
long long host_sync_count();
long long launch_count();
// While profiling is enabled, records one occurrence of the counter `name` with `value`
// (tucker_profile_query reports the occurrences as launches and the sum of values as flops).
void prof_count(const char* name, double value);

// Records CUDA events around its lifetime (or up to end()) on `s` when profiling is enabled
// (tucker_profile_enable), tagged with the launch's algorithmic FLOPs and bytes.
class ProfScope {
 public:
  ProfScope(const char* name, cudaStream_t s, double flops, double bytes);
  ~ProfScope() { end(); }
  // Closes the span now (the destructor then does nothing).
  void end();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  const char* name_;
  cudaStream_t s_;
  double flops_, bytes_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
  bool active_ = false;
};

// Device status word bits written by kernels (never trap: a kernel that finds a bad state
// records it and returns, so the context stays usable).
enum : int {
  DEV_OK = 0,
  DEV_BAD_INDEX = 1,
  DEV_TIMEOUT = 2,
  DEV_CHOL_BREAKDOWN = 4,
  DEV_NOT_CONVERGED = 8,
  DEV_CHOL_SHIFTED = 16,
};

// ---- stream-ordered work buffers ------------------------------------------------------------
// A Buf owns one cudaMallocAsync allocation and frees it on `stream` when it goes out of scope.
struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t s = 0;
  Buf() = default;
  Buf(const Buf&) = delete;
  Buf& operator=(const Buf&) = delete;
  ~Buf() { release(); }
  int alloc(size_t nbytes, cudaStream_t stream) {
    keep_pool_memory();
    release();
    s = stream;
    bytes = nbytes;
    if (nbytes == 0) return TUCKER_OK;
    cudaError_t e = cudaMallocAsync(&p, nbytes, stream);
    if (e != cudaSuccess) {
      p = nullptr;
      set_last_cuda_error(e, "cudaMallocAsync", __FILE__, __LINE__);
      return TUCKER_ENOMEM;
    }
    return TUCKER_OK;
  }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    bytes = 0;
  }
  template <class T>
  T* as() const { return static_cast<T*>(p); }
};

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

int num_sms();

// ---- device helpers -------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Grid-wide barrier for cooperative launches, with a bounded spin.  `*count` (zeroed before the
// launch) only grows: barrier number e (1, 2, ...) completes when it reaches e * nblocks, so
// each block makes one atomic per barrier and polls.  `*epoch` is the block's barrier count.
// Returns false (and sets DEV_TIMEOUT in *status) when the spin limit runs out; callers then
// leave their loops.  All blocks of a cooperative launch are co-resident, so in a healthy run
// every wait ends.
__device__ __forceinline__ bool grid_barrier(unsigned int* count, unsigned int nblocks,
                                             unsigned int* epoch, int* status) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok_s = 1;
    const unsigned int target = (*epoch + 1) * nblocks;
    __threadfence();
    atomicAdd(count, 1u);
    volatile unsigned int* vc = count;
    const long long t0 = clock64();
    while (*vc < target) {
      if (clock64() - t0 > 2000000000ll) {  // about a second: far beyond any healthy wait
        atomicOr(status, DEV_TIMEOUT);
        ok_s = 0;
        break;
      }
    }
    __threadfence();
  }
  ++*epoch;
  __syncthreads();
  return ok_s != 0;
}

}  // namespace tk
