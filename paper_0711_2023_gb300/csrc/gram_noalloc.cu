// Allocation-free variant of the FP64 Gram M = Y1 Y1^T (+ Y2 Y2^T) (tucker_gram).
//
// Some callers cannot let a library allocate device memory while they run: serving processes
// that reserve all device memory up front in their own pool and run under a fixed budget, and
// callers that must not risk the implicit device synchronisation that cudaMalloc/cudaFree can
// cause.  This entry point serves them: it takes its split-K workspace from one fixed
// file-scope __device__ array instead of cudaMallocAsync, and calls no allocating routine.
//
// Properties callers rely on:
//   * Scratch: NOALLOC_SCRATCH_DOUBLES doubles (16 MiB), present on every GPU that loads the
//     library, for the life of the process.  Size limit: rows * rows <= NOALLOC_SCRATCH_DOUBLES
//     (rows <= 1448); larger calls are rejected with TUCKER_EINVAL.
//   * Set-up: the first call on each device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current).  Make that first call before any stream
//     capture begins.
//   * No part of the scratch needs to start at zero: every element the reduction reads is
//     written earlier in the same call.  The array keeps the last call's contents.
//   * All calls on a device share the one array: calls whose executions overlap on the GPU
//     (different streams, no ordering between them) race on it.  Order them on one stream.
#include <mutex>

#include "internal.h"

namespace tk {

namespace {

constexpr int64_t NOALLOC_SCRATCH_DOUBLES = int64_t(1) << 21;
constexpr int NB = 64, NK = 16;
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) double g_gram_scratch[NOALLOC_SCRATCH_DOUBLES];

std::mutex g_mu;
double* g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once per device).
int scratch_address(double** out) {
  int dev = 0;
  TK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) return TUCKER_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    TK_CUDA(cudaGetSymbolAddress(&p, g_gram_scratch));
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return TUCKER_OK;
}

// Split-K SYRK partials like the allocating kernel, but the lower-triangle tile pair of block x
// is decoded from its index (ti >= tj) instead of read from a table.
__global__ void __launch_bounds__(256)
syrk_noalloc_kernel(int rows, const double* __restrict__ Y1, int64_t K1,
                    const double* __restrict__ Y2, int64_t K2, int64_t kchunk,
                    double* __restrict__ P) {
  __shared__ double As[NK][NB + 1];
  __shared__ double Bs[NK][NB + 1];
  const int64_t x = blockIdx.x;
  int ti = (int)((sqrt(8.0 * (double)x + 1.0) - 1.0) * 0.5);
  while ((int64_t)ti * (ti + 1) / 2 > x) --ti;
  while ((int64_t)(ti + 1) * (ti + 2) / 2 <= x) ++ti;
  const int tj = (int)(x - (int64_t)ti * (ti + 1) / 2);
  const int r0 = ti * NB, c0 = tj * NB;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t K = K1 + K2;
  const int64_t kb = (int64_t)blockIdx.y * kchunk;
  const int64_t ke = min64(K, kb + kchunk);
  double acc[4][4] = {};
  for (int64_t k0 = kb; k0 < ke; k0 += NK) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = threadIdx.x + 256 * e;
      const int rr = idx / NK, kk = idx % NK;
      const int64_t kg = k0 + kk;
      double va = 0.0, vb = 0.0;
      if (kg < ke) {
        const int ra = r0 + rr, rb = c0 + rr;
        if (kg < K1) {
          if (ra < rows) va = Y1[(int64_t)ra * K1 + kg];
          if (rb < rows) vb = Y1[(int64_t)rb * K1 + kg];
        } else {
          const int64_t k2 = kg - K1;
          if (ra < rows) va = Y2[(int64_t)ra * K2 + k2];
          if (rb < rows) vb = Y2[(int64_t)rb * K2 + k2];
        }
      }
      As[kk][rr] = va;
      Bs[kk][rr] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < NK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double* Pz = P + (int64_t)blockIdx.y * rows * rows;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + ty + 16 * i;
    if (r >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx + 16 * j;
      if (c < rows) Pz[(int64_t)r * rows + c] = acc[i][j];
    }
  }
}

// Sums the split partials of lower-triangle tiles in split order and mirrors them.
__global__ void syrk_noalloc_reduce(const double* __restrict__ P, int splits, int rows,
                                    double* __restrict__ M) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)rows * rows) return;
  const int r = (int)(t / rows), c = (int)(t % rows);
  if (r / NB < c / NB) return;
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += P[(int64_t)z * rows * rows + t];
  M[(int64_t)r * rows + c] = s;
  if (r / NB != c / NB) M[(int64_t)c * rows + r] = s;
}

__global__ void zero_kernel(double* __restrict__ M, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) M[t] = 0.0;
}

}  // namespace

}  // namespace tk

using namespace tk;

extern "C" int tucker_gram_noalloc(const double* d_Y1, int64_t K1, const double* d_Y2, int64_t K2,
                                   int32_t rows, double* d_M, void* stream) {
  if (!d_Y1 || !d_M || rows < 1 || K1 < 0 || (d_Y2 && K2 < 0)) return TUCKER_EINVAL;
  if ((int64_t)rows * rows > NOALLOC_SCRATCH_DOUBLES) {
    set_error_detail("tucker_gram_noalloc: rows * rows exceeds the fixed scratch of 2^21 "
                     "doubles (rows <= 1448)");
    return TUCKER_EINVAL;
  }
  if (!d_Y2) K2 = 0;
  cudaStream_t s = (cudaStream_t)stream;
  double* P = nullptr;
  TK_TRY(scratch_address(&P));
  const int64_t K = K1 + K2;
  const int64_t cells = (int64_t)rows * rows;
  if (K == 0) {
    zero_kernel<<<ceil_div(cells, 256), 256, 0, s>>>(d_M, cells);
    TK_LAUNCH();
    TK_CUDA(cudaStreamSynchronize(s));
    return TUCKER_OK;
  }
  const int nt = ceil_div(rows, NB);
  const int npairs = nt * (nt + 1) / 2;
  // As many K splits as the scratch holds, up to about three CTAs per SM.
  int splits = (3 * num_sms() + npairs - 1) / npairs;
  const int64_t by_k = (K + 127) / 128, by_scratch = NOALLOC_SCRATCH_DOUBLES / cells;
  if (splits > by_k) splits = (int)by_k;
  if (splits > by_scratch) splits = (int)by_scratch;
  if (splits < 1) splits = 1;
  int64_t kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + NK - 1) / NK * NK;
  const int nsplit = (int)((K + kchunk - 1) / kchunk);
  dim3 grid(npairs, nsplit);
  syrk_noalloc_kernel<<<grid, 256, 0, s>>>(rows, d_Y1, K1, d_Y2, K2, kchunk, P);
  TK_LAUNCH();
  syrk_noalloc_reduce<<<ceil_div(cells, 256), 256, 0, s>>>(P, nsplit, rows, d_M);
  TK_LAUNCH();
  TK_CUDA(cudaStreamSynchronize(s));
  return TUCKER_OK;
}
