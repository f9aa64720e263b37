// Tensor-core Gram M = sum_terms Y Y^T for the mixed-precision path (the "U_(1) U_(1)^T" and
// slice-sum matrices of Figures hooi3, sp3, mp3).  Y is given split into BF16 halves,
// Y = hi + lo, and each product is formed as hi hi^T + hi lo^T + lo hi^T (BF16x3) on the
// 5th-generation tensor cores with FP32 accumulation in tensor memory:
//
//   * one CTA computes one 128 x 128 tile (ti >= tj) of M over one K chunk of <= 4096;
//   * warp 0 / lane 0 streams 128 x 64 BF16 tiles of hi and lo through a 3-stage ring with
//     TMA (128-byte swizzle, mbarrier completion); diagonal tiles load A only;
//   * warp 1 / lane 0 issues tcgen05.mma (M=128, N=128, K=16, kind::f16, BF16 in, FP32 out)
//     and returns ring slots with tcgen05.commit;
//   * all four warps read the accumulator with tcgen05.ld and store the chunk's FP32 tile;
//   * a reduction kernel adds the chunks in FP64, in chunk order, and mirrors the lower
//     triangle, so M is exactly symmetric and bitwise reproducible.
// Every wait is bounded: on timeout the kernel records DEV_TIMEOUT, drains what it issued,
// frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <vector>

#include "internal.h"

namespace tk {

namespace {

constexpr int TM = 128, TK = 64, STAGES = 3, KCHUNK_MAX = 4096;
constexpr int TILE_BYTES = TM * TK * 2;           // 16 KB
constexpr int STAGE_BYTES = 4 * TILE_BYTES;       // Ah, Al, Bh, Bl
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr long long WAIT_CYCLES = 4000000000ll;   // ~2 s at 2 GHz

struct Job {
  int ti, tj;      // tile pair (ti >= tj)
  int term;        // 0 or 1
  int k0, nk;      // first K column and number of 64-wide K steps
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase; false (and DEV_TIMEOUT in *status) on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* status,
                                          volatile int* abort_flag) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicOr(status, DEV_TIMEOUT);
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(const void* p) {
  const uint64_t addr = (uint64_t)(smem_u32(p) & 0x3FFFFu) >> 4;
  const uint64_t lbo = 1;            // unused for swizzled K-major layouts
  const uint64_t sbo = 1024 >> 4;    // stride between 8-row core-matrix groups
  return addr | (lbo << 16) | (sbo << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor: kind::f16, A = B = BF16, D = F32, both K-major, M = 128, N = 128.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) |
                           ((128u >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(IDESC), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct TermMaps {
  CUtensorMap hi[2];
  CUtensorMap lo[2];
};

__global__ void __launch_bounds__(128, 1)
gram_bf16x3_kernel(const __grid_constant__ TermMaps maps, const Job* __restrict__ jobs,
                   float* __restrict__ partial, int* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Job job = jobs[blockIdx.x];
  const bool diag = job.ti == job.tj;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(128u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const CUtensorMap* mh = &maps.hi[job.term];
  const CUtensorMap* ml = &maps.lo[job.term];
  const int rowA = job.ti * TM, rowB = job.tj * TM;
  const uint32_t bytes = (diag ? 2 : 4) * TILE_BYTES;

  if (warp == 0 && lane == 0) {
    // TMA producer
    int issued = 0;
    for (int ks = 0; ks < job.nk; ++ks) {
      const int s = ks % STAGES;
      if (ks >= STAGES && !mbar_wait(&empty[s], ((ks / STAGES) - 1) & 1, status, abort_flag))
        break;
      uint8_t* st = smem + s * STAGE_BYTES;
      mbar_expect_tx(&full[s], bytes);
      const int kx = job.k0 + ks * TK;
      tma_load_2d(st, mh, &full[s], kx, rowA);
      tma_load_2d(st + TILE_BYTES, ml, &full[s], kx, rowA);
      if (!diag) {
        tma_load_2d(st + 2 * TILE_BYTES, mh, &full[s], kx, rowB);
        tma_load_2d(st + 3 * TILE_BYTES, ml, &full[s], kx, rowB);
      }
      ++issued;
    }
    if (*abort_flag) {
      // Drain: wait (bounded) until the copies this thread issued have landed.
      for (int ks = issued > STAGES ? issued - STAGES : 0; ks < issued; ++ks) {
        const long long t0 = clock64();
        while (!mbar_try_wait(&full[ks % STAGES], (ks / STAGES) & 1) &&
               clock64() - t0 < WAIT_CYCLES) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    int issued = 0;
    for (int ks = 0; ks < job.nk; ++ks) {
      const int s = ks % STAGES;
      if (!mbar_wait(&full[s], (ks / STAGES) & 1, status, abort_flag)) break;
      tc_fence_after();
      uint8_t* st = smem + s * STAGE_BYTES;
      const uint8_t* ah = st;
      const uint8_t* al = st + TILE_BYTES;
      const uint8_t* bh = diag ? ah : st + 2 * TILE_BYTES;
      const uint8_t* bl = diag ? al : st + 3 * TILE_BYTES;
      const uint64_t dah = sw128_desc(ah), dal = sw128_desc(al);
      const uint64_t dbh = sw128_desc(bh), dbl = sw128_desc(bl);
#pragma unroll
      for (int kk = 0; kk < TK / 16; ++kk) {
        const uint64_t off = (uint64_t)(kk * 32) >> 4;  // 16 BF16 = 32 bytes along K
        mma_bf16(tmem, dah + off, dbh + off, (ks | kk) ? 1u : 0u);
        mma_bf16(tmem, dah + off, dbl + off, 1u);
        mma_bf16(tmem, dal + off, dbh + off, 1u);
      }
      mma_commit(&empty[s]);
      ++issued;
    }
    mma_commit(done);  // arrives once all issued MMAs have completed (also when none were)
  }
  __syncwarp();
  // Everyone waits for the accumulator (bounded; an aborted run still drains the commit).
  bool ok = mbar_wait(done, 0, status, abort_flag);
  if (!ok) {
    const long long t0 = clock64();
    while (!mbar_try_wait(done, 0) && clock64() - t0 < WAIT_CYCLES) {
    }
  }
  tc_fence_after();
  // tcgen05.ld is warp-collective: take the decision per warp.
  if (__all_sync(0xffffffffu, ok && !*abort_flag)) {
    const int row = warp * 32 + lane;  // TMEM lane = tile row
    float* out = partial + (int64_t)blockIdx.x * TM * TM + (int64_t)row * TM;
#pragma unroll 1
    for (int c = 0; c < TM; c += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
#pragma unroll
      for (int i = 0; i < 32; i += 4)
        *reinterpret_cast<float4*>(out + c + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u)
                 : "memory");
  }
}

// M[r][c] (r >= c, lower triangle) = sum over the chunks of tile pair (r/128, c/128), in chunk
// order, in FP64; mirrored to M[c][r].
__global__ void gram_reduce_kernel(const float* __restrict__ partial,
                                   const int* __restrict__ pair_first,
                                   const int* __restrict__ pair_count, int stride, int rows,
                                   double* __restrict__ M) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)rows * rows) return;
  const int r = (int)(t / rows), c = (int)(t % rows);
  if (c > r) return;
  const int ti = r / TM, tj = c / TM;
  const int pr = ti * (ti + 1) / 2 + tj;
  const int rr = r - ti * TM, cc = c - tj * TM;
  double s = 0.0;
  const int j0 = pair_first[pr], nj = pair_count[pr];
  for (int j = 0; j < nj; ++j)
    s += (double)partial[((int64_t)j0 + (int64_t)j * stride) * TM * TM + rr * TM + cc];
  M[(int64_t)r * rows + c] = s;
  M[(int64_t)c * rows + r] = s;
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

int make_map(CUtensorMap* m, const __nv_bfloat16* base, int rows, int64_t ld) {
  auto enc = get_encode();
  if (!enc) {
    set_error_detail("cuTensorMapEncodeTiled is not available from the driver");
    return TUCKER_ECUDA;
  }
  cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)TM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error_detail("cuTensorMapEncodeTiled rejected the Gram operand layout");
    return TUCKER_ECUDA;
  }
  return TUCKER_OK;
}

}  // namespace

int64_t gram_ld(int64_t K) { return (K + TK - 1) / TK * TK; }

int gram_bf16x3(int rows, int nterms, const GramTerm* terms, double* M, cudaStream_t s) {
  if (rows <= 0) return TUCKER_OK;
  if (nterms < 1 || nterms > 2) return TUCKER_EINVAL;
  TermMaps maps;
  memset(&maps, 0, sizeof(maps));
  int64_t Ktot = 0;
  for (int t = 0; t < nterms; ++t) {
    if (terms[t].ld % TK != 0 || terms[t].K > terms[t].ld) return TUCKER_EINVAL;
    TK_TRY(make_map(&maps.hi[t], terms[t].hi, rows, terms[t].ld));
    TK_TRY(make_map(&maps.lo[t], terms[t].lo, rows, terms[t].ld));
    Ktot += terms[t].K;
  }
  const int nt = ceil_div(rows, TM);
  const int npairs = nt * (nt + 1) / 2;
  // K chunk: multiple of 64, at most 4096, small enough to give about two jobs per SM.
  int64_t chunk = (Ktot * npairs) / (2 * (int64_t)num_sms());
  chunk = (chunk + TK - 1) / TK * TK;
  if (chunk < 4 * TK) chunk = 4 * TK;
  if (chunk > KCHUNK_MAX) chunk = KCHUNK_MAX;
  // Jobs in chunk-major order: the CTAs that run together work on the same K range of every
  // tile pair, so each row tile's chunk comes from DRAM once and is re-read from L2 by the
  // other pairs (a 1000-row chunk of hi + lo is 16 MB).  Job c * npairs + pr is chunk c of
  // pair pr; the reduction adds a pair's chunks in chunk order.
  std::vector<Job> jobs;
  std::vector<int> first(npairs), count(npairs);
  int nchunks = 0;
  for (int t = 0; t < nterms; ++t)
    for (int64_t k0 = 0; k0 < terms[t].K; k0 += chunk, ++nchunks) {
      const int64_t k1 = std::min<int64_t>(terms[t].K, k0 + chunk);
      for (int ti = 0; ti < nt; ++ti)
        for (int tj = 0; tj <= ti; ++tj)
          jobs.push_back(Job{ti, tj, t, (int)k0, (int)((k1 - k0 + TK - 1) / TK)});
    }
  for (int pr = 0; pr < npairs; ++pr) {
    first[pr] = pr;
    count[pr] = nchunks;
  }
  const int64_t njobs = (int64_t)jobs.size();
  const double flops = 2.0 * 3.0 * (double)Ktot * TM * TM * npairs;
  ProfScope prof("gram_bf16x3", s, (double)rows * (rows + 1) * (double)Ktot,
                 4.0 * rows * (double)Ktot + 8.0 * rows * rows);
  (void)flops;
  Buf djobs, dfirst, dcount, part, st;
  TK_TRY(djobs.alloc(sizeof(Job) * njobs, s));
  TK_TRY(dfirst.alloc(sizeof(int) * npairs, s));
  TK_TRY(dcount.alloc(sizeof(int) * npairs, s));
  TK_TRY(part.alloc(sizeof(float) * (size_t)njobs * TM * TM, s));
  TK_TRY(st.alloc(sizeof(int), s));
  TK_CUDA(cudaMemcpyAsync(djobs.p, jobs.data(), sizeof(Job) * njobs, cudaMemcpyHostToDevice, s));
  TK_CUDA(cudaMemcpyAsync(dfirst.p, first.data(), sizeof(int) * npairs, cudaMemcpyHostToDevice, s));
  TK_CUDA(cudaMemcpyAsync(dcount.p, count.data(), sizeof(int) * npairs, cudaMemcpyHostToDevice, s));
  TK_CUDA(cudaMemsetAsync(st.p, 0, sizeof(int), s));
  static const cudaError_t attr = cudaFuncSetAttribute(
      gram_bf16x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  TK_CUDA(attr);
  gram_bf16x3_kernel<<<(unsigned)njobs, 128, SMEM_BYTES, s>>>(maps, djobs.as<Job>(),
                                                               part.as<float>(), st.as<int>());
  TK_LAUNCH();
  gram_reduce_kernel<<<ceil_div((int64_t)rows * rows, 256), 256, 0, s>>>(
      part.as<float>(), dfirst.as<int>(), dcount.as<int>(), npairs, rows, M);
  TK_LAUNCH();
  int h = 0;
  TK_CUDA(cudaMemcpyAsync(&h, st.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  if (h & DEV_TIMEOUT) {
    set_error_detail("tensor-core Gram: a bounded wait on an mbarrier gave up");
    return TUCKER_ETIMEOUT;
  }
  return TUCKER_OK;
}

}  // namespace tk
