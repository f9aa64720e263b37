// Fused slice projection and tensor-core Gram for the mixed form of SP and MP (Figures sp3,
// mp3): M = sum_terms Gram((X x_m U_m^T)_(n)) without writing the projection Y to memory.
//
// A Gram tile needs two row tiles of Y; when each CTA builds the Y rows it needs in shared
// memory, a mode with nt row tiles rebuilds every row nt times.  For modes of at most 256 rows
// (two row tiles: the batched workload's tensors, 30..300 per mode) one CTA holds all rows of a
// K chunk, so nothing is built twice:
//   * a CTA owns one term and a range of K stages of 64 columns (column c = i_o J_m + p);
//   * 8 producer warps build each stage of Y: warp w takes rows w, w + 8, ..., lane l columns
//     l and l + 32; entry (a, c) sums x U_m[i_m, p] over the leaves of fiber (a, i_o), found
//     through the ordering's dense fiber map (no fiber: zero); the FP32 value is split into
//     BF16 hi + lo and stored in the 128-byte-swizzled K-major layout the MMA reads, two stages
//     in flight;
//   * one thread issues the BF16x3 MMAs (hi hi^T + hi lo^T + lo hi^T, M = N = 128, K = 16) for
//     the tile pairs (0,0), (1,0), (1,1) into tensor memory (FP32), accumulating over the CTA's
//     K range;
//   * the CTA writes its FP32 tiles; a reduction adds the CTAs' tiles in FP64 in a fixed order
//     and mirrors the lower triangle (bitwise reproducible, exactly symmetric).
// Waits are bounded: on a timeout the kernel records DEV_TIMEOUT, drains and returns.
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "tc_ptx.cuh"

namespace tk {

namespace {

constexpr int TM = 128, TKF = 64, FSTAGES = 2, PROD_WARPS = 8;
constexpr int FTHREADS = 32 * (PROD_WARPS + 1);         // warp 0 MMA, warps 1..8 producers
constexpr int TILE_BYTES = TM * TKF * 2;                 // 16 KB: 128 rows x 64 BF16
constexpr int FSTAGE_BYTES = 4 * TILE_BYTES;             // hi and lo of two row tiles
constexpr int FSMEM_BYTES = FSTAGES * FSTAGE_BYTES + 1024 + 256;
constexpr uint32_t IDESC = tc::idesc_bf16(128, 128);

struct FusedTerm {
  const int32_t* fiber_map;   // [I_n x I_o] fiber id of (i_n, i_o) or -1
  const int64_t* fiber_ptr;
  const int32_t* leaf_idx;    // i_m
  const float* val;
  const float* Um;            // I_m x J_m, row stride ldm
  int64_t ldm;
  int Jm;
  int64_t Io;
  int64_t nst;                // stages of 64 columns: ceil(I_o J_m / 64)
};

struct FusedArgs {
  FusedTerm term[2];
  int rows, nt;               // rows of M (<= 256), row tiles (1 or 2)
  int chunk;                  // stages per CTA
  int jobs_t0;                // CTAs of term 0 (the rest belong to term 1)
};

// Byte offset of element (r, k) (r < 128, k < 64) in a 128 x 64 BF16 tile, K-major, 128-byte
// swizzle: 8-row groups of 1024 bytes, 16-byte chunks XORed with the row within the group.
__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
  const int kb = k * 2;
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((kb >> 4) ^ (r & 7)) & 7) << 4) +
                    (kb & 15));
}

__global__ void __launch_bounds__(FTHREADS, 1)
gram_fused_kernel(const __grid_constant__ FusedArgs args, float* __restrict__ partial,
                  int* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + FSTAGES * FSTAGE_BYTES);
  uint64_t* empty = full + FSTAGES;
  uint64_t* done = empty + FSTAGES;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  const int tsel = blockIdx.x < (unsigned)args.jobs_t0 ? 0 : 1;
  const FusedTerm& T = args.term[tsel];
  const int64_t jb = tsel == 0 ? blockIdx.x : blockIdx.x - args.jobs_t0;
  const int64_t s0 = jb * args.chunk;
  const int ns = (int)min64(args.chunk, T.nst - s0);
  const int nt = args.nt, npair = nt * (nt + 1) / 2;

  if (threadIdx.x == 0) {
    for (int s = 0; s < FSTAGES; ++s) {
      tc::mbar_init(&full[s], PROD_WARPS * 32);   // every producer thread arrives
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, 512);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- MMA issuer ----------------------------------------------------------------------
      for (int j = 0; j < ns; ++j) {
        const int s = j % FSTAGES;
        if (!tc::mbar_wait(&full[s], (j / FSTAGES) & 1, status, abort_flag)) break;
        tc::fence_after();
        const uint8_t* st = smem + s * FSTAGE_BYTES;
        // tile layout in a stage: hi0, lo0, hi1, lo1
        for (int p = 0; p < npair; ++p) {
          const int ti = p == 0 ? 0 : 1, tj = p == 2 ? 1 : 0;
          const uint64_t ah = tc::sw_desc(st + (2 * ti) * TILE_BYTES, 128);
          const uint64_t al = tc::sw_desc(st + (2 * ti + 1) * TILE_BYTES, 128);
          const uint64_t bh = tc::sw_desc(st + (2 * tj) * TILE_BYTES, 128);
          const uint64_t bl = tc::sw_desc(st + (2 * tj + 1) * TILE_BYTES, 128);
          const uint32_t d = tmem + (uint32_t)(p * 128);
#pragma unroll
          for (int kk = 0; kk < TKF / 16; ++kk) {
            const uint64_t off = (uint64_t)(kk * 32) >> 4;
            tc::mma_bf16<IDESC>(d, ah + off, bh + off, (j | kk) ? 1u : 0u);
            tc::mma_bf16<IDESC>(d, ah + off, bl + off, 1u);
            tc::mma_bf16<IDESC>(d, al + off, bh + off, 1u);
          }
        }
        tc::mma_commit(&empty[s]);
      }
      tc::mma_commit(done);
    }
  } else {
    // ---- producers: Y tiles in shared memory ---------------------------------------------
    const int pw = warp - 1;
    for (int j = 0; j < ns; ++j) {
      const int s = j % FSTAGES;
      if (j >= FSTAGES && !tc::mbar_wait(&empty[s], ((j / FSTAGES) - 1) & 1, status, abort_flag))
        break;
      uint8_t* st = smem + s * FSTAGE_BYTES;
      const int64_t k0 = (s0 + j) * TKF;
      for (int r = pw; r < nt * TM; r += PROD_WARPS) {
        const int ti = r >> 7, rr = r & 127;
        uint8_t* th = st + (2 * ti) * TILE_BYTES;
        uint8_t* tl = th + TILE_BYTES;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          const int kc = lane + 32 * half;
          const int64_t c = k0 + kc;
          float y = 0.f;
          if (r < args.rows && c < T.Io * T.Jm) {
            const int64_t io = c / T.Jm;
            const int p = (int)(c - io * T.Jm);
            const int32_t f = T.fiber_map[(int64_t)r * T.Io + io];
            if (f >= 0)
              for (int64_t l = T.fiber_ptr[f]; l < T.fiber_ptr[f + 1]; ++l)
                y = fmaf(T.val[l], T.Um[(int64_t)T.leaf_idx[l] * T.ldm + p], y);
          }
          const __nv_bfloat16 h = __float2bfloat16_rn(y);
          const __nv_bfloat16 lo = __float2bfloat16_rn(y - __bfloat162float(h));
          const uint32_t off = sw128_off(rr, kc);
          *reinterpret_cast<__nv_bfloat16*>(th + off) = h;
          *reinterpret_cast<__nv_bfloat16*>(tl + off) = lo;
        }
      }
      // make this thread's generic-proxy stores visible to the tensor cores, then report
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc::mbar_arrive(&full[s]);
    }
  }
  __syncwarp();
  if (!tc::mbar_wait(done, 0, status, abort_flag)) tc::mbar_drain(done, 0);
  tc::fence_after();
  // ---- epilogue: warps 1..4 (one per TMEM lane quarter) write the FP32 tiles ------------------
  if (warp >= 1 && warp <= 4 && __all_sync(0xffffffffu, !*abort_flag) && ns > 0) {
    const int q = warp & 3;
    const int row = q * 32 + lane;
    for (int p = 0; p < npair; ++p) {
      float* out = partial + ((int64_t)blockIdx.x * npair + p) * TM * TM + (int64_t)row * TM;
#pragma unroll 1
      for (int c = 0; c < TM; c += 32) {
        uint32_t v[32];
        tc::tmem_ld32_raw(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(p * 128 + c), v);
#pragma unroll
        for (int i = 0; i < 32; i += 4)
          *reinterpret_cast<float4*>(out + c + i) =
              make_float4(__uint_as_float(v[i]), __uint_as_float(v[i + 1]),
                          __uint_as_float(v[i + 2]), __uint_as_float(v[i + 3]));
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

// M[r][c] (r >= c) = sum over the CTAs, in CTA order, of their tile (r / 128, c / 128), in FP64;
// mirrored.  A CTA with no stages wrote nothing and is skipped.
__global__ void gram_fused_reduce(const float* __restrict__ partial, int njobs, int nt, int rows,
                                  const int* __restrict__ job_ns, double* __restrict__ M) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)rows * rows) return;
  const int r = (int)(t / rows), c = (int)(t % rows);
  if (c > r) return;
  const int ti = r / TM, tj = c / TM;
  const int p = ti == 0 ? 0 : (tj == 0 ? 1 : 2);
  const int npair = nt * (nt + 1) / 2;
  const int rr = r - ti * TM, cc = c - tj * TM;
  double s = 0.0;
  for (int j = 0; j < njobs; ++j)
    if (job_ns[j] > 0) s += (double)partial[((int64_t)j * npair + p) * TM * TM + rr * TM + cc];
  M[(int64_t)r * rows + c] = s;
  M[(int64_t)c * rows + r] = s;
}

}  // namespace

int gram_fused_mixed(const tucker_tensor_s* X, int n, int nterms, const Ordering* const ord[2],
                     const float* const Um[2], const int64_t ldm[2], const int Jm[2], double* M,
                     cudaStream_t s) {
  const int rows = (int)X->dims[n];
  if (rows < 1 || rows > FUSED_GRAM_MAX_ROWS || nterms < 1 || nterms > 2) return TUCKER_EINVAL;
  FusedArgs a;
  memset(&a, 0, sizeof(a));
  a.rows = rows;
  a.nt = rows > TM ? 2 : 1;
  int64_t nst_max = 0, Ktot = 0, nnz = 0;
  for (int t = 0; t < nterms; ++t) {
    const Ordering* o = ord[t];
    FusedTerm& T = a.term[t];
    T.fiber_map = o->fiber_map;
    T.fiber_ptr = o->fiber_ptr;
    T.leaf_idx = o->leaf_idx;
    T.val = o->val_f32;
    T.Um = Um[t];
    T.ldm = ldm[t];
    T.Jm = Jm[t];
    T.Io = X->dims[o->m];   // ordering (n, o, m): the middle mode indexes the slices
    T.nst = (T.Io * T.Jm + TKF - 1) / TKF;
    nst_max = std::max(nst_max, T.nst);
    Ktot += T.Io * T.Jm;
    nnz += X->nnz;
  }
  // Stages per CTA: about two CTAs per SM over both terms, at least 4 stages each.
  int64_t stages = 0;
  for (int t = 0; t < nterms; ++t) stages += a.term[t].nst;
  a.chunk = (int)std::max<int64_t>(4, (stages + 2 * num_sms() - 1) / (2 * num_sms()));
  const int j0 = (int)((a.term[0].nst + a.chunk - 1) / a.chunk);
  const int j1 = nterms == 2 ? (int)((a.term[1].nst + a.chunk - 1) / a.chunk) : 0;
  a.jobs_t0 = j0;
  const int njobs = j0 + j1;
  const int npair = a.nt * (a.nt + 1) / 2;
  std::vector<int> ns(njobs);
  for (int j = 0; j < njobs; ++j) {
    const int t = j < j0 ? 0 : 1;
    const int64_t jb = t == 0 ? j : j - j0;
    ns[j] = (int)std::max<int64_t>(0, std::min<int64_t>(a.chunk, a.term[t].nst - jb * a.chunk));
  }
  ProfScope prof("gram_fused", s, (double)rows * (rows + 1) * (double)Ktot,
                 16.0 * nnz + 8.0 * rows * (double)rows);
  Buf part, dns, st;
  TK_TRY(part.alloc(sizeof(float) * (size_t)njobs * npair * TM * TM, s));
  TK_TRY(dns.alloc(sizeof(int) * njobs, s));
  TK_TRY(st.alloc(sizeof(int), s));
  TK_CUDA(cudaMemcpyAsync(dns.p, ns.data(), sizeof(int) * njobs, cudaMemcpyHostToDevice, s));
  TK_CUDA(cudaMemsetAsync(st.p, 0, sizeof(int), s));
  static const cudaError_t attr = cudaFuncSetAttribute(
      gram_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, FSMEM_BYTES);
  TK_CUDA(attr);
  gram_fused_kernel<<<njobs, FTHREADS, FSMEM_BYTES, s>>>(a, part.as<float>(), st.as<int>());
  TK_LAUNCH();
  gram_fused_reduce<<<ceil_div((int64_t)rows * rows, 256), 256, 0, s>>>(
      part.as<float>(), njobs, a.nt, rows, dns.as<int>(), M);
  TK_LAUNCH();
  int h = 0;
  TK_CUDA(cudaMemcpyAsync(&h, st.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  if (h & DEV_TIMEOUT) {
    set_error_detail("fused tensor-core Gram: a bounded wait on an mbarrier gave up");
    return TUCKER_ETIMEOUT;
  }
  return TUCKER_OK;
}

}  // namespace tk
