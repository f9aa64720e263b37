// FP64-accurate matrix products on the BF16 tensor cores.  The GB300's FP64 rate is about
// 1.25 TFLOP/s; the products of this file reach FP64 accuracy on the BF16 tensor pipe by
// error-free splitting (the scheme of Ozaki, Ogita, Oishi and Rump, "Error-free transformations
// of matrix multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012).  They serve the FP64 Gram of the projections
// (the "U_(1) U_(1)^T" and slice-sum matrices of Figures hooi3, sp3, mp3) and the eigensolver's
// products with M.
//
//   * every row i of an operand (a row of A, or a column of B for A B) is scaled by a power of
//     two, u = y 2^-e_i with |u| < 1/2, and cut into S integer slices of 8 bits,
//     u = sum_s q_s 2^(-8(s+1)) + r with |q_s| <= 128 and |r| <= 2^-(8S+1) (each q_s exact in
//     BF16).  S = 6 (48 bits) for the Grams and the HOOI projection, S = 7 (56 bits) for the
//     eigensolver's products, whose rows can be dominated by a single entry, and S = 3 (24
//     bits, FP32-class) for the mixed form's filter products;
//   * u_i . v_j = 2^-16 sum_d L_d 2^(-8d), with the level sums L_d = sum_{s+t=d} q_s(i).q_t(j)
//     kept for d < S (S (S + 1) / 2 slice pairs).  For even S the first dropped level holds
//     the square pair (S/2, S/2), whose products q_s(k)^2 on a Gram's diagonal do not average
//     out: that one pair is kept as a level of its own (22 pairs for S = 6, 28 for S = 7).  The
//     remaining dropped pairs (products of different digits, zero on average) and r contribute
//     about 2^-(8S-1) per term;
//   * each level has its own FP32 accumulator in tensor memory.  Its products are integers of
//     at most 2^14, and a level is read out after at most 1024 / (d + 1) K columns, so every
//     partial sum is an integer of at most 2^24 and the FP32 accumulation is exact;
//   * the level chunks are read out on a staggered schedule (at most two levels per K stage,
//     while the tensor pipe works on the others), converted to integers and summed in 64-bit
//     integer registers: hi = sum_{d<=3} L_d 2^(8(3-d)), lo = sum_{d>=4} L_d 2^(8(6-d)).  The
//     integer sums are exact, so the result does not depend on the order of the K chunks;
//   * a reduction kernel adds the K splits' integer partials, scales them back to FP64 and
//     applies the epilogue alpha C + beta X + gamma Z.
//
// Two kernels.  A tcgen05.mma instruction costs about the same for N = 64 and N = 128 (its
// issue, not the tensor pipe, sets the rate), so the long symmetric Grams use 128 x 128 tiles
// (wk::): tensor memory then holds only four level accumulators of 128 columns, and the levels
// run in two passes over the job's K range (levels 0-3 from slices 0-3, then the lower levels
// from all slices; 16 epilogue warps, 32 columns each).  The other products (the eigensolver's,
// whose B has ~150 columns, and the per-slice HOOI products with few stages each) use 128 x 64
// tiles in one pass (nk::), described below.
//
// Layout (nk::): one CTA computes a 128 x 64 tile (rows of A = tile ti of 128 rows, rows of B^T =
// tile tj of 64 rows; for a symmetric product only tj <= 2 ti + 1, the lower triangle) over a
// range of K stages of 32 columns.  Warp 0 streams all S slices of A (128 x 32) and B (64 x 32)
// of a stage with two 3-D TMA loads (64-byte swizzle) through a 6-stage (S = 3), 3-stage (S = 6)
// or 2-stage (S = 7) ring; warps 1 and 2 issue the 12, 44 or 56 MMAs of a stage (M = 128,
// N = 64, K = 16, kind::f16), each for its own levels; warps 3-10 read the level accumulators
// out.  Every wait is bounded: on a timeout
// the kernel records DEV_TIMEOUT, drains and returns.
#include <cudaTypedefs.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "tc_ptx.cuh"

namespace tk {

namespace {

constexpr int BETA = 8;                              // bits per slice
constexpr int TM = 128, KS = 32;
// Issuing a tcgen05.mma costs its thread about 100 cycles -- three times what an M = 128, N = 64
// MMA takes on the tensor pipe, and about the same for N = 128 -- so the levels are split between
// NMMA issuing warps (balanced by slice pairs), each committing its own MMAs, and long products
// use N = 128.
constexpr int NMMA = 2;
// Lowest level kept for nslice slices (the lo sum is scaled by 2^-8 LT).
__host__ __device__ constexpr int oz_lowest_level(int nslice) {
  return nslice % 2 == 0 ? nslice : nslice - 1;
}
// Stages per K split or per batched job: at most 2^19 (2^24 columns), so that the integer
// sums of a job, |hi| <= K 2^14 (2^24 + 2^17 + 3 2^8 + 4), stay below 2^63.
constexpr int MAX_JOB_STAGES = 1 << 19;

// Grid geometry: CTA b computes tile pair b % npairs over K split b / npairs.  Tiles are
// 128 x tn (tn = 64 or 128).  Tile pairs are numbered row by row: (ti, tj) -> ti * ntj + tj, or
// for a symmetric product (the lower triangle: tj <= 2 ti + 1 when tn = 64, every row but
// possibly the last holding 2 ti + 2 pairs; tj <= ti when tn = 128) ti (ti + 1) + tj or
// ti (ti + 1) / 2 + tj.
struct Grid {
  int ntj, npairs, nsplit, nst;
  int sym;
  int tn;
  // Batched products (one product per slice, each over its own stage range): CTA b computes
  // tile pair b % npairs of slice b / npairs over stages [stage_start[i], stage_start[i + 1]).
  const int* stage_start;
};

struct Job {
  int ti, tj;   // 128-row tile of A, tn-row tile of B^T
  int s0, ns;   // first K stage and number of stages
};

__host__ __device__ inline void pair_tiles(const Grid& g, int p, int* ti, int* tj) {
  if (!g.sym) {
    *ti = p / g.ntj;
    *tj = p % g.ntj;
    return;
  }
  const int f = g.tn == 64 ? 2 : 1;   // row t starts at f t (t + 1) / 2
  int t = (int)((sqrt(8.0 / f * (double)p + 1.0) - 1.0) * 0.5);
  while (f * t * (t + 1) / 2 > p) --t;
  while (f * (t + 1) * (t + 2) / 2 <= p) ++t;
  *ti = t;
  *tj = p - f * t * (t + 1) / 2;
}

__host__ __device__ inline int pair_index(const Grid& g, int ti, int tj) {
  return g.sym ? (g.tn == 64 ? ti * (ti + 1) : ti * (ti + 1) / 2) + tj : ti * g.ntj + tj;
}

__device__ inline Job job_of(const Grid& g, int b) {
  Job j;
  if (g.stage_start) {
    const int i = b / g.npairs, p = b % g.npairs;
    j.ti = p / g.ntj;
    j.tj = p % g.ntj;
    j.s0 = g.stage_start[i];
    j.ns = g.stage_start[i + 1] - j.s0;
    return j;
  }
  const int z = b / g.npairs, p = b % g.npairs;
  pair_tiles(g, p, &j.ti, &j.tj);
  j.s0 = (int)((int64_t)g.nst * z / g.nsplit);
  j.ns = (int)((int64_t)g.nst * (z + 1) / g.nsplit) - j.s0;
  return j;
}

// ---- 128 x 64 tiles, one pass: every level has a 64-column accumulator in tensor memory ------
namespace nk {
constexpr int TN = 64;
constexpr int NTHREADS = 32 * (1 + NMMA + 8);   // warp 0 TMA, warps 1..NMMA MMA, then 8 epilogue
constexpr uint32_t IDESC = tc::idesc_bf16(TM, TN);

// Ring geometry for S slices per operand (S levels, S (S + 1) / 2 slice pairs): one stage holds
// all S slices of A (S x 8 KB) and of B (S x 4 KB); 3 stages for S <= 6 (221 KB), else 2.
// S <= 7: 7 levels x 64 columns fit in tensor memory, and 8 S bits fit the 64-bit split.
template <int S>
struct Geo {
  static_assert(S == 3 || (S >= 5 && S <= 7), "3 or 5 to 7 slices per operand");
  static constexpr int A_BYTES = S * TM * KS * 2;
  static constexpr int B_BYTES = S * TN * KS * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int NSTAGE = S <= 3 ? 6 : S <= 6 ? 3 : 2;
  static constexpr int SMEM_BYTES = NSTAGE * STAGE_BYTES + 1024 + 512;
  // Levels: d < S, plus for even S a level S holding the one pair (S/2, S/2) (see the file
  // comment); the lowest level is 6 for S = 6 and S = 7.
  static constexpr int NL = S % 2 == 0 ? S + 1 : S;
  static constexpr int PAIRS = S * (S + 1) / 2 + (S % 2 == 0 ? 1 : 0);
};

// Readout schedule of level d: its accumulator restarts at local stage j > 0 when
// j % CHUNK[d] == RESIDUE[d].  A chunk spans at most CHUNK[d] stages of 32 columns, and
// (d + 1) CHUNK[d] <= 32, so a chunk sums at most 32 x 32 products of magnitude <= 2^14: |L| <= 2^24,
// every partial sum is an integer that FP32 holds exactly.  The residues spread the readouts
// (at most two levels restart at one stage).
__host__ __device__ constexpr int level_chunk(int d) {
  return d == 0 ? 32 : d == 1 ? 16 : d <= 3 ? 8 : 4;
}
__host__ __device__ constexpr int level_residue(int d) {
  return d == 0 ? 0 : d == 1 ? 8 : d == 2 ? 2 : d == 3 ? 6 : d == 4 ? 1 : d == 5 ? 3 : 0;
}
// Issuing warp (0 .. NMMA - 1) of level d: pair counts per level are 1, 2, ..., S (and 1 for
// the square-pair level of an even S); the two halves hold 11 + 11 (S = 6), 14 + 14 (S = 7) and
// 3 + 3 (S = 3) pairs.
template <int S>
__host__ __device__ constexpr int level_owner(int d) {
  return S == 6 ? ((d == 4 || d == 5) ? 1 : 0)
       : S == 7 ? ((d == 0 || d == 5 || d == 6) ? 0 : 1)
                : (d == 2 ? 1 : 0);
}
__device__ __forceinline__ bool restarts(int d, int j) {
  return j > 0 && j % level_chunk(d) == level_residue(d);
}
// Bit d set: level d restarts at local stage j (the chunks are powers of two).
template <int S>
__device__ __forceinline__ uint32_t restart_mask(int j) {
  uint32_t m = 0;
  if (j > 0) {
#pragma unroll
    for (int d = 0; d < Geo<S>::NL; ++d)
      if ((j & (level_chunk(d) - 1)) == level_residue(d)) m |= 1u << d;
  }
  return m;
}

template <int S>
__global__ void __launch_bounds__(NTHREADS, 1)
gram_ozaki_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                  const Grid grid, long long* __restrict__ partial, int* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int STAGES = Geo<S>::NSTAGE, NL = Geo<S>::NL, LT = NL - 1;
  uint64_t* full = (uint64_t*)(smem + STAGES * Geo<S>::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;   // [NL] a level's chunk is complete in TMEM
  uint64_t* acc_free = acc_full + NL;    // [NL] the epilogue has read it
  uint64_t* done = acc_free + NL;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Job job = job_of(grid, blockIdx.x);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], NMMA);   // one commit per issuing warp
    }
    for (int d = 0; d < NL; ++d) {
      tc::mbar_init(&acc_full[d], 1);
      tc::mbar_init(&acc_free[d], 8);   // one arrival per epilogue warp
    }
    tc::mbar_init(done, NMMA);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, 512);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: all slices of A and B for one K stage per ring slot ------------------
    int issued = 0;
    for (int j = 0; j < job.ns; ++j) {
      const int s = j % STAGES;
      if (j >= STAGES && !tc::mbar_wait(&empty[s], ((j / STAGES) - 1) & 1, status, abort_flag))
        break;
      uint8_t* st = smem + s * Geo<S>::STAGE_BYTES;
      tc::mbar_expect_tx(&full[s], Geo<S>::STAGE_BYTES);
      const int kx = (job.s0 + j) * KS;
      tc::tma_load_3d(st, &mapA, &full[s], kx, job.ti * TM, 0);
      tc::tma_load_3d(st + Geo<S>::A_BYTES, &mapB, &full[s], kx, job.tj * TN, 0);
      ++issued;
    }
    if (*abort_flag)
      for (int j = issued > STAGES ? issued - STAGES : 0; j < issued; ++j)
        tc::mbar_drain(&full[j % STAGES], (j / STAGES) & 1);
  } else if (warp >= 1 && warp <= NMMA && lane == 0) {
    const int mi = warp - 1;   // this thread issues the levels d with level_owner<S>(d) == mi
    // ---- MMA issuer ----------------------------------------------------------------------------
    uint32_t free_phase = 0;   // bit d: parity of the next acc_free[d] phase to wait for
    bool ok = true;
    for (int j = 0; j < job.ns && ok; ++j) {
      const int s = j % STAGES;
      if (!tc::mbar_wait(&full[s], (j / STAGES) & 1, status, abort_flag)) break;
      tc::fence_after();
      const uint8_t* st = smem + s * Geo<S>::STAGE_BYTES;
      // Slice q of A (B) starts q * 8 KB (4 KB) after slice 0: descriptor address field + q *
      // bytes / 16 (the whole ring lies below 256 KB, so the 14-bit field does not overflow).
      const uint64_t da0 = tc::sw_desc(st, 64), db0 = tc::sw_desc(st + Geo<S>::A_BYTES, 64);
      constexpr uint64_t DA = (TM * KS * 2) >> 4, DB = (TN * KS * 2) >> 4;
      const uint32_t rm = restart_mask<S>(j);
      const uint32_t fresh = j == 0 ? 0xFFFFu : rm;
      // Levels that keep accumulating first, then the restarting ones (their accumulators
      // must first have been read out).  Fully unrolled: the issuing thread spends a few
      // instructions per MMA.
#pragma unroll
      for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
        for (int d = 0; d < NL; ++d) {
          if (level_owner<S>(d) != mi) continue;
          const bool rs = (rm >> d) & 1u;
          if (pass == 0 ? rs : !rs) continue;
          if (rs) {
            if (!tc::mbar_wait(&acc_free[d], (free_phase >> d) & 1u, status, abort_flag)) {
              ok = false;
              break;
            }
            free_phase ^= 1u << d;
            tc::fence_after();
          }
          const uint32_t dt = tmem + (uint32_t)(d * TN);
          const uint32_t acc0 = ((fresh >> d) & 1u) ? 0u : 1u;
#pragma unroll
          for (int kk = 0; kk < KS / 16; ++kk) {
            const uint64_t off = (uint64_t)(kk * 32) >> 4;   // 16 BF16 = 32 bytes along K
            if (d < S) {
#pragma unroll
              for (int q = 0; q <= d; ++q)
                tc::mma_bf16<IDESC>(dt, da0 + (q * DA + off), db0 + ((d - q) * DB + off),
                                    (kk == 0 && q == 0) ? acc0 : 1u);
            } else {   // level S: the pair (S/2, S/2) only
              tc::mma_bf16<IDESC>(dt, da0 + ((S / 2) * DA + off), db0 + ((S / 2) * DB + off),
                                  kk == 0 ? acc0 : 1u);
            }
          }
        }
        if (!ok) break;
      }
      if (!ok) break;
      tc::mma_commit(&empty[s]);
      const bool last = j + 1 == job.ns;
      for (int d = 0; d < NL; ++d)
        if (level_owner<S>(d) == mi && (last || restarts(d, j + 1)))
          tc::mma_commit(&acc_full[d]);
    }
    tc::mma_commit(done);   // arrives once every MMA issued above has completed
  } else if (warp > NMMA) {
    // ---- epilogue: level readouts into exact 64-bit integer sums -----------------------------
    const int q = warp & 3;              // TMEM lane quarter this warp may access
    const int h = (warp - NMMA - 1) >> 2;   // column half of the 64-column level accumulator
    long long hi[32], lo[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) hi[i] = lo[i] = 0;
    uint32_t full_phase = 0;   // bit d: parity of the next acc_full[d] phase to wait for
    bool ok = true;
    auto readout = [&](int d) {
      if (!ok) return;
      if (!tc::mbar_wait(&acc_full[d], (full_phase >> d) & 1u, status, abort_flag)) {
        ok = false;
        return;
      }
      full_phase ^= 1u << d;
      tc::fence_after();
      uint32_t r[32];
      tc::tmem_ld32_raw(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(d * TN + h * 32), r);
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acc_free[d]);
      // |L| <= 2^24 and integral: the conversion is exact.
      const int sh = d <= 3 ? BETA * (3 - d) : BETA * (LT - d);
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int v = __float2int_rn(__uint_as_float(r[i]));
        const long long w = (long long)v << sh;
        if (d <= 3)
          hi[i] += w;
        else
          lo[i] += w;
      }
    };
    for (int j = 1; j < job.ns && ok; ++j)
      for (int d = 0; d < NL; ++d)
        if (restarts(d, j)) readout(d);
    if (job.ns > 0)
      for (int d = 0; d < NL; ++d) readout(d);
    if (__all_sync(0xffffffffu, ok && !*abort_flag)) {
      const int row = q * 32 + lane;
      long long* ph = partial + (int64_t)blockIdx.x * 2 * TM * TN + (int64_t)row * TN + h * 32;
      long long* pl = ph + TM * TN;
#pragma unroll
      for (int i = 0; i < 32; i += 2) {
        *reinterpret_cast<longlong2*>(ph + i) = make_longlong2(hi[i], hi[i + 1]);
        *reinterpret_cast<longlong2*>(pl + i) = make_longlong2(lo[i], lo[i + 1]);
      }
    }
  }
  __syncwarp();
  // Nobody frees tensor memory while MMAs may still be in flight.
  if (!tc::mbar_wait(done, 0, status, abort_flag)) tc::mbar_drain(done, 0);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

}  // namespace nk

// ---- 128 x 128 tiles, two passes over K (the long Grams): four 128-column accumulators ------
namespace wk {
constexpr int TN = 128;
// 16 epilogue warps: four per TMEM lane quarter, each reading 32 columns of a 128-column slot
// (32 int64 sums per thread).
constexpr int NEPI = 16;
constexpr int NTHREADS = 32 * (1 + NMMA + NEPI);   // warp 0 TMA, warps 1..NMMA MMA, epilogue
constexpr uint32_t IDESC = tc::idesc_bf16(TM, TN);
constexpr int SLOT_COLS = TN;                    // one level accumulator: 128 FP32 columns
constexpr int RING_BYTES = 224 * 1024;

// Tensor memory holds four 128-column accumulators, so the levels run in two passes over the
// job's K range: pass 0 the levels d <= 3 (slices 0..3; levels 0..2 and slices 0..2 when S = 3),
// pass 1 the lower levels (all S slices).  A stage of a pass holds its slices of A and of B
// (8 KB each per slice); the ring of each pass fills RING_BYTES.
template <int S>
struct Geo {
  static_assert(S == 3 || (S >= 5 && S <= 7), "3 or 5 to 7 slices per operand");
  // Levels: d < S, plus for even S a level S holding the one pair (S/2, S/2) (see the file
  // comment); the lowest level is 6 for S = 6 and S = 7.
  static constexpr int NL = S % 2 == 0 ? S + 1 : S;
  static constexpr int PAIRS = S * (S + 1) / 2 + (S % 2 == 0 ? 1 : 0);
  static constexpr int NL0 = NL < 4 ? NL : 4;    // levels of pass 0
  static constexpr int NL1 = NL - NL0;           // levels of pass 1
  static constexpr int SL0 = NL0;                // slices of pass 0
  static constexpr int SL1 = S;                  // slices of pass 1
  static constexpr int SLICE_BYTES = TM * KS * 2;   // = TN * KS * 2
  static constexpr int STAGE0 = 2 * SL0 * SLICE_BYTES;
  static constexpr int STAGE1 = 2 * SL1 * SLICE_BYTES;
  static constexpr int NST0 = RING_BYTES / STAGE0 < 4 ? RING_BYTES / STAGE0 : 4;
  static constexpr int NST1 = RING_BYTES / STAGE1 < 4 ? RING_BYTES / STAGE1 : 4;
  static_assert(NST0 >= 2 && (NL1 == 0 || NST1 >= 2), "ring too small");
  static constexpr int SMEM_BYTES = RING_BYTES + 1024 + 512;
};

// Readout schedule of level d: its accumulator restarts at local stage j > 0 of its pass when
// j % CHUNK[d] == RESIDUE[d].  A chunk spans at most CHUNK[d] stages of 32 columns, and
// pairs(d) CHUNK[d] <= 32, so a chunk sums at most 32 x 32 products of magnitude <= 2^14:
// |L| <= 2^24, every partial sum is an integer that FP32 holds exactly (pairs(d) = d + 1, and 1
// for the square-pair level S of an even S).  The residues spread the restarts of a pass.
template <int S>
__host__ __device__ constexpr int level_chunk(int d) {
  return d == 0 ? 32 : d == 1 ? 16 : d <= 3 ? 8 : d <= 5 ? 4 : (S % 2 == 0 ? 32 : 4);
}
template <int S>
__host__ __device__ constexpr int level_residue(int d) {
  return d == 0 ? 8 : d == 1 ? 4 : d == 2 ? 2 : d == 3 ? 6 : d == 4 ? 1 : d == 5 ? 3 : 2;
}
// Issuing warp (0 .. NMMA - 1) of level d, balancing slice pairs within each pass: pass 0 puts
// levels {0, 3} (5 pairs) and {1, 2} (5) apart; pass 1 {4, S} (6) and {5} (6) for S = 6, {4, 5}
// (11) and {6} (7) for S = 7; S = 3 has {0, 1} (3) and {2} (3).
template <int S>
__host__ __device__ constexpr int level_owner(int d) {
  return S == 3 ? (d == 2 ? 1 : 0)
       : d <= 3 ? ((d == 0 || d == 3) ? 0 : 1)
       : S == 6 ? (d == 5 ? 1 : 0)
                : (d == 6 ? 1 : 0);
}
template <int S>
__device__ __forceinline__ bool restarts(int d, int j) {
  return j > 0 && (j & (level_chunk<S>(d) - 1)) == level_residue<S>(d);
}

// Barriers of one pass: ring full/empty, per-slot chunk complete / read out.
struct PassBars {
  uint64_t* full;
  uint64_t* empty;
  uint64_t* acc_full;
  uint64_t* acc_free;
};

template <int S>
__global__ void __launch_bounds__(NTHREADS, 1)
gram_ozaki_kernel(const __grid_constant__ CUtensorMap mapA0,
                  const __grid_constant__ CUtensorMap mapB0,
                  const __grid_constant__ CUtensorMap mapA1,
                  const __grid_constant__ CUtensorMap mapB1, const Grid grid,
                  long long* __restrict__ partial, int* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  using G = Geo<S>;
  constexpr int NL = G::NL, LT = NL - 1;
  uint64_t* bars = (uint64_t*)(smem + RING_BYTES);
  PassBars pb[2];
  pb[0].full = bars;                       // [NST0]
  pb[0].empty = pb[0].full + G::NST0;      // [NST0]
  pb[1].full = pb[0].empty + G::NST0;      // [NST1]
  pb[1].empty = pb[1].full + G::NST1;      // [NST1]
  pb[0].acc_full = pb[1].empty + G::NST1;  // [4] slots of pass 0
  pb[0].acc_free = pb[0].acc_full + 4;
  pb[1].acc_full = pb[0].acc_free + 4;     // [4] slots of pass 1
  pb[1].acc_free = pb[1].acc_full + 4;
  uint64_t* pass_free = pb[1].acc_free + 4;   // the epilogue has read pass 0 out
  uint64_t* done = pass_free + 1;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Job job = job_of(grid, blockIdx.x);

  if (threadIdx.x == 0) {
    for (int p = 0; p < 2; ++p) {
      const int nst = p == 0 ? G::NST0 : G::NST1;
      for (int s = 0; s < nst; ++s) {
        tc::mbar_init(&pb[p].full[s], 1);
        tc::mbar_init(&pb[p].empty[s], NMMA);   // one commit per issuing warp
      }
      for (int t = 0; t < 4; ++t) {
        tc::mbar_init(&pb[p].acc_full[t], 1);
        tc::mbar_init(&pb[p].acc_free[t], NEPI);   // one arrival per epilogue warp
      }
    }
    tc::mbar_init(pass_free, NEPI);
    tc::mbar_init(done, NMMA);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, 512);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: the pass's slices of A and B for one K stage per ring slot -----------
    bool ok = true;
    for (int p = 0; p < 2 && ok; ++p) {
      if (p == 1 && G::NL1 == 0) break;
      const int nst = p == 0 ? G::NST0 : G::NST1;
      const int stage_bytes = p == 0 ? G::STAGE0 : G::STAGE1;
      const int a_bytes = stage_bytes / 2;
      const CUtensorMap* mA = p == 0 ? &mapA0 : &mapA1;
      const CUtensorMap* mB = p == 0 ? &mapB0 : &mapB1;
      int issued = 0;
      for (int j = 0; j < job.ns; ++j) {
        const int s = j % nst;
        if (j >= nst &&
            !tc::mbar_wait(&pb[p].empty[s], ((j / nst) - 1) & 1, status, abort_flag)) {
          ok = false;
          break;
        }
        uint8_t* st = smem + s * stage_bytes;
        tc::mbar_expect_tx(&pb[p].full[s], stage_bytes);
        const int kx = (job.s0 + j) * KS;
        tc::tma_load_3d(st, mA, &pb[p].full[s], kx, job.ti * TM, 0);
        tc::tma_load_3d(st + a_bytes, mB, &pb[p].full[s], kx, job.tj * TN, 0);
        ++issued;
      }
      if (!ok) {
        for (int j = issued > nst ? issued - nst : 0; j < issued; ++j)
          tc::mbar_drain(&pb[p].full[j % nst], (j / nst) & 1);
        break;
      }
      // The ring is reused by the next pass with another layout: wait until the MMAs have read
      // every stage of this one.
      for (int j = job.ns > nst ? job.ns - nst : 0; j < job.ns; ++j)
        if (!tc::mbar_wait(&pb[p].empty[j % nst], (j / nst) & 1, status, abort_flag)) {
          ok = false;
          break;
        }
    }
  } else if (warp >= 1 && warp <= NMMA && lane == 0) {
    const int mi = warp - 1;   // this thread issues the levels d with level_owner<S>(d) == mi
    // ---- MMA issuers ---------------------------------------------------------------------------
    bool ok = true;
    for (int p = 0; p < 2 && ok; ++p) {
      if (p == 1 && G::NL1 == 0) break;
      const int nst = p == 0 ? G::NST0 : G::NST1;
      const int stage_bytes = p == 0 ? G::STAGE0 : G::STAGE1;
      const int d0 = p == 0 ? 0 : G::NL0, d1 = p == 0 ? G::NL0 : NL;   // levels [d0, d1)
      if (p == 1) {
        // pass 1 writes the slots pass 0's last chunks are read from
        if (!tc::mbar_wait(pass_free, 0, status, abort_flag)) break;
        tc::fence_after();
      }
      uint32_t free_phase = 0;   // bit t: parity of the next acc_free[t] phase to wait for
      for (int j = 0; j < job.ns && ok; ++j) {
        const int s = j % nst;
        if (!tc::mbar_wait(&pb[p].full[s], (j / nst) & 1, status, abort_flag)) {
          ok = false;
          break;
        }
        tc::fence_after();
        const uint8_t* st = smem + s * stage_bytes;
        // Slice q of A (B) starts q * 8 KB after the first: descriptor address field + q * 512
        // (the ring lies below 256 KB, so the 14-bit field does not overflow).
        const uint64_t da0 = tc::sw_desc(st, 64), db0 = tc::sw_desc(st + stage_bytes / 2, 64);
        constexpr uint64_t DS = G::SLICE_BYTES >> 4;
        // Levels that keep accumulating first, then the restarting ones (their slot must first
        // have been read out).
#pragma unroll
        for (int ph = 0; ph < 2; ++ph) {
#pragma unroll
          for (int d = 0; d < NL; ++d) {
            if (d < d0 || d >= d1 || level_owner<S>(d) != mi) continue;
            const bool rs = restarts<S>(d, j);
            if (ph == 0 ? rs : !rs) continue;
            const int t = d - d0;
            if (rs) {
              if (!tc::mbar_wait(&pb[p].acc_free[t], (free_phase >> t) & 1u, status,
                                 abort_flag)) {
                ok = false;
                break;
              }
              free_phase ^= 1u << t;
              tc::fence_after();
            }
            const uint32_t dt = tmem + (uint32_t)(t * SLOT_COLS);
            const uint32_t acc0 = (j == 0 || rs) ? 0u : 1u;
#pragma unroll
            for (int kk = 0; kk < KS / 16; ++kk) {
              const uint64_t off = (uint64_t)(kk * 32) >> 4;   // 16 BF16 = 32 bytes along K
              if (d < S) {
#pragma unroll
                for (int q = 0; q <= d; ++q)
                  tc::mma_bf16<IDESC>(dt, da0 + (q * DS + off), db0 + ((d - q) * DS + off),
                                      (kk == 0 && q == 0) ? acc0 : 1u);
              } else {   // level S: the pair (S/2, S/2) only
                tc::mma_bf16<IDESC>(dt, da0 + ((S / 2) * DS + off), db0 + ((S / 2) * DS + off),
                                    kk == 0 ? acc0 : 1u);
              }
            }
          }
          if (!ok) break;
        }
        if (!ok) break;
        tc::mma_commit(&pb[p].empty[s]);
        const bool last = j + 1 == job.ns;
#pragma unroll
        for (int d = 0; d < NL; ++d)
          if (d >= d0 && d < d1 && level_owner<S>(d) == mi && (last || restarts<S>(d, j + 1)))
            tc::mma_commit(&pb[p].acc_full[d - d0]);
      }
    }
    tc::mma_commit(done);   // arrives once every MMA issued above has completed
  } else if (warp > NMMA) {
    // ---- epilogue: level readouts into exact 64-bit integer sums, one pass at a time --------
    const int q = warp & 3;                   // TMEM lane quarter this warp may access
    const int c4 = (warp - NMMA - 1) >> 2;    // 32-column quarter of a 128-column slot
    const int row = q * 32 + lane;
    long long* out = partial + (int64_t)blockIdx.x * 2 * TM * TN + (int64_t)row * TN + c4 * 32;
    bool ok = true;
    for (int p = 0; p < 2; ++p) {
      long long acc[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) acc[i] = 0;
      const int d0 = p == 0 ? 0 : G::NL0, d1 = p == 0 ? G::NL0 : NL;
      uint32_t full_phase = 0;   // bit t: parity of the next acc_full[t] phase to wait for
      auto readout = [&](int d) {
        if (!ok) return;
        const int t = d - d0;
        if (!tc::mbar_wait(&pb[p].acc_full[t], (full_phase >> t) & 1u, status, abort_flag)) {
          ok = false;
          return;
        }
        full_phase ^= 1u << t;
        tc::fence_after();
        const uint32_t ta =
            tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(t * SLOT_COLS + c4 * 32);
        // |L| <= 2^24 and integral: the conversion is exact.
        const int sh = d <= 3 ? BETA * (3 - d) : BETA * (LT - d);
        uint32_t r[16];
        tc::tmem_ld16_raw(ta, r);
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[i] += (long long)__float2int_rn(__uint_as_float(r[i])) << sh;
        tc::tmem_ld16_raw(ta + 16, r);
        tc::fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&pb[p].acc_free[t]);
#pragma unroll
        for (int i = 0; i < 16; ++i)
          acc[16 + i] += (long long)__float2int_rn(__uint_as_float(r[i])) << sh;
      };
      if (!(p == 1 && G::NL1 == 0)) {
        for (int j = 1; j < job.ns && ok; ++j)
          for (int d = d0; d < d1; ++d)
            if (restarts<S>(d, j)) readout(d);
        if (job.ns > 0)
          for (int d = d0; d < d1; ++d) readout(d);
      }
      if (p == 0) {
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(pass_free);
      }
      // pass 0 gives hi = sum_{d<=3} L_d 2^(8(3-d)), pass 1 lo = sum_{d>=4} L_d 2^(8(6-d))
      if (__all_sync(0xffffffffu, ok && !*abort_flag)) {
        long long* o = out + (p == 0 ? 0 : TM * TN);
#pragma unroll
        for (int i = 0; i < 32; i += 2)
          *reinterpret_cast<longlong2*>(o + i) = make_longlong2(acc[i], acc[i + 1]);
      }
    }
  }
  __syncwarp();
  // Nobody frees tensor memory while MMAs may still be in flight.
  if (!tc::mbar_wait(done, 0, status, abort_flag)) tc::mbar_drain(done, 0);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

}  // namespace wk

// The splitting runs in integer arithmetic on the FP64 bit patterns (this part's FP64 pipe
// is far too slow for it).  A row's scale exponent e satisfies |y 2^-e| < 1/2 for every y in
// the row: e = frexp exponent of max |y| + 1, computed from the largest |y| bit pattern (for
// non-negative doubles the bit patterns order like the values).  A zero row gets OZ_ZERO_EXP
// (its slices are zero, and two such exponents still add without overflow).
constexpr int OZ_ZERO_EXP = -1100;
__device__ __forceinline__ int oz_exponent_bits(unsigned long long a) {
  if (a == 0ull) return OZ_ZERO_EXP;
  const int be = (int)(a >> 52);
  if (be > 0) return be - 1021;                 // a = 1.f 2^(be - 1023): frexp exponent be - 1022
  return (63 - __clzll((long long)a)) - 1072;   // subnormal
}
__device__ __forceinline__ unsigned long long abs_bits(double y) {
  return (unsigned long long)__double_as_longlong(y) & 0x7FFFFFFFFFFFFFFFull;
}

// Z = round(y 2^(7 S - e)) as a signed integer; |Z| <= 2^(7 S - 1) when |y| < 2^(e-1).
template <int S>
__device__ __forceinline__ long long oz_fixed(double y, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(y);
  const int be = (int)((b >> 52) & 0x7FF);
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (be > 0) m |= 1ull << 52;
  if (m == 0ull) return 0;
  const int sh = (be > 0 ? be - 1075 : -1074) + BETA * S - e;   // Z = m 2^sh
  long long z;
  if (sh >= 0)
    z = (long long)(m << sh);                      // subnormal rows only; still below 2^55
  else if (sh > -64)
    z = (long long)((m + (1ull << (-sh - 1))) >> (-sh));
  else
    z = 0;
  return (b >> 63) ? -z : z;
}

// Cuts Z into S balanced base-256 digits, Z = sum_s q_s 256^(S-1-s) with q_(S-1)..q_1 in
// [-128, 127] and |q_0| <= 128, and stores slice s (q_s as a BF16 integer) at out[s * plane].
template <int S>
__device__ __forceinline__ void oz_cut(long long z, __nv_bfloat16* out, int64_t plane) {
  int q[S];
#pragma unroll
  for (int s = S - 1; s > 0; --s) {
    const int d = (int)((z + 128) & 255) - 128;
    q[s] = d;
    z = (z - d) >> 8;                             // exact: z - d is a multiple of 256
  }
  q[0] = (int)z;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    __nv_bfloat16_raw r;
    r.x = (unsigned short)(__float_as_uint((float)q[s]) >> 16);   // exact: at most 8 bits
    out[s * plane] = r;
  }
}

// Row exponents of [A | A2] (A: rows x K1, ld lda; A2: rows x K2, ld lda2): one block per row.
__global__ void oz_scale_rows(const double* __restrict__ A, int64_t lda, int64_t K1,
                              const double* __restrict__ A2, int64_t lda2, int64_t K2,
                              int* __restrict__ ex) {
  __shared__ unsigned long long ws[8];
  const int r = blockIdx.x;
  unsigned long long m = 0ull;
  for (int64_t k = threadIdx.x; k < K1; k += blockDim.x) {
    const unsigned long long a = abs_bits(A[(int64_t)r * lda + k]);
    m = a > m ? a : m;
  }
  for (int64_t k = threadIdx.x; k < K2; k += blockDim.x) {
    const unsigned long long a = abs_bits(A2[(int64_t)r * lda2 + k]);
    m = a > m ? a : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t > m ? t : m;
  }
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0ull;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = ws[w] > t ? ws[w] : t;
    ex[r] = oz_exponent_bits(t);
  }
}

// Slices of the rows of [A | A2]: Q[s][r][k], r < rows_pad, k < ldK; columns [0, K1) from A,
// [K1p, K1p + K2) from A2 (K1p = K1 rounded up to a stage), zero elsewhere.  Each thread cuts
// 4 consecutive columns.
template <int S>
__global__ void oz_split_rows_kernel(int rows, int rows_pad, const double* __restrict__ A,
                                     int64_t lda, int64_t K1, int64_t K1p,
                                     const double* __restrict__ A2, int64_t lda2, int64_t K2,
                                     int64_t ldK, const int* __restrict__ ex,
                                     __nv_bfloat16* __restrict__ Q) {
  const int64_t quads = ldK / 4;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)rows_pad * quads) return;
  const int r = (int)(t / quads);
  const int64_t k0 = (t % quads) * 4;
  const int e = r < rows ? ex[r] : 0;
  const int64_t plane = (int64_t)rows_pad * ldK;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t k = k0 + i;
    double y = 0.0;
    if (r < rows) {
      if (k < K1)
        y = A[(int64_t)r * lda + k];
      else if (k >= K1p && k - K1p < K2)
        y = A2[(int64_t)r * lda2 + (k - K1p)];
    }
    oz_cut<S>(oz_fixed<S>(y, e), Q + (int64_t)r * ldK + k, plane);
  }
}

// Column exponents of B (K x cols, ld ldb): blocks of 32 columns x 256 rows, combined with
// atomicMax (ex starts at INT_MIN).
__global__ void oz_scale_cols(const double* __restrict__ B, int64_t ldb, int64_t K, int cols,
                              int* __restrict__ ex) {
  const int c = blockIdx.x * 32 + threadIdx.x;
  const int64_t k0 = (int64_t)blockIdx.y * 256;
  unsigned long long m = 0ull;
  if (c < cols)
    for (int64_t k = k0 + threadIdx.y; k < K && k < k0 + 256; k += 8) {
      const unsigned long long a = abs_bits(B[k * ldb + c]);
      m = a > m ? a : m;
    }
  if (c < cols && m != 0ull) atomicMax(&ex[c], oz_exponent_bits(m));
}

__global__ void oz_fix_zero_cols(int cols, int* __restrict__ ex) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < cols && ex[c] < OZ_ZERO_EXP) ex[c] = OZ_ZERO_EXP;
}

// Slices of the columns of B (K x cols, ld ldb), i.e. of the rows of B^T: Q[s][c][k] for
// c < rows_pad, k < ldK, through a 32 x 32 shared-memory transpose.
template <int S>
__global__ void oz_split_cols_kernel(const double* __restrict__ B, int64_t ldb, int64_t K,
                                     int cols, int rows_pad, int64_t ldK,
                                     const int* __restrict__ ex, __nv_bfloat16* __restrict__ Q) {
  __shared__ double tile[32][33];
  const int c0 = blockIdx.x * 32;
  const int64_t k0 = (int64_t)blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t k = k0 + i;
    const int c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (k < K && c < cols) ? B[k * ldb + c] : 0.0;
  }
  __syncthreads();
  const int64_t plane = (int64_t)rows_pad * ldK;
  const int64_t k = k0 + threadIdx.x;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int c = c0 + i;
    const int e = c < cols ? ex[c] : 0;
    oz_cut<S>(oz_fixed<S>(tile[threadIdx.x][i], e), Q + (int64_t)c * ldK + k, plane);
  }
}

// C[r][c] = alpha 2^(e_r + f_c - 16) (hi 2^-24 + lo 2^-48) + beta X[r][c] + gamma Z[r][c],
// with hi and lo summed over the K splits in integers (as high and low 32-bit halves, so that
// many splits cannot overflow).  A symmetric product fills r >= c and mirrors.
__global__ void oz_reduce(const long long* __restrict__ partial, const Grid g, int nslice, int m,
                          int n,
                          const int* __restrict__ exA, const int* __restrict__ exB, double alpha,
                          double beta, const double* X, int64_t ldx, double gamma, const double* Z,
                          int64_t ldz, double* C, int64_t ldc) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * n) return;
  const int r = (int)(t / n), c = (int)(t % n);
  if (g.sym && c > r) return;
  const int tn = g.tn;
  const int ti = r / TM, tj = c / tn;
  const int p = pair_index(g, ti, tj);
  const int rr = r - ti * TM, cc = c - tj * tn;
  long long hh = 0, hl = 0, lh = 0, ll = 0;
  for (int z = 0; z < g.nsplit; ++z) {
    const long long* P = partial + ((int64_t)z * g.npairs + p) * 2 * TM * tn;
    const long long a = P[rr * tn + cc], b = P[TM * tn + rr * tn + cc];
    hh += a >> 32;
    hl += a & 0xFFFFFFFFll;
    lh += b >> 32;
    ll += b & 0xFFFFFFFFll;
  }
  const double hi = ldexp((double)hh, 32) + (double)hl;
  const double lo = ldexp((double)lh, 32) + (double)ll;
  const int E = exA[r] + exB[c] - 2 * BETA;
  double v = alpha * (ldexp(hi, E - 3 * BETA) + ldexp(lo, E - oz_lowest_level(nslice) * BETA));
  if (X) v += beta * X[(int64_t)r * ldx + c];
  if (Z) v += gamma * Z[(int64_t)r * ldz + c];
  C[(int64_t)r * ldc + c] = v;
  if (g.sym) C[(int64_t)c * ldc + r] = v;
}

__global__ void zero_f64(double* __restrict__ M, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) M[t] = 0.0;
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

// 3-D map over the slice planes: (k, row, slice), box (32, box_rows, box_slices) -- the first
// box_slices slices of a stage -- with 64-byte swizzle.
int make_slice_map(CUtensorMap* m, const OzSlices& S, int box_rows, int box_slices) {
  auto enc = get_encode();
  if (!enc) {
    set_error_detail("cuTensorMapEncodeTiled is not available from the driver");
    return TUCKER_ECUDA;
  }
  cuuint64_t dims[3] = {(cuuint64_t)S.ldK, (cuuint64_t)S.rows_pad, (cuuint64_t)S.nslice};
  cuuint64_t strides[2] = {(cuuint64_t)S.ldK * 2, (cuuint64_t)S.rows_pad * (cuuint64_t)S.ldK * 2};
  cuuint32_t box[3] = {(cuuint32_t)KS, (cuuint32_t)box_rows, (cuuint32_t)box_slices};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, S.Q.p, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error_detail("cuTensorMapEncodeTiled rejected the slice layout of an FP64 product");
    return TUCKER_ECUDA;
  }
  return TUCKER_OK;
}

int reserve(OzSlices* out, int rows, int64_t ldK, int nslice, cudaStream_t s) {
  if (nslice != 3 && nslice != 6 && nslice != 7) return TUCKER_EINVAL;
  out->nslice = nslice;
  out->rows = rows;
  out->rows_pad = ceil_div(rows, TM) * TM;
  out->ldK = ldK;
  const size_t qb = sizeof(__nv_bfloat16) * nslice * (size_t)out->rows_pad * (size_t)ldK;
  if (out->Q.bytes < qb || out->Q.s != s) TK_TRY(out->Q.alloc(qb, s));
  if (out->ex.bytes < sizeof(int) * out->rows_pad || out->ex.s != s)
    TK_TRY(out->ex.alloc(sizeof(int) * out->rows_pad, s));
  return TUCKER_OK;
}

}  // namespace

int64_t oz_ldk(int64_t K) { return (K + KS - 1) / KS * KS; }

int oz_split_rows(const double* A, int64_t lda, int rows, int64_t K1, const double* A2,
                  int64_t lda2, int64_t K2, int nslice, OzSlices* out, cudaStream_t s) {
  if (rows < 1 || K1 < 0 || K2 < 0) return TUCKER_EINVAL;
  if (!A2) K2 = 0;
  const int64_t K1p = oz_ldk(K1);
  TK_TRY(reserve(out, rows, K1p + oz_ldk(K2), nslice, s));
  ProfScope prof("ozaki_split", s, 0.0,
                 8.0 * rows * (double)(K1 + K2) * 2 +
                     2.0 * nslice * out->rows_pad * (double)out->ldK);
  oz_scale_rows<<<rows, 256, 0, s>>>(A, lda, K1, A2, lda2, K2, out->ex.as<int>());
  TK_LAUNCH();
  if (out->ldK == 0) return TUCKER_OK;   // no columns: nothing to cut
  const int64_t quads = (int64_t)out->rows_pad * (out->ldK / 4);
  auto kern = nslice == 7 ? oz_split_rows_kernel<7>
              : nslice == 6 ? oz_split_rows_kernel<6> : oz_split_rows_kernel<3>;
  kern<<<ceil_div(quads, 256), 256, 0, s>>>(rows, out->rows_pad, A, lda, K1, K1p, A2, lda2, K2,
                                            out->ldK, out->ex.as<int>(),
                                            out->Q.as<__nv_bfloat16>());
  TK_LAUNCH();
  return TUCKER_OK;
}

int oz_split_cols(const double* B, int64_t ldb, int64_t K, int cols, int nslice, OzSlices* out,
                  cudaStream_t s) {
  if (cols < 1 || K < 0) return TUCKER_EINVAL;
  TK_TRY(reserve(out, cols, oz_ldk(K), nslice, s));
  ProfScope prof("ozaki_split", s, 0.0,
                 8.0 * cols * (double)K * 2 + 2.0 * nslice * out->rows_pad * (double)out->ldK);
  TK_CUDA(cudaMemsetAsync(out->ex.p, 0x80, sizeof(int) * cols, s));   // INT_MIN-like start
  if (K > 0) {
    oz_scale_cols<<<dim3(ceil_div(cols, 32), ceil_div(K, 256)), dim3(32, 8), 0, s>>>(
        B, ldb, K, cols, out->ex.as<int>());
    TK_LAUNCH();
  }
  oz_fix_zero_cols<<<ceil_div(cols, 256), 256, 0, s>>>(cols, out->ex.as<int>());
  TK_LAUNCH();
  if (out->ldK == 0) return TUCKER_OK;   // no rows of B: nothing to cut
  auto kern = nslice == 7 ? oz_split_cols_kernel<7>
              : nslice == 6 ? oz_split_cols_kernel<6> : oz_split_cols_kernel<3>;
  kern<<<dim3(out->rows_pad / 32, (unsigned)(out->ldK / 32)), dim3(32, 8), 0, s>>>(
      B, ldb, K, cols, out->rows_pad, out->ldK, out->ex.as<int>(), out->Q.as<__nv_bfloat16>());
  TK_LAUNCH();
  return TUCKER_OK;
}

namespace {

// The tensor maps and the products: 128 x 64 tiles in one pass (tensor maps of all S slices), or
// 128 x 128 tiles in two passes (pass 0 loads the first wk::Geo<S>::SL0 slices of a stage, pass 1
// all of them).
template <int S>
int launch_products(const OzSlices& A, const OzSlices& B, const Grid& g, int64_t njobs,
                    long long* part, int* status, cudaStream_t s) {
  if (g.tn == nk::TN) {
    CUtensorMap mA, mB;
    TK_TRY(make_slice_map(&mA, A, TM, S));
    TK_TRY(make_slice_map(&mB, B, nk::TN, S));
    static const cudaError_t attr = cudaFuncSetAttribute(
        nk::gram_ozaki_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        nk::Geo<S>::SMEM_BYTES);
    TK_CUDA(attr);
    nk::gram_ozaki_kernel<S><<<(unsigned)njobs, nk::NTHREADS, nk::Geo<S>::SMEM_BYTES, s>>>(
        mA, mB, g, part, status);
    TK_LAUNCH();
    return TUCKER_OK;
  }
  CUtensorMap mA0, mB0, mA1, mB1;
  TK_TRY(make_slice_map(&mA0, A, TM, wk::Geo<S>::SL0));
  TK_TRY(make_slice_map(&mB0, B, wk::TN, wk::Geo<S>::SL0));
  TK_TRY(make_slice_map(&mA1, A, TM, wk::Geo<S>::SL1));
  TK_TRY(make_slice_map(&mB1, B, wk::TN, wk::Geo<S>::SL1));
  static const cudaError_t attr = cudaFuncSetAttribute(
      wk::gram_ozaki_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      wk::Geo<S>::SMEM_BYTES);
  TK_CUDA(attr);
  wk::gram_ozaki_kernel<S><<<(unsigned)njobs, wk::NTHREADS, wk::Geo<S>::SMEM_BYTES, s>>>(
      mA0, mB0, mA1, mB1, g, part, status);
  TK_LAUNCH();
  return TUCKER_OK;
}

}  // namespace

int oz_gemm_nt(const OzSlices& A, const OzSlices& B, bool sym, double alpha, double beta,
               const double* X, int64_t ldx, double gamma, const double* Z, int64_t ldz,
               double* C, int64_t ldc, int* status, cudaStream_t s, const char* prof_name) {
  if (A.ldK != B.ldK || A.nslice != B.nslice || (sym && &A != &B)) return TUCKER_EINVAL;
  const int S = A.nslice;
  const int m = A.rows, n = B.rows;
  // The long symmetric Grams take 128 x 128 tiles (half the MMA instructions per output); the
  // eigensolver's products, whose B has ~150 columns, waste less with 128 x 64.
  const int TN = (sym && S == OZ_GRAM_SLICES) ? wk::TN : nk::TN;
  const int nti = ceil_div(m, TM), ntj = ceil_div(n, TN);
  const int nst = (int)(A.ldK / KS);
  Grid g{ntj, 0, 1, nst, sym ? 1 : 0, TN, nullptr};
  g.npairs = !sym ? nti * ntj
             : TN == nk::TN ? nti * (nti + 1) - (ntj < 2 * nti ? 1 : 0) : nti * (nti + 1) / 2;
  // K splits: the fewest that fill the SMs' waves to 90 %, each at least 8 stages long and at
  // most MAX_JOB_STAGES.
  const int sms = num_sms();
  const int min_split = std::max(1, (nst + MAX_JOB_STAGES - 1) / MAX_JOB_STAGES);
  const int max_split = std::max(min_split, std::min(64, nst / 8));
  double best = 0.0;
  g.nsplit = min_split;
  for (int z = min_split; z <= max_split; ++z) {
    const int64_t jobs = (int64_t)g.npairs * z;
    const double eff = (double)jobs / (double)(((jobs + sms - 1) / sms) * sms);
    if (eff > best + 1e-9) {
      best = eff;
      g.nsplit = z;
    }
    if (eff >= 0.9) break;
  }
  const int64_t njobs = (int64_t)g.npairs * g.nsplit;
  if (nst == 0) {
    // empty K: C = beta X + gamma Z
    Buf zero;
    TK_TRY(zero.alloc(sizeof(long long) * 2 * TM * TN * (size_t)std::max<int64_t>(njobs, 1), s));
    TK_CUDA(cudaMemsetAsync(zero.p, 0, zero.bytes, s));
    g.nsplit = 1;
    oz_reduce<<<ceil_div((int64_t)m * n, 256), 256, 0, s>>>(zero.as<long long>(), g, S, m, n,
                                                             A.ex.as<int>(), B.ex.as<int>(), alpha,
                                                             beta, X, ldx, gamma, Z, ldz, C, ldc);
    TK_LAUNCH();
    return TUCKER_OK;
  }
  Buf part;
  TK_TRY(part.alloc(sizeof(long long) * 2 * TM * TN * (size_t)njobs, s));
  {
    // flops: the BF16 tensor-core FLOPs issued (S (S + 1) / 2 slice pairs per output tile and
    // K column); bytes: the slices read once plus the integer partials written.
    const int pairs = S * (S + 1) / 2 + (S % 2 == 0 ? 1 : 0);
    ProfScope pk(prof_name, s, 2.0 * pairs * TM * TN * (double)KS * nst * g.npairs,
                 2.0 * S * ((double)A.rows_pad + (sym ? 0.0 : (double)B.rows_pad)) * A.ldK +
                     16.0 * TM * TN * (double)njobs);
    if (S == 7)
      TK_TRY(launch_products<7>(A, B, g, njobs, part.as<long long>(), status, s));
    else if (S == 6)
      TK_TRY(launch_products<6>(A, B, g, njobs, part.as<long long>(), status, s));
    else
      TK_TRY(launch_products<3>(A, B, g, njobs, part.as<long long>(), status, s));
  }
  oz_reduce<<<ceil_div((int64_t)m * n, 256), 256, 0, s>>>(part.as<long long>(), g, S, m, n,
                                                           A.ex.as<int>(), B.ex.as<int>(), alpha,
                                                           beta, X, ldx, gamma, Z, ldz, C, ldc);
  TK_LAUNCH();
  return TUCKER_OK;
}

int gram_f64_tc(int rows, const double* Y1, int64_t K1, const double* Y2, int64_t K2, double* M,
                cudaStream_t s) {
  if (rows <= 0) return TUCKER_OK;
  if (!Y2) K2 = 0;
  const int64_t Ktot = K1 + K2;
  ProfScope prof("gram_f64_tc", s, (double)rows * (rows + 1) * (double)Ktot,
                 8.0 * rows * (double)Ktot + 8.0 * rows * rows);
  const int64_t cells = (int64_t)rows * rows;
  if (Ktot == 0) {
    zero_f64<<<ceil_div(cells, 256), 256, 0, s>>>(M, cells);
    TK_LAUNCH();
    return TUCKER_OK;
  }
  OzSlices S;
  TK_TRY(oz_split_rows(Y1, K1, rows, K1, Y2, K2, K2, OZ_GRAM_SLICES, &S, s));
  Buf st;
  TK_TRY(st.alloc(sizeof(int), s));
  TK_CUDA(cudaMemsetAsync(st.p, 0, sizeof(int), s));
  TK_TRY(oz_gemm_nt(S, S, true, 1.0, 0.0, nullptr, 0, 0.0, nullptr, 0, M, rows, st.as<int>(), s,
                    "gram_ozaki"));
  int h = 0;
  TK_CUDA(cudaMemcpyAsync(&h, st.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  if (h & DEV_TIMEOUT) {
    set_error_detail("FP64 tensor-core Gram: a bounded wait on an mbarrier gave up");
    return TUCKER_ETIMEOUT;
  }
  return TUCKER_OK;
}

namespace {

// Slices of a gathered, transposed operand for the batched HOOI projection: the K position of
// fiber f is pos(f) = f + pad[slice of f] (every slice's fibers start on a stage boundary);
// out[s][j][pos(f)] = digit s of S[src(f)][j] scaled by 2^-ex[j] (src(f) = rows[f], or f when
// rows is NULL) for j < J, and 0 for J <= j < rows_pad (grid.y = rows_pad / 32).  The positions
// of no fiber (the tail of each slice's last stage) are cleared by oz_zero_tails.  Tiles of
// 32 fibers x 32 columns through shared memory keep reads and writes coalesced.
template <int S>
__global__ void oz_split_gather_kernel(const double* __restrict__ Src, int64_t ld, int J,
                                       const int32_t* __restrict__ rows, int64_t F,
                                       const int32_t* __restrict__ fiber_root,
                                       const int64_t* __restrict__ pad, const int* __restrict__ ex,
                                       int rows_pad, int64_t ldK, __nv_bfloat16* __restrict__ Q) {
  __shared__ double tile[32][33];
  __shared__ int64_t pos_s[32];
  const int64_t f0 = (int64_t)blockIdx.x * 32;
  const int j0 = blockIdx.y * 32;
  if (threadIdx.y == 0) {
    const int64_t f = f0 + threadIdx.x;
    pos_s[threadIdx.x] = f < F ? f + pad[fiber_root[f]] : -1;
  }
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t f = f0 + i;
    const int j = j0 + threadIdx.x;
    double v = 0.0;
    if (f < F && j < J) v = Src[(rows ? (int64_t)rows[f] : f) * ld + j];
    tile[i][threadIdx.x] = v;
  }
  __syncthreads();
  const int64_t plane = (int64_t)rows_pad * ldK;
  const int64_t pos = pos_s[threadIdx.x];
  if (pos < 0) return;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int j = j0 + i;
    oz_cut<S>(j < J ? oz_fixed<S>(tile[threadIdx.x][i], ex[j]) : 0ll, Q + (int64_t)j * ldK + pos,
              plane);
  }
}

// Zeros at the positions of no fiber: slice i's fibers fill [sst[i] 32, sst[i] 32 + F_i) of its
// stages [sst[i], sst[i + 1]); the rest (at most 31 columns) of every row and slice plane.
__global__ void oz_zero_tails(const int64_t* __restrict__ root_ptr, const int* __restrict__ sst,
                              int rows_pad, int64_t ldK, int nslice,
                              __nv_bfloat16* __restrict__ Q) {
  const int64_t i = blockIdx.x;
  const int64_t a = (int64_t)sst[i] * KS + (root_ptr[i + 1] - root_ptr[i]);
  const int len = (int)((int64_t)sst[i + 1] * KS - a);
  if (len <= 0) return;
  const int64_t plane = (int64_t)rows_pad * ldK;
  __nv_bfloat16_raw z;
  z.x = 0;
  for (int t = threadIdx.x; t < nslice * rows_pad * len; t += blockDim.x) {
    const int c = t % len, r = (t / len) % rows_pad, sl = t / (len * rows_pad);
    Q[(int64_t)sl * plane + (int64_t)r * ldK + a + c] = z;
  }
}

// Y[i, p J_o + q] = 2^(ex_a[p] + ex_b[q] - 16) (hi 2^-24 + lo 2^-48) of slice i's product.
__global__ void oz_reduce_batched(const long long* __restrict__ partial, int ntj, int npairs,
                                  int nslice, int64_t nslices, int Jm, int Jo,
                                  const int* __restrict__ exA, const int* __restrict__ exB,
                                  double* __restrict__ Y) {
  constexpr int TN = nk::TN;   // the batched products use 128 x 64 tiles
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)Jm * Jo;
  if (t >= nslices * per) return;
  const int64_t i = t / per;
  const int p = (int)((t % per) / Jo), q = (int)(t % Jo);
  const int ti = p / TM, tj = q / TN;
  const long long* P = partial + (i * npairs + (int64_t)ti * ntj + tj) * 2 * TM * TN;
  const int rr = p - ti * TM, cc = q - tj * TN;
  const long long hi = P[rr * TN + cc], lo = P[TM * TN + rr * TN + cc];
  const int E = exA[p] + exB[q] - 2 * BETA;
  Y[t] = ldexp((double)hi, E - 3 * BETA) + ldexp((double)lo, E - oz_lowest_level(nslice) * BETA);
}

// Padded K layout of a TTMc ordering: pad[i] = (stage start of slice i) * 32 - root_ptr[i],
// stage_start[i + 1] = stage_start[i] + ceil(F_i / 32).
__global__ void slice_stages(const int64_t* __restrict__ root_ptr, int64_t In,
                             int* __restrict__ nstage) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < In) nstage[i] = (int)((root_ptr[i + 1] - root_ptr[i] + KS - 1) / KS);
}
__global__ void slice_pads(const int64_t* __restrict__ root_ptr, const int* __restrict__ stage_start,
                           int64_t In, int64_t* __restrict__ pad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < In) pad[i] = (int64_t)stage_start[i] * KS - root_ptr[i];
}

template <int S>
int split_gather(const double* Src, int64_t ld, int J, const int32_t* rows, int64_t F,
                 const int32_t* fiber_root, const int64_t* pad, const int* ex, int rows_pad,
                 int64_t ldK, __nv_bfloat16* Q, cudaStream_t s) {
  dim3 grid((unsigned)ceil_div(F, 32), (unsigned)(rows_pad / 32));
  oz_split_gather_kernel<S><<<grid, dim3(32, 8), 0, s>>>(Src, ld, J, rows, F, fiber_root, pad, ex,
                                                         rows_pad, ldK, Q);
  TK_LAUNCH();
  return TUCKER_OK;
}

}  // namespace

int ttmc_f64_tc(const tucker_tensor_s* X, const Ordering* o, const double* Um, int Jm,
                const double* Uo, int Jo, double* Y, cudaStream_t s) {
  const int64_t In = X->dims[o->n], F = o->F;
  constexpr int S = OZ_GRAM_SLICES;
  constexpr int TN = nk::TN;   // short per-slice products: 128 x 64 tiles in one pass
  if (In == 0) return TUCKER_OK;
  ProfScope prof("ttmc_f64_tc", s, 2.0 * ((double)X->nnz * Jo + (double)F * Jm * Jo),
                 12.0 * X->nnz + 16.0 * F + 8.0 * In * (double)Jm * Jo);
  // stage 1 on the CUDA cores: T[f, q] = sum over fiber f's leaves of x U_o[i_o, q]
  Buf T, nst, sst, pad, exA, exB, tot, part, st;
  TK_TRY(T.alloc(sizeof(double) * (size_t)std::max<int64_t>(F, 1) * Jo, s));
  TK_TRY(slice_proj_f64_fibers(F, nullptr, nullptr, o->fiber_ptr, o->leaf_idx, o->val, Uo, Jo, 0,
                               T.as<double>(), s));
  // padded stage layout: slice i's fibers start at stage sst[i]
  TK_TRY(nst.alloc(sizeof(int) * (In + 1), s));
  TK_TRY(sst.alloc(sizeof(int) * (In + 1), s));
  TK_TRY(pad.alloc(sizeof(int64_t) * In, s));
  TK_TRY(tot.alloc(sizeof(unsigned), s));
  slice_stages<<<ceil_div(In, 256), 256, 0, s>>>(o->root_ptr, In, nst.as<int>());
  TK_LAUNCH();
  TK_TRY(exclusive_scan_u32(nst.as<unsigned>(), sst.as<unsigned>(), In, tot.as<unsigned>(), s));
  unsigned stages = 0;
  TK_CUDA(cudaMemcpyAsync(&stages, tot.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaMemcpyAsync(sst.as<unsigned>() + In, tot.p, sizeof(unsigned),
                          cudaMemcpyDeviceToDevice, s));
  slice_pads<<<ceil_div(In, 256), 256, 0, s>>>(o->root_ptr, sst.as<int>(), In, pad.as<int64_t>());
  TK_LAUNCH();
  TK_CUDA(cudaStreamSynchronize(s));
  const int64_t ldK = std::max<int64_t>((int64_t)stages * KS, KS);
  // operands: A^T rows p (the fibers' U_m rows), B^T rows q (T); per-column scale exponents
  OzSlices A, B;
  A.nslice = B.nslice = S;
  A.rows = Jm;
  A.rows_pad = ceil_div(Jm, TM) * TM;
  B.rows = Jo;
  B.rows_pad = ceil_div(Jo, TM) * TM;
  A.ldK = B.ldK = ldK;
  TK_TRY(A.Q.alloc(sizeof(__nv_bfloat16) * S * (size_t)A.rows_pad * ldK, s));
  TK_TRY(B.Q.alloc(sizeof(__nv_bfloat16) * S * (size_t)B.rows_pad * ldK, s));
  TK_TRY(A.ex.alloc(sizeof(int) * A.rows_pad, s));
  TK_TRY(B.ex.alloc(sizeof(int) * B.rows_pad, s));
  if (F == 0) {   // no fiber: every position is padding
    TK_CUDA(cudaMemsetAsync(A.Q.p, 0, A.Q.bytes, s));
    TK_CUDA(cudaMemsetAsync(B.Q.p, 0, B.Q.bytes, s));
  } else {
    oz_zero_tails<<<(unsigned)In, 256, 0, s>>>(o->root_ptr, sst.as<int>(), A.rows_pad, ldK, S,
                                                A.Q.as<__nv_bfloat16>());
    TK_LAUNCH();
    oz_zero_tails<<<(unsigned)In, 256, 0, s>>>(o->root_ptr, sst.as<int>(), B.rows_pad, ldK, S,
                                                B.Q.as<__nv_bfloat16>());
    TK_LAUNCH();
  }
  TK_CUDA(cudaMemsetAsync(A.ex.p, 0x80, sizeof(int) * Jm, s));
  TK_CUDA(cudaMemsetAsync(B.ex.p, 0x80, sizeof(int) * Jo, s));
  const int64_t Im = X->dims[o->m];
  oz_scale_cols<<<dim3(ceil_div(Jm, 32), ceil_div(Im, 256)), dim3(32, 8), 0, s>>>(
      Um, Jm, Im, Jm, A.ex.as<int>());
  TK_LAUNCH();
  if (F > 0) {
    oz_scale_cols<<<dim3(ceil_div(Jo, 32), ceil_div(F, 256)), dim3(32, 8), 0, s>>>(
        T.as<double>(), Jo, F, Jo, B.ex.as<int>());
    TK_LAUNCH();
  }
  oz_fix_zero_cols<<<ceil_div(Jm, 256), 256, 0, s>>>(Jm, A.ex.as<int>());
  TK_LAUNCH();
  oz_fix_zero_cols<<<ceil_div(Jo, 256), 256, 0, s>>>(Jo, B.ex.as<int>());
  TK_LAUNCH();
  if (F > 0) {
    TK_TRY(split_gather<S>(Um, Jm, Jm, o->fiber_idx, F, o->fiber_root, pad.as<int64_t>(),
                           A.ex.as<int>(), A.rows_pad, ldK, A.Q.as<__nv_bfloat16>(), s));
    TK_TRY(split_gather<S>(T.as<double>(), Jo, Jo, nullptr, F, o->fiber_root, pad.as<int64_t>(),
                           B.ex.as<int>(), B.rows_pad, ldK, B.Q.as<__nv_bfloat16>(), s));
  }
  // one product per slice: (J_m x J_o) = A_i^T B_i over the slice's stages
  const int nti = ceil_div(Jm, TM), ntj = ceil_div(Jo, TN);
  Grid g{ntj, nti * ntj, 1, (int)stages, 0, TN, sst.as<int>()};
  const int64_t njobs = In * g.npairs;
  TK_TRY(part.alloc(sizeof(long long) * 2 * TM * TN * (size_t)njobs, s));
  TK_TRY(st.alloc(sizeof(int), s));
  TK_CUDA(cudaMemsetAsync(st.p, 0, sizeof(int), s));
  {
    ProfScope pk("ttmc_ozaki", s,
                 2.0 * nk::Geo<S>::PAIRS * TM * TN * (double)KS * stages * g.npairs,
                 2.0 * S * ((double)A.rows_pad + B.rows_pad) * ldK + 16.0 * TM * TN * (double)njobs);
    TK_TRY(launch_products<S>(A, B, g, njobs, part.as<long long>(), st.as<int>(), s));
  }
  oz_reduce_batched<<<ceil_div(In * Jm * Jo, 256), 256, 0, s>>>(
      part.as<long long>(), ntj, g.npairs, S, In, Jm, Jo, A.ex.as<int>(), B.ex.as<int>(), Y);
  TK_LAUNCH();
  int h = 0;
  TK_CUDA(cudaMemcpyAsync(&h, st.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  if (h & DEV_TIMEOUT) {
    set_error_detail("FP64 tensor-core projection: a bounded wait on an mbarrier gave up");
    return TUCKER_ETIMEOUT;
  }
  return TUCKER_OK;
}

}  // namespace tk
