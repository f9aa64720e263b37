// Small dense symmetric eigenproblems (order m <= SYEV_REFINED_MAX_M): the Rayleigh-Ritz
// matrix H = V^T M V of the subspace iteration and, for small unfoldings, M itself.
//
// FP64 arithmetic is a narrow pipe on this part (about 2 FMA per clock per SM), so a cyclic
// Jacobi in FP64 is bound by the latency of its m - 1 rounds per sweep.  Instead:
//   1. a cyclic round-robin Jacobi in FP32, all of it in one CTA's shared memory, gives an
//      approximate eigenvector matrix X (accurate to ~1e-7 of |A|);
//   2. Ogita & Aishima's iterative refinement for the symmetric eigenproblem (Japan J. Indust.
//      Appl. Math. 35, 2018) brings X to FP64 accuracy.  One step, all in FP64:
//          R = I - X^T X,  S = X^T A X,  lambda_i = s_ii / (1 - r_ii),
//          E_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i)   (i != j, separated pair),
//          E_ij = r_ij / 2                                          (i == j, or unresolved),
//          X <- X + X E.
//      A pair counts as separated when its first-order correction is small against its gap,
//      |s_ij + lambda_j r_ij| <= 0.1 |lambda_j - lambda_i|, and the gap is above the FP64 noise
//      floor; the products are FP64 GEMMs spread over the whole GPU.  Convergence is quadratic.
//   3. The result is accepted once every column's off-diagonal mass |S_{:,j}|_offdiag is below
//      the caller's threshold and the loss of orthogonality max |R| is below 1e-12.  S and G
//      are symmetrised before use (see oa_column_kernel).  A near-degenerate
//      cluster that the first-order step cannot split (and that would matter at the caller's
//      tolerance) sends the problem to the FP64 Jacobi instead.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace tk {

namespace {

constexpr int JAC32_MAX_H = SYEV_REFINED_MAX_M / 2;


// Cyclic Jacobi on FP32(0.5 (A + A^T)) in shared memory (scaled by a power of two when its
// entries lie outside FP32's comfortable range), round-robin ordering: round r rotates the m/2
// disjoint pairs at once.  A rotation is applied when |a_pq| exceeds both tol_abs * max |a_ii|
// and tol_rel * sqrt|a_pp a_qq|; the sweep loop ends after a sweep without one, or once a
// sweep fails to halve the off-diagonal mass (the FP32 rounding floor).  The
// update is in place: block (I, K) of J^T A J reads and writes only rows {p_I, q_I} x columns
// {p_K, q_K}, which no other block touches.  Q is kept transposed so that the rows of a pair's
// two columns are contiguous for the lanes.  X (m x m, FP64, ld ldx) receives Q.
__global__ void __launch_bounds__(1024)
jacobi32_kernel(const double* __restrict__ A, int m, int64_t lda, float tol_rel, float tol_abs,
                int max_sweeps, double* __restrict__ X, int64_t ldx, int* __restrict__ info) {
  extern __shared__ float smf[];
  const int mp = m + (m & 1), h = mp / 2;
  float* a = smf;             // mp x mp
  float* qt = a + mp * mp;    // qt[c * mp + r] = Q[r][c]
  __shared__ float cs[JAC32_MAX_H], sn[JAC32_MAX_H], dp[JAC32_MAX_H], dq[JAC32_MAX_H];
  __shared__ int pi[JAC32_MAX_H], qi[JAC32_MAX_H], on_s[JAC32_MAX_H];
  __shared__ float dmax_s;
  __shared__ unsigned long long amax_s;
  __shared__ double pow2_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // max |a_ij| from the bit patterns (integer compares keep this off the FP64 pipe)
  if (tid == 0) amax_s = 0ull;
  __syncthreads();
  unsigned long long mb = 0ull;
  for (int t = tid; t < m * m; t += blockDim.x) {
    const int r = t / m, c = t - r * m;
    const unsigned long long b =
        (unsigned long long)__double_as_longlong(A[(int64_t)r * lda + c]) & 0x7fffffffffffffffull;
    mb = b > mb ? b : mb;
  }
  atomicMax(&amax_s, mb);
  __syncthreads();
  if (tid == 0) {
    // A power of two that brings max |a_ij| near 1 when FP32 could not hold it as it is.
    const double amax = __longlong_as_double((long long)amax_s);
    int e = 0;
    if (amax > 0.0) frexp(amax, &e);
    pow2_s = (amax > 1e30 || (amax > 0.0 && amax < 1e-30)) ? ldexp(1.0, -e) : 1.0;
  }
  __syncthreads();
  const double pw = pow2_s;
  for (int t = tid; t < mp * mp; t += blockDim.x) {
    const int r = t / mp, c = t - r * mp;
    float v = 0.0f;
    if (r < m && c < m) {
      double x = A[(int64_t)r * lda + c], y = A[(int64_t)c * lda + r];
      if (pw != 1.0) { x *= pw; y *= pw; }
      v = 0.5f * ((float)x + (float)y);
    }
    a[t] = v;
    qt[t] = (r == c) ? 1.0f : 0.0f;
  }
  __syncthreads();
  if (warp == 0) {
    float mx = 0.0f;
    for (int i = lane; i < m; i += 32) mx = fmaxf(mx, fabsf(a[i * mp + i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) dmax_s = mx;
  }
  __syncthreads();
  const float abs_thr = tol_abs * dmax_s;
  // Fixed work assignment of the update phase (no divisions inside the sweep loop).
  const int sa = blockDim.x / h, kb = tid % h, ib = tid / h;
  const int sq = blockDim.x / mp, rq = tid % mp, iq = tid / mp;
  __shared__ float off_s;
  float prev_off2 = 3.0e38f;
  int sweep = 0, converged = 0;
  for (; sweep < max_sweeps; ++sweep) {
    int active_sweep = 0;
    // Round-robin slots of pair tid (slot 0 stays, the others step through 1..mp-1).
    int sx = tid == 0 ? 0 : 1 + (tid - 1) % (mp - 1);
    int sy = 1 + (mp - 2 - tid) % (mp - 1);
    for (int r = 0; r < mp - 1; ++r, sx = (sx == 0 ? 0 : (sx == mp - 1 ? 1 : sx + 1)),
                                     sy = (sy == mp - 1 ? 1 : sy + 1)) {
      int on = 0;
      if (tid < h) {
        const int x = sx, y = sy;
        const int p = min(x, y), q = max(x, y);
        const float app = a[p * mp + p], aqq = a[q * mp + q], apq = a[p * mp + q];
        float c = 1.0f, s = 0.0f, np_ = app, nq_ = aqq;
        if (fabsf(apq) > abs_thr && fabsf(apq) > tol_rel * sqrtf(fabsf(app)) * sqrtf(fabsf(aqq))) {
          // Symmetric 2x2 Schur decomposition (Golub & Van Loan, Algorithm 8.4.1).
          // Approximate division and square root suffice: any (c, s) with c^2 + s^2 = 1 to
          // FP32 precision is a rotation, and the FP64 refinement removes what it leaves.
          const float tau = __fdividef(aqq - app, 2.0f * apq);
          const float w = fmaf(tau, tau, 1.0f);
          const float t = fabsf(tau) < 1e18f
                              ? copysignf(__frcp_rn(fabsf(tau) + w * rsqrtf(w)), tau)
                              : __frcp_rn(2.0f * tau);
          c = rsqrtf(fmaf(t, t, 1.0f));
          s = t * c;
          np_ = app - t * apq;
          nq_ = aqq + t * apq;
          on = 1;
        }
        cs[tid] = c; sn[tid] = s; dp[tid] = np_; dq[tid] = nq_;
        pi[tid] = p; qi[tid] = q; on_s[tid] = on;
      }
      if (!__syncthreads_or(on)) continue;  // nothing to rotate this round (uniform)
      active_sweep = 1;
      // 2x2 blocks (I, K): thread t takes K = t mod h and I = t / h, t / h + sa, ...
      if (tid < sa * h) {
        const int K = kb;
        const float c2 = cs[K], s2 = sn[K];
        const int u = pi[K], v = qi[K];
        for (int I = ib; I < h; I += sa) {
          const float c1 = cs[I], s1 = sn[I];
          const int p = pi[I], q = qi[I];
          if (K == I) {
            if (on_s[I]) {
              a[p * mp + p] = dp[I];
              a[q * mp + q] = dq[I];
              a[p * mp + q] = 0.0f;
              a[q * mp + p] = 0.0f;
            }
            continue;
          }
          if (s1 == 0.0f && s2 == 0.0f) continue;
          const float x0 = a[p * mp + u], x1 = a[p * mp + v];
          const float x2 = a[q * mp + u], x3 = a[q * mp + v];
          const float rpu = c1 * x0 - s1 * x2, rpv = c1 * x1 - s1 * x3;
          const float rqu = s1 * x0 + c1 * x2, rqv = s1 * x1 + c1 * x3;
          a[p * mp + u] = c2 * rpu - s2 * rpv;
          a[p * mp + v] = s2 * rpu + c2 * rpv;
          a[q * mp + u] = c2 * rqu - s2 * rqv;
          a[q * mp + v] = s2 * rqu + c2 * rqv;
        }
      }
      // Q <- Q J: thread t takes row t mod mp of the column pairs I = t / mp, t / mp + sq, ...
      // (columns p and q of Q are rows p and q of qt: consecutive threads, consecutive words).
      if (tid < sq * mp) {
        for (int I = iq; I < h; I += sq) {
          const float c1 = cs[I], s1 = sn[I];
          if (s1 == 0.0f) continue;
          const int p = pi[I], q = qi[I];
          const float y0 = qt[p * mp + rq], y1 = qt[q * mp + rq];
          qt[p * mp + rq] = c1 * y0 - s1 * y1;
          qt[q * mp + rq] = s1 * y0 + c1 * y1;
        }
      }
      __syncthreads();
    }
    if (!active_sweep) {
      converged = 1;
      ++sweep;
      break;
    }
    // Off-diagonal mass after the sweep.  Jacobi converges quadratically until FP32 rounding
    // sets a floor; a sweep that does not halve the mass has reached it, and the FP64
    // refinement takes over from there.
    if (tid == 0) off_s = 0.0f;
    __syncthreads();
    float o2 = 0.0f;
    for (int t = tid; t < mp * mp; t += blockDim.x) {
      const int r = t / mp, c = t - r * mp;
      if (r != c) o2 = fmaf(a[t], a[t], o2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) o2 += __shfl_xor_sync(0xffffffffu, o2, o);
    if (lane == 0) atomicAdd(&off_s, o2);
    __syncthreads();
    const float off2 = off_s;
    const bool stalled = sweep >= 2 && off2 > 0.25f * prev_off2;
    prev_off2 = off2;
    if (stalled) {
      converged = 1;
      ++sweep;
      break;
    }
  }
  for (int t = tid; t < m * m; t += blockDim.x) {
    const int r = t / m, c = t - r * m;
    X[(int64_t)r * ldx + c] = (double)qt[c * mp + r];
  }
  if (tid == 0) {
    info[0] = sweep;
    info[1] = converged;
  }
}

// lambda_i = s_ii / g_ii (g = X^T X, so 1 - r_ii = g_ii), one thread per i.
__global__ void oa_lambda_kernel(const double* __restrict__ SG, int m, int64_t ld,
                                 double* __restrict__ lam) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) lam[i] = SG[(int64_t)i * ld + i] / SG[(int64_t)i * ld + m + i];
}

// One block per column j of the refinement: E[:, j], and the column's statistics
//   stats[3j]     = sum_{i != j} s_ij^2,
//   stats[3j + 1] = max_i |r_ij|,
//   stats[3j + 2] = pairs (i, j) left unresolved with |s_ij| > bad_thr_rel * max(nA, scale).
// nA = max_i |lambda_i| is recomputed by every block (m values).
__global__ void __launch_bounds__(256)
oa_column_kernel(const double* __restrict__ SG, int m, int64_t ld, const double* __restrict__ lam,
                 double scale, double bad_thr_rel, double* __restrict__ E,
                 double* __restrict__ stats) {
  __shared__ double red[3][8];
  __shared__ double nA_s;
  const int j = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double mx = 0.0;
  for (int i = tid; i < m; i += blockDim.x) mx = fmax(mx, fabs(lam[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) red[0][warp] = mx;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[0][w]);
    nA_s = t;
  }
  __syncthreads();
  const double nA = nA_s;
  const double lj = lam[j];
  const double floor_gap = 1e-13 * nA;
  const double bad_thr = bad_thr_rel * fmax(nA, scale);
  double off2 = 0.0, orth = 0.0, bad = 0.0;
  for (int i = tid; i < m; i += blockDim.x) {
    // S and G are symmetric in exact arithmetic; their rounded products are not, and an
    // asymmetry divided by a small gap would leave an orthogonality floor far above eps.
    const double s = 0.5 * (SG[(int64_t)i * ld + j] + SG[(int64_t)j * ld + i]);
    const double g = 0.5 * (SG[(int64_t)i * ld + m + j] + SG[(int64_t)j * ld + m + i]);
    const double r = (i == j ? 1.0 : 0.0) - g;
    orth = fmax(orth, fabs(r));
    double e = 0.5 * r;
    if (i != j) {
      off2 = fma(s, s, off2);
      const double num = fma(lj, r, s), den = lj - lam[i];
      if (fabs(den) > floor_gap && fabs(num) <= 0.1 * fabs(den)) {
        e = num / den;
      } else if (fabs(s) > bad_thr) {
        bad += 1.0;
      }
    }
    E[(int64_t)i * m + j] = e;
  }
  off2 = warp_sum(off2);
  bad = warp_sum(bad);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) orth = fmax(orth, __shfl_xor_sync(0xffffffffu, orth, o));
  __syncthreads();
  if (lane == 0) {
    red[0][warp] = off2;
    red[1][warp] = orth;
    red[2][warp] = bad;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b = fmax(b, red[1][w]);
      c += red[2][w];
    }
    stats[3 * j] = a;
    stats[3 * j + 1] = b;
    stats[3 * j + 2] = c;
  }
}

// Jacobi rotations for the pairs a first-order refinement step cannot split (near-degenerate
// clusters of eigenvalues).  B = 0.5 (S + S^T) with S = X^T A X (m x m, ld lds) is held in
// shared memory; X (m x m, ld ldx) is rotated in place.  Each round: every thread scans its
// share of B's strict upper triangle for entries above thr_rel * max |b_ii| (magnitudes compared
// as bit patterns, off the FP64 pipe) that are not small against their diagonal gap
// (|b_pq| > 0.05 |b_qq - b_pp|; the refinement's first-order step resolves the others); one
// thread picks disjoint pairs greedily; their
// symmetric Schur rotations (Golub & Van Loan, Algorithm 8.4.1) are applied to the rows of B,
// then to its columns and to the columns of X, and the rotated entries are set to zero.  The
// loop ends after a round without such an entry (info[0] = rounds, info[1] = 1) or after
// max_rounds (info[1] = 0).  The clusters are small, so a round touches a few rows of B only.
constexpr int ROT_MAX_CAND = 512;
__global__ void __launch_bounds__(512)
cluster_rotate_kernel(const double* __restrict__ S, int64_t lds, int m, double thr_rel,
                      int max_rounds, double* __restrict__ X, int64_t ldx, int* __restrict__ info) {
  extern __shared__ double b[];   // m x m
  __shared__ int cp[ROT_MAX_CAND], cq[ROT_MAX_CAND];
  __shared__ int sp[SYEV_REFINED_MAX_M / 2], sq[SYEV_REFINED_MAX_M / 2];
  __shared__ double sc[SYEV_REFINED_MAX_M / 2], ss[SYEV_REFINED_MAX_M / 2];
  __shared__ unsigned char used[SYEV_REFINED_MAX_M];
  __shared__ int ncand, nsel;
  __shared__ unsigned long long dmax_s;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) dmax_s = 0ull;
  __syncthreads();
  unsigned long long mb = 0ull;
  for (int t = tid; t < m * m; t += nt) {
    const int i = t / m, j = t - i * m;
    const double v = 0.5 * (S[(int64_t)i * lds + j] + S[(int64_t)j * lds + i]);
    b[t] = v;
    if (i == j) {
      const unsigned long long a = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
      mb = a > mb ? a : mb;
    }
  }
  atomicMax(&dmax_s, mb);
  __syncthreads();
  const unsigned long long thr_bits = (unsigned long long)__double_as_longlong(
      thr_rel * __longlong_as_double((long long)dmax_s));
  int round = 0, done = 0;
  for (; round < max_rounds; ++round) {
    if (tid == 0) ncand = 0;
    __syncthreads();
    for (int t = tid; t < m * m; t += nt) {
      const int i = t / m, j = t - i * m;
      if (j <= i) continue;
      const unsigned long long a = (unsigned long long)__double_as_longlong(b[t]) & 0x7fffffffffffffffull;
      // pairs a first-order step resolves (|b_pq| <= 0.1 |b_qq - b_pp|) are left to it
      if (a > thr_bits && fabs(b[t]) > 0.05 * fabs(b[j * m + j] - b[i * m + i])) {
        const int c = atomicAdd(&ncand, 1);
        if (c < ROT_MAX_CAND) {
          cp[c] = i;
          cq[c] = j;
        }
      }
    }
    __syncthreads();
    if (ncand == 0) {   // uniform: read after the barrier
      done = 1;
      break;
    }
    if (tid == 0) {
      for (int i = 0; i < m; ++i) used[i] = 0;
      int n = 0;
      const int nc = min(ncand, ROT_MAX_CAND);
      for (int c = 0; c < nc && n < SYEV_REFINED_MAX_M / 2; ++c) {
        const int p = cp[c], q = cq[c];
        if (used[p] || used[q]) continue;
        used[p] = used[q] = 1;
        sp[n] = p;
        sq[n] = q;
        ++n;
      }
      nsel = n;
    }
    __syncthreads();
    const int ns = nsel;
    if (tid < ns) {
      const int p = sp[tid], q = sq[tid];
      const double apq = b[p * m + q];
      const double tau = (b[q * m + q] - b[p * m + p]) / (2.0 * apq);
      const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      const double c = 1.0 / sqrt(1.0 + t * t);
      sc[tid] = c;
      ss[tid] = t * c;
    }
    __syncthreads();
    for (int t = tid; t < ns * m; t += nt) {   // rows p, q of B <- J^T B
      const int r = t / m, k = t - r * m;
      const int p = sp[r], q = sq[r];
      const double c = sc[r], sn = ss[r];
      const double bp = b[p * m + k], bq = b[q * m + k];
      b[p * m + k] = c * bp - sn * bq;
      b[q * m + k] = sn * bp + c * bq;
    }
    __syncthreads();
    for (int t = tid; t < ns * m; t += nt) {   // columns p, q of B <- B J, and of X <- X J
      const int r = t / m, k = t - r * m;
      const int p = sp[r], q = sq[r];
      const double c = sc[r], sn = ss[r];
      const double bp = b[k * m + p], bq = b[k * m + q];
      b[k * m + p] = c * bp - sn * bq;
      b[k * m + q] = sn * bp + c * bq;
      double* xr = X + (int64_t)k * ldx;
      const double xp = xr[p], xq = xr[q];
      xr[p] = c * xp - sn * xq;
      xr[q] = sn * xp + c * xq;
    }
    __syncthreads();
    if (tid < ns) {
      const int p = sp[tid], q = sq[tid];
      b[p * m + q] = 0.0;
      b[q * m + p] = 0.0;
    }
    __syncthreads();
  }
  if (tid == 0) {
    info[0] = round;
    info[1] = done;
  }
}

}  // namespace

int syev_refined(const double* A, int m, int64_t lda, double* Qout, double* evals_out,
                 double scale, double acc_rel, cudaStream_t s, SyevStats* st) {
  SyevStats local;
  if (!st) st = &local;
  *st = SyevStats();
  if (m <= 0) return TUCKER_EINVAL;
  if (m > SYEV_REFINED_MAX_M) {
    st->fallback = true;
    prof_count("syev_fallback", 3.0);
    return jacobi_eig(A, m, lda, Qout, evals_out, s, &st->fp64_sweeps);
  }
  ProfScope prof("syev_refined", s, 0.0, 0.0);
  const int mp = m + (m & 1);
  const int64_t ld = 2 * (int64_t)m;  // [W | X] and [S | G] side by side
  // misc: per-column statistics [3m], lambda [m], the FP32 Jacobi's info [2 ints]: one
  // device-to-host copy reads all of them.
  Buf WX0, WX1, SG, E, misc;
  TK_TRY(WX0.alloc(sizeof(double) * m * ld, s));
  TK_TRY(WX1.alloc(sizeof(double) * m * ld, s));
  TK_TRY(SG.alloc(sizeof(double) * m * ld, s));
  TK_TRY(E.alloc(sizeof(double) * m * m, s));
  TK_TRY(misc.alloc(sizeof(double) * (4 * (size_t)m + 2), s));
  double* stats = misc.as<double>();
  double* lam = stats + 3 * m;
  int* info = reinterpret_cast<int*>(lam + m);
  double* cur = WX0.as<double>();
  double* nxt = WX1.as<double>();
  {
    const size_t smem = 2 * sizeof(float) * (size_t)mp * mp;
    static const cudaError_t attr = cudaFuncSetAttribute(
        jacobi32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)(2 * sizeof(float) * SYEV_REFINED_MAX_M * SYEV_REFINED_MAX_M));
    TK_CUDA(attr);
    {
      ProfScope pj("syev_jacobi32", s, 0.0, 0.0);
      jacobi32_kernel<<<1, 1024, smem, s>>>(A, m, lda, 1e-6f, 1e-7f, 40, cur + m, ld, info);
    }
    TK_LAUNCH();
  }
  // Refinement.  The statistics are read back (one host synchronisation each) from the step
  // `first_check` on: from an FP32 start two steps rarely, and three steps usually, meet the
  // bars, so checking from step 3 needs one synchronisation in the common case.
  const int max_steps = 8;
  const int first_check = 3;
  const double bad_rel = acc_rel;
  std::vector<double> hs(4 * (size_t)m + 2);
  int hinfo[2] = {0, 0};
  bool accepted = false, cluster = false;
  int rotations = 0;
  int step = 0;
  for (; step <= max_steps; ++step) {
    double* X = cur + m;
    TK_TRY(gemm_nn_f64(m, m, m, 1.0, A, lda, X, ld, 0.0, nullptr, 0, 0.0, nullptr, 0, cur, ld, s));
    TK_TRY(gemm_tn_f64(m, 2 * m, m, X, ld, cur, ld, SG.as<double>(), ld, s));
    oa_lambda_kernel<<<ceil_div(m, 128), 128, 0, s>>>(SG.as<double>(), m, ld, lam);
    TK_LAUNCH();
    oa_column_kernel<<<m, 256, 0, s>>>(SG.as<double>(), m, ld, lam, scale, bad_rel,
                                       E.as<double>(), stats);
    TK_LAUNCH();
    if (step >= first_check) {
      TK_CUDA(cudaMemcpyAsync(hs.data(), misc.p, misc.bytes, cudaMemcpyDeviceToHost, s));
      TK_TRY(host_sync(s));
      memcpy(hinfo, hs.data() + 4 * m, sizeof(hinfo));
      double hl_max = 0.0;
      for (int j = 0; j < m; ++j) hl_max = std::max(hl_max, fabs(hs[3 * m + j]));
      const double thr = acc_rel * std::max(hl_max, scale);
      double off = 0.0, orth = 0.0, bad = 0.0;
      for (int j = 0; j < m; ++j) {
        off = std::max(off, sqrt(hs[3 * j]));
        orth = std::max(orth, hs[3 * j + 1]);
        bad += hs[3 * j + 2];
      }
      st->offdiag = off / std::max(std::max(hl_max, scale), 1e-300);
      st->orth = orth;
      if (off <= thr && orth <= 1e-12) {
        accepted = true;
        break;
      }
      // An unresolved cluster that matters does not get better by more first-order steps: its
      // pairs are rotated by Jacobi on S = X^T A X (at most twice; the rotations are orthogonal,
      // so X keeps its orthogonality error, which the following steps remove), and the
      // refinement goes on from the rotated X.  If that does not settle it, the FP64 Jacobi
      // takes over.
      if (bad > 0.0) {
        if (rotations == 2 || orth > 1e-4) {
          if (rotations > 0) {
            int rinfo[2];
            memcpy(rinfo, hs.data() + 4 * m + 1, sizeof(rinfo));
            prof_count("syev_rotation_unconverged", rinfo[1] ? 0.0 : 1.0);
          }
          cluster = true;
          break;
        }
        ++rotations;
        const size_t rsm = sizeof(double) * (size_t)m * m;
        static const cudaError_t rattr = cudaFuncSetAttribute(
            cluster_rotate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
            (int)(sizeof(double) * SYEV_REFINED_MAX_M * SYEV_REFINED_MAX_M));
        TK_CUDA(rattr);
        cluster_rotate_kernel<<<1, 512, rsm, s>>>(SG.as<double>(), ld, m, 0.25 * acc_rel, 4 * m,
                                                  X, ld, info + 2);
        TK_LAUNCH();
        prof_count("syev_cluster_rotations", 1.0);
        continue;
      }
    }
    if (step == max_steps) break;
    // X <- X + X E into the other buffer.
    TK_TRY(gemm_nn_f64(m, m, m, 1.0, X, ld, E.as<double>(), m, 1.0, X, ld, 0.0, nullptr, 0,
                       nxt + m, ld, s));
    std::swap(cur, nxt);
  }
  st->steps = step;
  st->fp32_sweeps = hinfo[0];
  prof_count("syev_fp32_sweeps", (double)hinfo[0]);
  prof_count("syev_steps", (double)step);
  if (!accepted) {
    st->fallback = true;
    prof_count("syev_fallback", cluster ? 1.0 : 2.0);
    return jacobi_eig(A, m, lda, Qout, evals_out, s, &st->fp64_sweeps);
  }
  return sort_eig_desc(cur + m, ld, m, lam, Qout, m, evals_out, s);
}

}  // namespace tk
