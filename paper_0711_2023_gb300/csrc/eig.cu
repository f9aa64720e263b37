// Leading-J eigenvectors of a symmetric positive semi-definite matrix M (n x n, FP64): the
// "J_n leading eigenvectors of ..." step of every method (Figures HO-SVD3, hooi3, sp3, mp3).
//
// Method:
//   * small n: all eigenpairs of M at once (syev.cu: FP32 Jacobi refined in FP64, or the FP64
//     cyclic Jacobi below: Golub & Van Loan, Sec. 8.5, parallel round-robin ordering);
//   * otherwise block subspace iteration on k = J + max(16, J/2) columns:
//       - four power steps from the start block (warm start: the previous pass's factor);
//       - Rayleigh-Ritz (FP64): H = V^T M V, eigenpairs of H to a tenth of the locking
//         tolerance (syev.cu), V <- V Q; residuals |M v - theta v| in FP64;
//       - locking: leading Ritz pairs with residual <= tol * theta_1 are frozen and removed
//         from the filter's operator, M_d = M - L diag(theta_L) L^T;
//       - Chebyshev filtering (Zhou & Saad's filtered subspace iteration): p_d(M_d) with the
//         unwanted interval [0, theta_k] mapped to [-1, 1], the degree d capped so that the
//         block stays well conditioned, two filter applications per Rayleigh-Ritz step (four
//         power steps while an outlier eigenvalue pins d to 1); optionally the filter's
//         products run in FP32 until the residuals near the FP32 noise floor;
//       - Cholesky-QR2 orthonormalisation in FP64 (R = chol(V^T V), factored by blocks over one
//         thread-block cluster, then x R = v solved for every row v of V, twice), with a
//         shifted pass when the Gram matrix is not numerically positive definite.
//   The returned columns are sorted by eigenvalue (largest first) and sign-normalised: the
//   entry of largest magnitude in each column is positive.
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace tk {

namespace {

__device__ __forceinline__ int rr_index(int j, int r, int m) {
  return j == 0 ? 0 : 1 + (j - 1 + r) % (m - 1);
}

struct JacobiArgs {
  double* A0;         // m x m, symmetric, padded rows/cols beyond mreal are zero
  double* A1;         // m x m scratch
  double* Q;          // m x m, initialised to the identity
  double* evals;      // m (output: final diagonal)
  int m, mreal, max_sweeps;
  double tol;         // relative rotation threshold
  unsigned* bar;      // grid barrier words (2)
  unsigned* rot;      // rotations applied per sweep [max_sweeps]
  int* status;
  int* sweeps_out;
  int cluster;        // 1: the grid is one thread-block cluster, rounds end with its barrier
};

// End of a Jacobi round for a grid that is a single cluster: the hardware cluster barrier
// (release/acquire at cluster scope orders the round's global-memory writes).
__device__ __forceinline__ void cluster_round_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

struct Rot {
  double c, s, np, nq;
  bool on;
};

// Symmetric 2x2 Schur decomposition (Golub & Van Loan, Algorithm 8.4.1): the rotation that
// zeroes a_pq.  Kept out of line so every thread computing the same pair gets the same bits.
__device__ __noinline__ Rot sym_schur2(double app, double aqq, double apq, bool active,
                                       double tol, double abs_tol) {
  Rot r{1.0, 0.0, app, aqq, false};
  // The threshold compares squares: FP64 square roots and divisions are long instruction
  // sequences on this part and this runs on every round's critical path.
  if (active && fabs(apq) > abs_tol && apq * apq > tol * tol * fabs(app * aqq)) {
    const double tau = (aqq - app) * (0.5 / apq);
    const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(fma(tau, tau, 1.0)));
    r.c = rsqrt(fma(t, t, 1.0));
    r.s = t * r.c;
    r.np = app - t * apq;
    r.nq = aqq + t * apq;
    r.on = true;
  }
  return r;
}

__device__ __forceinline__ void pair_of(int I, int r, int m, int* p, int* q) {
  const int a = rr_index(I, r, m), b = rr_index(m - 1 - I, r, m);
  *p = min(a, b);
  *q = max(a, b);
}

// Cyclic two-sided Jacobi, round-robin ordering: in round r the m/2 disjoint pairs are rotated
// at once.  Work items of a round: the 2x2 blocks (I <= K) of A' = J^T A J (double-buffered),
// then the (row, pair) items of Q <- Q J.  Each block first issues the loads of its first work
// item, then computes the round's rotations into shared memory (one thread per pair, from the
// diagonal 2x2 blocks of the current A) while those loads are in flight, then applies them; a
// round ends with one grid barrier.
constexpr int CLUSTER_JACOBI_MAX_M = 128;

__global__ void __launch_bounds__(512) jacobi_kernel(JacobiArgs g) {
  extern __shared__ double sh[];
  const int m = g.m, h = m / 2;
  double* cs = sh;
  double* sn = cs + h;
  double* dp = sn + h;
  double* dq = dp + h;
  int* pi = (int*)(dq + h);
  int* qi = pi + h;
  __shared__ double normA_s;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gsize = (int64_t)gridDim.x * blockDim.x;
  double* Acur = g.A0;
  double* Anext = g.A1;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int i = 0; i < g.mreal; ++i) mx = fmax(mx, fabs(g.A0[(int64_t)i * m + i]));
    normA_s = mx;
  }
  __syncthreads();
  const double abs_tol = 1e-17 * normA_s + 1e-300;
  const int64_t ntri = (int64_t)h * (h + 1) / 2;
  const int64_t nwork = ntri + (int64_t)m * h;
  unsigned int epoch = 0;
  int sweep = 0;
  bool alive = true;
  for (; sweep < g.max_sweeps && alive; ++sweep) {
    for (int r = 0; r < m - 1 && alive; ++r) {
      bool first = true;
      for (int64_t t0 = (int64_t)blockIdx.x * blockDim.x; t0 < nwork || first; t0 += gsize) {
        const int64_t t = t0 + threadIdx.x;
        // ---- decode the item and issue its loads -------------------------------------------
        int I = 0, K = 0, row = -1, p = 0, q = 0, u = 0, v = 0;
        double x0 = 0.0, x1 = 0.0, x2 = 0.0, x3 = 0.0;
        const bool valid = t < nwork;
        const bool is_a = valid && t < ntri;
        if (is_a) {
          // triangular index from an FP32 estimate, corrected exactly in integers below
          K = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
          while ((int64_t)K * (K + 1) / 2 > t) --K;
          while ((int64_t)(K + 1) * (K + 2) / 2 <= t) ++K;
          I = (int)(t - (int64_t)K * (K + 1) / 2);
          pair_of(I, r, m, &p, &q);
          if (I != K) {
            pair_of(K, r, m, &u, &v);
            x0 = Acur[(int64_t)p * m + u];
            x1 = Acur[(int64_t)p * m + v];
            x2 = Acur[(int64_t)q * m + u];
            x3 = Acur[(int64_t)q * m + v];
          }
        } else if (valid) {
          const int64_t t2 = t - ntri;
          row = (int)(t2 / h);
          I = (int)(t2 % h);
          pair_of(I, r, m, &p, &q);
          x0 = g.Q[(int64_t)row * m + p];
          x1 = g.Q[(int64_t)row * m + q];
        }
        // ---- the round's rotations (once per block) ------------------------------------------
        if (first) {
          for (int i = threadIdx.x; i < h; i += blockDim.x) {
            int pp, qq;
            pair_of(i, r, m, &pp, &qq);
            const Rot R = sym_schur2(Acur[(int64_t)pp * m + pp], Acur[(int64_t)qq * m + qq],
                                     Acur[(int64_t)pp * m + qq], qq < g.mreal, g.tol, abs_tol);
            if (R.on && blockIdx.x == 0) atomicAdd(&g.rot[sweep], 1u);
            cs[i] = R.c; sn[i] = R.s; dp[i] = R.np; dq[i] = R.nq; pi[i] = pp; qi[i] = qq;
          }
          __syncthreads();
          first = false;
        }
        // ---- apply ---------------------------------------------------------------------------
        if (is_a) {
          if (I == K) {
            Anext[(int64_t)p * m + p] = dp[I];
            Anext[(int64_t)q * m + q] = dq[I];
            Anext[(int64_t)p * m + q] = 0.0;
            Anext[(int64_t)q * m + p] = 0.0;
          } else {
            const double c1 = cs[I], s1 = sn[I], c2 = cs[K], s2 = sn[K];
            const double rpu = c1 * x0 - s1 * x2, rpv = c1 * x1 - s1 * x3;
            const double rqu = s1 * x0 + c1 * x2, rqv = s1 * x1 + c1 * x3;
            const double bpu = c2 * rpu - s2 * rpv, bpv = s2 * rpu + c2 * rpv;
            const double bqu = c2 * rqu - s2 * rqv, bqv = s2 * rqu + c2 * rqv;
            Anext[(int64_t)p * m + u] = bpu; Anext[(int64_t)u * m + p] = bpu;
            Anext[(int64_t)p * m + v] = bpv; Anext[(int64_t)v * m + p] = bpv;
            Anext[(int64_t)q * m + u] = bqu; Anext[(int64_t)u * m + q] = bqu;
            Anext[(int64_t)q * m + v] = bqv; Anext[(int64_t)v * m + q] = bqv;
          }
        } else if (valid) {
          const double c = cs[I], s = sn[I];
          if (s != 0.0) {
            g.Q[(int64_t)row * m + p] = c * x0 - s * x1;
            g.Q[(int64_t)row * m + q] = s * x0 + c * x1;
          }
        }
      }
      if (g.cluster) {
        cluster_round_barrier();
      } else {
        alive = grid_barrier(g.bar, gridDim.x, &epoch, g.status);
      }
      double* tmp = Acur; Acur = Anext; Anext = tmp;
    }
    if (!alive) break;
    const unsigned cnt = *((volatile unsigned*)&g.rot[sweep]);
    if (cnt == 0) { ++sweep; break; }
  }
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) g.evals[i] = Acur[(int64_t)i * m + i];
    if (threadIdx.x == 0) {
      *g.sweeps_out = sweep;
      if (alive && sweep >= g.max_sweeps &&
          *((volatile unsigned*)&g.rot[g.max_sweeps - 1]) != 0)
        atomicOr(g.status, DEV_NOT_CONVERGED);
    }
  }
}

__global__ void set_identity(double* Q, int m) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < (int64_t)m * m) Q[t] = (t / m == t % m) ? 1.0 : 0.0;
}

__global__ void pad_copy(const double* __restrict__ src, int n, int64_t lds, double* __restrict__ dst,
                         int m) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * m) return;
  const int r = (int)(t / m), c = (int)(t % m);
  dst[t] = (r < n && c < n) ? 0.5 * (src[(int64_t)r * lds + c] + src[(int64_t)c * lds + r]) : 0.0;
}

// order[rank] = index, ranking by value descending (ties: lower index first).
__global__ void rank_desc(const double* __restrict__ d, int n, int* __restrict__ order) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double di = d[i];
  int rank = 0;
  for (int j = 0; j < n; ++j) {
    const double dj = d[j];
    rank += (dj > di) || (dj == di && j < i);
  }
  order[rank] = i;
}

// dst[:, j] = src[:, order[j]] for j < cols; evals_out[j] = evals[order[j]].
__global__ void permute_cols(const double* __restrict__ src, int64_t lds, int rows, int cols,
                             const int* __restrict__ order, double* __restrict__ dst,
                             int64_t ldd, const double* __restrict__ evals,
                             double* __restrict__ evals_out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < (int64_t)rows * cols) {
    const int r = (int)(t / cols), c = (int)(t % cols);
    dst[(int64_t)r * ldd + c] = src[(int64_t)r * lds + order[c]];
  }
  if (evals_out && t < cols) evals_out[t] = evals[order[t]];
}

// U_out[:, j] = sign_j * V[:, j], sign_j making the largest-magnitude entry positive
// (first row on ties).  One block per column.
__global__ void sign_fix_out(const double* __restrict__ V, int64_t ldv, int n,
                             double* __restrict__ U, int J) {
  __shared__ double bv[256];
  __shared__ int bi[256];
  const int j = blockIdx.x;
  double best = -1.0;
  int besti = 0x7fffffff;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double a = fabs(V[(int64_t)i * ldv + j]);
    if (a > best || (a == best && i < besti)) { best = a; besti = i; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = besti;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double a = bv[threadIdx.x + s];
      const int ai = bi[threadIdx.x + s];
      if (a > bv[threadIdx.x] || (a == bv[threadIdx.x] && ai < bi[threadIdx.x])) {
        bv[threadIdx.x] = a;
        bi[threadIdx.x] = ai;
      }
    }
    __syncthreads();
  }
  const double sg = (bi[0] < n && V[(int64_t)bi[0] * ldv + j] < 0.0) ? -1.0 : 1.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) U[(int64_t)i * J + j] = sg * V[(int64_t)i * ldv + j];
}

// Cholesky G = R^T R (R upper) and R^{-1}, one CTA; G is k x k symmetric (upper part read).
// shift is added to the diagonal first.  On a non-positive pivot sets DEV_CHOL_BREAKDOWN.
__global__ void __launch_bounds__(1024)
chol_inv_kernel(const double* __restrict__ G, int k, double shift, double* __restrict__ R,
                double* __restrict__ Rinv, int* status) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int64_t t = threadIdx.x; t < (int64_t)k * k; t += blockDim.x) {
    const int r = (int)(t / k), c = (int)(t % k);
    R[t] = (c >= r) ? G[t] + (r == c ? shift : 0.0) : 0.0;
  }
  __syncthreads();
  __shared__ double inv_s;
  for (int j = 0; j < k; ++j) {
    const double d = R[(int64_t)j * k + j];
    if (!(d > 0.0)) {
      if (threadIdx.x == 0) bad = 1;
      __syncthreads();
      break;
    }
    if (threadIdx.x == 0) inv_s = rsqrt(d);  // one thread: FP64 rsqrt is a long sequence
    __syncthreads();
    const double inv = inv_s;
    for (int c = j + threadIdx.x; c < k; c += blockDim.x)
      R[(int64_t)j * k + c] = (c == j) ? d * inv : R[(int64_t)j * k + c] * inv;
    __syncthreads();
    const int rem = k - j - 1;
    for (int64_t t = threadIdx.x; t < (int64_t)rem * rem; t += blockDim.x) {
      const int r = j + 1 + (int)(t / rem), c = j + 1 + (int)(t % rem);
      if (c >= r) R[(int64_t)r * k + c] -= R[(int64_t)j * k + r] * R[(int64_t)j * k + c];
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) atomicOr(status, DEV_CHOL_BREAKDOWN);
    return;
  }
  // Column c of R^{-1} by back substitution (one thread per column), with the reciprocal
  // diagonal formed once per row.
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    for (int i = 0; i < k; ++i) Rinv[(int64_t)i * k + c] = 0.0;
    Rinv[(int64_t)c * k + c] = 1.0 / R[(int64_t)c * k + c];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    for (int i = c - 1; i >= 0; --i) {
      double s = 0.0;
      for (int l = i + 1; l <= c; ++l) s = fma(R[(int64_t)i * k + l], Rinv[(int64_t)l * k + c], s);
      Rinv[(int64_t)i * k + c] = -s * Rinv[(int64_t)i * k + i];
    }
  }
}

// Cholesky G + shift I = R^T R without the inverse, for Cholesky-QR by triangular solves
// (k <= TRSM_MAX_K), spread over one cluster of CL CTAs (16 where the GPU can co-schedule them,
// else 8).  FP64 arithmetic on this part retires under two lanes per cycle per SM with a 64-cycle
// dependent latency, so a factorisation on one SM is bound by that rate; the cluster multiplies
// it by CL, and the serial pivot chain is kept to five dependent FP64 operations per pivot.  R is
// built in place in Rout (global memory, L2-resident).
//   A G within 2^-27 of the identity takes the first-order factor R = I + triu(F, 1) + diag(F)/2
// (G = I + F; exact to O(|F|^2) < eps) with no serial factorisation.
//   Otherwise right-looking by blocks of CHOL_NB rows.  For block row J (rows J0..J1-1):
//   1. every CTA factors the diagonal block and its own share of the panel columns (columns
//      J1 + b + CL s for CTA b), one or two elements of the block row per thread, by jb unscaled
//      elimination steps a[r][c] -= a[j][r] a[j][c] / d_j; the diagonal block is factored
//      redundantly by every CTA from identical data, so all CTAs take the same branches.  Row j+1
//      is published in shared memory as soon as step j has finished it; the thread holding the
//      next pivot forms its reciprocal (pivot_recip).  The rows are then scaled by
//      1 / sqrt(d_r) and the panel written back;
//   2. after a cluster barrier every CTA reads the whole panel P (jb x m) and the trailing upper
//      triangle takes W[q][c] -= sum_i P[i][q] P[i][c], its elements spread over all threads of
//      the cluster (rows q and m - 1 - q folded together so that every fold has m + 1 elements);
//      CTA 0 stores the diagonal block; a second cluster barrier ends the block.
// A non-positive pivot restarts the factorisation once with the shift
// 11 (n k + k (k + 1)) eps tr(G) (shifted Cholesky-QR, Fukaya et al. 2020) and sets
// DEV_CHOL_SHIFTED; if that fails too, DEV_CHOL_BREAKDOWN.  Outputs: R (k x k, upper, zero
// below) and rdinv[j] = 1 / R[j][j].
constexpr int TRSM_MAX_K = 384;
constexpr int CHOL_NB = 16;
constexpr int CHOL_THREADS = 512;
// Block-row elements per thread: jb (jb + 1) / 2 + jb ceil(m / CL) over CHOL_THREADS threads.
template <int CL>
__host__ __device__ constexpr int chol_slots() {
  return (CHOL_NB * (CHOL_NB + 1) / 2 + CHOL_NB * ((TRSM_MAX_K - CHOL_NB + CL - 1) / CL) +
          CHOL_THREADS - 1) / CHOL_THREADS;
}

// d > 0 (and not NaN) decided on the bit pattern with integer compares.
__device__ __forceinline__ bool positive_f64(double d) {
  const long long bits = __double_as_longlong(d);
  return bits > 0 && bits <= 0x7ff0000000000000ll;
}

// 1 / d for a normal d > 0: a seed x from the FP32 reciprocal of d's leading mantissa bits
// (relative error below 2^-22, formed with integer operations and one rcp.approx), then one
// third-order step x <- x (1 + e + e^2) with e = 1 - d x, which cubes the relative error (the
// Newton-Raphson step x (1 + e) only squares it), to FP64 rounding level in three dependent FMAs.
// Exponents outside [1, 2044] take the division.
__device__ __forceinline__ double pivot_recip(double d) {
  const long long bits = __double_as_longlong(d);
  const int e = (int)((bits >> 52) & 0x7ff);
  if (e < 1 || e > 2044) return 1.0 / d;
  const unsigned fm = 0x3f800000u | (unsigned)((bits >> 29) & 0x7fffff);  // mantissa in [1, 2)
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(__uint_as_float(fm)));
  const unsigned yb = __float_as_uint(y);                                  // y in (0.5, 1]
  const long long ye = (long long)((yb >> 23) & 0xff) - 127 + 1023 + (1023 - e);
  double x = __longlong_as_double((ye << 52) | ((long long)(yb & 0x7fffff) << 29));
  const double e1 = fma(-d, x, 1.0);
  return fma(x, fma(e1, e1, e1), x);
}

template <int CL>
__global__ void __launch_bounds__(CHOL_THREADS)
chol_cluster_kernel(const double* __restrict__ G, int k, int64_t nrows, double* Rout,
                    double* __restrict__ rdinv, int* __restrict__ status) {
  extern __shared__ double panel[];  // jb x m, row stride m
  __shared__ double rowbuf[2][CHOL_NB + 48];
  __shared__ double dinv_s[2];
  __shared__ double piv_s[CHOL_NB], ri_s[CHOL_NB];
  __shared__ double shift_s;
  __shared__ unsigned long long fmax_s;
  double* W = Rout;
  const int b = blockIdx.x, tid = threadIdx.x;
  constexpr int SLOTS = chol_slots<CL>();
  const int gtid = b * CHOL_THREADS + tid, gthreads = CL * CHOL_THREADS;
  // Whole-matrix passes: a row per warp, columns over the lanes (no index divisions).
  const int lane = tid & 31, nw = CHOL_THREADS / 32, gwarp = b * nw + (tid >> 5);
  {
    if (tid == 0) fmax_s = 0ull;
    __syncthreads();
    unsigned long long mb = 0ull;
    for (int r = tid >> 5; r < k; r += nw) {
      const double* Gr = G + (int64_t)r * k;
      for (int c = r + lane; c < k; c += 32) {
        double f = Gr[c];
        if (c == r) f -= 1.0;  // the only FP64 operation of the test
        const unsigned long long bb =
            (unsigned long long)__double_as_longlong(f) & 0x7fffffffffffffffull;
        mb = bb > mb ? bb : mb;
      }
    }
    atomicMax(&fmax_s, mb);
    __syncthreads();
    if (__longlong_as_double((long long)fmax_s) <= 7.450580596923828e-9) {
      for (int r = gwarp; r < k; r += CL * nw) {
        const double* Gr = G + (int64_t)r * k;
        double* Wr = W + (int64_t)r * k;
        for (int c = lane; c < k; c += 32) {
          double v = c > r ? Gr[c] : 0.0;
          if (c == r) {
            v = 0.5 * (1.0 + Gr[c]);
            rdinv[r] = 1.0 / v;
          }
          Wr[c] = v;
        }
      }
      return;  // uniform over the cluster: every CTA read the same G
    }
  }
  int attempt = 0;
  for (; attempt < 2; ++attempt) {
    if (tid == 0) {
      double sh = 0.0;
      if (attempt == 1) {
        double tr = 0.0;
        for (int i = 0; i < k; ++i) tr += G[(int64_t)i * k + i];
        sh = 11.0 * ((double)nrows * k + (double)k * (k + 1)) * 2.220446049250313e-16 * tr;
      }
      shift_s = sh;
    }
    __syncthreads();
    const double shift = shift_s;
    for (int r = gwarp; r < k; r += CL * nw) {
      const double* Gr = G + (int64_t)r * k;
      double* Wr = W + (int64_t)r * k;
      for (int c = lane; c < k; c += 32) {
        double v = c >= r ? Gr[c] : 0.0;
        if (c == r && attempt == 1) v += shift;
        Wr[c] = v;
      }
    }
    cluster_round_barrier();
    bool bad = false;
    for (int J0 = 0; J0 < k; J0 += CHOL_NB) {
      const int jb = min(CHOL_NB, k - J0), J1 = J0 + jb, m = k - J1;
      const int nc = m > b ? (m - b + CL - 1) / CL : 0;
      const int nelem = jb * nc + jb * (jb + 1) / 2;
      // This thread's elements of the block row: row r, rowbuf slot x (x < CHOL_NB: diagonal
      // column J0 + x; otherwise panel column J1 + b + CL (x - CHOL_NB)).
      int er[SLOTS], ex[SLOTS];
      double a[SLOTS];
#pragma unroll
      for (int e = 0; e < SLOTS; ++e) {
        const int idx = tid + e * CHOL_THREADS;
        er[e] = -1;
        ex[e] = 0;
        a[e] = 0.0;
        if (idx < nelem) {
          int rem = idx;
          for (int rr = 0; rr < jb; ++rr) {
            const int len = jb - rr + nc;
            if (rem < len) {
              er[e] = rr;
              ex[e] = rem < jb - rr ? rr + rem : CHOL_NB + rem - (jb - rr);
              break;
            }
            rem -= len;
          }
          const int col = ex[e] < CHOL_NB ? J0 + ex[e] : J1 + b + CL * (ex[e] - CHOL_NB);
          a[e] = __ldcg(W + (int64_t)(J0 + er[e]) * k + col);
          if (er[e] == 0) {
            rowbuf[0][ex[e]] = a[e];
            if (ex[e] == 0) {
              piv_s[0] = a[e];
              dinv_s[0] = pivot_recip(a[e]);
            }
          }
        }
      }
      for (int j = 0; j < jb; ++j) {
        __syncthreads();
        if (!positive_f64(rowbuf[j & 1][j])) {  // every thread of every CTA reads the same pivot
          bad = true;
          break;
        }
        const double dinv = dinv_s[j & 1];
#pragma unroll
        for (int e = 0; e < SLOTS; ++e) {
          if (er[e] > j) {
            const double f = rowbuf[j & 1][er[e]] * dinv;
            a[e] = fma(-f, rowbuf[j & 1][ex[e]], a[e]);
            if (er[e] == j + 1) {
              rowbuf[(j + 1) & 1][ex[e]] = a[e];
              if (ex[e] == j + 1) {
                piv_s[j + 1] = a[e];
                dinv_s[(j + 1) & 1] = pivot_recip(a[e]);
              }
            }
          }
        }
      }
      if (bad) break;
      __syncthreads();
      if (tid < jb) ri_s[tid] = rsqrt(piv_s[tid]);
      __syncthreads();
#pragma unroll
      for (int e = 0; e < SLOTS; ++e) {
        if (er[e] >= 0) {
          a[e] *= ri_s[er[e]];
          if (ex[e] >= CHOL_NB)
            W[(int64_t)(J0 + er[e]) * k + J1 + b + CL * (ex[e] - CHOL_NB)] = a[e];
        }
      }
      if (b == 0 && tid < jb) rdinv[J0 + tid] = ri_s[tid];
      cluster_round_barrier();
      for (int t = tid; t < jb * m; t += CHOL_THREADS) {
        const int i = t / m, c = t % m;
        panel[t] = __ldcg(W + (int64_t)(J0 + i) * k + J1 + c);
      }
      if (b == 0) {
#pragma unroll
        for (int e = 0; e < SLOTS; ++e)
          if (er[e] >= 0 && ex[e] < CHOL_NB) W[(int64_t)(J0 + er[e]) * k + J0 + ex[e]] = a[e];
      }
      __syncthreads();
      const int m1 = m + 1;
      const int total = ((m + 1) / 2) * m1;
      for (int f = gtid; f < total; f += gthreads) {
        const int p = f / m1, xx = f % m1;
        int q = p, c = p + xx;
        if (xx >= m - p) {
          q = m - 1 - p;
          if (q == p) continue;
          c = q + xx - (m - p);
        }
        double* w = W + (int64_t)(J1 + q) * k + J1 + c;
        double acc = __ldcg(w);
#pragma unroll
        for (int i = 0; i < CHOL_NB; ++i)
          if (i < jb) acc = fma(-panel[i * m + q], panel[i * m + c], acc);
        *w = acc;
      }
      cluster_round_barrier();
    }
    if (!bad) break;
    cluster_round_barrier();  // every CTA has stopped reading W before the restart rewrites it
  }
  if (b == 0 && tid == 0) {
    if (attempt == 2) atomicOr(status, DEV_CHOL_BREAKDOWN);
    else if (attempt == 1) atomicOr(status, DEV_CHOL_SHIFTED);
  }
}

// V <- V R^{-1} in place (x R = v for every row v of V), R upper k x k with rdinv = 1/diag(R).
// One warp per RW rows; lane l holds entries l, l + 32, ... of each row in registers, and the
// RW independent substitution chains are interleaved to hide their latency.  Skipped when the
// factorisation that made R broke down.
template <int KT, int RW>
__global__ void __launch_bounds__(64)
trsm_rows_kernel(double* __restrict__ V, int64_t ldv, int n, int k, const double* __restrict__ R,
                 const double* __restrict__ rdinv, const int* __restrict__ status) {
  if (*status & DEV_CHOL_BREAKDOWN) return;
  const int lane = threadIdx.x & 31;
  const int64_t row0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * RW;
  if (row0 >= n) return;
  double x[RW][KT];
#pragma unroll
  for (int w = 0; w < RW; ++w) {
    const bool valid = row0 + w < n;
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int l = 32 * t + lane;
      x[w][t] = (valid && l < k) ? V[(row0 + w) * ldv + l] : 0.0;
    }
  }
#pragma unroll
  for (int t = 0; t < KT; ++t) {
    const int jend = min(32, k - 32 * t);
    for (int jj = 0; jj < jend; ++jj) {
      const int j = 32 * t + jj;
      const double rd = __ldg(rdinv + j);
      double xj[RW];
#pragma unroll
      for (int w = 0; w < RW; ++w) {
        xj[w] = __shfl_sync(0xffffffffu, x[w][t], jj) * rd;
        if (lane == jj) x[w][t] = xj[w];
      }
      const double* Rj = R + (int64_t)j * k;
#pragma unroll
      for (int t2 = t; t2 < KT; ++t2) {
        const int l = 32 * t2 + lane;
        if (l > j && l < k) {
          const double r = __ldg(Rj + l);
#pragma unroll
          for (int w = 0; w < RW; ++w) x[w][t2] = fma(-xj[w], r, x[w][t2]);
        }
      }
    }
  }
#pragma unroll
  for (int w = 0; w < RW; ++w) {
    if (row0 + w >= n) break;
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int l = 32 * t + lane;
      if (l < k) V[(row0 + w) * ldv + l] = x[w][t];
    }
  }
}

// One row per warp, two warps per CTA: every row is a serial chain of k FP64 steps, and FP64
// issue is per SM sub-partition, so the rows are spread over as many sub-partitions as possible
// (8-warp CTAs left most of the SMs idle for n of a few hundred).
template <int KT>
void launch_trsm(double* V, int64_t ldv, int n, int k, const double* R, const double* rdinv,
                 const int* status, cudaStream_t s) {
  trsm_rows_kernel<KT, 1><<<ceil_div(n, 2), 64, 0, s>>>(V, ldv, n, k, R, rdinv, status);
}

int trsm_rows(double* V, int64_t ldv, int n, int k, const double* R, const double* rdinv,
              const int* status, cudaStream_t s) {
  if (n <= 0) return TUCKER_OK;
  switch ((k + 31) / 32) {
    case 1: launch_trsm<1>(V, ldv, n, k, R, rdinv, status, s); break;
    case 2: launch_trsm<2>(V, ldv, n, k, R, rdinv, status, s); break;
    case 3: launch_trsm<3>(V, ldv, n, k, R, rdinv, status, s); break;
    case 4: launch_trsm<4>(V, ldv, n, k, R, rdinv, status, s); break;
    case 5: launch_trsm<5>(V, ldv, n, k, R, rdinv, status, s); break;
    case 6: launch_trsm<6>(V, ldv, n, k, R, rdinv, status, s); break;
    case 7: launch_trsm<7>(V, ldv, n, k, R, rdinv, status, s); break;
    case 8: launch_trsm<8>(V, ldv, n, k, R, rdinv, status, s); break;
    case 9: launch_trsm<9>(V, ldv, n, k, R, rdinv, status, s); break;
    case 10: launch_trsm<10>(V, ldv, n, k, R, rdinv, status, s); break;
    case 11: launch_trsm<11>(V, ldv, n, k, R, rdinv, status, s); break;
    case 12: launch_trsm<12>(V, ldv, n, k, R, rdinv, status, s); break;
    default: return TUCKER_EINVAL;
  }
  TK_LAUNCH();
  return TUCKER_OK;
}

// r[j] = |W[:, j] - theta[j] V[:, j]|_2, one block per column.
__global__ void residual_norms(const double* __restrict__ W, const double* __restrict__ V,
                               int64_t ld, int n, const double* __restrict__ theta,
                               double* __restrict__ r) {
  __shared__ double ws[8];
  const int j = blockIdx.x;
  const double th = theta[j];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double d = W[(int64_t)i * ld + j] - th * V[(int64_t)i * ld + j];
    s = fma(d, d, s);
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    r[j] = sqrt(t);
  }
}

// Scales every column of V (n x cols, ld) to unit 2-norm (zero columns are left alone).
// One block per column.
__global__ void normalize_cols_inplace(double* V, int64_t ld, int n) {
  __shared__ double ws[8];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = V[(int64_t)i * ld + j];
    s = fma(v, v, s);
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    ws[0] = t > 0.0 ? 1.0 / sqrt(t) : 1.0;
  }
  __syncthreads();
  const double inv = ws[0];
  for (int i = threadIdx.x; i < n; i += blockDim.x) V[(int64_t)i * ld + j] *= inv;
}

// LS = L diag(lam) (n x nl, ld nl) and Lt = L^T (nl x n) from the first nl columns L of V.
__global__ void scaled_transpose(const double* __restrict__ V, int64_t ldv, int n, int nl,
                                 const double* __restrict__ lam, double* __restrict__ LS,
                                 double* __restrict__ Lt) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * nl) return;
  const int64_t i = t / nl, l = t % nl;
  const double v = V[i * ldv + l];
  LS[i * nl + l] = v * lam[l];
  Lt[l * n + i] = v;
}

// y += a * x over n contiguous elements.
__global__ void add_scaled(double* __restrict__ y, const double* __restrict__ x, double a,
                           int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) y[t] = fma(a, x[t], y[t]);
}

// Columns [c0, c1) of V (n x ld) from a counter-based hash: uniform in [-1, 1).
__global__ void random_cols(double* V, int64_t ld, int n, int c0, int c1, uint64_t seed) {
  const int64_t w = c1 - c0;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * w) return;
  const int64_t r = t / w, c = c0 + t % w;
  uint64_t z = seed + (uint64_t)(r * 1315423911ull + c * 2654435761ull + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  V[r * ld + c] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

int cooperative_grid(int work, size_t smem) {
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, jacobi_kernel, 256, smem);
  const int dev_max = per * num_sms();
  int want = (work + 255) / 256;
  if (want < 1) want = 1;
  return std::min(want, std::max(dev_max, 1));
}

// Chebyshev T_d(x) for x >= 1.
double cheb(int d, double x) { return cosh((double)d * acosh(std::max(x, 1.0))); }

}  // namespace

// Eigen-decomposition of the symmetric m_real x m_real matrix A (device, leading dimension
// lda) by Jacobi.  On return Qout (mreal x mreal, ld mreal) holds eigenvectors as columns in
// descending eigenvalue order and evals_out (mreal) the eigenvalues.
int jacobi_eig(const double* A, int mreal, int64_t lda, double* Qout, double* evals_out,
               cudaStream_t s, int* sweeps) {
  const int m = mreal + (mreal & 1);
  const int h = m / 2;
  Buf A0, A1, Q, ev, ord, ctl, rot;
  const int max_sweeps = 40;
  TK_TRY(A0.alloc(sizeof(double) * m * m, s));
  TK_TRY(A1.alloc(sizeof(double) * m * m, s));
  TK_TRY(Q.alloc(sizeof(double) * m * m, s));
  TK_TRY(ev.alloc(sizeof(double) * m, s));
  TK_TRY(ord.alloc(sizeof(int) * m, s));
  TK_TRY(ctl.alloc(sizeof(int) * 4, s));
  TK_TRY(rot.alloc(sizeof(unsigned) * max_sweeps, s));
  const int nb = ceil_div((int64_t)m * m, 256);
  pad_copy<<<nb, 256, 0, s>>>(A, mreal, lda, A0.as<double>(), m);
  TK_LAUNCH();
  TK_CUDA(cudaMemsetAsync(A1.p, 0, sizeof(double) * m * m, s));
  set_identity<<<nb, 256, 0, s>>>(Q.as<double>(), m);
  TK_LAUNCH();
  TK_CUDA(cudaMemsetAsync(ctl.p, 0, sizeof(int) * 4, s));
  TK_CUDA(cudaMemsetAsync(rot.p, 0, sizeof(unsigned) * max_sweeps, s));
  JacobiArgs g;
  g.A0 = A0.as<double>();
  g.A1 = A1.as<double>();
  g.Q = Q.as<double>();
  g.evals = ev.as<double>();
  g.m = m;
  g.mreal = mreal;
  g.max_sweeps = max_sweeps;
  g.tol = 1e-14;
  g.bar = (unsigned*)ctl.as<int>();   // words 0, 1
  g.status = ctl.as<int>() + 2;
  g.sweeps_out = ctl.as<int>() + 3;
  g.rot = rot.as<unsigned>();
  const size_t smem = (size_t)h * (4 * sizeof(double) + 2 * sizeof(int));
  if (smem > 48 * 1024)
    TK_CUDA(cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  const int work = h * (h + 1) / 2 + m * h;
  {
    ProfScope prof("jacobi_f64", s, 0.0, 0.0);
    count_launch();
    if (m <= CLUSTER_JACOBI_MAX_M) {
      // One cluster of 8 CTAs x 512 threads: rounds end with the hardware cluster barrier.
      g.cluster = 1;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(8, 1, 1);
      cfg.blockDim = dim3(512, 1, 1);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 8;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      TK_CUDA(cudaLaunchKernelEx(&cfg, jacobi_kernel, g));
    } else {
      g.cluster = 0;
      const int grid = cooperative_grid(std::min(work, 1 << 22), smem);
      void* args[] = {&g};
      TK_CUDA(cudaLaunchCooperativeKernel((void*)jacobi_kernel, grid, 256, args, smem, s));
    }
  }
  rank_desc<<<ceil_div(mreal, 256), 256, 0, s>>>(ev.as<double>(), mreal, ord.as<int>());
  TK_LAUNCH();
  permute_cols<<<ceil_div((int64_t)mreal * mreal, 256), 256, 0, s>>>(
      Q.as<double>(), m, mreal, mreal, ord.as<int>(), Qout, mreal, ev.as<double>(), evals_out);
  TK_LAUNCH();
  int hctl[4];
  TK_CUDA(cudaMemcpyAsync(hctl, ctl.p, sizeof(hctl), cudaMemcpyDeviceToHost, s));
  TK_TRY(host_sync(s));
  if (sweeps) *sweeps = hctl[3];
  if (hctl[2] & DEV_TIMEOUT) return TUCKER_ETIMEOUT;
  if (hctl[2] & DEV_NOT_CONVERGED) return TUCKER_ENOTCONV;
  return TUCKER_OK;
}

int sort_eig_desc(const double* Q, int64_t ldq, int m, const double* ev, double* Qout,
                  int64_t ldo, double* evals_out, cudaStream_t s) {
  Buf ord;
  TK_TRY(ord.alloc(sizeof(int) * m, s));
  rank_desc<<<ceil_div(m, 256), 256, 0, s>>>(ev, m, ord.as<int>());
  TK_LAUNCH();
  permute_cols<<<ceil_div((int64_t)m * m, 256), 256, 0, s>>>(Q, ldq, m, m, ord.as<int>(), Qout,
                                                             ldo, ev, evals_out);
  TK_LAUNCH();
  return TUCKER_OK;
}

namespace {

// The eigensolver's dense products.  Those of at least OZ_MIN_FLOPS run FP64-accurate on the
// tensor cores (gram_ozaki.cu: error-free slices, exact integer sums), with the slices of the
// filter operator cut once per operator; smaller ones run on the CUDA cores (FP32 in the mixed
// form's filter, FP64 otherwise).
constexpr double OZ_MIN_FLOPS = 2e7;

struct EigOps {
  cudaStream_t s = 0;
  int n = 0;
  const double* mop = nullptr;    // operator whose row slices are in msl (nullptr: none)
  const double* mop3 = nullptr;   // operator whose 3-slice row slices are in msl3
  OzSlices msl, msl3, a, b;
  int* status = nullptr;          // device word: DEV_TIMEOUT from the tensor-core kernels
  void invalidate() { mop = mop3 = nullptr; }
};

// FP32-class filter products (the mixed form) of at least this many flops run as 3-slice
// products on the tensor cores, smaller ones in FP32 on the CUDA cores.
constexpr double OZ3_MIN_FLOPS = 1e8;

// C (n x cols) = alpha Mop V + beta X + gamma Z, V n x cols (ld ldv).  With Mop32 (the mixed
// form's filter, which needs only FP32 accuracy) the product is FP32-class: 3-slice products of
// Mop on the tensor cores, or FP32 on the CUDA cores with Mop32.
int op_mv(EigOps& e, const double* Mop, const float* Mop32, const double* V, int64_t ldv,
          int cols, double alpha, double beta, const double* X, int64_t ldx, double gamma,
          const double* Z, int64_t ldz, double* C, int64_t ldc) {
  const int n = e.n;
  if (Mop32 && 2.0 * n * (double)n * cols >= OZ3_MIN_FLOPS) {
    if (e.mop3 != Mop) {
      TK_TRY(oz_split_rows(Mop, n, n, n, nullptr, 0, 0, OZ_F32_SLICES, &e.msl3, e.s));
      e.mop3 = Mop;
    }
    TK_TRY(oz_split_cols(V, ldv, n, cols, OZ_F32_SLICES, &e.b, e.s));
    return oz_gemm_nt(e.msl3, e.b, false, alpha, beta, X, ldx, gamma, Z, ldz, C, ldc, e.status,
                      e.s, "eig_mv_ozaki3");
  }
  if (Mop32)
    return gemm_nn_f32a(n, cols, n, alpha, Mop32, n, V, ldv, beta, X, ldx, gamma, Z, ldz, C, ldc,
                        e.s);
  if (2.0 * n * (double)n * cols >= OZ_MIN_FLOPS) {
    if (e.mop != Mop) {
      TK_TRY(oz_split_rows(Mop, n, n, n, nullptr, 0, 0, OZ_GEMM_SLICES, &e.msl, e.s));
      e.mop = Mop;
    }
    TK_TRY(oz_split_cols(V, ldv, n, cols, OZ_GEMM_SLICES, &e.b, e.s));
    return oz_gemm_nt(e.msl, e.b, false, alpha, beta, X, ldx, gamma, Z, ldz, C, ldc, e.status,
                      e.s, "eig_mv_ozaki");
  }
  return gemm_nn_f64(n, cols, n, alpha, Mop, n, V, ldv, beta, X, ldx, gamma, Z, ldz, C, ldc, e.s);
}

// C (ka x kb, ld ldc) = A^T B with A: K x ka (ld lda), B: K x kb (ld ldb).
int op_tn(EigOps& e, int ka, int kb, int64_t K, const double* A, int64_t lda, const double* B,
          int64_t ldb, double* C, int64_t ldc) {
  if (2.0 * ka * (double)kb * K >= OZ_MIN_FLOPS) {
    TK_TRY(oz_split_cols(A, lda, K, ka, OZ_GEMM_SLICES, &e.a, e.s));
    if (A == B && lda == ldb && ka == kb)
      return oz_gemm_nt(e.a, e.a, true, 1.0, 0.0, nullptr, 0, 0.0, nullptr, 0, C, ldc, e.status,
                        e.s, "eig_tn_ozaki");
    TK_TRY(oz_split_cols(B, ldb, K, kb, OZ_GEMM_SLICES, &e.b, e.s));
    return oz_gemm_nt(e.a, e.b, false, 1.0, 0.0, nullptr, 0, 0.0, nullptr, 0, C, ldc, e.status,
                      e.s, "eig_tn_ozaki");
  }
  return gemm_tn_f64(ka, kb, K, A, lda, B, ldb, C, ldc, e.s);
}

// C (m x cols) = alpha A B + beta X + gamma Z with A: m x K (ld lda), B: K x cols (ld ldb).
// The tensor-core products scale every row of A by its largest entry, so their error in C[i][j]
// is relative to max_k |A[i][k]| max_k |B[k][j]|.  In the solver's N-N products (V Q, W Q, the
// deflation) the rows of A mix columns of very different size (W = M V: row i is dominated by
// the theta_1 column), and the Ritz residuals of the small-theta columns need accuracy relative
// to their own size; those products have K <= k (small), so they run on the CUDA cores in FP64.
// Only long-K N-N products (not used by the solver today) go to the tensor cores.
constexpr int OZ_NN_MIN_K = 1024;
int op_nn(EigOps& e, int m, int cols, int K, double alpha, const double* A, int64_t lda,
          const double* B, int64_t ldb, double beta, const double* X, int64_t ldx, double gamma,
          const double* Z, int64_t ldz, double* C, int64_t ldc) {
  if (K >= OZ_NN_MIN_K && 2.0 * m * (double)cols * K >= OZ_MIN_FLOPS) {
    TK_TRY(oz_split_rows(A, lda, m, K, nullptr, 0, 0, OZ_GEMM_SLICES, &e.a, e.s));
    TK_TRY(oz_split_cols(B, ldb, K, cols, OZ_GEMM_SLICES, &e.b, e.s));
    return oz_gemm_nt(e.a, e.b, false, alpha, beta, X, ldx, gamma, Z, ldz, C, ldc, e.status,
                      e.s, "gemm_ozaki");
  }
  return gemm_nn_f64(m, cols, K, alpha, A, lda, B, ldb, beta, X, ldx, gamma, Z, ldz, C, ldc, e.s);
}

// Work arrays of cholqr2.
struct CholWork {
  double* T;     // n x k (only for k > TRSM_MAX_K)
  double* Gk;    // k x k
  double* R;     // k x k
  double* Ri;    // k x k (only for k > TRSM_MAX_K)
  double* rd;    // k
  int* stat;     // 8 status words, one per pass
};

// One pass for k > TRSM_MAX_K: explicit inverse and a GEMM (the factorisation then runs in
// global memory on one CTA; such k occur only for very large cores).
int cholqr_pass_inverse(EigOps& e, double* V, int64_t ldv, int n, int k, const CholWork& w,
                        int* stat, cudaStream_t s, bool* shifted) {
  TK_TRY(op_tn(e, k, k, n, V, ldv, V, ldv, w.Gk, k));
  double shift = 0.0;
  *shifted = false;
  for (int attempt = 0; attempt < 2; ++attempt) {
    TK_CUDA(cudaMemsetAsync(stat, 0, sizeof(int), s));
    {
      ProfScope prof("chol_f64", s, (double)k * k * k, 0.0);
      chol_inv_kernel<<<1, 1024, 0, s>>>(w.Gk, k, shift, w.R, w.Ri, stat);
    }
    TK_LAUNCH();
    int h = 0;
    TK_CUDA(cudaMemcpyAsync(&h, stat, sizeof(int), cudaMemcpyDeviceToHost, s));
    TK_TRY(host_sync(s));
    if (!(h & DEV_CHOL_BREAKDOWN)) break;
    if (attempt == 1) return TUCKER_EINTERNAL;
    std::vector<double> diag(k);
    TK_CUDA(cudaMemcpy2DAsync(diag.data(), sizeof(double), w.Gk, sizeof(double) * (k + 1),
                              sizeof(double), k, cudaMemcpyDeviceToHost, s));
    TK_TRY(host_sync(s));
    double tr = 0.0;
    for (double d : diag) tr += d;
    shift = 11.0 * ((double)n * k + (double)k * (k + 1)) * 2.220446049250313e-16 * tr;
    *shifted = true;
  }
  TK_TRY(op_nn(e, n, k, k, 1.0, V, ldv, w.Ri, k, 0.0, nullptr, 0, 0.0, nullptr, 0, w.T, k));
  TK_TRY(copy_cols_f64(n, k, w.T, k, V, ldv, s));
  return TUCKER_OK;
}

// Launch shape of chol_cluster_kernel<cl> (cluster dimension attached by the caller).
cudaLaunchConfig_t chol_launch_config(int cl, int k, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl, 1, 1);
  cfg.blockDim = dim3(CHOL_THREADS, 1, 1);
  cfg.dynamicSmemBytes = sizeof(double) * CHOL_NB * (size_t)std::max(k - 1, 1);
  cfg.stream = s;
  return cfg;
}

// Cluster size of the Cholesky: 16 CTAs (a non-portable size) when the GPU reports that such a
// cluster of this kernel fits, else the portable 8; 0 when neither can be configured.
int chol_cluster_size() {
  const int max_smem = (int)(sizeof(double) * CHOL_NB * (TRSM_MAX_K - 1));
  if (cudaFuncSetAttribute(chol_cluster_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           max_smem) != cudaSuccess)
    return 0;
  if (cudaFuncSetAttribute(chol_cluster_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           max_smem) == cudaSuccess &&
      cudaFuncSetAttribute(chol_cluster_kernel<16>,
                           cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = chol_launch_config(16, TRSM_MAX_K, nullptr);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, chol_cluster_kernel<16>, &cfg) == cudaSuccess &&
        clusters >= 1)
      return 16;
  }
  (void)cudaGetLastError();  // a refused non-portable size leaves no sticky error
  return 8;
}

// One pass for k <= TRSM_MAX_K, all on the device: G = V^T V, R = chol(G) (shifted on
// breakdown, flagged in *stat), V <- V R^{-1} by row-wise triangular solves.
int cholqr_pass(EigOps& e, double* V, int64_t ldv, int n, int k, const CholWork& w, int* stat,
                cudaStream_t s) {
  TK_TRY(op_tn(e, k, k, n, V, ldv, V, ldv, w.Gk, k));
  {
    ProfScope prof("chol_f64", s, (double)k * k * k / 3.0, 0.0);
    static const int cl = chol_cluster_size();
    TK_CUDA(cl > 0 ? cudaSuccess : cudaErrorLaunchOutOfResources);
    cudaLaunchConfig_t cfg = chol_launch_config(cl, k, s);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cl == 16)
      TK_CUDA(cudaLaunchKernelEx(&cfg, chol_cluster_kernel<16>, (const double*)w.Gk, k,
                                 (int64_t)n, w.R, w.rd, stat));
    else
      TK_CUDA(cudaLaunchKernelEx(&cfg, chol_cluster_kernel<8>, (const double*)w.Gk, k,
                                 (int64_t)n, w.R, w.rd, stat));
  }
  TK_LAUNCH();
  return trsm_rows(V, ldv, n, k, w.R, w.rd, stat, s);
}

// Cholesky-QR of the n x k block V (ld ldv), in place, until two clean passes (CholQR2).  A
// pass whose Gram matrix is not numerically positive definite is redone with a diagonal shift
// and does not count as clean.  Two passes are issued before the one host synchronisation that
// reads their status words.
int cholqr2(EigOps& e, double* V, int64_t ldv, int n, int k, const CholWork& w, cudaStream_t s) {
  if (k > TRSM_MAX_K) {
    int clean = 0;
    for (int pass = 0; pass < 8 && clean < 2; ++pass) {
      bool shifted = false;
      TK_TRY(cholqr_pass_inverse(e, V, ldv, n, k, w, w.stat, s, &shifted));
      if (!shifted) ++clean;
    }
    return clean >= 2 ? TUCKER_OK : TUCKER_EINTERNAL;
  }
  TK_CUDA(cudaMemsetAsync(w.stat, 0, sizeof(int) * 8, s));
  int issued = 0, clean = 0, checked = 0;
  int hs[8];
  while (clean < 2) {
    const int want = std::min(8, issued + (2 - clean));
    if (want <= issued) break;
    for (; issued < want; ++issued) TK_TRY(cholqr_pass(e, V, ldv, n, k, w, w.stat + issued, s));
    TK_CUDA(cudaMemcpyAsync(hs, w.stat, sizeof(int) * issued, cudaMemcpyDeviceToHost, s));
    TK_TRY(host_sync(s));
    for (; checked < issued; ++checked) {
      if (hs[checked] & DEV_CHOL_BREAKDOWN) return TUCKER_EINTERNAL;
      if (!(hs[checked] & DEV_CHOL_SHIFTED)) ++clean;
    }
  }
  return clean >= 2 ? TUCKER_OK : TUCKER_EINTERNAL;
}

// Va <- Va - L (L^T Va): the n x ka block Va (ld ldv) against nl locked columns L (ld ldl).
int deflate(EigOps& e, const double* L, int64_t ldl, double* Va, int64_t ldv, int n, int nl,
            int ka, double* P) {
  if (nl <= 0 || ka <= 0) return TUCKER_OK;
  TK_TRY(op_tn(e, nl, ka, n, L, ldl, Va, ldv, P, ka));
  TK_TRY(op_nn(e, n, ka, nl, -1.0, L, ldl, P, ka, 1.0, Va, ldv, 0.0, nullptr, 0, Va, ldv));
  return TUCKER_OK;
}

}  // namespace

namespace {
// Records the launches and host synchronisations of one solve as profile counters.
struct EigCounters {
  long long l0 = launch_count(), s0 = host_sync_count();
  ~EigCounters() {
    prof_count("eig_launches", (double)(launch_count() - l0));
    prof_count("eig_host_syncs", (double)(host_sync_count() - s0));
  }
};
}  // namespace

int eig_topk_f64(const double* M, int n, int J, const double* U0, double* U, double* lambda,
                 cudaStream_t s, EigStats* st, const float* M32, double tol) {
  EigCounters counters;
  ProfScope prof("eig_topk", s, 0.0, 0.0);
  EigStats local;
  if (!st) st = &local;
  *st = EigStats();
  if (n <= 0 || J <= 0 || J > n) return TUCKER_EINVAL;
  const int p = std::max(16, J / 2);
  const int k = std::min(n, J + p);
  if (n <= std::max(160, 2 * k)) {
    // All eigenpairs of M at once.
    st->direct = true;
    Buf Qf, ev;
    TK_TRY(Qf.alloc(sizeof(double) * n * n, s));
    TK_TRY(ev.alloc(sizeof(double) * n, s));
    SyevStats ss;
    TK_TRY(syev_refined(M, n, n, Qf.as<double>(), ev.as<double>(), 0.0, 0.1 * tol, s, &ss));
    st->jacobi_sweeps += ss.fp32_sweeps + ss.fp64_sweeps;
    st->refine_steps += ss.steps;
    st->fp64_fallbacks += ss.fallback;
    sign_fix_out<<<J, 256, 0, s>>>(Qf.as<double>(), n, n, U, J);
    TK_LAUNCH();
    std::vector<double> hev(n);
    TK_CUDA(cudaMemcpyAsync(hev.data(), ev.p, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    if (lambda) TK_CUDA(cudaMemcpyAsync(lambda, ev.p, sizeof(double) * J, cudaMemcpyDeviceToDevice, s));
    TK_TRY(host_sync(s));
    st->rank_deficient = !(hev[J - 1] > 1e-13 * std::max(hev[0], 1e-300));
    return TUCKER_OK;
  }

  bool use32 = M32 != nullptr;
  const int max_outer = 120, dmax = 24;
  const double growth_cap = 1e4, abs_cap = 1e8;
  Buf Vb, T1, T2, T3, H, Qh, evrn, Gk, R, Ri, rd, Tc, P, stat;
  Buf Md, Md32, LS, Lt, lamd;  // deflated filter operator and its factors
  TK_TRY(Md.alloc(sizeof(double) * n * n, s));
  if (M32) TK_TRY(Md32.alloc(sizeof(float) * n * n, s));
  TK_TRY(LS.alloc(sizeof(double) * n * k, s));
  TK_TRY(Lt.alloc(sizeof(double) * n * k, s));
  TK_TRY(lamd.alloc(sizeof(double) * k, s));
  const double* Mf = M;    // operator of the filter: M, then M with the locked pairs removed
  const float* Mf32 = M32;
  const size_t nk = sizeof(double) * (size_t)n * k;
  TK_TRY(Vb.alloc(nk, s));
  TK_TRY(T1.alloc(nk, s));
  TK_TRY(T2.alloc(nk, s));
  TK_TRY(T3.alloc(nk, s));
  TK_TRY(H.alloc(sizeof(double) * k * k, s));
  TK_TRY(Qh.alloc(sizeof(double) * k * k, s));
  TK_TRY(evrn.alloc(sizeof(double) * 2 * k, s));  // Ritz values [k], residual norms [k]
  double* evh = evrn.as<double>();
  double* rn = evh + k;
  TK_TRY(Gk.alloc(sizeof(double) * k * k, s));
  TK_TRY(R.alloc(sizeof(double) * k * k, s));
  TK_TRY(rd.alloc(sizeof(double) * k, s));
  if (k > TRSM_MAX_K) {
    TK_TRY(Ri.alloc(sizeof(double) * k * k, s));
    TK_TRY(Tc.alloc(nk, s));
  }
  TK_TRY(P.alloc(sizeof(double) * k * k, s));
  TK_TRY(stat.alloc(sizeof(int) * 8, s));
  const CholWork cw{Tc.as<double>(), Gk.as<double>(), R.as<double>(), Ri.as<double>(),
                    rd.as<double>(), stat.as<int>()};
  Buf ozst;
  TK_TRY(ozst.alloc(sizeof(int), s));
  TK_CUDA(cudaMemsetAsync(ozst.p, 0, sizeof(int), s));
  EigOps ops;
  ops.s = s;
  ops.n = n;
  ops.status = ozst.as<int>();
  double* V = Vb.as<double>();
  int c0 = 0;
  if (U0) {
    TK_TRY(copy_cols_f64(n, J, U0, J, V, k, s));
    c0 = J;
  }
  random_cols<<<ceil_div((int64_t)n * (k - c0), 256), 256, 0, s>>>(V, k, n, c0, k,
                                                                   0x5EEDull + (uint64_t)n * 131 + J);
  TK_LAUNCH();
  TK_TRY(cholqr2(ops, V, k, n, k, cw, s));
  // Power steps before the first Rayleigh-Ritz solve (which on a random block would buy
  // nothing): V <- orth(normalise(M V) + 1e-3 V).  The small multiple of V keeps the block of
  // full rank when M has fewer than k nonzero eigenvalues.  (A warm start with a single power
  // step costs more Rayleigh-Ritz iterations than the three steps it saves.)
  const int power_steps = 4;
  ProfScope prof_power("eig_power", s, 0.0, 0.0);
  for (int rep = 0; rep < power_steps; ++rep) {
    double* W = T1.as<double>();
    TK_TRY(op_mv(ops, M, use32 ? M32 : nullptr, V, k, k, 1.0, 0.0, nullptr, 0, 0.0, nullptr, 0, W,
                 k));
    st->matvecs++;
    normalize_cols_inplace<<<k, 256, 0, s>>>(W, k, n);
    TK_LAUNCH();
    add_scaled<<<ceil_div((int64_t)n * k, 256), 256, 0, s>>>(W, V, 1e-3, (int64_t)n * k);
    TK_LAUNCH();
    TK_TRY(copy_cols_f64(n, k, W, k, V, k, s));
    const int qs = cholqr2(ops, V, k, n, k, cw, s);
    if (qs != TUCKER_OK) {
      set_error_detail("eigensolver: Cholesky-QR failed in the initial power steps");
      return qs;
    }
  }

  prof_power.end();
  int nl = 0;
  double theta1 = 0.0;
  std::vector<double> locked_theta;
  std::vector<double> thrr(2 * (size_t)k);
  double* th = thrr.data();
  double* rr = th + k;
  bool done = false;
  for (int outer = 0; outer < max_outer; ++outer) {
    st->outer_iters = outer + 1;
    const int ka = k - nl;
    double* Va = V + nl;
    double* W = T1.as<double>();
    // Rayleigh-Ritz on the active block.
    ProfScope prof_rr("eig_rr", s, 0.0, 0.0);
    TK_TRY(op_mv(ops, M, nullptr, Va, k, ka, 1.0, 0.0, nullptr, 0, 0.0, nullptr, 0, W, ka));
    st->matvecs++;
    TK_TRY(op_tn(ops, ka, ka, n, Va, k, W, ka, H.as<double>(), ka));
    // Eigenpairs of H to a tenth of the locking tolerance (relative to the largest Ritz value
    // seen so far, or to |H| on the first solve).
    SyevStats ss;
    const int js = syev_refined(H.as<double>(), ka, ka, Qh.as<double>(), evh,
                                theta1, 0.1 * tol, s, &ss);
    st->jacobi_sweeps += ss.fp32_sweeps + ss.fp64_sweeps;
    st->refine_steps += ss.steps;
    st->fp64_fallbacks += ss.fallback;
    if (js != TUCKER_OK) return js;
    TK_TRY(op_nn(ops, n, ka, ka, 1.0, Va, k, Qh.as<double>(), ka, 0.0, nullptr, 0, 0.0, nullptr,
                 0, T2.as<double>(), ka));
    TK_TRY(op_nn(ops, n, ka, ka, 1.0, W, ka, Qh.as<double>(), ka, 0.0, nullptr, 0, 0.0, nullptr,
                 0, T3.as<double>(), ka));
    TK_TRY(copy_cols_f64(n, ka, T2.as<double>(), ka, Va, k, s));
    residual_norms<<<ka, 256, 0, s>>>(T3.as<double>(), T2.as<double>(), ka, n, evh, rn);
    TK_LAUNCH();
    // one copy of both (Ritz values in [0, k), residuals in [k, 2k))
    TK_CUDA(cudaMemcpyAsync(thrr.data(), evh, sizeof(double) * 2 * k, cudaMemcpyDeviceToHost, s));
    int ozs = 0;
    TK_CUDA(cudaMemcpyAsync(&ozs, ozst.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    TK_TRY(host_sync(s));
    if (ozs & DEV_TIMEOUT) {
      set_error_detail("eigensolver: a bounded wait in a tensor-core product gave up");
      return TUCKER_ETIMEOUT;
    }
    prof_rr.end();
    theta1 = std::max(theta1, th[0]);
    const double thr = tol * std::max(theta1, 1e-300);
    int nlock = 0;
    while (nlock < ka && nl + nlock < J && rr[nlock] <= thr) {
      locked_theta.push_back(th[nlock]);
      ++nlock;
    }
    nl += nlock;
    if (nl >= J) { done = true; break; }
    if (nlock > 0) {
      // Filter operator with the locked pairs removed: Md = M - L diag(theta_L) L^T.  Their
      // eigenvalues drop to ~0, inside the damped interval, so the filter needs no projection
      // at every step (only the final one below).
      ProfScope prof_lock("eig_lock", s, 0.0, 0.0);
      TK_CUDA(cudaMemcpyAsync(lamd.p, locked_theta.data(), sizeof(double) * nl,
                              cudaMemcpyHostToDevice, s));
      scaled_transpose<<<ceil_div((int64_t)n * nl, 256), 256, 0, s>>>(V, k, n, nl,
                                                                    lamd.as<double>(),
                                                                    LS.as<double>(),
                                                                    Lt.as<double>());
      TK_LAUNCH();
      TK_TRY(op_nn(ops, n, n, nl, -1.0, LS.as<double>(), nl, Lt.as<double>(), n, 1.0, M, n, 0.0,
                   nullptr, 0, Md.as<double>(), n));
      ops.invalidate();   // Md was rewritten: its slices must be cut again
      if (M32) TK_TRY(f64_to_f32(Md.as<double>(), Md32.as<float>(), (int64_t)n * n, s));
      Mf = Md.as<double>();
      Mf32 = M32 ? Md32.as<float>() : nullptr;
    }
    // Chebyshev filter on the remaining active columns.
    const int ka2 = k - nl;
    const double* tha = th + nlock;
    // Unwanted interval [0, b]; when M has fewer than k nonzero eigenvalues the smallest Ritz
    // value is ~0, so b is floored to keep the map (x - c) / e finite.
    const double b = std::max(tha[ka2 - 1], 1e-10 * theta1);
    const double cc = 0.5 * b, e = std::max(0.5 * b, 1e-300);
    const int jw = std::min(J - nl, ka2) - 1;  // last wanted active column
    const double gmax = (tha[0] - cc) / e, gw = (tha[jw] - cc) / e;
    // Degree: wanted columns may not outgrow the last wanted one by more than growth_cap, and
    // no column may grow by more than abs_cap (unwanted columns are not rescaled, so their
    // pollution by the largest active directions must stay far below 1/eps).
    int d = 1;
    while (d < dmax && cheb(d + 1, gmax) / cheb(d + 1, gw) <= growth_cap &&
           cheb(d + 1, gmax) <= abs_cap)
      ++d;
    // In the FP32-filter mode, switch the products to FP64 once the wanted residuals approach
    // the FP32 noise floor.
    if (use32) {
      double mres = 0.0;
      for (int i = nlock; i < ka && i < nlock + (J - nl); ++i) mres = std::max(mres, rr[i]);
      if (mres < 1e-5 * theta1) use32 = false;
    }
    // Filter-and-orthonormalise several times per Rayleigh-Ritz step: the product of two degree-d
    // filters grows like one of degree 2d, at the price of a Cholesky-QR2 instead of a Jacobi
    // eigensolve.  While an outlier holds the degree at 1 these are plain power steps.
    const int reps = d == 1 ? 4 : 2;
    double* Xa = V + nl;
    for (int rep = 0; rep < reps; ++rep) {
      double* Y0 = T1.as<double>();
      double* Y1 = T2.as<double>();
      ProfScope prof_filter("eig_filter", s, 0.0, 0.0);
      TK_TRY(copy_cols_f64(n, ka2, Xa, k, Y0, ka2, s));
      TK_TRY(op_mv(ops, Mf, use32 ? Mf32 : nullptr, Y0, ka2, ka2, 1.0 / e, -cc / e, Y0, ka2, 0.0,
                   nullptr, 0, Y1, ka2));
      st->matvecs++;
      for (int j = 2; j <= d; ++j) {
        // Y0 <- (2/e) M Y1 - (2c/e) Y1 - Y0, then swap roles.
        TK_TRY(op_mv(ops, Mf, use32 ? Mf32 : nullptr, Y1, ka2, ka2, 2.0 / e, -2.0 * cc / e, Y1,
                     ka2, -1.0, Y0, ka2, Y0, ka2));
        st->matvecs++;
        double* t = Y0; Y0 = Y1; Y1 = t;
      }
      TK_TRY(copy_cols_f64(n, ka2, Y1, ka2, Xa, k, s));
      prof_filter.end();
      ProfScope prof_orth("eig_orth", s, 0.0, 0.0);
      for (int dd = 0; dd < 2; ++dd) TK_TRY(deflate(ops, V, k, Xa, k, n, nl, ka2, P.as<double>()));
      normalize_cols_inplace<<<ka2, 256, 0, s>>>(Xa, k, n);
      TK_LAUNCH();
      const int qs = cholqr2(ops, Xa, k, n, ka2, cw, s);
      if (qs != TUCKER_OK) {
        char msg[256];
        snprintf(msg, sizeof(msg),
                 "eigensolver: Cholesky-QR failed (n=%d J=%d k=%d outer=%d locked=%d degree=%d)",
                 n, J, k, outer, nl, d);
        set_error_detail(msg);
        return qs;
      }
    }
  }
  prof_count("eig_outer", (double)st->outer_iters);
  if (!done) {
    char msg[160];
    snprintf(msg, sizeof(msg), "eigensolver: %d outer iterations, %d of %d locked (n=%d)",
             max_outer, nl, J, n);
    set_error_detail(msg);
    return TUCKER_ENOTCONV;
  }
  sign_fix_out<<<J, 256, 0, s>>>(V, k, n, U, J);
  TK_LAUNCH();
  if (lambda)
    TK_CUDA(cudaMemcpyAsync(lambda, locked_theta.data(), sizeof(double) * J,
                            cudaMemcpyHostToDevice, s));
  TK_TRY(host_sync(s));
  st->rank_deficient = !(locked_theta[J - 1] > 1e-13 * std::max(theta1, 1e-300));
  return TUCKER_OK;
}

}  // namespace tk
