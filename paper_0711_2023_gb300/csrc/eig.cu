// Leading-J eigenvectors of a symmetric positive semi-definite matrix M (n x n, FP64): the
// "J_n leading eigenvectors of ..." step of every method (Figures HO-SVD3, hooi3, sp3, mp3).
//
// Method (all FP64):
//   * small n: cyclic two-sided Jacobi on M itself (Golub & Van Loan, Sec. 8.5, parallel
//     round-robin ordering) in one cooperative launch;
//   * otherwise block subspace iteration on k = J + p columns with
//       - Rayleigh-Ritz: H = V^T M V, eigenpairs of H by the same Jacobi kernel, V <- V Q;
//       - locking: leading Ritz pairs with residual |M v - theta v| <= tol * theta_1 are
//         frozen; later products are projected against them;
//       - Chebyshev filtering (Zhou & Saad's filtered subspace iteration): p_d(M) with the
//         unwanted interval [0, theta_k] mapped to [-1, 1]; each column is rescaled by
//         1/T_d of its Ritz value and d is capped so that no column outgrows the last wanted
//         one by more than a fixed factor, which keeps the block well conditioned;
//       - Cholesky-QR2 orthonormalisation (R = chol(V^T V), V <- V R^-1, twice), with a
//         shifted first pass if the Gram matrix is not numerically positive definite.
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
};

__global__ void __launch_bounds__(256) jacobi_kernel(JacobiArgs g) {
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
  unsigned int epoch = 0;
  int sweep = 0;
  bool alive = true;
  for (; sweep < g.max_sweeps && alive; ++sweep) {
    for (int r = 0; r < m - 1 && alive; ++r) {
      for (int i = threadIdx.x; i < h; i += blockDim.x) {
        const int a = rr_index(i, r, m), b = rr_index(m - 1 - i, r, m);
        const int p = min(a, b), q = max(a, b);
        const double app = Acur[(int64_t)p * m + p], aqq = Acur[(int64_t)q * m + q];
        const double apq = Acur[(int64_t)p * m + q];
        double c = 1.0, s = 0.0, np = app, nq = aqq;
        if (q < g.mreal && fabs(apq) > abs_tol && fabs(apq) > g.tol * sqrt(fabs(app * aqq))) {
          const double tau = (aqq - app) / (2.0 * apq);
          const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + t * t);
          s = t * c;
          np = app - t * apq;
          nq = aqq + t * apq;
          if (blockIdx.x == 0) atomicAdd(&g.rot[sweep], 1u);
        }
        cs[i] = c; sn[i] = s; dp[i] = np; dq[i] = nq; pi[i] = p; qi[i] = q;
      }
      __syncthreads();
      for (int64_t t = gtid; t < ntri; t += gsize) {
        int K = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
        while ((int64_t)K * (K + 1) / 2 > t) --K;
        while ((int64_t)(K + 1) * (K + 2) / 2 <= t) ++K;
        const int I = (int)(t - (int64_t)K * (K + 1) / 2);
        const int p = pi[I], q = qi[I];
        if (I == K) {
          Anext[(int64_t)p * m + p] = dp[I];
          Anext[(int64_t)q * m + q] = dq[I];
          Anext[(int64_t)p * m + q] = 0.0;
          Anext[(int64_t)q * m + p] = 0.0;
        } else {
          const int u = pi[K], v = qi[K];
          const double c1 = cs[I], s1 = sn[I], c2 = cs[K], s2 = sn[K];
          const double apu = Acur[(int64_t)p * m + u], apv = Acur[(int64_t)p * m + v];
          const double aqu = Acur[(int64_t)q * m + u], aqv = Acur[(int64_t)q * m + v];
          const double rpu = c1 * apu - s1 * aqu, rpv = c1 * apv - s1 * aqv;
          const double rqu = s1 * apu + c1 * aqu, rqv = s1 * apv + c1 * aqv;
          const double bpu = c2 * rpu - s2 * rpv, bpv = s2 * rpu + c2 * rpv;
          const double bqu = c2 * rqu - s2 * rqv, bqv = s2 * rqu + c2 * rqv;
          Anext[(int64_t)p * m + u] = bpu; Anext[(int64_t)u * m + p] = bpu;
          Anext[(int64_t)p * m + v] = bpv; Anext[(int64_t)v * m + p] = bpv;
          Anext[(int64_t)q * m + u] = bqu; Anext[(int64_t)u * m + q] = bqu;
          Anext[(int64_t)q * m + v] = bqv; Anext[(int64_t)v * m + q] = bqv;
        }
      }
      for (int64_t t = gtid; t < (int64_t)m * h; t += gsize) {
        const int row = (int)(t / h), I = (int)(t % h);
        const double c = cs[I], s = sn[I];
        if (s == 0.0) continue;
        double* Qr = g.Q + (int64_t)row * m;
        const double qp = Qr[pi[I]], qq = Qr[qi[I]];
        Qr[pi[I]] = c * qp - s * qq;
        Qr[qi[I]] = s * qp + c * qq;
      }
      alive = grid_barrier(g.bar, gridDim.x, &epoch, g.status);
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
  for (int j = 0; j < k; ++j) {
    const double d = R[(int64_t)j * k + j];
    if (!(d > 0.0)) {
      if (threadIdx.x == 0) bad = 1;
      __syncthreads();
      break;
    }
    const double rjj = sqrt(d);
    __syncthreads();
    for (int c = j + threadIdx.x; c < k; c += blockDim.x)
      R[(int64_t)j * k + c] = (c == j) ? rjj : R[(int64_t)j * k + c] / rjj;
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
  // Column c of R^{-1} by back substitution (one thread per column).
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    for (int i = 0; i < k; ++i) Rinv[(int64_t)i * k + c] = 0.0;
    Rinv[(int64_t)c * k + c] = 1.0 / R[(int64_t)c * k + c];
    for (int i = c - 1; i >= 0; --i) {
      double s = 0.0;
      for (int l = i + 1; l <= c; ++l) s = fma(R[(int64_t)i * k + l], Rinv[(int64_t)l * k + c], s);
      Rinv[(int64_t)i * k + c] = -s / R[(int64_t)i * k + i];
    }
  }
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
  static int dev_max = 0;
  static size_t dev_smem = (size_t)-1;
  if (dev_smem != smem) {
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, jacobi_kernel, 256, smem);
    dev_max = per * num_sms();
    dev_smem = smem;
  }
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
  const int work = std::max(h * (h + 1) / 2, m * h);
  const int grid = cooperative_grid(std::min(work, 1 << 22), smem);
  void* args[] = {&g};
  {
    ProfScope prof("jacobi_f64", s, 0.0, 0.0);
    count_launch();
    TK_CUDA(cudaLaunchCooperativeKernel((void*)jacobi_kernel, grid, 256, args, smem, s));
  }
  rank_desc<<<ceil_div(mreal, 256), 256, 0, s>>>(ev.as<double>(), mreal, ord.as<int>());
  TK_LAUNCH();
  permute_cols<<<ceil_div((int64_t)mreal * mreal, 256), 256, 0, s>>>(
      Q.as<double>(), m, mreal, mreal, ord.as<int>(), Qout, mreal, ev.as<double>(), evals_out);
  TK_LAUNCH();
  int hctl[4];
  TK_CUDA(cudaMemcpyAsync(hctl, ctl.p, sizeof(hctl), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  if (sweeps) *sweeps = hctl[3];
  if (hctl[2] & DEV_TIMEOUT) return TUCKER_ETIMEOUT;
  if (hctl[2] & DEV_NOT_CONVERGED) return TUCKER_ENOTCONV;
  return TUCKER_OK;
}

namespace {

// Cholesky-QR of the n x k block V (ld ldv), in place, until two clean passes (CholQR2).
// A pass whose Gram matrix is not numerically positive definite is redone with a diagonal
// shift (shifted Cholesky-QR, Fukaya et al. 2020) and does not count as clean.
int cholqr2(double* V, int64_t ldv, int n, int k, double* T, double* Gk, double* R, double* Ri,
            int* dstat, cudaStream_t s) {
  int clean = 0;
  for (int pass = 0; pass < 8 && clean < 2; ++pass) {
    TK_TRY(gemm_tn_f64(k, k, n, V, ldv, V, ldv, Gk, k, s));
    double shift = 0.0;
    bool shifted = false;
    for (int attempt = 0; attempt < 2; ++attempt) {
      TK_CUDA(cudaMemsetAsync(dstat, 0, sizeof(int), s));
      chol_inv_kernel<<<1, 1024, 0, s>>>(Gk, k, shift, R, Ri, dstat);
      TK_LAUNCH();
      int h = 0;
      TK_CUDA(cudaMemcpyAsync(&h, dstat, sizeof(int), cudaMemcpyDeviceToHost, s));
      TK_CUDA(cudaStreamSynchronize(s));
      if (!(h & DEV_CHOL_BREAKDOWN)) break;
      if (attempt == 1) return TUCKER_EINTERNAL;
      // shift = 11 (n k + k (k + 1)) eps |G|_2, with |G|_2 bounded by the trace.
      std::vector<double> diag(k);
      TK_CUDA(cudaMemcpy2DAsync(diag.data(), sizeof(double), Gk, sizeof(double) * (k + 1),
                                sizeof(double), k, cudaMemcpyDeviceToHost, s));
      TK_CUDA(cudaStreamSynchronize(s));
      double tr = 0.0;
      for (double d : diag) tr += d;
      shift = 11.0 * ((double)n * k + (double)k * (k + 1)) * 2.220446049250313e-16 * tr;
      shifted = true;
    }
    TK_TRY(gemm_nn_f64(n, k, k, 1.0, V, ldv, Ri, k, 0.0, nullptr, 0, 0.0, nullptr, 0, T, k, s));
    TK_TRY(copy_cols_f64(n, k, T, k, V, ldv, s));
    if (!shifted) ++clean;
  }
  return clean >= 2 ? TUCKER_OK : TUCKER_EINTERNAL;
}

// Va <- Va - L (L^T Va): the n x ka block Va (ld ldv) against nl locked columns L (ld ldl).
int deflate(const double* L, int64_t ldl, double* Va, int64_t ldv, int n, int nl, int ka,
            double* P, cudaStream_t s) {
  if (nl <= 0 || ka <= 0) return TUCKER_OK;
  TK_TRY(gemm_tn_f64(nl, ka, n, L, ldl, Va, ldv, P, ka, s));
  TK_TRY(gemm_nn_f64(n, ka, nl, -1.0, L, ldl, P, ka, 1.0, Va, ldv, 0.0, nullptr, 0, Va, ldv, s));
  return TUCKER_OK;
}

}  // namespace

int eig_topk_f64(const double* M, int n, int J, const double* U0, double* U, double* lambda,
                 cudaStream_t s, EigStats* st, const float* M32, double tol) {
  EigStats local;
  if (!st) st = &local;
  *st = EigStats();
  if (n <= 0 || J <= 0 || J > n) return TUCKER_EINVAL;
  const int p = std::max(16, J / 2);
  const int k = std::min(n, J + p);
  if (n <= std::max(160, 2 * k)) {
    // Full Jacobi on M.
    st->direct = true;
    Buf Qf, ev;
    TK_TRY(Qf.alloc(sizeof(double) * n * n, s));
    TK_TRY(ev.alloc(sizeof(double) * n, s));
    TK_TRY(jacobi_eig(M, n, n, Qf.as<double>(), ev.as<double>(), s, &st->jacobi_sweeps));
    sign_fix_out<<<J, 256, 0, s>>>(Qf.as<double>(), n, n, U, J);
    TK_LAUNCH();
    std::vector<double> hev(n);
    TK_CUDA(cudaMemcpyAsync(hev.data(), ev.p, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    if (lambda) TK_CUDA(cudaMemcpyAsync(lambda, ev.p, sizeof(double) * J, cudaMemcpyDeviceToDevice, s));
    TK_CUDA(cudaStreamSynchronize(s));
    st->rank_deficient = !(hev[J - 1] > 1e-13 * std::max(hev[0], 1e-300));
    return TUCKER_OK;
  }

  bool use32 = M32 != nullptr;
  const int max_outer = 120, dmax = 24;
  const double growth_cap = 1e4, abs_cap = 1e8;
  Buf Vb, T1, T2, T3, H, Qh, evh, Gk, R, Ri, P, rn, stat;
  const size_t nk = sizeof(double) * (size_t)n * k;
  TK_TRY(Vb.alloc(nk, s));
  TK_TRY(T1.alloc(nk, s));
  TK_TRY(T2.alloc(nk, s));
  TK_TRY(T3.alloc(nk, s));
  TK_TRY(H.alloc(sizeof(double) * k * k, s));
  TK_TRY(Qh.alloc(sizeof(double) * k * k, s));
  TK_TRY(evh.alloc(sizeof(double) * k, s));
  TK_TRY(Gk.alloc(sizeof(double) * k * k, s));
  TK_TRY(R.alloc(sizeof(double) * k * k, s));
  TK_TRY(Ri.alloc(sizeof(double) * k * k, s));
  TK_TRY(P.alloc(sizeof(double) * k * k, s));
  TK_TRY(rn.alloc(sizeof(double) * k, s));
  TK_TRY(stat.alloc(sizeof(int), s));
  double* V = Vb.as<double>();
  int c0 = 0;
  if (U0) {
    TK_TRY(copy_cols_f64(n, J, U0, J, V, k, s));
    c0 = J;
  }
  random_cols<<<ceil_div((int64_t)n * (k - c0), 256), 256, 0, s>>>(V, k, n, c0, k,
                                                                   0x5EEDull + (uint64_t)n * 131 + J);
  TK_LAUNCH();
  TK_TRY(cholqr2(V, k, n, k, T1.as<double>(), Gk.as<double>(), R.as<double>(), Ri.as<double>(),
                 stat.as<int>(), s));

  int nl = 0;
  double theta1 = 0.0;
  std::vector<double> locked_theta;
  std::vector<double> th(k), rr(k);
  bool done = false;
  for (int outer = 0; outer < max_outer; ++outer) {
    st->outer_iters = outer + 1;
    const int ka = k - nl;
    double* Va = V + nl;
    double* W = T1.as<double>();
    // Rayleigh-Ritz on the active block.
    TK_TRY(gemm_nn_f64(n, ka, n, 1.0, M, n, Va, k, 0.0, nullptr, 0, 0.0, nullptr, 0, W, ka, s));
    st->matvecs++;
    TK_TRY(gemm_tn_f64(ka, ka, n, Va, k, W, ka, H.as<double>(), ka, s));
    int sw = 0;
    const int js = jacobi_eig(H.as<double>(), ka, ka, Qh.as<double>(), evh.as<double>(), s, &sw);
    st->jacobi_sweeps += sw;
    if (js != TUCKER_OK) return js;
    TK_TRY(gemm_nn_f64(n, ka, ka, 1.0, Va, k, Qh.as<double>(), ka, 0.0, nullptr, 0, 0.0, nullptr,
                       0, T2.as<double>(), ka, s));
    TK_TRY(gemm_nn_f64(n, ka, ka, 1.0, W, ka, Qh.as<double>(), ka, 0.0, nullptr, 0, 0.0, nullptr,
                       0, T3.as<double>(), ka, s));
    TK_TRY(copy_cols_f64(n, ka, T2.as<double>(), ka, Va, k, s));
    residual_norms<<<ka, 256, 0, s>>>(T3.as<double>(), T2.as<double>(), ka, n, evh.as<double>(),
                                      rn.as<double>());
    TK_LAUNCH();
    TK_CUDA(cudaMemcpyAsync(th.data(), evh.p, sizeof(double) * ka, cudaMemcpyDeviceToHost, s));
    TK_CUDA(cudaMemcpyAsync(rr.data(), rn.p, sizeof(double) * ka, cudaMemcpyDeviceToHost, s));
    TK_CUDA(cudaStreamSynchronize(s));
    theta1 = std::max(theta1, th[0]);
    const double thr = tol * std::max(theta1, 1e-300);
    int nlock = 0;
    while (nlock < ka && nl + nlock < J && rr[nlock] <= thr) {
      locked_theta.push_back(th[nlock]);
      ++nlock;
    }
    nl += nlock;
    if (nl >= J) { done = true; break; }
    // Chebyshev filter on the remaining active columns.
    const int ka2 = k - nl;
    const double* tha = th.data() + nlock;
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
      TK_TRY(copy_cols_f64(n, ka2, Xa, k, Y0, ka2, s));
      if (use32)
        TK_TRY(gemm_nn_f32a(n, ka2, n, 1.0 / e, M32, n, Y0, ka2, -cc / e, Y0, ka2, 0.0, nullptr,
                            0, Y1, ka2, s));
      else
        TK_TRY(gemm_nn_f64(n, ka2, n, 1.0 / e, M, n, Y0, ka2, -cc / e, Y0, ka2, 0.0, nullptr, 0,
                           Y1, ka2, s));
      st->matvecs++;
      TK_TRY(deflate(V, k, Y1, ka2, n, nl, ka2, P.as<double>(), s));
      for (int j = 2; j <= d; ++j) {
        // Y0 <- (2/e) M Y1 - (2c/e) Y1 - Y0, then swap roles.
        if (use32)
          TK_TRY(gemm_nn_f32a(n, ka2, n, 2.0 / e, M32, n, Y1, ka2, -2.0 * cc / e, Y1, ka2, -1.0,
                              Y0, ka2, Y0, ka2, s));
        else
          TK_TRY(gemm_nn_f64(n, ka2, n, 2.0 / e, M, n, Y1, ka2, -2.0 * cc / e, Y1, ka2, -1.0, Y0,
                             ka2, Y0, ka2, s));
        st->matvecs++;
        TK_TRY(deflate(V, k, Y0, ka2, n, nl, ka2, P.as<double>(), s));
        double* t = Y0; Y0 = Y1; Y1 = t;
      }
      TK_TRY(copy_cols_f64(n, ka2, Y1, ka2, Xa, k, s));
      for (int dd = 0; dd < 2; ++dd) TK_TRY(deflate(V, k, Xa, k, n, nl, ka2, P.as<double>(), s));
      normalize_cols_inplace<<<ka2, 256, 0, s>>>(Xa, k, n);
      TK_LAUNCH();
      const int qs = cholqr2(Xa, k, n, ka2, T3.as<double>(), Gk.as<double>(), R.as<double>(),
                             Ri.as<double>(), stat.as<int>(), s);
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
  TK_CUDA(cudaStreamSynchronize(s));
  st->rank_deficient = !(locked_theta[J - 1] > 1e-13 * std::max(theta1, 1e-300));
  return TUCKER_OK;
}

}  // namespace tk
