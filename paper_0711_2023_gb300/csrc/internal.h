// Internal host-side interfaces between the translation units of the Tucker library.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>

#include "common.cuh"

namespace tk {

// One compressed mode ordering (n, m, o): nonzeros sorted by (i_n, i_m, i_o).
struct Ordering {
  bool built = false;
  int n = 0, m = 0, o = 0;
  int64_t F = 0;               // fibers (runs of equal (i_n, i_m))
  int64_t* root_ptr = nullptr; // [I_n + 1]
  int32_t* fiber_idx = nullptr;// [F]   i_m
  int32_t* fiber_root = nullptr;// [F]  i_n
  int64_t* fiber_ptr = nullptr;// [F + 1]
  int32_t* leaf_idx = nullptr; // [nnz] i_o
  double* val = nullptr;       // [nnz]
  float* val_f32 = nullptr;    // [nnz] (mixed path, built on demand)
  int32_t* fiber_map = nullptr;// [I_n * I_m] fiber id of (i_n, i_m) or -1 (built on demand)
};

}  // namespace tk

struct tucker_tensor_s {
  int64_t dims[3] = {0, 0, 0};
  int64_t nnz = 0;              // distinct nonzeros
  int32_t* idx[3] = {nullptr, nullptr, nullptr};  // canonical COO sorted by (i1, i2, i3)
  double* val = nullptr;
  double norm2 = 0.0;
  int device = 0;
  tk::Ordering ord[6];
};

namespace tk {

int ordering_slot(int n, int m, int o);  // 0..5, or -1 if not a permutation
int ensure_ordering(tucker_tensor_s* X, int n, int m, int o, cudaStream_t s, Ordering** out);
int ensure_fiber_map(tucker_tensor_s* X, Ordering* ord, cudaStream_t s);
int ensure_val_f32(tucker_tensor_s* X, Ordering* ord, cudaStream_t s);

// csf.cu
int build_canonical(tucker_tensor_s* X, const int32_t* d_i0, const int32_t* d_i1,
                    const int32_t* d_i2, const double* d_v, int64_t nnz_in, cudaStream_t s);
int build_ordering(tucker_tensor_s* X, Ordering* ord, cudaStream_t s);
int sum_squares(const double* d_v, int64_t n, double* d_out, cudaStream_t s);
// Exclusive prefix sum of n unsigned values (in may equal out); *d_total (device) gets the sum.
int exclusive_scan_u32(const unsigned* in, unsigned* out, int64_t n, unsigned* d_total,
                       cudaStream_t s);
int build_fiber_map(tucker_tensor_s* X, Ordering* ord, cudaStream_t s);

// sparse.cu (FP64)
int ttmc_f64(const tucker_tensor_s* X, const Ordering* ord, const double* Um, int Jm,
             const double* Uo, int Jo, double* Y, cudaStream_t s);
int slice_proj_f64(const tucker_tensor_s* X, const Ordering* ord, const double* Um, int Jm,
                   double* Y, cudaStream_t s);
// The same HOOI projection with the fibers' rank updates as per-slice FP64-accurate products on
// the tensor cores (gram_ozaki.cu), and the dispatcher between the two.
int ttmc_f64_tc(const tucker_tensor_s* X, const Ordering* ord, const double* Um, int Jm,
                const double* Uo, int Jo, double* Y, cudaStream_t s);
int ttmc_fp64(const tucker_tensor_s* X, const Ordering* ord, const double* Um, int Jm,
              const double* Uo, int Jo, double* Y, cudaStream_t s);
int unfolding_gram_f64(const tucker_tensor_s* X, const Ordering* rows, const Ordering* fibers,
                       double* M, cudaStream_t s);

// The slice projection and the HOOI projection on an explicit fiber list (a chunk of an
// ordering): Y[row[f] * ncol * Jm + col[f] * Jm + p] = sum over fiber f's leaves of x U_m[leaf, p];
// and Y[i] (i < nroots, Jm x Jo) from roots -> fibers (U_m rows) -> leaves (U_o rows).
int slice_proj_f64_fibers(int64_t F, const int32_t* row, const int32_t* col,
                          const int64_t* fiber_ptr, const int32_t* leaf_idx, const double* val,
                          const double* Um, int Jm, int64_t ncol, double* Y, cudaStream_t s);
int ttmc_f64_roots(int64_t nroots, const int64_t* root_ptr, const int32_t* fiber_idx,
                   const int64_t* fiber_ptr, const int32_t* leaf_idx, const double* val,
                   const double* Um, int Jm, const double* Uo, int Jo, double* Y, cudaStream_t s);

// dense.cu (FP64)
// C[m x n] = alpha * A[m x k] B[k x n] + beta * Xm + gamma * Zm (Xm, Zm optional, same shape
// as C; Xm may alias C).  All row-major with leading dimensions.
int gemm_nn_f64(int m, int n, int k, double alpha, const double* A, int64_t lda, const double* B,
                int64_t ldb, double beta, const double* Xm, int64_t ldx, double gamma,
                const double* Zm, int64_t ldz, double* C, int64_t ldc, cudaStream_t s);
// The same with A in FP32 and the products and sums in FP32 (B converted on load).
int gemm_nn_f32a(int m, int n, int k, double alpha, const float* A, int64_t lda, const double* B,
                 int64_t ldb, double beta, const double* Xm, int64_t ldx, double gamma,
                 const double* Zm, int64_t ldz, double* C, int64_t ldc, cudaStream_t s);
// C[m x n] = A^T B with A: k x m, B: k x n (row-major), deterministic split-K.
int gemm_tn_f64(int m, int n, int64_t k, const double* A, int64_t lda, const double* B,
                int64_t ldb, double* C, int64_t ldc, cudaStream_t s);
// M = Y1 Y1^T (+ Y2 Y2^T): rows x rows from row-major rows x K inputs; deterministic.
int syrk_f64(int rows, const double* Y1, int64_t K1, const double* Y2, int64_t K2, double* M,
             cudaStream_t s);
int copy_cols_f64(int rows, int cols, const double* src, int64_t lds, double* dst, int64_t ldd,
                  cudaStream_t s);
int scale_f64(int64_t n, double alpha, double* x, cudaStream_t s);

// mixed.cu (FP32 projections written as BF16 hi/lo pairs for the tensor-core Gram)
int f64_to_f32(const double* a, float* b, int64_t n, cudaStream_t s);
int f32_to_f64(const float* a, double* b, int64_t n, cudaStream_t s);
// a (rows x cols, dense) to FP32 rows of stride ldb >= cols, padding columns zeroed.
int f64_to_f32_rows(const double* a, int64_t rows, int cols, float* b, int64_t ldb,
                    cudaStream_t s);
// Factor row strides ldm, ldo (in floats).  Rows padded to a multiple of 4 floats, 16-byte
// aligned, let the slice projection load them as float4 (factor_ld32 gives that stride).
inline int64_t factor_ld32(int J) { return (J + 3) / 4 * 4; }
int ttmc_mixed(const tucker_tensor_s* X, const Ordering* o, const float* Um, int64_t ldm, int Jm,
               const float* Uo, int64_t ldo, int Jo, __nv_bfloat16* Yh, __nv_bfloat16* Yl,
               int64_t ldY, float* Y32, cudaStream_t s);
int slice_proj_mixed(const tucker_tensor_s* X, const Ordering* o, const float* Um, int64_t ldm,
                     int Jm, __nv_bfloat16* Yh, __nv_bfloat16* Yl, int64_t ldY, cudaStream_t s);

// gram_ozaki.cu: FP64-accurate products on the BF16 tensor cores (error-free splitting into
// 8-bit slices, exact integer level sums).  An operand is first cut into OzSlices: nslice BF16
// planes of a K-major (rows_pad x ldK) matrix and one scale exponent per row.
// nslice = 6 keeps 48 bits of every row's largest entry (error about 2^-47 max|a_i| max|b_j| per
// term); nslice = 7 keeps 56 bits, for products whose rows are dominated by one entry and whose
// small terms must stay accurate (the eigensolver's M V: M is strongly diagonal-dominant).
struct OzSlices {
  Buf Q, ex;
  int nslice = 6;
  int rows = 0, rows_pad = 0;
  int64_t ldK = 0;
};
// nslice = 3 keeps 24 bits (an FP32-class product, for the mixed form's filter).
constexpr int OZ_GRAM_SLICES = 6, OZ_GEMM_SLICES = 7, OZ_F32_SLICES = 3;
int64_t oz_ldk(int64_t K);
// Slices of the rows of [A | A2] (A: rows x K1, ld lda; A2 optional: rows x K2, ld lda2).
int oz_split_rows(const double* A, int64_t lda, int rows, int64_t K1, const double* A2,
                  int64_t lda2, int64_t K2, int nslice, OzSlices* out, cudaStream_t s);
// Slices of the columns of B (K x cols, ld ldb), i.e. of the rows of B^T.
int oz_split_cols(const double* B, int64_t ldb, int64_t K, int cols, int nslice, OzSlices* out,
                  cudaStream_t s);
// C (A.rows x B.rows, ld ldc) = alpha A B^T + beta X + gamma Z (X, Z optional; Z may alias C).
// sym: B is A, only the lower triangle is computed and it is mirrored (X, Z must be NULL or
// symmetric).  Timeouts set DEV_TIMEOUT in *status (device); prof_name names the profile record.
int oz_gemm_nt(const OzSlices& A, const OzSlices& B, bool sym, double alpha, double beta,
               const double* X, int64_t ldx, double gamma, const double* Z, int64_t ldz,
               double* C, int64_t ldc, int* status, cudaStream_t s, const char* prof_name);
// M = Y1 Y1^T (+ Y2 Y2^T), FP64-accurate; same arguments and result as syrk_f64.
int gram_f64_tc(int rows, const double* Y1, int64_t K1, const double* Y2, int64_t K2, double* M,
                cudaStream_t s);

// gram_fused.cu: M = sum over 1 or 2 terms of Gram((X x_m U_m^T)_(n)) in the mixed form, the
// projection built in shared memory and fed to the tensor cores (BF16x3), for I_n <= 256.
// ord[t] is ordering (n, o, m_t) with its FP32 values and fiber map; Um[t] FP32 (row stride ldm).
constexpr int FUSED_GRAM_MAX_ROWS = 256;
int gram_fused_mixed(const tucker_tensor_s* X, int n, int nterms, const Ordering* const ord[2],
                     const float* const Um[2], const int64_t ldm[2], const int Jm[2], double* M,
                     cudaStream_t s);

// gram_tc.cu: M = sum_t Y_t Y_t^T on tcgen05 with Y_t = hi + lo (BF16x3), FP64 result.
struct GramTerm {
  const __nv_bfloat16* hi;
  const __nv_bfloat16* lo;
  int64_t K;   // columns used
  int64_t ld;  // row stride in elements, a multiple of 64; columns K..ld-1 are zero
};
int64_t gram_ld(int64_t K);
int gram_bf16x3(int rows, int nterms, const GramTerm* terms, double* M, cudaStream_t s);

// eig.cu
struct EigStats {
  int outer_iters = 0;
  int matvecs = 0;
  int jacobi_sweeps = 0;     // FP32 pre-solve sweeps plus any FP64 Jacobi sweeps
  int refine_steps = 0;      // refinement steps of the small eigensolver
  int fp64_fallbacks = 0;    // small eigenproblems handed to the FP64 Jacobi
  bool direct = false;
  bool rank_deficient = false;
};
// Eigen-decomposition of the symmetric m x m matrix A (device, ld lda) by FP64 cyclic Jacobi:
// Qout (m x m, ld m) gets the eigenvectors as columns in descending eigenvalue order and
// evals_out (m) the eigenvalues.
int jacobi_eig(const double* A, int m, int64_t lda, double* Qout, double* evals_out,
               cudaStream_t s, int* sweeps);
// Columns of Q (m x m, ld ldq) reordered by descending ev into Qout (ld ldo), ev into evals_out.
int sort_eig_desc(const double* Q, int64_t ldq, int m, const double* ev, double* Qout,
                  int64_t ldo, double* evals_out, cudaStream_t s);

// autotune.cu: runs run(v) for the variant v kept for the shape class (family, a, b, c); on the
// class's first call (while tuning is enabled) times variants 0 and 1 once each on s, keeps the
// faster and runs it again.  With tuning disabled and no decision yet, runs variant 0.
enum { TUNE_TTMC_MIXED = 1, TUNE_SLICE_MIXED = 2 };
int autotune_run(int family, int a, int b, int c, const std::function<int(int)>& run,
                 cudaStream_t s);

// syev.cu: the same contract as jacobi_eig, solved in FP32 and refined in FP64 until every
// column's off-diagonal mass of X^T A X is below acc_rel * max(|A|_2, scale) and X is
// orthonormal to 1e-12; falls back to jacobi_eig for m > SYEV_REFINED_MAX_M or when a
// near-degenerate cluster does not resolve.
constexpr int SYEV_REFINED_MAX_M = 160;
struct SyevStats {
  int steps = 0;
  int fp32_sweeps = 0;
  int fp64_sweeps = 0;
  bool fallback = false;
  double offdiag = 0.0;  // accepted off-diagonal mass relative to max(|A|_2, scale)
  double orth = 0.0;
};
int syev_refined(const double* A, int m, int64_t lda, double* Qout, double* evals_out,
                 double scale, double acc_rel, cudaStream_t s, SyevStats* st);
// Leading J eigenvectors of the symmetric PSD n x n matrix M (device).  U0 (n x J, may be
// NULL) warm-starts; U (n x J) and lambda (J, may be NULL) receive the result.  Locking
// residual |M v - theta v| <= tol * theta_1.  With M32 (an FP32 copy of M) the Chebyshev
// filter's products run in FP32 until the residuals near the FP32 noise floor; Rayleigh-Ritz,
// residuals and Cholesky-QR2 are always FP64.
constexpr double EIG_TOL_FP64 = 3e-13;
constexpr double EIG_TOL_MIXED = 1e-6;
int eig_topk_f64(const double* M, int n, int J, const double* U0, double* U, double* lambda,
                 cudaStream_t s, EigStats* st, const float* M32 = nullptr,
                 double tol = EIG_TOL_FP64);

// core / fit (api.cu)
// dst (rows x cols, row-major) = src with every column scaled to unit length (zero columns
// stay zero): the random start of Figures sp3 and sp4.
int normalize_columns(const double* src, int rows, int cols, double* dst, cudaStream_t s);
// *fit_dev = 1 - sqrt(max(0, nX2 - *g2_dev)) / sqrt(nX2) (fit equation, norm identity).
int fit_on_device(double nX2, const double* g2_dev, double* fit_dev, cudaStream_t s);
int core_from_ttmc3(const double* Y3, int I3, int J1, int J2, const double* C, int J3,
                    double* G, double* g2_dev, cudaStream_t s);

}  // namespace tk
