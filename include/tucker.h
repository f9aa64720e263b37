/*
 * tucker.h -- C ABI of the GB300 sparse third-order Tucker library.
 *
 * The library computes the four decompositions evaluated in Turney, "Empirical Evaluation of
 * Four Tensor Decomposition Algorithms" (2007): HO-SVD (Figure HO-SVD3), HOOI (Figure hooi3),
 * Slice Projection (Figure sp3) and Multislice Projection (Figure mp3), on a sparse tensor
 * X of size I1 x I2 x I3, returning a core G of size J1 x J2 x J3 and factors A, B, C with
 * orthonormal columns such that X ~ [[G; A, B, C]] (Tucker operator, Section 2), plus the
 * fit 1 - |X - Xhat|_F / |X|_F (fit equation, Section 2).  Every step runs in CUDA kernels
 * on the current GPU; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 *   - Status: every function returns TUCKER_OK (0) or a negative tucker_status;
 *     tucker_strerror() names it.  On error no output is guaranteed to be written.
 *   - Indices are 0-based.  Dense matrices are row-major: factor U_n is I_n x J_n with
 *     element (i, p) at U[i * J_n + p].  The core is row-major: g[(p * J2 + q) * J3 + r].
 *   - Memory: a `where` field / argument says whether a pointer is host (TUCKER_HOST) or
 *     device (TUCKER_DEVICE) memory.  Pointers named d_* are always device memory.
 *   - Ownership: the library never keeps a caller pointer after a call returns.  Outputs are
 *     allocated by the caller; sizes follow from dims and J.  Library work buffers are taken
 *     from the device with stream-ordered allocation and returned before the call returns.
 *   - Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).  All entry
 *     points are synchronous: when they return, results are in the output buffers.
 *   - Duplicates in a COO input are summed in their input order (as MATLAB sparse() does in
 *     the paper's appendix); explicit zeros are kept.
 *   - Index linearisation uses 64-bit keys: I1 * I2 * I3 must be below 2^62.
 */
#ifndef TUCKER_H
#define TUCKER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TUCKER_OK = 0,
  TUCKER_EINVAL = -1,    /* bad argument: dims, core size, index out of range, NULL pointer */
  TUCKER_ENOMEM = -2,    /* a device allocation failed */
  TUCKER_ECUDA = -3,     /* a CUDA runtime call or kernel launch failed */
  TUCKER_EEMPTY = -4,    /* |X|_F = 0: the fit is undefined */
  TUCKER_ETIMEOUT = -5,  /* a bounded device-side wait gave up */
  TUCKER_EINTERNAL = -6, /* an internal consistency check failed (e.g. Cholesky breakdown) */
  TUCKER_ENOTCONV = -7   /* the eigensolver hit its iteration limit before its tolerance */
} tucker_status;

typedef enum { TUCKER_FP64 = 0, TUCKER_MIXED = 1 } tucker_precision;
typedef enum { TUCKER_HOST = 0, TUCKER_DEVICE = 1 } tucker_mem;

/* Sparse input tensor in coordinate form.  idx[a][t] is the mode-a index of nonzero t. */
typedef struct {
  int64_t dims[3];
  int64_t nnz;
  const int32_t* idx[3];
  const double* val;
  int32_t where; /* tucker_mem of idx[] and val */
} tucker_coo;

typedef struct {
  int32_t precision;     /* tucker_precision */
  double tol;            /* stop threshold of the Delta_fit / Delta_G test; -INFINITY = never */
  int32_t max_iter;      /* passes of the main loop (>= 1; ignored by HO-SVD) */
  const double* init[3]; /* optional starting factors, I_n x J_n (NULL = the method's own).
                            HOOI, MP: init[1], init[2] replace the start of B and C
                                  (HOOI's HO-SVD start, MP's pseudo HO-SVD start).
                            SP:   init[2] is the REQUIRED raw random I3 x J3 matrix of
                                  Figure sp3; the library normalises its columns. */
  int32_t init_where;    /* tucker_mem of init[] */
  void* stream;          /* cudaStream_t */
  uint32_t flags;        /* reserved, must be 0 */
} tucker_opts;

typedef struct {
  double* G;             /* J1*J2*J3 (output) */
  double* U[3];          /* I_n * J_n (output) */
  double* fit_history;   /* optional, max_iter entries: fit after each pass */
  int32_t where;         /* tucker_mem of G, U[], fit_history */
  double fit;            /* fit of the returned decomposition */
  int32_t iters;         /* passes of the main loop run (1 for HO-SVD) */
  int32_t rank_deficient;/* bit n set: J_n exceeded the numerical rank of mode n's matrix */
} tucker_result;

typedef struct tucker_tensor_s* tucker_tensor;

/* ---- tensor handle -------------------------------------------------------------------
 * tucker_tensor_create copies X to the device, checks every index against dims (EINVAL),
 * sums duplicates and computes |X|_F^2.  Mode orderings (compressed sorted forms, the
 * counterpart of the paper's sorted slice files, Section 3 "Slice Projection" and the
 * appendix functions sort_index / slice) are built on first use and kept in the handle. */
int tucker_tensor_create(const tucker_coo* X, void* stream, tucker_tensor* out);
int tucker_tensor_destroy(tucker_tensor X);
/* Number of distinct nonzeros after duplicate summation, and |X|_F^2 (fit equation). */
int tucker_tensor_info(tucker_tensor X, int64_t* nnz, double* norm2);

/* ---- the four methods -----------------------------------------------------------------
 * J: core size (1 <= J_n <= I_n).  opts may be NULL for FP64, tol 1e-4, max_iter 50.
 * HO-SVD: Figure HO-SVD3.  HOOI: Figure hooi3 + Delta_fit stop (signed, fit_0 = 0).
 * SP: Figure sp3 + Delta_G stop (tested from the second pass).  MP: Figure mp3 + Delta_fit
 * stop; its pseudo HO-SVD start equals 2 X_(n) X_(n)^T, whose leading eigenvectors are
 * HO-SVD's. */
int tucker_hosvd(tucker_tensor X, const int32_t J[3], const tucker_opts* opts, tucker_result* out);
int tucker_hooi(tucker_tensor X, const int32_t J[3], const tucker_opts* opts, tucker_result* out);
int tucker_sp(tucker_tensor X, const int32_t J[3], const tucker_opts* opts, tucker_result* out);
int tucker_mp(tucker_tensor X, const int32_t J[3], const tucker_opts* opts, tucker_result* out);

/* ---- batched form -------------------------------------------------------------------------
 * HOOI (Figure hooi3) or MP (Figure mp3) on `count` independent tensors Xs[t] with core sizes
 * J[3t .. 3t+2]; results in out[t] (each with its own buffers and `where`).  opts applies to
 * all tensors (its init[] must be NULL).  The tensors' decompositions run concurrently on the
 * GPU (a pool of host threads, one non-blocking stream each, on the calling thread's device);
 * every ordering of every tensor is built first on opts->stream.  Each result equals what the
 * single-tensor call returns.  Returns the first failing tensor's status (lowest index). */
int tucker_hooi_batched(int32_t count, const tucker_tensor* Xs, const int32_t* J,
                        const tucker_opts* opts, tucker_result* out);
int tucker_mp_batched(int32_t count, const tucker_tensor* Xs, const int32_t* J,
                      const tucker_opts* opts, tucker_result* out);

/* ---- fourth-order tensors -------------------------------------------------------------------
 * HO-SVD and HOOI for N = 4 (Figures HO-SVDn and hooin), Slice Projection and Multislice
 * Projection for fourth-order tensors (Figures sp4 and mp4), in the FP64 form (precision must be
 * TUCKER_FP64, else EINVAL).  Conventions as above with four modes: factor n is I_n x J_n
 * row-major, the core g[((p J2 + q) J3 + r) J4 + s].  Stop tests as for third order (HOOI, MP:
 * signed Delta_fit with fit_0 = 0; SP: Delta_G from the second pass).  SP's init[3] is the
 * REQUIRED raw random I4 x J4 matrix of Figure sp4 (columns normalised by the library); for
 * HOOI and MP, init[1..3] may replace the start of B, C, D (HO-SVD's; MP's pseudo HO-SVD matrices
 * equal 3 X_(n) X_(n)^T and have the same leading eigenvectors).  Limits: every I_a I_b < 2^31
 * (two modes are merged into one index internally), I1 I2 I3 I4 < 2^62. */
typedef struct {
  int64_t dims[4];
  int64_t nnz;
  const int32_t* idx[4];
  const double* val;
  int32_t where;
} tucker4_coo;

typedef struct {
  int32_t precision;
  double tol;
  int32_t max_iter;
  const double* init[4];
  int32_t init_where;
  void* stream;
  uint32_t flags;
} tucker4_opts;

typedef struct {
  double* G;             /* J1*J2*J3*J4 */
  double* U[4];          /* I_n * J_n */
  double* fit_history;   /* optional, max_iter entries */
  int32_t where;
  double fit;
  int32_t iters;
  int32_t rank_deficient;
} tucker4_result;

typedef struct tucker4_tensor_s* tucker4_tensor;

/* Copies X to the device, checks every index (EINVAL), sums duplicates, computes |X|_F^2. */
int tucker4_tensor_create(const tucker4_coo* X, void* stream, tucker4_tensor* out);
int tucker4_tensor_destroy(tucker4_tensor X);
int tucker4_tensor_info(tucker4_tensor X, int64_t* nnz, double* norm2);
int tucker4_hosvd(tucker4_tensor X, const int32_t J[4], const tucker4_opts* opts,
                  tucker4_result* out);
int tucker4_hooi(tucker4_tensor X, const int32_t J[4], const tucker4_opts* opts,
                 tucker4_result* out);
int tucker4_sp(tucker4_tensor X, const int32_t J[4], const tucker4_opts* opts, tucker4_result* out);
int tucker4_mp(tucker4_tensor X, const int32_t J[4], const tucker4_opts* opts, tucker4_result* out);
/* HOOI's projection of Figure hooin for N = 4: Z = [[X; U_1^T, ..., I_n, ..., U_4^T]] written as
 * Z_(n), I_n x (J_a J_b J_c) row-major with column (p J_b + q) J_c + r for the other modes
 * a < b < c.  d_U[n] is not read (may be NULL).  Device pointers; synchronous on stream. */
int tucker4_ttmc(tucker4_tensor X, int32_t n, const double* const d_U[4], const int32_t J[4],
                 double* d_Y, void* stream);

/* ---- tensors streamed from host memory ---------------------------------------------------
 * Slice Projection and Multislice Projection for tensors whose orderings do not fit in device
 * memory (the paper's reason for SP and MP: their matrices are sums over slices, so the tensor
 * can be read one slice after another; Section 3 "Slice Projection").  tucker_stream_create
 * keeps the slice-major orderings of X in pinned host memory, building them chunk by chunk on
 * the GPU so that at most `budget` bytes of device memory are used for one chunk (budget >= 64
 * KiB; duplicates summed, indices checked: EINVAL).  tucker_sp_streamed / tucker_mp_streamed run
 * the methods with the same arguments and results as tucker_sp / tucker_mp (FP64 form only),
 * streaming the chunks over NVLink-C2C with copies overlapped with the work on the previous
 * chunk; *bytes_streamed (may be NULL) receives the host-to-device bytes moved.
 * tucker_stream_info reports the distinct nonzeros, |X|_F^2 and the number of chunks. */
typedef struct tucker_stream_s* tucker_stream_tensor;
int tucker_stream_create(const tucker_coo* X, int64_t budget, void* stream,
                         tucker_stream_tensor* out);
int tucker_stream_destroy(tucker_stream_tensor X);
int tucker_stream_info(tucker_stream_tensor X, int64_t* nnz, double* norm2, int64_t* chunks);
int tucker_sp_streamed(tucker_stream_tensor X, const int32_t J[3], const tucker_opts* opts,
                       tucker_result* out, double* bytes_streamed);
int tucker_mp_streamed(tucker_stream_tensor X, const int32_t J[3], const tucker_opts* opts,
                       tucker_result* out, double* bytes_streamed);

const char* tucker_strerror(int status);
/* Text of the last CUDA failure seen by the calling thread (empty if none). */
const char* tucker_last_error_detail(void);

/* ---- hot-path steps, exposed for verification and profiling ---------------------------
 * All pointers d_* are device memory; all calls are synchronous on `stream`. */

/* Mode ordering (n, m, o) of the nonzeros: stable sort by (i_n, i_m, i_o); a fiber is a run
 * with equal (i_n, i_m).  (n, m, o) must be a permutation of (0, 1, 2).  Returns the fiber
 * count; with non-NULL outputs (`where` memory) also copies root_ptr[I_n+1] (first fiber of
 * each i_n), fiber_idx[F] (i_m), fiber_ptr[F+1] (first nonzero), leaf_idx[nnz] (i_o) and
 * val[nnz] (values in sorted order). */
int tucker_ordering(tucker_tensor X, int32_t n, int32_t m, int32_t o, int64_t* nfibers,
                    int64_t* root_ptr, int32_t* fiber_idx, int64_t* fiber_ptr,
                    int32_t* leaf_idx, double* val, int32_t where);

/* Unfolding Gram M = X_(n) X_(n)^T, I_n x I_n (Figure HO-SVD3). */
int tucker_unfolding_gram(tucker_tensor X, int32_t n, double* d_M, void* stream);

/* HOOI projection Y = X x_m U_m^T x_o U_o^T (Figure hooi3), m < o the other modes, written
 * as Y_(n): I_n x (J_m J_o) row-major, column p * J_o + q.  d_Um is I_m x J_m, d_Uo I_o x J_o. */
int tucker_ttmc(tucker_tensor X, int32_t n, const double* d_Um, int32_t Jm, const double* d_Uo,
                int32_t Jo, double* d_Y, void* stream);

/* Slice projection Y = X x_m U_m^T (Figures sp3, mp3) written as Y_(n), n != m, with o the
 * remaining mode: I_n x (I_o J_m) row-major, column i_o * J_m + p.  Sum over slices of
 * X_s U U^T X_s^T equals Y_(n) Y_(n)^T. */
int tucker_slice_proj(tucker_tensor X, int32_t n, int32_t m, const double* d_Um, int32_t Jm,
                      double* d_Y, void* stream);

/* Gram M = Y1 Y1^T (+ Y2 Y2^T when d_Y2 != NULL): Y1 is rows x K1, Y2 rows x K2, row-major;
 * M is rows x rows (both triangles written).  Computed on the BF16 tensor cores to FP64
 * accuracy: every row is scaled by a power of two and cut into six 8-bit integer slices
 * (error-free splitting, Ozaki et al. 2012); the 22 slice products that reach 2^-47 of the
 * leading term (with the one square pair of the next level, whose sum on the diagonal does not
 * average out) are summed exactly (integer-valued FP32 chunks, 64-bit integer totals), so the
 * error is a few units of 2^-47 max|y_i| max|y_j| per term (max over each row), zero on
 * average, and the result does not depend on how K is split.  d_Y1 may be NULL when K1 = 0 (M = 0).  ETIMEOUT if a bounded wait inside the
 * kernel gave up. */
int tucker_gram(const double* d_Y1, int64_t K1, const double* d_Y2, int64_t K2, int32_t rows,
                double* d_M, void* stream);

/* C = A B (A: m x K, ld lda; B: K x n, ld ldb; C: m x n, ld ldc; row-major, device), computed
 * on the BF16 tensor cores with the error-free slicing of tucker_gram: every row of A and every
 * column of B is scaled by a power of two and cut into seven 8-bit slices (28 slice
 * products), so the error of C[i][j] is a few units of 2^-55 max_k |A[i][k]| max_k |B[k][j]|
 * (times sqrt(K) at most for uncorrelated errors).  The eigensolver's products with M (M V) use it.  d_A, d_B may be NULL
 * when K = 0 (C = 0). */
int tucker_gemm(const double* d_A, int64_t lda, const double* d_B, int64_t ldb, int32_t m,
                int32_t n, int64_t K, double* d_C, int64_t ldc, void* stream);

/* Allocation-free tucker_gram (the paper has no counterpart: this serves callers that cannot
 * let a library allocate device memory while they run, such as serving processes that reserve
 * all device memory in their own pool, or callers that must avoid the implicit synchronisation
 * cudaMalloc/cudaFree can cause).  Same arguments and result as tucker_gram; the split-K
 * workspace is one fixed array of 2^21 doubles (16 MiB) that every GPU loading the library
 * holds until exit, so rows * rows must be <= 2^21 (rows <= 1448), else TUCKER_EINVAL.  The
 * first call on a device looks up the array's address (cudaGetSymbolAddress): make it before
 * any stream capture.  The address is kept for the life of the process, so the library does
 * not support a cudaDeviceReset between calls.  Like every entry point, the call is
 * synchronous: it returns once M is written.  Calls share the array: calls that overlap on the
 * GPU race; order them on one stream. */
int tucker_gram_noalloc(const double* d_Y1, int64_t K1, const double* d_Y2, int64_t K2,
                        int32_t rows, double* d_M, void* stream);

/* ---- mixed-precision steps (TUCKER_MIXED form) ---------------------------------------------
 * BF16 matrices are passed as uint16_t bit patterns.  A "split" matrix Y is stored as two
 * BF16 matrices hi = bf16(y), lo = bf16(y - hi), row-major with row stride ld (elements, a
 * multiple of 64, columns K..ld-1 zero), base addresses 16-byte aligned. */

/* tucker_ttmc in FP32 from FP32 factors: writes the split Y_(n) (rows I_n, K = J_m J_o, stride
 * ldY) when d_Yhi/d_Ylo are given, and/or the FP32 Y_(n) (stride J_m J_o) when d_Y32 is. */
int tucker_ttmc_mixed(tucker_tensor X, int32_t n, const float* d_Um, int32_t Jm,
                      const float* d_Uo, int32_t Jo, uint16_t* d_Yhi, uint16_t* d_Ylo,
                      int64_t ldY, float* d_Y32, void* stream);

/* tucker_slice_proj in FP32 from an FP32 factor, written split (K = I_o J_m, stride ldY). */
int tucker_slice_proj_mixed(tucker_tensor X, int32_t n, int32_t m, const float* d_Um, int32_t Jm,
                            uint16_t* d_Yhi, uint16_t* d_Ylo, int64_t ldY, void* stream);

/* Gram M = Y1 Y1^T (+ Y2 Y2^T) of split matrices on the tensor cores: each product is
 * hi hi^T + hi lo^T + lo hi^T in BF16 with FP32 accumulation over K chunks of at most 4096,
 * chunks summed in FP64.  M (rows x rows, FP64) is exactly symmetric.  Pass d_Y2hi = NULL for
 * one term.  ETIMEOUT if a bounded wait inside the kernel gave up. */
int tucker_gram_bf16x3(const uint16_t* d_Y1hi, const uint16_t* d_Y1lo, int64_t K1, int64_t ld1,
                       const uint16_t* d_Y2hi, const uint16_t* d_Y2lo, int64_t K2, int64_t ld2,
                       int32_t rows, double* d_M, void* stream);

/* M = sum over one or two terms of Gram((X x_m U_m^T)_(n)) (Figures sp3, mp3) in the mixed form,
 * fused: the FP32 projection is built in shared memory, split into BF16 hi + lo and fed to the
 * tensor cores (hi hi^T + hi lo^T + lo hi^T, FP32 accumulation per K range, FP64 sum), so the
 * projection never goes to memory.  For modes of at most 256 rows (EINVAL above); the methods'
 * mixed form uses it for such modes.  d_U1 (I_m1 x J1), d_U2 (I_m2 x J2) FP32 row-major; pass
 * m2 = -1 for one term.  M rows x rows FP64, exactly symmetric. */
int tucker_gram_fused(tucker_tensor X, int32_t n, int32_t m1, const float* d_U1, int32_t J1,
                      int32_t m2, const float* d_U2, int32_t J2, double* d_M, void* stream);

/* J leading eigenvectors of the symmetric positive semi-definite n x n matrix M (largest
 * eigenvalue first; in each column the entry of largest magnitude is positive).  d_U0
 * (n x J, may be NULL) is a starting guess.  Outputs d_U (n x J) and d_lambda (J).
 * Block subspace iteration with Chebyshev filtering, Cholesky-QR2 and Rayleigh-Ritz, locking a
 * Ritz pair once its residual |M u - lambda u| is at most 3e-13 lambda_1; when n is small all
 * eigenpairs of M at once.  Its larger products (M V, V^T W, ...) run FP64-accurate on the
 * tensor cores, like tucker_gram.  The small symmetric eigenproblems (the Rayleigh-Ritz matrix, or M)
 * are solved by an FP32 Jacobi refined to FP64 accuracy (Ogita-Aishima iterative refinement),
 * with an FP64 Jacobi as fallback; every other step is FP64.  ENOTCONV / EINTERNAL carry a
 * detail string (tucker_last_error_detail). */
int tucker_eig_topk(const double* d_M, int32_t n, int32_t J, const double* d_U0, double* d_U,
                    double* d_lambda, void* stream);

/* Core G = [[X; A^T, B^T, C^T]] (row-major J1 x J2 x J3) and |G|_F^2. */
int tucker_core(tucker_tensor X, const double* d_A, const double* d_B, const double* d_C,
                const int32_t J[3], double* d_G, double* g_norm2, void* stream);

/* ---- profiling (no counterpart in the paper; the paper reports wall time only) ----------
 * tucker_profile_enable(1) clears previous records and starts recording CUDA events on the
 * launching stream around the hot-path kernels; 0 stops.  tucker_profile_query sums, for the
 * record `name`, the launches recorded, their device time in milliseconds and their
 * algorithmic FLOPs and bytes (what the method must compute and move, not what the kernel
 * happens to do).  Timed records: "gram_f64_tc" (the whole FP64 Gram: splitting, tensor-core
 * products, reduction) with its kernels "ozaki_split" and "gram_ozaki" (flops: the BF16 FLOPs
 * its tensor cores issue), "gemm_ozaki" (tucker_gemm's tensor-core products, flops likewise),
 * "eig_mv_ozaki" and "eig_tn_ozaki" (the eigensolver's products M V and A^T B on the tensor
 * cores), "eig_mv_ozaki3" (the mixed form's FP32-class filter products M V, 3 slices), "ttmc_f64_tc" (the FP64 HOOI projection with its rank updates on the tensor cores)
 * with its kernel "ttmc_ozaki", the kernels "syrk_f64", "gram_bf16x3", "gram_fused", "ttmc_f64",
 * "ttmc_mixed", "slice_proj_f64", "slice_proj_mixed", "unfold_gram_f64", "gemm_nn_f64",
 * "gemm_nn_f32", "gemm_tn_f64", "chol_f64", "jacobi_f64", "csf_build", and the stages
 * "eig_topk" (one leading-eigenvector solve: "eig_power" its initial power steps, "eig_rr" its
 * Rayleigh-Ritz solves, "eig_lock" its deflation updates, "eig_filter" its Chebyshev filters,
 * "eig_orth" its re-orthonormalisations) and "syev_refined" (one small eigenproblem) with
 * "syev_jacobi32" (its FP32 Jacobi).
 * Counters (occurrences as launches, summed values as flops, no time): "syev_steps" (value:
 * refinement steps of one small eigenproblem), "syev_fp32_sweeps" (value: sweeps of its FP32
 * Jacobi), "syev_cluster_rotations" (value 1: near-degenerate clusters split by Jacobi
 * rotations inside the refinement), "syev_rotation_unconverged" (value 1: those rotations hit
 * their round limit before a fallback), "syev_fallback" (value 1: unresolved cluster,
 * 2: step limit, 3: order above the shared-memory limit), "eig_outer" (value: Rayleigh-Ritz
 * iterations of one solve), "eig_launches" and "eig_host_syncs" (value: the kernel launches and
 * host synchronisations of one solve).  Every name and the argument order are fixed; unknown names
 * report zero.  tucker_launch_count returns the number of kernels this library has launched
 * in the process. */
/* ---- autotuning (no counterpart in the paper) -------------------------------------------
 * The mixed-precision projections have two kernels each that compute the same result up to the
 * order of FP32 sums: variant 0 gives each fiber a group of 8 lanes that loads factor rows as
 * float4 (rows padded to 16 bytes), variant 1 gives each fiber a warp.  On the first call for a
 * shape class (family; core sizes; rounded log2 of the mean fiber length) the library times both
 * once on the caller's stream and keeps the faster for the rest of the process, so every later
 * call, single-tensor or batched, runs the same kernel.  tucker_autotune_enable(0) stops new
 * timing (classes without a decision then use variant 0).  tucker_autotune_count returns the
 * number of decisions; tucker_autotune_decision reads decision i (0-based): family (1 HOOI
 * projection, 2 SP/MP slice projection), key[3] (J_m, J_o or 0, fiber-length class), the kept
 * variant and both measured times in milliseconds (kept first); EINVAL for i out of range. */
void tucker_autotune_enable(int on);
int tucker_autotune_count(void);
int tucker_autotune_decision(int32_t i, int32_t* family, int32_t key[3], int32_t* variant,
                             double* ms_kept, double* ms_other);

void tucker_profile_enable(int on);
int tucker_profile_query(const char* name, int64_t* launches, double* total_ms, double* flops,
                         double* bytes);
int64_t tucker_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* TUCKER_H */
