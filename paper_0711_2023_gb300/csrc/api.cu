// C ABI and host orchestration of the four methods (Figures HO-SVD3, hooi3, sp3, mp3) on the
// GPU kernels of this library.  The host only sequences kernels, sizes buffers and reads back
// the scalars its loop tests need (the fit after each pass, Ritz values in the eigensolver).
//
// Two precision forms share one driver:
//   FP64   every step in FP64 (CUDA cores);
//   MIXED  projections in FP32 from FP32 factors, written as BF16 hi/lo pairs; the Gram on the
//          tensor cores (BF16x3, FP32 accumulation per K chunk, FP64 chunk sum); the
//          eigensolver (Cholesky-QR2, Rayleigh-Ritz), the core and the fit in FP64.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace tk {

namespace {
thread_local std::string g_last_error;
}

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  g_last_error = buf;
}

void set_error_detail(const char* msg) { g_last_error = msg; }

int num_sms() {
  static std::atomic<int> cached{0};
  int n = cached.load(std::memory_order_relaxed);
  if (n == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    n = v > 0 ? v : 1;
    cached.store(n, std::memory_order_relaxed);
  }
  return n;
}

namespace {
// Work buffers come from the device's default stream-ordered pool.  By default the pool hands
// freed memory back to the driver at every synchronisation, so the next allocation has to map
// it again; the library synchronises often (the eigensolver reads Ritz values back), so keep
// freed blocks in the pool instead.
std::mutex g_pool_mu;
bool g_pool_ready[64] = {};
}  // namespace

void keep_pool_memory() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (g_pool_ready[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  g_pool_ready[dev] = true;
}

int ordering_slot(int n, int m, int o) {
  if (n < 0 || m < 0 || o < 0 || n > 2 || m > 2 || o > 2 || n == m || m == o || n == o) return -1;
  return n * 2 + (m < o ? 0 : 1);
}

int ensure_ordering(tucker_tensor_s* X, int n, int m, int o, cudaStream_t s, Ordering** out) {
  const int slot = ordering_slot(n, m, o);
  if (slot < 0) return TUCKER_EINVAL;
  Ordering* ord = &X->ord[slot];
  if (!ord->built) {
    ord->n = n;
    ord->m = m;
    ord->o = o;
    TK_TRY(build_ordering(X, ord, s));
  }
  *out = ord;
  return TUCKER_OK;
}

int ensure_fiber_map(tucker_tensor_s* X, Ordering* ord, cudaStream_t s) {
  if (!ord->fiber_map) TK_TRY(build_fiber_map(X, ord, s));
  return TUCKER_OK;
}

namespace {

__global__ void fit_kernel(double nX2, const double* __restrict__ g2, double* __restrict__ fit) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    *fit = 1.0 - sqrt(fmax(0.0, nX2 - *g2)) / sqrt(nX2);
}

__global__ void normalize_cols(const double* __restrict__ src, int rows, int cols,
                              double* __restrict__ dst) {
  __shared__ double ws[8];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) {
    const double v = src[(int64_t)i * cols + j];
    s = fma(v, v, s);
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    ws[0] = sqrt(t);
  }
  __syncthreads();
  const double nrm = ws[0];
  for (int i = threadIdx.x; i < rows; i += blockDim.x)
    dst[(int64_t)i * cols + j] = nrm > 0.0 ? src[(int64_t)i * cols + j] / nrm : 0.0;
}

cudaMemcpyKind kind_to_device(int where) {
  return where == TUCKER_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
cudaMemcpyKind kind_from_device(int where) {
  return where == TUCKER_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

void other_modes(int n, int* m, int* o) {
  *m = n == 0 ? 1 : 0;
  *o = n == 2 ? 1 : 2;
}

}  // namespace

int fit_on_device(double nX2, const double* g2_dev, double* fit_dev, cudaStream_t s) {
  fit_kernel<<<1, 32, 0, s>>>(nX2, g2_dev, fit_dev);
  TK_LAUNCH();
  return TUCKER_OK;
}

int normalize_columns(const double* src, int rows, int cols, double* dst, cudaStream_t s) {
  normalize_cols<<<cols, 256, 0, s>>>(src, rows, cols, dst);
  TK_LAUNCH();
  return TUCKER_OK;
}

int core_from_ttmc3(const double* Y3, int I3, int J1, int J2, const double* C, int J3, double* G,
                    double* g2_dev, cudaStream_t s) {
  // G[(p J2 + q) J3 + r] = sum_k Y3[k, p J2 + q] C[k, r]  (G = W x_3 C^T, Figure hooi3).
  TK_TRY(gemm_tn_f64(J1 * J2, J3, I3, Y3, (int64_t)J1 * J2, C, J3, G, J3, s));
  TK_TRY(sum_squares(G, (int64_t)J1 * J2 * J3, g2_dev, s));
  return TUCKER_OK;
}

// ----------------------------------------------------------------------------------------------
// Method driver
// ----------------------------------------------------------------------------------------------
namespace {

enum class Method { HOSVD, HOOI, SP, MP };

// (n, m) pairs of Figure sp3: A from X x_3 C^T, B from X x_1 A^T, C from X x_2 B^T.
const int SP_PAIRS[3][2] = {{0, 2}, {1, 0}, {2, 1}};

struct Run {
  tucker_tensor_s* X = nullptr;
  Method method = Method::HOOI;
  int J[3] = {0, 0, 0};
  cudaStream_t s = 0;
  tucker_opts o;
  bool mixed = false;
  Buf U[3], U32[3];
  Buf Y, Y2;                  // FP64 projections; Y also stages the core input
  Buf Yh, Yl, Y2h, Y2l, Y32;  // mixed projections
  Buf M, M32, G, sc;          // sc: [0] |G|^2, [1] fit; M32: FP32 copy for the eigensolver
  int rank_def = 0;
  std::vector<double> fits;
  int64_t dim(int a) const { return X->dims[a]; }
};

size_t bf16_bytes(int64_t rows, int64_t K) { return 2 * (size_t)rows * (size_t)gram_ld(K); }

int alloc_buffers(Run& r) {
  const int* J = r.J;
  for (int a = 0; a < 3; ++a) {
    TK_TRY(r.U[a].alloc(sizeof(double) * r.dim(a) * J[a], r.s));
    if (r.mixed) TK_TRY(r.U32[a].alloc(sizeof(float) * r.dim(a) * factor_ld32(J[a]), r.s));
  }
  const int64_t maxI = std::max(r.dim(0), std::max(r.dim(1), r.dim(2)));
  TK_TRY(r.M.alloc(sizeof(double) * maxI * maxI, r.s));
  if (r.mixed) TK_TRY(r.M32.alloc(sizeof(float) * maxI * maxI, r.s));
  TK_TRY(r.G.alloc(sizeof(double) * J[0] * J[1] * J[2], r.s));
  TK_TRY(r.sc.alloc(sizeof(double) * 2, r.s));
  const size_t core_in = (size_t)(r.dim(2) * J[0] * J[1]);  // W_(3): I3 x J1 J2
  size_t y = core_in * sizeof(double), y2 = 0, yb = 0, yb2 = 0;
  for (int n = 0; n < 3; ++n) {
    int m, o;
    other_modes(n, &m, &o);
    if (r.method == Method::HOOI) {
      y = std::max(y, sizeof(double) * (size_t)(r.dim(n) * J[m] * J[o]));
      yb = std::max(yb, bf16_bytes(r.dim(n), (int64_t)J[m] * J[o]));
    } else if (r.method == Method::SP) {
      const int nn = SP_PAIRS[n][0], mm = SP_PAIRS[n][1], oo = 3 - nn - mm;
      y = std::max(y, sizeof(double) * (size_t)(r.dim(nn) * r.dim(oo) * J[mm]));
      yb = std::max(yb, bf16_bytes(r.dim(nn), r.dim(oo) * J[mm]));
    } else if (r.method == Method::MP) {
      y = std::max(y, sizeof(double) * (size_t)(r.dim(n) * r.dim(o) * J[m]));
      y2 = std::max(y2, sizeof(double) * (size_t)(r.dim(n) * r.dim(m) * J[o]));
      yb = std::max(yb, bf16_bytes(r.dim(n), r.dim(o) * J[m]));
      yb2 = std::max(yb2, bf16_bytes(r.dim(n), r.dim(m) * J[o]));
    }
  }
  if (r.mixed) {
    TK_TRY(r.Y.alloc(core_in * sizeof(double), r.s));
    TK_TRY(r.Y32.alloc(core_in * sizeof(float), r.s));
    // yb, yb2: bytes of one BF16 matrix (hi or lo) of the largest projection
    if (yb) {
      TK_TRY(r.Yh.alloc(yb, r.s));
      TK_TRY(r.Yl.alloc(yb, r.s));
    }
    if (yb2) {
      TK_TRY(r.Y2h.alloc(yb2, r.s));
      TK_TRY(r.Y2l.alloc(yb2, r.s));
    }
  } else {
    TK_TRY(r.Y.alloc(y, r.s));
    if (y2) TK_TRY(r.Y2.alloc(y2, r.s));
  }
  return TUCKER_OK;
}

int refresh32(Run& r, int n) {
  if (!r.mixed) return TUCKER_OK;
  return f64_to_f32_rows(r.U[n].as<double>(), r.dim(n), r.J[n], r.U32[n].as<float>(),
                         factor_ld32(r.J[n]), r.s);
}

int eig_update(Run& r, int n, bool warm) {
  EigStats st;
  const float* m32 = nullptr;
  if (r.mixed) {
    TK_TRY(f64_to_f32(r.M.as<double>(), r.M32.as<float>(), r.dim(n) * r.dim(n), r.s));
    m32 = r.M32.as<float>();
  }
  TK_TRY(eig_topk_f64(r.M.as<double>(), (int)r.dim(n), r.J[n], warm ? r.U[n].as<double>() : nullptr,
                      r.U[n].as<double>(), nullptr, r.s, &st, m32,
                      r.mixed ? EIG_TOL_MIXED : EIG_TOL_FP64));
  if (st.rank_deficient) r.rank_def |= 1 << n;
  return refresh32(r, n);
}

int unfolding_gram(Run& r, int n, double* M) {
  int m, o;
  other_modes(n, &m, &o);
  Ordering *rows, *fib;
  TK_TRY(ensure_ordering(r.X, n, m, o, r.s, &rows));
  TK_TRY(ensure_ordering(r.X, m, o, n, r.s, &fib));
  TK_TRY(ensure_fiber_map(r.X, fib, r.s));
  return unfolding_gram_f64(r.X, rows, fib, M, r.s);
}

int ordering(Run& r, int n, int m, int o, Ordering** ord) {
  TK_TRY(ensure_ordering(r.X, n, m, o, r.s, ord));
  if (r.mixed) TK_TRY(ensure_val_f32(r.X, *ord, r.s));
  return TUCKER_OK;
}

// Mode-n matrix of HOOI (Figure hooi3): Gram of (X x_m U_m^T x_o U_o^T)_(n).  For n = 2 the
// projection W is kept for the core.
int hooi_matrix(Run& r, int n) {
  int m, o;
  other_modes(n, &m, &o);
  Ordering* ord;
  TK_TRY(ordering(r, n, m, o, &ord));
  const int64_t K = (int64_t)r.J[m] * r.J[o];
  if (!r.mixed) {
    TK_TRY(ttmc_fp64(r.X, ord, r.U[m].as<double>(), r.J[m], r.U[o].as<double>(), r.J[o],
                    r.Y.as<double>(), r.s));
    return gram_f64_tc((int)r.dim(n), r.Y.as<double>(), K, nullptr, 0, r.M.as<double>(), r.s);
  }
  const int64_t ld = gram_ld(K);
  __nv_bfloat16 *yh = r.Yh.as<__nv_bfloat16>(), *yl = r.Yl.as<__nv_bfloat16>();
  TK_TRY(ttmc_mixed(r.X, ord, r.U32[m].as<float>(), factor_ld32(r.J[m]), r.J[m],
                    r.U32[o].as<float>(), factor_ld32(r.J[o]), r.J[o], yh, yl, ld,
                    n == 2 ? r.Y32.as<float>() : nullptr, r.s));
  GramTerm t{yh, yl, K, ld};
  return gram_bf16x3((int)r.dim(n), 1, &t, r.M.as<double>(), r.s);
}

// One slice-projection term (X x_m U_m^T)_(n), on ordering (n, o, m); K = I_o J_m.
int slice_term(Run& r, int n, int m, int which, GramTerm* t) {
  const int o = 3 - n - m;
  Ordering* ord;
  TK_TRY(ordering(r, n, o, m, &ord));
  const int64_t K = r.dim(o) * r.J[m];
  if (!r.mixed) {
    double* Y = which == 0 ? r.Y.as<double>() : r.Y2.as<double>();
    TK_TRY(slice_proj_f64(r.X, ord, r.U[m].as<double>(), r.J[m], Y, r.s));
    *t = GramTerm{nullptr, nullptr, K, K};
    return TUCKER_OK;
  }
  const int64_t ld = gram_ld(K);
  __nv_bfloat16* yh = which == 0 ? r.Yh.as<__nv_bfloat16>() : r.Y2h.as<__nv_bfloat16>();
  __nv_bfloat16* yl = which == 0 ? r.Yl.as<__nv_bfloat16>() : r.Y2l.as<__nv_bfloat16>();
  TK_TRY(slice_proj_mixed(r.X, ord, r.U32[m].as<float>(), factor_ld32(r.J[m]), r.J[m], yh, yl,
                          ld, r.s));
  *t = GramTerm{yh, yl, K, ld};
  return TUCKER_OK;
}

// Mode-n matrix of SP (one term, Figure sp3) or MP (two terms, Figure mp3).  In the mixed form
// a mode of at most 256 rows takes the fused kernel (the projection never leaves shared memory).
int slice_matrix(Run& r, int n, int m1, int m2) {
  if (r.mixed && r.dim(n) <= FUSED_GRAM_MAX_ROWS) {
    const int nt = m2 >= 0 ? 2 : 1;
    const int ms[2] = {m1, m2};
    const Ordering* ords[2] = {nullptr, nullptr};
    const float* U[2] = {nullptr, nullptr};
    int64_t ld[2] = {0, 0};
    int J[2] = {0, 0};
    for (int t = 0; t < nt; ++t) {
      Ordering* ord;
      TK_TRY(ordering(r, n, 3 - n - ms[t], ms[t], &ord));
      TK_TRY(ensure_fiber_map(r.X, ord, r.s));
      ords[t] = ord;
      U[t] = r.U32[ms[t]].as<float>();
      ld[t] = factor_ld32(r.J[ms[t]]);
      J[t] = r.J[ms[t]];
    }
    return gram_fused_mixed(r.X, n, nt, ords, U, ld, J, r.M.as<double>(), r.s);
  }
  GramTerm t[2];
  TK_TRY(slice_term(r, n, m1, 0, &t[0]));
  const int nt = m2 >= 0 ? 2 : 1;
  if (nt == 2) TK_TRY(slice_term(r, n, m2, 1, &t[1]));
  if (!r.mixed)
    return gram_f64_tc((int)r.dim(n), r.Y.as<double>(), t[0].K,
                       nt == 2 ? r.Y2.as<double>() : nullptr, nt == 2 ? t[1].K : 0,
                       r.M.as<double>(), r.s);
  return gram_bf16x3((int)r.dim(n), nt, t, r.M.as<double>(), r.s);
}

// G = [[X; A^T, B^T, C^T]] from W = [[X; A^T, B^T, I]] (computed unless w_ready), then the fit.
int core_and_fit(Run& r, bool w_ready, double* fit, double* g2) {
  Ordering* ord;
  TK_TRY(ordering(r, 2, 0, 1, &ord));
  const int64_t nW = r.dim(2) * r.J[0] * r.J[1];
  if (!r.mixed) {
    if (!w_ready)
      TK_TRY(ttmc_fp64(r.X, ord, r.U[0].as<double>(), r.J[0], r.U[1].as<double>(), r.J[1],
                      r.Y.as<double>(), r.s));
  } else {
    if (!w_ready)
      TK_TRY(ttmc_mixed(r.X, ord, r.U32[0].as<float>(), factor_ld32(r.J[0]), r.J[0],
                        r.U32[1].as<float>(), factor_ld32(r.J[1]), r.J[1], nullptr, nullptr, 0,
                        r.Y32.as<float>(), r.s));
    TK_TRY(f32_to_f64(r.Y32.as<float>(), r.Y.as<double>(), nW, r.s));
  }
  TK_TRY(core_from_ttmc3(r.Y.as<double>(), (int)r.dim(2), r.J[0], r.J[1], r.U[2].as<double>(),
                         r.J[2], r.G.as<double>(), r.sc.as<double>(), r.s));
  fit_kernel<<<1, 32, 0, r.s>>>(r.X->norm2, r.sc.as<double>(), r.sc.as<double>() + 1);
  TK_LAUNCH();
  double h[2];
  TK_CUDA(cudaMemcpyAsync(h, r.sc.p, sizeof(h), cudaMemcpyDeviceToHost, r.s));
  TK_CUDA(cudaStreamSynchronize(r.s));
  // fit = 1 - sqrt(|X|^2 - |G|^2) / |X| turns a relative error d in |G|^2 into a fit error of
  // about d |G|^2 / (2 |X| |X - X^|).  With an FP32 projection (d ~ 1e-7) that stays far below
  // 1e-5 while the residual |X - X^| is above 1% of |X|; closer to exact recovery the mixed
  // form recomputes the core from the FP64 factors with the FP64 projection.
  if (r.mixed && h[1] > 0.99) {
    TK_TRY(ttmc_fp64(r.X, ord, r.U[0].as<double>(), r.J[0], r.U[1].as<double>(), r.J[1],
                    r.Y.as<double>(), r.s));
    TK_TRY(core_from_ttmc3(r.Y.as<double>(), (int)r.dim(2), r.J[0], r.J[1], r.U[2].as<double>(),
                           r.J[2], r.G.as<double>(), r.sc.as<double>(), r.s));
    fit_kernel<<<1, 32, 0, r.s>>>(r.X->norm2, r.sc.as<double>(), r.sc.as<double>() + 1);
    TK_LAUNCH();
    TK_CUDA(cudaMemcpyAsync(h, r.sc.p, sizeof(h), cudaMemcpyDeviceToHost, r.s));
    TK_CUDA(cudaStreamSynchronize(r.s));
  }
  *g2 = h[0];
  *fit = h[1];
  return TUCKER_OK;
}

int finish(Run& r, tucker_result* out) {
  const int where = out->where;
  TK_CUDA(cudaMemcpyAsync(out->G, r.G.p, sizeof(double) * r.J[0] * r.J[1] * r.J[2],
                          kind_from_device(where), r.s));
  for (int a = 0; a < 3; ++a)
    TK_CUDA(cudaMemcpyAsync(out->U[a], r.U[a].p, sizeof(double) * r.dim(a) * r.J[a],
                            kind_from_device(where), r.s));
  if (out->fit_history && !r.fits.empty())
    TK_CUDA(cudaMemcpyAsync(out->fit_history, r.fits.data(), sizeof(double) * r.fits.size(),
                            where == TUCKER_DEVICE ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost,
                            r.s));
  TK_CUDA(cudaStreamSynchronize(r.s));
  out->fit = r.fits.empty() ? 0.0 : r.fits.back();
  out->iters = (int32_t)r.fits.size();
  out->rank_deficient = r.rank_def;
  return TUCKER_OK;
}

int check_args(tucker_tensor_s* X, const int32_t J[3], const tucker_opts* opts,
               const tucker_result* out, bool needs_iter) {
  if (!X || !J || !out || !out->G || !out->U[0] || !out->U[1] || !out->U[2]) return TUCKER_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (J[a] < 1 || J[a] > X->dims[a]) return TUCKER_EINVAL;
  if (out->where != TUCKER_HOST && out->where != TUCKER_DEVICE) return TUCKER_EINVAL;
  if (opts) {
    if (opts->precision != TUCKER_FP64 && opts->precision != TUCKER_MIXED) return TUCKER_EINVAL;
    if (needs_iter && opts->max_iter < 1) return TUCKER_EINVAL;
    if (isnan(opts->tol) || opts->tol == INFINITY) return TUCKER_EINVAL;
    if (opts->flags != 0) return TUCKER_EINVAL;
    if (opts->init_where != TUCKER_HOST && opts->init_where != TUCKER_DEVICE) return TUCKER_EINVAL;
  }
  if (X->nnz == 0 || !(X->norm2 > 0.0)) return TUCKER_EEMPTY;
  return TUCKER_OK;
}

tucker_opts default_opts() {
  tucker_opts o;
  memset(&o, 0, sizeof(o));
  o.precision = TUCKER_FP64;
  o.tol = 1e-4;
  o.max_iter = 50;
  return o;
}

int load_init(Run& r, int n) {
  if (!r.o.init[n]) return 0;
  if (cudaMemcpyAsync(r.U[n].p, r.o.init[n], sizeof(double) * r.dim(n) * r.J[n],
                      kind_to_device(r.o.init_where), r.s) != cudaSuccess)
    return -1;
  return refresh32(r, n) == TUCKER_OK ? 1 : -1;
}

int run_method(Method method, tucker_tensor_s* X, const int32_t J[3], const tucker_opts* opts,
               tucker_result* out) {
  TK_TRY(check_args(X, J, opts, out, method != Method::HOSVD));
  if (method == Method::SP && (!opts || !opts->init[2])) return TUCKER_EINVAL;  // random C
  Run r;
  r.X = X;
  r.method = method;
  for (int a = 0; a < 3; ++a) r.J[a] = J[a];
  r.o = opts ? *opts : default_opts();
  r.s = (cudaStream_t)r.o.stream;
  r.mixed = r.o.precision == TUCKER_MIXED;
  TK_TRY(alloc_buffers(r));
  bool have[3] = {false, false, false};

  // ---- initialisation -------------------------------------------------------------------
  if (method == Method::HOSVD) {
    for (int n = 0; n < 3; ++n) {
      TK_TRY(unfolding_gram(r, n, r.M.as<double>()));
      TK_TRY(eig_update(r, n, false));
    }
    double fit, g2;
    TK_TRY(core_and_fit(r, false, &fit, &g2));
    r.fits.push_back(fit);
    return finish(r, out);
  }
  if (method == Method::SP) {
    // Figure sp3: C is a random I3 x J3 matrix with its columns normalised.
    Buf raw;
    TK_TRY(raw.alloc(sizeof(double) * r.dim(2) * J[2], r.s));
    TK_CUDA(cudaMemcpyAsync(raw.p, r.o.init[2], sizeof(double) * r.dim(2) * J[2],
                            kind_to_device(r.o.init_where), r.s));
    TK_TRY(normalize_columns(raw.as<double>(), (int)r.dim(2), J[2], r.U[2].as<double>(), r.s));
    TK_TRY(refresh32(r, 2));
    TK_CUDA(cudaStreamSynchronize(r.s));
  } else {
    // HOOI: B, C from HO-SVD.  MP: pseudo HO-SVD; each of its two slice sums equals
    // X_(n) X_(n)^T (Figure mp3), so the matrix is 2 X_(n) X_(n)^T.  Either start is replaced by
    // the caller's B, C when given.
    for (int n = 1; n < 3; ++n) {
      {
        const int li = load_init(r, n);
        if (li < 0) return TUCKER_ECUDA;
        if (li > 0) {
          have[n] = true;
          continue;
        }
      }
      TK_TRY(unfolding_gram(r, n, r.M.as<double>()));
      if (method == Method::MP) TK_TRY(scale_f64(r.dim(n) * r.dim(n), 2.0, r.M.as<double>(), r.s));
      TK_TRY(eig_update(r, n, false));
      have[n] = true;
    }
  }

  // ---- main loop ------------------------------------------------------------------------
  double old = 0.0, gprev = 0.0;
  for (int it = 0; it < r.o.max_iter; ++it) {
    for (int step = 0; step < 3; ++step) {
      int n = step;
      if (method == Method::HOOI) {
        TK_TRY(hooi_matrix(r, n));
      } else if (method == Method::SP) {
        n = SP_PAIRS[step][0];
        TK_TRY(slice_matrix(r, n, SP_PAIRS[step][1], -1));
      } else {
        int m, o;
        other_modes(n, &m, &o);
        TK_TRY(slice_matrix(r, n, m, o));
      }
      TK_TRY(eig_update(r, n, have[n]));
      have[n] = true;
    }
    double fit, g2;
    TK_TRY(core_and_fit(r, method == Method::HOOI, &fit, &g2));
    r.fits.push_back(fit);
    if (method == Method::SP) {
      const double gn = sqrt(g2);
      if (it >= 1 && (1.0 - gprev / gn) < r.o.tol) break;  // Delta_G test
      gprev = gn;
    } else {
      if (fit - old < r.o.tol) break;                      // Delta_fit test (signed)
      old = fit;
    }
  }
  return finish(r, out);
}

// ----------------------------------------------------------------------------------------------
// Batched driver: many independent tensors.  Every ordering (with its fiber map and FP32
// values) of every tensor is built first, on the caller's stream, so that the worker threads
// only read the handles; then a pool of host threads, each with its own non-blocking stream,
// runs the tensors' decompositions concurrently on the GPU.
// ----------------------------------------------------------------------------------------------
// Host threads (one stream each).  Measured on the 256-tensor batch: 4 -> 400, 8 -> 467,
// 16 -> 415, 32 -> 345 tensor-sweeps/s (more threads contend for the driver and the GPU).
constexpr int BATCH_STREAMS = 8;

int prepare_all_orderings(tucker_tensor_s* X, bool mixed, cudaStream_t s) {
  for (int n = 0; n < 3; ++n)
    for (int m = 0; m < 3; ++m) {
      if (m == n) continue;
      const int o = 3 - n - m;
      Ordering* ord;
      TK_TRY(ensure_ordering(X, n, m, o, s, &ord));
      TK_TRY(ensure_fiber_map(X, ord, s));
      if (mixed) TK_TRY(ensure_val_f32(X, ord, s));
    }
  return TUCKER_OK;
}

int run_batched(Method method, int32_t count, const tucker_tensor* Xs, const int32_t* J,
                const tucker_opts* opts, tucker_result* out) {
  if (count < 0 || (count > 0 && (!Xs || !J || !out))) return TUCKER_EINVAL;
  if (count == 0) return TUCKER_OK;
  const tucker_opts base = opts ? *opts : default_opts();
  if (base.init[0] || base.init[1] || base.init[2]) return TUCKER_EINVAL;  // no per-tensor starts
  cudaStream_t s0 = (cudaStream_t)base.stream;
  const bool mixed = base.precision == TUCKER_MIXED;
  for (int t = 0; t < count; ++t) {
    if (!Xs[t]) return TUCKER_EINVAL;
    TK_TRY(prepare_all_orderings(Xs[t], mixed, s0));
  }
  TK_CUDA(cudaStreamSynchronize(s0));
  int dev = 0;
  TK_CUDA(cudaGetDevice(&dev));
  const int nthreads = std::min<int>(count, BATCH_STREAMS);
  std::vector<cudaStream_t> streams(nthreads, nullptr);
  for (int i = 0; i < nthreads; ++i)
    TK_CUDA(cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking));
  std::vector<int> status(count, TUCKER_OK);
  // The error detail is per thread: a worker keeps the text of each failing tensor so that the
  // caller's thread can report the one whose status it returns.
  std::vector<std::string> detail(count);
  std::vector<std::thread> pool;
  for (int i = 0; i < nthreads; ++i)
    pool.emplace_back([&, i]() {
      if (cudaSetDevice(dev) != cudaSuccess) {
        for (int t = i; t < count; t += nthreads) status[t] = TUCKER_ECUDA;
        return;
      }
      tucker_opts o = base;
      o.stream = streams[i];
      for (int t = i; t < count; t += nthreads) {
        g_last_error.clear();
        status[t] = run_method(method, Xs[t], J + 3 * (int64_t)t, &o, &out[t]);
        if (status[t] != TUCKER_OK) detail[t] = g_last_error;
      }
    });
  for (auto& th : pool) th.join();
  for (auto st : streams) cudaStreamDestroy(st);
  for (int t = 0; t < count; ++t)
    if (status[t] != TUCKER_OK) {
      g_last_error = detail[t];
      return status[t];
    }
  return TUCKER_OK;
}

}  // namespace
}  // namespace tk

using namespace tk;

extern "C" {

int tucker_hooi_batched(int32_t count, const tucker_tensor* Xs, const int32_t* J,
                        const tucker_opts* opts, tucker_result* out) {
  return run_batched(Method::HOOI, count, Xs, J, opts, out);
}

int tucker_mp_batched(int32_t count, const tucker_tensor* Xs, const int32_t* J,
                      const tucker_opts* opts, tucker_result* out) {
  return run_batched(Method::MP, count, Xs, J, opts, out);
}

const char* tucker_strerror(int status) {
  switch (status) {
    case TUCKER_OK: return "ok";
    case TUCKER_EINVAL: return "invalid argument";
    case TUCKER_ENOMEM: return "device memory allocation failed";
    case TUCKER_ECUDA: return "CUDA error";
    case TUCKER_EEMPTY: return "empty tensor (|X| = 0): fit undefined";
    case TUCKER_ETIMEOUT: return "a bounded device-side wait gave up";
    case TUCKER_EINTERNAL: return "internal consistency check failed";
    case TUCKER_ENOTCONV: return "eigensolver did not converge";
    default: return "unknown status";
  }
}

const char* tucker_last_error_detail(void) { return g_last_error.c_str(); }

int tucker_tensor_create(const tucker_coo* X, void* stream, tucker_tensor* out) {
  if (!X || !out) return TUCKER_EINVAL;
  *out = nullptr;
  for (int a = 0; a < 3; ++a)
    if (X->dims[a] < 1 || X->dims[a] > 2147483647ll) return TUCKER_EINVAL;
  const double cells = (double)X->dims[0] * (double)X->dims[1] * (double)X->dims[2];
  if (cells >= 4.6e18) return TUCKER_EINVAL;
  if (X->nnz < 0 || X->nnz > 2147483647ll) return TUCKER_EINVAL;
  if (X->where != TUCKER_HOST && X->where != TUCKER_DEVICE) return TUCKER_EINVAL;
  if (X->nnz > 0 && (!X->idx[0] || !X->idx[1] || !X->idx[2] || !X->val)) return TUCKER_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  tucker_tensor_s* T = new (std::nothrow) tucker_tensor_s();
  if (!T) return TUCKER_ENOMEM;
  for (int a = 0; a < 3; ++a) T->dims[a] = X->dims[a];
  cudaGetDevice(&T->device);
  int st = TUCKER_OK;
  {
    const int64_t n = X->nnz;
    Buf bi[3], bv;
    const int32_t* di[3] = {X->idx[0], X->idx[1], X->idx[2]};
    const double* dv = X->val;
    if (X->where == TUCKER_HOST && n > 0) {
      for (int a = 0; a < 3 && st == TUCKER_OK; ++a) {
        st = bi[a].alloc(sizeof(int32_t) * n, s);
        if (st == TUCKER_OK &&
            cudaMemcpyAsync(bi[a].p, X->idx[a], sizeof(int32_t) * n, cudaMemcpyHostToDevice, s) !=
                cudaSuccess)
          st = TUCKER_ECUDA;
        di[a] = bi[a].as<int32_t>();
      }
      if (st == TUCKER_OK) st = bv.alloc(sizeof(double) * n, s);
      if (st == TUCKER_OK &&
          cudaMemcpyAsync(bv.p, X->val, sizeof(double) * n, cudaMemcpyHostToDevice, s) != cudaSuccess)
        st = TUCKER_ECUDA;
      dv = bv.as<double>();
    }
    if (st == TUCKER_OK) st = build_canonical(T, di[0], di[1], di[2], dv, n, s);
    if (st == TUCKER_OK && cudaStreamSynchronize(s) != cudaSuccess) st = TUCKER_ECUDA;
  }
  if (st != TUCKER_OK) {
    tucker_tensor_destroy(T);
    return st;
  }
  *out = T;
  return TUCKER_OK;
}

int tucker_tensor_destroy(tucker_tensor T) {
  if (!T) return TUCKER_OK;
  cudaDeviceSynchronize();
  for (int a = 0; a < 3; ++a) cudaFree(T->idx[a]);
  cudaFree(T->val);
  for (auto& o : T->ord) {
    cudaFree(o.root_ptr);
    cudaFree(o.fiber_idx);
    cudaFree(o.fiber_root);
    cudaFree(o.fiber_ptr);
    cudaFree(o.leaf_idx);
    cudaFree(o.val);
    cudaFree(o.val_f32);
    cudaFree(o.fiber_map);
  }
  delete T;
  return TUCKER_OK;
}

int tucker_tensor_info(tucker_tensor X, int64_t* nnz, double* norm2) {
  if (!X) return TUCKER_EINVAL;
  if (nnz) *nnz = X->nnz;
  if (norm2) *norm2 = X->norm2;
  return TUCKER_OK;
}

int tucker_hosvd(tucker_tensor X, const int32_t J[3], const tucker_opts* opts, tucker_result* out) {
  return run_method(Method::HOSVD, X, J, opts, out);
}
int tucker_hooi(tucker_tensor X, const int32_t J[3], const tucker_opts* opts, tucker_result* out) {
  return run_method(Method::HOOI, X, J, opts, out);
}
int tucker_sp(tucker_tensor X, const int32_t J[3], const tucker_opts* opts, tucker_result* out) {
  return run_method(Method::SP, X, J, opts, out);
}
int tucker_mp(tucker_tensor X, const int32_t J[3], const tucker_opts* opts, tucker_result* out) {
  return run_method(Method::MP, X, J, opts, out);
}

// ---- step entry points -----------------------------------------------------------------------

int tucker_ordering(tucker_tensor X, int32_t n, int32_t m, int32_t o, int64_t* nfibers,
                    int64_t* root_ptr, int32_t* fiber_idx, int64_t* fiber_ptr, int32_t* leaf_idx,
                    double* val, int32_t where) {
  if (!X || ordering_slot(n, m, o) < 0) return TUCKER_EINVAL;
  if (where != TUCKER_HOST && where != TUCKER_DEVICE) return TUCKER_EINVAL;
  cudaStream_t s = 0;
  Ordering* ord;
  TK_TRY(ensure_ordering(X, n, m, o, s, &ord));
  if (nfibers) *nfibers = ord->F;
  const cudaMemcpyKind k = kind_from_device(where);
  if (root_ptr) TK_CUDA(cudaMemcpy(root_ptr, ord->root_ptr, sizeof(int64_t) * (X->dims[n] + 1), k));
  if (fiber_idx && ord->F) TK_CUDA(cudaMemcpy(fiber_idx, ord->fiber_idx, sizeof(int32_t) * ord->F, k));
  if (fiber_ptr) TK_CUDA(cudaMemcpy(fiber_ptr, ord->fiber_ptr, sizeof(int64_t) * (ord->F + 1), k));
  if (leaf_idx && X->nnz) TK_CUDA(cudaMemcpy(leaf_idx, ord->leaf_idx, sizeof(int32_t) * X->nnz, k));
  if (val && X->nnz) TK_CUDA(cudaMemcpy(val, ord->val, sizeof(double) * X->nnz, k));
  return TUCKER_OK;
}

int tucker_unfolding_gram(tucker_tensor X, int32_t n, double* d_M, void* stream) {
  if (!X || n < 0 || n > 2 || !d_M) return TUCKER_EINVAL;
  Run r;
  r.X = X;
  r.s = (cudaStream_t)stream;
  TK_TRY(unfolding_gram(r, n, d_M));
  TK_CUDA(cudaStreamSynchronize(r.s));
  return TUCKER_OK;
}

int tucker_ttmc(tucker_tensor X, int32_t n, const double* d_Um, int32_t Jm, const double* d_Uo,
                int32_t Jo, double* d_Y, void* stream) {
  if (!X || n < 0 || n > 2 || !d_Um || !d_Uo || !d_Y || Jm < 1 || Jo < 1) return TUCKER_EINVAL;
  int m, o;
  other_modes(n, &m, &o);
  cudaStream_t s = (cudaStream_t)stream;
  Ordering* ord;
  TK_TRY(ensure_ordering(X, n, m, o, s, &ord));
  TK_TRY(ttmc_fp64(X, ord, d_Um, Jm, d_Uo, Jo, d_Y, s));
  TK_CUDA(cudaStreamSynchronize(s));
  return TUCKER_OK;
}

int tucker_slice_proj(tucker_tensor X, int32_t n, int32_t m, const double* d_Um, int32_t Jm,
                      double* d_Y, void* stream) {
  if (!X || n < 0 || n > 2 || m < 0 || m > 2 || n == m || !d_Um || !d_Y || Jm < 1)
    return TUCKER_EINVAL;
  const int o = 3 - n - m;
  cudaStream_t s = (cudaStream_t)stream;
  Ordering* ord;
  TK_TRY(ensure_ordering(X, n, o, m, s, &ord));
  TK_TRY(slice_proj_f64(X, ord, d_Um, Jm, d_Y, s));
  TK_CUDA(cudaStreamSynchronize(s));
  return TUCKER_OK;
}

int tucker_gram(const double* d_Y1, int64_t K1, const double* d_Y2, int64_t K2, int32_t rows,
                double* d_M, void* stream) {
  if ((!d_Y1 && K1 != 0) || !d_M || rows < 1 || K1 < 0 || (d_Y2 && K2 < 0)) return TUCKER_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  TK_TRY(gram_f64_tc(rows, d_Y1, K1, d_Y2, d_Y2 ? K2 : 0, d_M, s));
  TK_CUDA(cudaStreamSynchronize(s));
  return TUCKER_OK;
}

int tucker_gram_fused(tucker_tensor X, int32_t n, int32_t m1, const float* d_U1, int32_t J1,
                      int32_t m2, const float* d_U2, int32_t J2, double* d_M, void* stream) {
  if (!X || n < 0 || n > 2 || m1 < 0 || m1 > 2 || m1 == n || !d_U1 || J1 < 1 || !d_M)
    return TUCKER_EINVAL;
  const int nt = m2 >= 0 ? 2 : 1;
  if (nt == 2 && (m2 > 2 || m2 == n || m2 == m1 || !d_U2 || J2 < 1)) return TUCKER_EINVAL;
  if (X->dims[n] > FUSED_GRAM_MAX_ROWS) return TUCKER_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int ms[2] = {m1, m2};
  const Ordering* ords[2] = {nullptr, nullptr};
  for (int t = 0; t < nt; ++t) {
    Ordering* ord;
    TK_TRY(ensure_ordering(X, n, 3 - n - ms[t], ms[t], s, &ord));
    TK_TRY(ensure_val_f32(X, ord, s));
    TK_TRY(ensure_fiber_map(X, ord, s));
    ords[t] = ord;
  }
  const float* U[2] = {d_U1, d_U2};
  const int64_t ld[2] = {J1, J2};
  const int J[2] = {J1, J2};
  TK_TRY(gram_fused_mixed(X, n, nt, ords, U, ld, J, d_M, s));
  TK_CUDA(cudaStreamSynchronize(s));
  return TUCKER_OK;
}

int tucker_gemm(const double* d_A, int64_t lda, const double* d_B, int64_t ldb, int32_t m,
                int32_t n, int64_t K, double* d_C, int64_t ldc, void* stream) {
  if (!d_C || m < 1 || n < 1 || K < 0 || (K > 0 && (!d_A || !d_B)) || lda < K || ldb < n ||
      ldc < n)
    return TUCKER_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  OzSlices a, b;
  TK_TRY(oz_split_rows(d_A, lda, m, K, nullptr, 0, 0, OZ_GEMM_SLICES, &a, s));
  TK_TRY(oz_split_cols(d_B, ldb, K, n, OZ_GEMM_SLICES, &b, s));
  Buf st;
  TK_TRY(st.alloc(sizeof(int), s));
  TK_CUDA(cudaMemsetAsync(st.p, 0, sizeof(int), s));
  TK_TRY(oz_gemm_nt(a, b, false, 1.0, 0.0, nullptr, 0, 0.0, nullptr, 0, d_C, ldc, st.as<int>(), s,
                    "gemm_ozaki"));
  int h = 0;
  TK_CUDA(cudaMemcpyAsync(&h, st.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  if (h & DEV_TIMEOUT) {
    set_error_detail("tensor-core product: a bounded wait on an mbarrier gave up");
    return TUCKER_ETIMEOUT;
  }
  return TUCKER_OK;
}

int tucker_ttmc_mixed(tucker_tensor X, int32_t n, const float* d_Um, int32_t Jm, const float* d_Uo,
                      int32_t Jo, uint16_t* d_Yhi, uint16_t* d_Ylo, int64_t ldY, float* d_Y32,
                      void* stream) {
  if (!X || n < 0 || n > 2 || !d_Um || !d_Uo || Jm < 1 || Jo < 1) return TUCKER_EINVAL;
  if ((!d_Yhi) != (!d_Ylo) || (!d_Yhi && !d_Y32)) return TUCKER_EINVAL;
  if (d_Yhi && (ldY < (int64_t)Jm * Jo || ldY % 64 != 0)) return TUCKER_EINVAL;
  int m, o;
  other_modes(n, &m, &o);
  cudaStream_t s = (cudaStream_t)stream;
  Ordering* ord;
  TK_TRY(ensure_ordering(X, n, m, o, s, &ord));
  TK_TRY(ensure_val_f32(X, ord, s));
  TK_TRY(ttmc_mixed(X, ord, d_Um, Jm, Jm, d_Uo, Jo, Jo, (__nv_bfloat16*)d_Yhi,
                    (__nv_bfloat16*)d_Ylo, ldY, d_Y32, s));
  TK_CUDA(cudaStreamSynchronize(s));
  return TUCKER_OK;
}

int tucker_slice_proj_mixed(tucker_tensor X, int32_t n, int32_t m, const float* d_Um, int32_t Jm,
                            uint16_t* d_Yhi, uint16_t* d_Ylo, int64_t ldY, void* stream) {
  if (!X || n < 0 || n > 2 || m < 0 || m > 2 || n == m || !d_Um || !d_Yhi || !d_Ylo || Jm < 1)
    return TUCKER_EINVAL;
  const int o = 3 - n - m;
  if (ldY < X->dims[o] * Jm || ldY % 64 != 0) return TUCKER_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  Ordering* ord;
  TK_TRY(ensure_ordering(X, n, o, m, s, &ord));
  TK_TRY(ensure_val_f32(X, ord, s));
  TK_TRY(slice_proj_mixed(X, ord, d_Um, Jm, Jm, (__nv_bfloat16*)d_Yhi, (__nv_bfloat16*)d_Ylo, ldY,
                          s));
  TK_CUDA(cudaStreamSynchronize(s));
  return TUCKER_OK;
}

int tucker_gram_bf16x3(const uint16_t* d_Y1hi, const uint16_t* d_Y1lo, int64_t K1, int64_t ld1,
                       const uint16_t* d_Y2hi, const uint16_t* d_Y2lo, int64_t K2, int64_t ld2,
                       int32_t rows, double* d_M, void* stream) {
  if (!d_Y1hi || !d_Y1lo || !d_M || rows < 1 || K1 < 1 || ld1 < K1 || ld1 % 64) return TUCKER_EINVAL;
  const bool two = d_Y2hi != nullptr;
  if (two && (!d_Y2lo || K2 < 1 || ld2 < K2 || ld2 % 64)) return TUCKER_EINVAL;
  const uintptr_t al = (uintptr_t)d_Y1hi | (uintptr_t)d_Y1lo | (uintptr_t)d_Y2hi | (uintptr_t)d_Y2lo;
  if (al % 16) return TUCKER_EINVAL;  // TMA needs 16-byte aligned bases
  GramTerm t[2] = {{(const __nv_bfloat16*)d_Y1hi, (const __nv_bfloat16*)d_Y1lo, K1, ld1},
                   {(const __nv_bfloat16*)d_Y2hi, (const __nv_bfloat16*)d_Y2lo, K2, ld2}};
  cudaStream_t s = (cudaStream_t)stream;
  TK_TRY(gram_bf16x3(rows, two ? 2 : 1, t, d_M, s));
  TK_CUDA(cudaStreamSynchronize(s));
  return TUCKER_OK;
}

int tucker_eig_topk(const double* d_M, int32_t n, int32_t J, const double* d_U0, double* d_U,
                    double* d_lambda, void* stream) {
  if (!d_M || !d_U || n < 1 || J < 1 || J > n) return TUCKER_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  TK_TRY(eig_topk_f64(d_M, n, J, d_U0, d_U, d_lambda, s, nullptr));
  TK_CUDA(cudaStreamSynchronize(s));
  return TUCKER_OK;
}

int tucker_core(tucker_tensor X, const double* d_A, const double* d_B, const double* d_C,
                const int32_t J[3], double* d_G, double* g_norm2, void* stream) {
  if (!X || !d_A || !d_B || !d_C || !J || !d_G) return TUCKER_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (J[a] < 1 || J[a] > X->dims[a]) return TUCKER_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  Ordering* ord;
  TK_TRY(ensure_ordering(X, 2, 0, 1, s, &ord));
  Buf Y, g2;
  TK_TRY(Y.alloc(sizeof(double) * X->dims[2] * J[0] * J[1], s));
  TK_TRY(g2.alloc(sizeof(double), s));
  TK_TRY(ttmc_fp64(X, ord, d_A, J[0], d_B, J[1], Y.as<double>(), s));
  TK_TRY(core_from_ttmc3(Y.as<double>(), (int)X->dims[2], J[0], J[1], d_C, J[2], d_G,
                         g2.as<double>(), s));
  double h = 0.0;
  TK_CUDA(cudaMemcpyAsync(&h, g2.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  if (g_norm2) *g_norm2 = h;
  return TUCKER_OK;
}

}  // extern "C"
