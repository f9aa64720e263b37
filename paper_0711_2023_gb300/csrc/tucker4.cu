// Fourth-order tensors: HO-SVD and HOOI (Figures HO-SVDn and hooin with N = 4), Slice
// Projection (Figure sp4) and Multislice Projection (Figure mp4), FP64.
//
// Every matrix these methods build is a Gram matrix of a projected unfolding, and most of them
// are third-order quantities of a "view" of the tensor that merges two of its modes:
//   * the slice sums of SP4 / MP4 for output mode n and projecting mode m equal
//     Gram((X x_m U_m^T)_(n)); with the other two modes a < b merged into one index
//     i_a I_b + i_b, that is exactly the third-order slice projection of the view
//     (n, m, merged) — so those terms run on the third-order kernels (sparse.cu);
//   * X_(n) X_(n)^T (HO-SVD, HOOI's start, MP4's pseudo HO-SVD start, which equals
//     3 X_(n) X_(n)^T) is the third-order unfolding Gram of any view that keeps n;
//   * HOOI's projection Z = X x_a U_a^T x_b U_b^T x_c U_c^T (all modes but n) is not: merging
//     b, c would turn U_b (x) U_c into one I_b I_c x J_b J_c factor and lose the factorisation.
//     It runs as a three-level tree on the view (n, a, merged(b, c)) sorted by
//     (i_n, i_a, i_b, i_c): runs (i_n, i_a, i_b) with leaves i_c, groups (i_n, i_a), slices i_n:
//       t_run  = sum_leaves x U_c[i_c, :]                      (nnz J_c FMAs)
//       s_grp  = sum_runs  U_b[i_b, :]^T (x) t_run               (runs J_b J_c)
//       Y[i_n] = sum_grps  U_a[i_a, :]^T (x) s_grp               (groups J_a J_b J_c)
// The Grams run on the tensor cores (gram_f64_tc) and the eigensolver is eig_topk_f64, as for
// third-order tensors.  The views and the run structure are built on first use and kept.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace tk {

// Runs of a TTMc ordering: sub-fibers of equal (i_n, i_a, i_b) inside each group (i_n, i_a).
struct Runs {
  bool built = false;
  int64_t R = 0;
  int32_t* run_b = nullptr;      // [R] i_b of each run
  int64_t* run_ptr = nullptr;    // [R + 1] first leaf of each run
  int64_t* group_run = nullptr;  // [G + 1] first run of each group
};

}  // namespace tk

struct tucker4_tensor_s {
  int64_t dims[4] = {0, 0, 0, 0};
  int64_t nnz = 0;
  int32_t* idx[4] = {nullptr, nullptr, nullptr, nullptr};  // canonical COO, sorted by (i1..i4)
  double* val = nullptr;
  double norm2 = 0.0;
  tucker_tensor_s* view[6] = {};  // third-order views, one per pair of modes kept separate
  tk::Runs runs[4];               // run structure of each mode's TTMc ordering
};

namespace tk {

namespace {

// Pair index of the separate modes (lo < hi) of a view; the two other modes (a < b) are merged.
int pair_id(int lo, int hi) {
  static const int ids[4][4] = {{-1, 0, 1, 2}, {0, -1, 3, 4}, {1, 3, -1, 5}, {2, 4, 5, -1}};
  return ids[lo][hi];
}
void merged_modes(int lo, int hi, int* a, int* b) {
  int m[2], k = 0;
  for (int x = 0; x < 4; ++x)
    if (x != lo && x != hi) m[k++] = x;
  *a = m[0];
  *b = m[1];
}

__global__ void check_and_merge(const int32_t* __restrict__ i0, const int32_t* __restrict__ i1,
                                const int32_t* __restrict__ i2, const int32_t* __restrict__ i3,
                                int64_t n, int64_t d0, int64_t d1, int64_t d2, int64_t d3,
                                int32_t* __restrict__ merged, int* status) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int32_t a = i0[t], b = i1[t], c = i2[t], d = i3[t];
  if (a < 0 || a >= d0 || b < 0 || b >= d1 || c < 0 || c >= d2 || d < 0 || d >= d3) {
    atomicOr(status, DEV_BAD_INDEX);
    merged[t] = 0;
    return;
  }
  merged[t] = (int32_t)((int64_t)c * d3 + d);
}

__global__ void unmerge(const int32_t* __restrict__ merged, int64_t n, int64_t d3,
                        int32_t* __restrict__ ia, int32_t* __restrict__ ib) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  ia[t] = (int32_t)(merged[t] / d3);
  ib[t] = (int32_t)(merged[t] % d3);
}

__global__ void merge_pair(const int32_t* __restrict__ ia, const int32_t* __restrict__ ib,
                           int64_t n, int64_t db, int32_t* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = (int32_t)((int64_t)ia[t] * db + ib[t]);
}

void free_view(tucker_tensor_s* T) {
  if (!T) return;
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
}

// The view with modes lo < hi kept and the other two merged: dims (I_lo, I_hi, I_a I_b).
int ensure_view(tucker4_tensor_s* X, int lo, int hi, cudaStream_t s, tucker_tensor_s** out) {
  const int id = pair_id(lo, hi);
  if (!X->view[id]) {
    int a, b;
    merged_modes(lo, hi, &a, &b);
    tucker_tensor_s* V = new (std::nothrow) tucker_tensor_s();
    if (!V) return TUCKER_ENOMEM;
    V->dims[0] = X->dims[lo];
    V->dims[1] = X->dims[hi];
    V->dims[2] = X->dims[a] * X->dims[b];
    cudaGetDevice(&V->device);
    Buf mg;
    int st = mg.alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(X->nnz, 1), s);
    if (st == TUCKER_OK && X->nnz > 0) {
      merge_pair<<<ceil_div(X->nnz, 256), 256, 0, s>>>(X->idx[a], X->idx[b], X->nnz, X->dims[b],
                                                        mg.as<int32_t>());
      if (cudaGetLastError() != cudaSuccess) st = TUCKER_ECUDA;
      count_launch();
    }
    if (st == TUCKER_OK)
      st = build_canonical(V, X->idx[lo], X->idx[hi], mg.as<int32_t>(), X->val, X->nnz, s);
    if (st != TUCKER_OK) {
      free_view(V);
      return st;
    }
    X->view[id] = V;
  }
  *out = X->view[id];
  return TUCKER_OK;
}

// ---- TTMc of order four ------------------------------------------------------------------------

__global__ void run_heads(const int32_t* __restrict__ leaf, int64_t nnz, int64_t dc,
                          unsigned* __restrict__ head) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnz) return;
  head[t] = (t == 0 || leaf[t] / dc != leaf[t - 1] / dc) ? 1u : 0u;
}

__global__ void group_heads(const int64_t* __restrict__ fiber_ptr, int64_t G,
                            unsigned* __restrict__ head) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < G) head[fiber_ptr[g]] = 1u;
}

__global__ void fill_runs(const unsigned* __restrict__ head, const unsigned* __restrict__ rid,
                          const int32_t* __restrict__ leaf, int64_t nnz, int64_t dc,
                          int64_t* __restrict__ run_ptr, int32_t* __restrict__ run_b) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnz || !head[t]) return;
  run_ptr[rid[t]] = t;
  run_b[rid[t]] = (int32_t)(leaf[t] / dc);
}

__global__ void fill_group_runs(const int64_t* __restrict__ fiber_ptr, int64_t G,
                                const unsigned* __restrict__ rid, int64_t R, int64_t nnz,
                                int64_t* __restrict__ group_run, int64_t* __restrict__ run_ptr) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < G) group_run[g] = rid[fiber_ptr[g]];
  if (g == G) {
    group_run[G] = R;
    run_ptr[R] = nnz;
  }
}

// The ordering (n, a, merged(b, c)) of mode n's TTMc (a < b < c the other modes) and its runs.
int ensure_ttmc_ordering(tucker4_tensor_s* X, int n, cudaStream_t s, tucker_tensor_s** view,
                         Ordering** ord, Runs** runs, int* abc) {
  int o[3], k = 0;
  for (int x = 0; x < 4; ++x)
    if (x != n) o[k++] = x;
  abc[0] = o[0];
  abc[1] = o[1];
  abc[2] = o[2];
  const int lo = std::min(n, o[0]), hi = std::max(n, o[0]);
  TK_TRY(ensure_view(X, lo, hi, s, view));
  const int pn = n == lo ? 0 : 1, pa = 1 - pn;
  TK_TRY(ensure_ordering(*view, pn, pa, 2, s, ord));
  Runs* R = &X->runs[n];
  if (!R->built) {
    const int64_t nnz = (*view)->nnz, G = (*ord)->F, dc = X->dims[o[2]];
    const size_t nn = (size_t)std::max<int64_t>(nnz, 1);
    Buf head, rid, tot;
    TK_TRY(head.alloc(4 * nn, s));
    TK_TRY(rid.alloc(4 * nn, s));
    TK_TRY(tot.alloc(sizeof(unsigned), s));
    unsigned Rn = 0;
    if (nnz > 0) {
      run_heads<<<ceil_div(nnz, 256), 256, 0, s>>>((*ord)->leaf_idx, nnz, dc, head.as<unsigned>());
      TK_LAUNCH();
      group_heads<<<ceil_div(G, 256), 256, 0, s>>>((*ord)->fiber_ptr, G, head.as<unsigned>());
      TK_LAUNCH();
      TK_TRY(exclusive_scan_u32(head.as<unsigned>(), rid.as<unsigned>(), nnz, tot.as<unsigned>(),
                                s));
      TK_CUDA(cudaMemcpyAsync(&Rn, tot.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
      TK_CUDA(cudaStreamSynchronize(s));
    }
    R->R = Rn;
    TK_CUDA(cudaMalloc(&R->run_b, sizeof(int32_t) * std::max<size_t>(Rn, 1)));
    TK_CUDA(cudaMalloc(&R->run_ptr, sizeof(int64_t) * (Rn + 1)));
    TK_CUDA(cudaMalloc(&R->group_run, sizeof(int64_t) * (G + 1)));
    if (nnz > 0) {
      fill_runs<<<ceil_div(nnz, 256), 256, 0, s>>>(head.as<unsigned>(), rid.as<unsigned>(),
                                                   (*ord)->leaf_idx, nnz, dc, R->run_ptr,
                                                   R->run_b);
      TK_LAUNCH();
    }
    fill_group_runs<<<ceil_div(G + 1, 256), 256, 0, s>>>((*ord)->fiber_ptr, G, rid.as<unsigned>(),
                                                         Rn, nnz, R->group_run, R->run_ptr);
    TK_LAUNCH();
    TK_CUDA(cudaStreamSynchronize(s));
    R->built = true;
  }
  *runs = R;
  return TUCKER_OK;
}

// t_run[r] = sum over the run's leaves of x U_c[i_c, r]: one warp per run.
__global__ void ttmc4_runs(const int64_t* __restrict__ run_ptr, int64_t R,
                           const int32_t* __restrict__ leaf, const double* __restrict__ val,
                           int64_t dc, const double* __restrict__ Uc, int Jc,
                           double* __restrict__ T) {
  const int64_t run = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (run >= R) return;
  const int64_t l0 = run_ptr[run], l1 = run_ptr[run + 1];
  for (int r0 = 0; r0 < Jc; r0 += 32) {
    const int r = r0 + lane;
    double acc = 0.0;
    if (r < Jc)
      for (int64_t l = l0; l < l1; ++l) acc = fma(val[l], Uc[(int64_t)(leaf[l] % dc) * Jc + r], acc);
    if (r < Jc) T[run * Jc + r] = acc;
  }
}

// s_grp[q J_c + r] = sum over the group's runs of U_b[i_b, q] t_run[r]: one CTA per group.
__global__ void ttmc4_groups(const int64_t* __restrict__ group_run, int64_t G,
                             const int32_t* __restrict__ run_b, const double* __restrict__ T,
                             const double* __restrict__ Ub, int Jb, int Jc,
                             double* __restrict__ Sg) {
  const int64_t g = blockIdx.x;
  if (g >= G) return;
  const int64_t r0 = group_run[g], r1 = group_run[g + 1];
  const int JbJc = Jb * Jc;
  for (int c = threadIdx.x; c < JbJc; c += blockDim.x) {
    const int q = c / Jc, r = c - q * Jc;
    double acc = 0.0;
    for (int64_t u = r0; u < r1; ++u)
      acc = fma(Ub[(int64_t)run_b[u] * Jb + q], T[u * Jc + r], acc);
    Sg[g * JbJc + c] = acc;
  }
}

// Y[i_n, p J_b J_c + c] = sum over the slice's groups of U_a[i_a, p] s_grp[c]; a CTA covers 256
// columns c and PT rows p of one slice.
constexpr int PT = 16;
__global__ void __launch_bounds__(256)
ttmc4_slices(const int64_t* __restrict__ root_ptr, const int32_t* __restrict__ group_a,
             const double* __restrict__ Sg, const double* __restrict__ Ua, int Ja, int JbJc,
             double* __restrict__ Y) {
  const int64_t i = blockIdx.x;
  const int c = blockIdx.y * 256 + threadIdx.x;
  const int p0 = blockIdx.z * PT;
  __shared__ double ua[32][PT];
  double acc[PT];
#pragma unroll
  for (int p = 0; p < PT; ++p) acc[p] = 0.0;
  const int64_t g0 = root_ptr[i], g1 = root_ptr[i + 1];
  for (int64_t gb = g0; gb < g1; gb += 32) {
    const int ng = (int)min64(32, g1 - gb);
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * PT; e += 256) {
      const int gi = e / PT, p = e % PT;
      ua[gi][p] = (gi < ng && p0 + p < Ja) ? Ua[(int64_t)group_a[gb + gi] * Ja + p0 + p] : 0.0;
    }
    __syncthreads();
    if (c < JbJc)
      for (int gi = 0; gi < ng; ++gi) {
        const double sv = Sg[(gb + gi) * JbJc + c];
#pragma unroll
        for (int p = 0; p < PT; ++p) acc[p] = fma(ua[gi][p], sv, acc[p]);
      }
  }
  if (c >= JbJc) return;
  const int64_t row = (int64_t)Ja * JbJc;
#pragma unroll
  for (int p = 0; p < PT; ++p)
    if (p0 + p < Ja) Y[i * row + (int64_t)(p0 + p) * JbJc + c] = acc[p];
}

}  // namespace

// Y_(n) = (X x_a U_a^T x_b U_b^T x_c U_c^T)_(n): I_n x (J_a J_b J_c), column (p J_b + q) J_c + r.
int ttmc4_f64(tucker4_tensor_s* X, int n, const double* const U[4], const int J[4], double* Y,
              cudaStream_t s) {
  tucker_tensor_s* V;
  Ordering* ord;
  Runs* R;
  int abc[3];
  TK_TRY(ensure_ttmc_ordering(X, n, s, &V, &ord, &R, abc));
  const int a = abc[0], b = abc[1], c = abc[2];
  const int Ja = J[a], Jb = J[b], Jc = J[c];
  const int64_t JbJc = (int64_t)Jb * Jc;
  const int64_t G = ord->F, nnz = V->nnz;
  ProfScope prof("ttmc4_f64", s,
                 2.0 * ((double)nnz * Jc + (double)R->R * JbJc + (double)G * Ja * JbJc),
                 20.0 * nnz + 12.0 * R->R + 12.0 * G + 8.0 * X->dims[n] * Ja * (double)JbJc);
  Buf T, Sg;
  TK_TRY(T.alloc(sizeof(double) * (size_t)std::max<int64_t>(R->R, 1) * Jc, s));
  TK_TRY(Sg.alloc(sizeof(double) * (size_t)std::max<int64_t>(G, 1) * JbJc, s));
  if (R->R > 0) {
    ttmc4_runs<<<ceil_div(R->R * 32, 256), 256, 0, s>>>(R->run_ptr, R->R, ord->leaf_idx, ord->val,
                                                         X->dims[c], U[c], Jc, T.as<double>());
    TK_LAUNCH();
  }
  if (G > 0) {
    ttmc4_groups<<<(unsigned)G, 256, 0, s>>>(R->group_run, G, R->run_b, T.as<double>(), U[b], Jb,
                                             Jc, Sg.as<double>());
    TK_LAUNCH();
  }
  dim3 grid((unsigned)X->dims[n], (unsigned)ceil_div(JbJc, 256), (unsigned)ceil_div(Ja, PT));
  ttmc4_slices<<<grid, 256, 0, s>>>(ord->root_ptr, ord->fiber_idx, Sg.as<double>(), U[a], Ja,
                                    (int)JbJc, Y);
  TK_LAUNCH();
  return TUCKER_OK;
}

// ---- the four methods ----------------------------------------------------------------------

namespace {

enum class Method4 { HOSVD, HOOI, SP, MP };

// Figure sp4: A from X x_4 D^T, B from X x_1 A^T, C from X x_2 B^T, D from X x_3 C^T.
const int SP4_PAIRS[4][2] = {{0, 3}, {1, 0}, {2, 1}, {3, 2}};

__global__ void add_f64(double* __restrict__ y, const double* __restrict__ x, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) y[t] += x[t];
}

struct Run4 {
  tucker4_tensor_s* X = nullptr;
  Method4 method = Method4::HOOI;
  int J[4] = {0, 0, 0, 0};
  cudaStream_t s = 0;
  tucker4_opts o;
  Buf U[4], Y, M, Mt, G, sc;   // sc: [0] |G|^2, [1] fit
  int rank_def = 0;
  std::vector<double> fits;
  int64_t dim(int a) const { return X->dims[a]; }
  const double* u(int a) const { return U[a].as<double>(); }
};

int slice_term4(Run4& r, int n, int m, double* Y, int64_t* K) {
  const int lo = std::min(n, m), hi = std::max(n, m);
  tucker_tensor_s* V;
  TK_TRY(ensure_view(r.X, lo, hi, r.s, &V));
  const int pn = n == lo ? 0 : 1, pm = 1 - pn;
  Ordering* ord;
  TK_TRY(ensure_ordering(V, pn, 2, pm, r.s, &ord));   // root n, fibers (i_n, merged), leaves i_m
  TK_TRY(slice_proj_f64(V, ord, r.u(m), r.J[m], Y, r.s));
  *K = V->dims[2] * r.J[m];
  return TUCKER_OK;
}

int unfolding_gram4(Run4& r, int n, double* M) {
  const int a = n == 0 ? 1 : 0;
  const int lo = std::min(n, a), hi = std::max(n, a);
  tucker_tensor_s* V;
  TK_TRY(ensure_view(r.X, lo, hi, r.s, &V));
  const int pn = n == lo ? 0 : 1, pa = 1 - pn;
  Ordering *rows, *fib;
  TK_TRY(ensure_ordering(V, pn, pa, 2, r.s, &rows));
  TK_TRY(ensure_ordering(V, pa, 2, pn, r.s, &fib));
  TK_TRY(ensure_fiber_map(V, fib, r.s));
  return unfolding_gram_f64(V, rows, fib, M, r.s);
}

int eig4(Run4& r, int n, bool warm) {
  EigStats st;
  TK_TRY(eig_topk_f64(r.M.as<double>(), (int)r.dim(n), r.J[n], warm ? r.u(n) : nullptr,
                      r.U[n].as<double>(), nullptr, r.s, &st));
  if (st.rank_deficient) r.rank_def |= 1 << n;
  return TUCKER_OK;
}

int ttmc4_run(Run4& r, int n) {
  const double* U[4] = {r.u(0), r.u(1), r.u(2), r.u(3)};
  return ttmc4_f64(r.X, n, U, r.J, r.Y.as<double>(), r.s);
}

// G from Z = [[X; A^T, B^T, C^T, I]] (in Y; computed unless z_ready), then the fit.
int core_and_fit4(Run4& r, bool z_ready, double* fit, double* g2) {
  if (!z_ready) TK_TRY(ttmc4_run(r, 3));
  TK_TRY(core_from_ttmc3(r.Y.as<double>(), (int)r.dim(3), r.J[0] * r.J[1], r.J[2], r.u(3),
                         r.J[3], r.G.as<double>(), r.sc.as<double>(), r.s));
  TK_TRY(fit_on_device(r.X->norm2, r.sc.as<double>(), r.sc.as<double>() + 1, r.s));
  double h[2];
  TK_CUDA(cudaMemcpyAsync(h, r.sc.p, sizeof(h), cudaMemcpyDeviceToHost, r.s));
  TK_CUDA(cudaStreamSynchronize(r.s));
  *g2 = h[0];
  *fit = h[1];
  return TUCKER_OK;
}

int run_method4(Method4 method, tucker4_tensor_s* X, const int32_t J[4], const tucker4_opts* opts,
                tucker4_result* out) {
  if (!X || !J || !out || !out->G) return TUCKER_EINVAL;
  for (int a = 0; a < 4; ++a)
    if (!out->U[a] || J[a] < 1 || J[a] > X->dims[a]) return TUCKER_EINVAL;
  if (out->where != TUCKER_HOST && out->where != TUCKER_DEVICE) return TUCKER_EINVAL;
  Run4 r;
  r.X = X;
  r.method = method;
  for (int a = 0; a < 4; ++a) r.J[a] = J[a];
  if (opts) {
    r.o = *opts;
  } else {
    memset(&r.o, 0, sizeof(r.o));
    r.o.precision = TUCKER_FP64;
    r.o.tol = 1e-4;
    r.o.max_iter = 50;
  }
  if (r.o.precision != TUCKER_FP64) {
    set_error_detail("fourth-order methods run in the FP64 form only");
    return TUCKER_EINVAL;
  }
  if (method != Method4::HOSVD && r.o.max_iter < 1) return TUCKER_EINVAL;
  if (isnan(r.o.tol) || r.o.tol == INFINITY || r.o.flags != 0) return TUCKER_EINVAL;
  if (r.o.init_where != TUCKER_HOST && r.o.init_where != TUCKER_DEVICE) return TUCKER_EINVAL;
  if (method == Method4::SP && !r.o.init[3]) return TUCKER_EINVAL;   // random D of Figure sp4
  if (X->nnz == 0 || !(X->norm2 > 0.0)) return TUCKER_EEMPTY;
  r.s = (cudaStream_t)r.o.stream;
  const cudaMemcpyKind to_dev =
      r.o.init_where == TUCKER_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;

  // Buffers: factors, the largest mode matrix, the core, the projections.
  int64_t maxI = 0, ymax = 0;
  for (int a = 0; a < 4; ++a) {
    TK_TRY(r.U[a].alloc(sizeof(double) * r.dim(a) * J[a], r.s));
    maxI = std::max(maxI, r.dim(a));
    const int64_t jprod = (int64_t)J[(a + 1) % 4] * J[(a + 2) % 4] * J[(a + 3) % 4];
    ymax = std::max(ymax, r.dim(a) * jprod);                       // HOOI / core projections
    for (int m = 0; m < 4; ++m)
      if (m != a) ymax = std::max(ymax, r.dim(0) * r.dim(1) * r.dim(2) * r.dim(3) / r.dim(m) * J[m]);
  }
  TK_TRY(r.M.alloc(sizeof(double) * maxI * maxI, r.s));
  TK_TRY(r.Mt.alloc(sizeof(double) * maxI * maxI, r.s));
  TK_TRY(r.G.alloc(sizeof(double) * J[0] * J[1] * J[2] * J[3], r.s));
  TK_TRY(r.sc.alloc(sizeof(double) * 2, r.s));
  TK_TRY(r.Y.alloc(sizeof(double) * (size_t)ymax, r.s));
  bool have[4] = {false, false, false, false};

  if (method == Method4::HOSVD) {
    for (int n = 0; n < 4; ++n) {
      TK_TRY(unfolding_gram4(r, n, r.M.as<double>()));
      TK_TRY(eig4(r, n, false));
    }
    double fit, g2;
    TK_TRY(core_and_fit4(r, false, &fit, &g2));
    r.fits.push_back(fit);
  } else {
    if (method == Method4::SP) {
      Buf raw;
      TK_TRY(raw.alloc(sizeof(double) * r.dim(3) * J[3], r.s));
      TK_CUDA(cudaMemcpyAsync(raw.p, r.o.init[3], sizeof(double) * r.dim(3) * J[3], to_dev, r.s));
      TK_TRY(normalize_columns(raw.as<double>(), (int)r.dim(3), J[3], r.U[3].as<double>(), r.s));
      TK_CUDA(cudaStreamSynchronize(r.s));
    } else {
      // HOOI: B, C, D from HO-SVD; MP: the pseudo HO-SVD matrices 3 X_(n) X_(n)^T have the same
      // leading eigenvectors.  A caller's start replaces either.
      for (int n = 1; n < 4; ++n) {
        if (r.o.init[n]) {
          TK_CUDA(cudaMemcpyAsync(r.U[n].p, r.o.init[n], sizeof(double) * r.dim(n) * J[n], to_dev,
                                  r.s));
        } else {
          TK_TRY(unfolding_gram4(r, n, r.M.as<double>()));
          if (method == Method4::MP) TK_TRY(scale_f64(r.dim(n) * r.dim(n), 3.0, r.M.as<double>(), r.s));
          TK_TRY(eig4(r, n, false));
        }
        have[n] = true;
      }
    }
    double old = 0.0, gprev = 0.0;
    for (int it = 0; it < r.o.max_iter; ++it) {
      for (int step = 0; step < 4; ++step) {
        int n = step;
        if (method == Method4::HOOI) {
          TK_TRY(ttmc4_run(r, n));
          TK_TRY(gram_f64_tc((int)r.dim(n), r.Y.as<double>(),
                             (int64_t)J[(n + 1) % 4] * J[(n + 2) % 4] * J[(n + 3) % 4], nullptr,
                             0, r.M.as<double>(), r.s));
        } else if (method == Method4::SP) {
          n = SP4_PAIRS[step][0];
          int64_t K;
          TK_TRY(slice_term4(r, n, SP4_PAIRS[step][1], r.Y.as<double>(), &K));
          TK_TRY(gram_f64_tc((int)r.dim(n), r.Y.as<double>(), K, nullptr, 0, r.M.as<double>(),
                             r.s));
        } else {
          // Figure mp4: the sum over the three other modes m of Gram((X x_m U_m^T)_(n))
          bool first = true;
          for (int m = 0; m < 4; ++m) {
            if (m == n) continue;
            int64_t K;
            TK_TRY(slice_term4(r, n, m, r.Y.as<double>(), &K));
            double* dst = first ? r.M.as<double>() : r.Mt.as<double>();
            TK_TRY(gram_f64_tc((int)r.dim(n), r.Y.as<double>(), K, nullptr, 0, dst, r.s));
            if (!first) {
              add_f64<<<ceil_div(r.dim(n) * r.dim(n), 256), 256, 0, r.s>>>(
                  r.M.as<double>(), r.Mt.as<double>(), r.dim(n) * r.dim(n));
              TK_LAUNCH();
            }
            first = false;
          }
        }
        TK_TRY(eig4(r, n, have[n]));
        have[n] = true;
      }
      double fit, g2;
      // HOOI's last projection (mode 4) is the core's input.
      TK_TRY(core_and_fit4(r, method == Method4::HOOI, &fit, &g2));
      r.fits.push_back(fit);
      if (method == Method4::SP) {
        const double gn = sqrt(g2);
        if (it >= 1 && (1.0 - gprev / gn) < r.o.tol) break;   // Delta_G test
        gprev = gn;
      } else {
        if (fit - old < r.o.tol) break;                        // Delta_fit test (signed)
        old = fit;
      }
    }
  }
  // results
  const cudaMemcpyKind from_dev =
      out->where == TUCKER_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  TK_CUDA(cudaMemcpyAsync(out->G, r.G.p, sizeof(double) * J[0] * J[1] * J[2] * J[3], from_dev,
                          r.s));
  for (int a = 0; a < 4; ++a)
    TK_CUDA(cudaMemcpyAsync(out->U[a], r.U[a].p, sizeof(double) * r.dim(a) * J[a], from_dev, r.s));
  if (out->fit_history && !r.fits.empty())
    TK_CUDA(cudaMemcpyAsync(out->fit_history, r.fits.data(), sizeof(double) * r.fits.size(),
                            out->where == TUCKER_DEVICE ? cudaMemcpyHostToDevice
                                                        : cudaMemcpyHostToHost,
                            r.s));
  TK_CUDA(cudaStreamSynchronize(r.s));
  out->fit = r.fits.empty() ? 0.0 : r.fits.back();
  out->iters = (int32_t)r.fits.size();
  out->rank_deficient = r.rank_def;
  return TUCKER_OK;
}

}  // namespace
}  // namespace tk

using namespace tk;

extern "C" {

int tucker4_tensor_create(const tucker4_coo* X, void* stream, tucker4_tensor* out) {
  if (!X || !out) return TUCKER_EINVAL;
  *out = nullptr;
  double cells = 1.0;
  for (int a = 0; a < 4; ++a) {
    if (X->dims[a] < 1 || X->dims[a] > 2147483647ll) return TUCKER_EINVAL;
    cells *= (double)X->dims[a];
  }
  if (cells >= 4.6e18) return TUCKER_EINVAL;
  // every view merges two modes into one 32-bit index
  for (int a = 0; a < 4; ++a)
    for (int b = a + 1; b < 4; ++b)
      if (X->dims[a] * X->dims[b] > 2147483647ll) return TUCKER_EINVAL;
  if (X->nnz < 0 || X->nnz > 2147483647ll) return TUCKER_EINVAL;
  if (X->where != TUCKER_HOST && X->where != TUCKER_DEVICE) return TUCKER_EINVAL;
  for (int a = 0; a < 4; ++a)
    if (X->nnz > 0 && !X->idx[a]) return TUCKER_EINVAL;
  if (X->nnz > 0 && !X->val) return TUCKER_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  tucker4_tensor_s* T = new (std::nothrow) tucker4_tensor_s();
  if (!T) return TUCKER_ENOMEM;
  for (int a = 0; a < 4; ++a) T->dims[a] = X->dims[a];
  const int64_t n = X->nnz;
  int st = TUCKER_OK;
  {
    Buf bi[4], bv, mg, stat;
    const int32_t* di[4] = {X->idx[0], X->idx[1], X->idx[2], X->idx[3]};
    const double* dv = X->val;
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    if (X->where == TUCKER_HOST && n > 0) {
      for (int a = 0; a < 4 && st == TUCKER_OK; ++a) {
        st = bi[a].alloc(sizeof(int32_t) * n, s);
        if (st == TUCKER_OK && cudaMemcpyAsync(bi[a].p, X->idx[a], sizeof(int32_t) * n,
                                               cudaMemcpyHostToDevice, s) != cudaSuccess)
          st = TUCKER_ECUDA;
        di[a] = bi[a].as<int32_t>();
      }
      if (st == TUCKER_OK) st = bv.alloc(sizeof(double) * n, s);
      if (st == TUCKER_OK &&
          cudaMemcpyAsync(bv.p, X->val, sizeof(double) * n, cudaMemcpyHostToDevice, s) != cudaSuccess)
        st = TUCKER_ECUDA;
      dv = bv.as<double>();
    }
    if (st == TUCKER_OK) st = mg.alloc(sizeof(int32_t) * nn, s);
    if (st == TUCKER_OK) st = stat.alloc(sizeof(int), s);
    int hstat = 0;
    if (st == TUCKER_OK && cudaMemsetAsync(stat.p, 0, sizeof(int), s) != cudaSuccess) st = TUCKER_ECUDA;
    if (st == TUCKER_OK && n > 0) {
      check_and_merge<<<ceil_div(n, 256), 256, 0, s>>>(di[0], di[1], di[2], di[3], n, T->dims[0],
                                                        T->dims[1], T->dims[2], T->dims[3],
                                                        mg.as<int32_t>(), stat.as<int>());
      count_launch();
      if (cudaGetLastError() != cudaSuccess) st = TUCKER_ECUDA;
    }
    if (st == TUCKER_OK &&
        (cudaMemcpyAsync(&hstat, stat.p, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
         cudaStreamSynchronize(s) != cudaSuccess))
      st = TUCKER_ECUDA;
    if (st == TUCKER_OK && (hstat & DEV_BAD_INDEX)) st = TUCKER_EINVAL;
    // The view (1, 2 | 3 4 merged) sums the duplicates and sorts by (i1, i2, i3 I4 + i4), which is
    // the canonical order of the fourth-order COO.
    tucker_tensor_s* V = nullptr;
    if (st == TUCKER_OK) {
      V = new (std::nothrow) tucker_tensor_s();
      if (!V) st = TUCKER_ENOMEM;
    }
    if (st == TUCKER_OK) {
      V->dims[0] = T->dims[0];
      V->dims[1] = T->dims[1];
      V->dims[2] = T->dims[2] * T->dims[3];
      cudaGetDevice(&V->device);
      st = build_canonical(V, di[0], di[1], mg.as<int32_t>(), dv, n, s);
      if (st != TUCKER_OK) {
        free_view(V);
      } else {
        T->view[pair_id(0, 1)] = V;
        T->nnz = V->nnz;
        T->norm2 = V->norm2;
        const size_t nu = (size_t)std::max<int64_t>(T->nnz, 1);
        for (int a = 0; a < 4 && st == TUCKER_OK; ++a)
          if (cudaMalloc(&T->idx[a], sizeof(int32_t) * nu) != cudaSuccess) st = TUCKER_ENOMEM;
        if (st == TUCKER_OK && cudaMalloc(&T->val, sizeof(double) * nu) != cudaSuccess)
          st = TUCKER_ENOMEM;
        if (st == TUCKER_OK && T->nnz > 0) {
          cudaMemcpyAsync(T->idx[0], V->idx[0], sizeof(int32_t) * T->nnz, cudaMemcpyDeviceToDevice, s);
          cudaMemcpyAsync(T->idx[1], V->idx[1], sizeof(int32_t) * T->nnz, cudaMemcpyDeviceToDevice, s);
          cudaMemcpyAsync(T->val, V->val, sizeof(double) * T->nnz, cudaMemcpyDeviceToDevice, s);
          unmerge<<<ceil_div(T->nnz, 256), 256, 0, s>>>(V->idx[2], T->nnz, T->dims[3], T->idx[2],
                                                         T->idx[3]);
          count_launch();
          if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
            st = TUCKER_ECUDA;
        }
      }
    }
  }
  if (st != TUCKER_OK) {
    tucker4_tensor_destroy(T);
    return st;
  }
  *out = T;
  return TUCKER_OK;
}

int tucker4_tensor_destroy(tucker4_tensor T) {
  if (!T) return TUCKER_OK;
  cudaDeviceSynchronize();
  for (int a = 0; a < 4; ++a) cudaFree(T->idx[a]);
  cudaFree(T->val);
  for (auto* V : T->view) free_view(V);
  for (auto& R : T->runs) {
    cudaFree(R.run_b);
    cudaFree(R.run_ptr);
    cudaFree(R.group_run);
  }
  delete T;
  return TUCKER_OK;
}

int tucker4_tensor_info(tucker4_tensor X, int64_t* nnz, double* norm2) {
  if (!X) return TUCKER_EINVAL;
  if (nnz) *nnz = X->nnz;
  if (norm2) *norm2 = X->norm2;
  return TUCKER_OK;
}

int tucker4_hosvd(tucker4_tensor X, const int32_t J[4], const tucker4_opts* opts,
                  tucker4_result* out) {
  return run_method4(Method4::HOSVD, X, J, opts, out);
}
int tucker4_hooi(tucker4_tensor X, const int32_t J[4], const tucker4_opts* opts,
                 tucker4_result* out) {
  return run_method4(Method4::HOOI, X, J, opts, out);
}
int tucker4_sp(tucker4_tensor X, const int32_t J[4], const tucker4_opts* opts, tucker4_result* out) {
  return run_method4(Method4::SP, X, J, opts, out);
}
int tucker4_mp(tucker4_tensor X, const int32_t J[4], const tucker4_opts* opts, tucker4_result* out) {
  return run_method4(Method4::MP, X, J, opts, out);
}

int tucker4_ttmc(tucker4_tensor X, int32_t n, const double* const d_U[4], const int32_t J[4],
                 double* d_Y, void* stream) {
  if (!X || n < 0 || n > 3 || !d_U || !J || !d_Y) return TUCKER_EINVAL;
  for (int a = 0; a < 4; ++a)
    if (a != n && (!d_U[a] || J[a] < 1 || J[a] > X->dims[a])) return TUCKER_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int Jc[4] = {J[0], J[1], J[2], J[3]};
  TK_TRY(ttmc4_f64(X, n, d_U, Jc, d_Y, s));
  TK_CUDA(cudaStreamSynchronize(s));
  return TUCKER_OK;
}

}  // extern "C"
