// FP64 sparse kernels of the hot path:
//   ttmc_f64        HOOI projection Y = X x_m U_m^T x_o U_o^T (Figure hooi3: the U, V, W
//                   tensors), fiber-factored in two stages on ordering (n, m, o);
//   slice_proj_f64  SP/MP projection Y = X x_m U_m^T (Figures sp3, mp3) on ordering (n, o, m);
//   unfolding_gram  X_(n) X_(n)^T (Figure HO-SVD3), row-owned and deterministic.
// Every output element has exactly one writer and a fixed summation order, so results are
// bitwise reproducible run to run.
#include "internal.h"

namespace tk {

namespace {

// Output tile (16*AP) x (16*AQ) of Y[i_n, p, q] for one root slice i_n per CTA.  Stage 1
// (one warp per fiber): t_f[q] = sum over the fiber's leaves of x * U_o[i_o, q]; the factor
// row U_m[i_m, :] of the fiber is staged beside it.  Stage 2: Y[i_n] += U_m[i_m,:] (x) t_f,
// a rank-FC update of the register tile.
template <int AP, int AQ>
__global__ void __launch_bounds__(256)
ttmc_f64_kernel(const int64_t* __restrict__ root_ptr, const int32_t* __restrict__ fiber_idx,
                const int64_t* __restrict__ fiber_ptr, const int32_t* __restrict__ leaf_idx,
                const double* __restrict__ val, const double* __restrict__ Um, int Jm,
                const double* __restrict__ Uo, int Jo, double* __restrict__ Y) {
  constexpr int TP = 16 * AP, TQ = 16 * AQ, FC = 32, RQ = (TQ + 31) / 32;
  __shared__ double su[FC][TP];
  __shared__ double st[FC][TQ];
  const int i = blockIdx.x;
  const int p0 = blockIdx.y * TP, q0 = blockIdx.z * TQ;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc[AP][AQ];
#pragma unroll
  for (int a = 0; a < AP; ++a)
#pragma unroll
    for (int b = 0; b < AQ; ++b) acc[a][b] = 0.0;
  const int64_t fb = root_ptr[i], fe = root_ptr[i + 1];
  for (int64_t fc = fb; fc < fe; fc += FC) {
    const int nc = (int)min64(FC, fe - fc);
    for (int c = warp; c < nc; c += 8) {
      const int64_t f = fc + c;
      const int64_t l0 = fiber_ptr[f], l1 = fiber_ptr[f + 1];
      const int64_t im = fiber_idx[f];
      for (int tp = lane; tp < TP; tp += 32)
        su[c][tp] = (p0 + tp < Jm) ? Um[im * Jm + p0 + tp] : 0.0;
      double t[RQ];
#pragma unroll
      for (int r = 0; r < RQ; ++r) t[r] = 0.0;
      for (int64_t l = l0; l < l1; ++l) {
        const double x = val[l];
        const double* row = Uo + (int64_t)leaf_idx[l] * Jo + q0;
#pragma unroll
        for (int r = 0; r < RQ; ++r) {
          const int q = lane + 32 * r;
          if (q < TQ && q0 + q < Jo) t[r] = fma(x, row[q], t[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < RQ; ++r) {
        const int q = lane + 32 * r;
        if (q < TQ) st[c][q] = t[r];
      }
    }
    __syncthreads();
    for (int c = 0; c < nc; ++c) {
      double uu[AP], tt[AQ];
#pragma unroll
      for (int a = 0; a < AP; ++a) uu[a] = su[c][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < AQ; ++b) tt[b] = st[c][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < AP; ++a)
#pragma unroll
        for (int b = 0; b < AQ; ++b) acc[a][b] = fma(uu[a], tt[b], acc[a][b]);
    }
    __syncthreads();
  }
  double* Yi = Y + (int64_t)i * Jm * Jo;
#pragma unroll
  for (int a = 0; a < AP; ++a) {
    const int p = p0 + ty + 16 * a;
    if (p >= Jm) continue;
#pragma unroll
    for (int b = 0; b < AQ; ++b) {
      const int q = q0 + tx + 16 * b;
      if (q < Jo) Yi[(int64_t)p * Jo + q] = acc[a][b];
    }
  }
}

template <int AP, int AQ>
void launch_ttmc(const tucker_tensor_s* X, const Ordering* o, const double* Um, int Jm,
                 const double* Uo, int Jo, double* Y, cudaStream_t s) {
  dim3 grid((unsigned)X->dims[o->n], ceil_div(Jm, 16 * AP), ceil_div(Jo, 16 * AQ));
  ttmc_f64_kernel<AP, AQ><<<grid, 256, 0, s>>>(o->root_ptr, o->fiber_idx, o->fiber_ptr,
                                               o->leaf_idx, o->val, Um, Jm, Uo, Jo, Y);
}

int tile_code(int J) { return J <= 16 ? 1 : (J <= 32 ? 2 : 4); }

// One warp per fiber (i_n, i_o): Y[i_n, i_o*Jm + p] = sum over leaves of x * U_m[i_m, p].
template <int NP>
__global__ void __launch_bounds__(256)
slice_proj_f64_kernel(int64_t F, const int32_t* __restrict__ fiber_root,
                      const int32_t* __restrict__ fiber_idx, const int64_t* __restrict__ fiber_ptr,
                      const int32_t* __restrict__ leaf_idx, const double* __restrict__ val,
                      const double* __restrict__ Um, int Jm, int64_t Io, double* __restrict__ Y) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t f = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); f < F;
       f += (int64_t)gridDim.x * wpb) {
    const int64_t l0 = fiber_ptr[f], l1 = fiber_ptr[f + 1];
    // without a (row, column) map, fiber f's sums form row f of Y (F x Jm)
    double* out = fiber_root ? Y + (int64_t)fiber_root[f] * Io * Jm + (int64_t)fiber_idx[f] * Jm
                             : Y + f * Jm;
    for (int pc = 0; pc < Jm; pc += 32 * NP) {
      double acc[NP];
#pragma unroll
      for (int r = 0; r < NP; ++r) acc[r] = 0.0;
      for (int64_t l = l0; l < l1; ++l) {
        const double x = val[l];
        const double* row = Um + (int64_t)leaf_idx[l] * Jm + pc;
#pragma unroll
        for (int r = 0; r < NP; ++r) {
          const int p = lane + 32 * r;
          if (pc + p < Jm) acc[r] = fma(x, row[p], acc[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < NP; ++r) {
        const int p = lane + 32 * r;
        if (pc + p < Jm) out[pc + p] = acc[r];
      }
    }
  }
}

// Row a of X_(n) X_(n)^T: for every nonzero (a, i_m, i_o) with value x (ordering (n, m, o)),
// the mode-n fiber (i_m, i_o) (ordering (m, o, n), located through the dense fiber map)
// contributes x * x_b to entry b for each of its nonzeros b.  Warps own disjoint sets of
// row-a fibers and accumulate into private shared-memory rows, summed in warp order.
__global__ void unfold_gram_f64_kernel(const int64_t* __restrict__ r_root_ptr,
                                       const int32_t* __restrict__ r_fiber_idx,
                                       const int64_t* __restrict__ r_fiber_ptr,
                                       const int32_t* __restrict__ r_leaf,
                                       const double* __restrict__ r_val,
                                       const int32_t* __restrict__ fmap, int64_t Io,
                                       const int64_t* __restrict__ f_fiber_ptr,
                                       const int32_t* __restrict__ f_leaf,
                                       const double* __restrict__ f_val, int In,
                                       double* __restrict__ M, int* status) {
  extern __shared__ double part[];  // [nwarps][In]
  const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int a = blockIdx.x;
  for (int t = threadIdx.x; t < nw * In; t += blockDim.x) part[t] = 0.0;
  __syncthreads();
  double* mine = part + (int64_t)w * In;
  const int64_t rb = r_root_ptr[a], re = r_root_ptr[a + 1];
  for (int64_t rf = rb + w; rf < re; rf += nw) {
    const int64_t im = r_fiber_idx[rf];
    const int64_t t0 = r_fiber_ptr[rf], t1 = r_fiber_ptr[rf + 1];
    for (int64_t tc = t0; tc < t1; tc += 32) {
      const int cnt = (int)min64(32, t1 - tc);
      double x = 0.0;
      int64_t lo = 0, hi = 0;
      if (lane < cnt) {
        x = r_val[tc + lane];
        const int32_t fid = fmap[im * Io + r_leaf[tc + lane]];
        if (fid < 0) {
          atomicOr(status, DEV_BAD_INDEX);
        } else {
          lo = f_fiber_ptr[fid];
          hi = f_fiber_ptr[fid + 1];
        }
      }
      for (int j = 0; j < cnt; ++j) {
        const double xj = __shfl_sync(0xffffffffu, x, j);
        const int64_t lj = __shfl_sync(0xffffffffu, lo, j);
        const int64_t hj = __shfl_sync(0xffffffffu, hi, j);
        for (int64_t l = lj + lane; l < hj; l += 32) {
          const int b = f_leaf[l];
          mine[b] = fma(xj, f_val[l], mine[b]);
        }
        __syncwarp();
      }
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < In; b += blockDim.x) {
    double sum = 0.0;
    for (int j = 0; j < nw; ++j) sum += part[(int64_t)j * In + b];
    M[(int64_t)a * In + b] = sum;
  }
}

}  // namespace

int ttmc_f64(const tucker_tensor_s* X, const Ordering* o, const double* Um, int Jm,
             const double* Uo, int Jo, double* Y, cudaStream_t s) {
  if (X->dims[o->n] == 0) return TUCKER_OK;
  const double nnz = (double)X->nnz, F = (double)o->F;
  ProfScope prof("ttmc_f64", s, 2.0 * (nnz * Jo + F * Jm * Jo),
                 12.0 * nnz + 12.0 * F + 8.0 * X->dims[o->n] * (double)Jm * Jo +
                     8.0 * (X->dims[o->m] * (double)Jm + X->dims[o->o] * (double)Jo));
  const int cp = tile_code(Jm), cq = tile_code(Jo);
#define TK_TT(A, B) \
  if (cp == A && cq == B) launch_ttmc<A, B>(X, o, Um, Jm, Uo, Jo, Y, s);
  TK_TT(1, 1) TK_TT(1, 2) TK_TT(1, 4) TK_TT(2, 1) TK_TT(2, 2) TK_TT(2, 4) TK_TT(4, 1)
  TK_TT(4, 2) TK_TT(4, 4)
#undef TK_TT
  TK_LAUNCH();
  return TUCKER_OK;
}

int slice_proj_f64(const tucker_tensor_s* X, const Ordering* o, const double* Um, int Jm,
                   double* Y, cudaStream_t s) {
  // ordering (n, o, m): fibers are (i_n, i_o), leaves i_m.
  const int64_t In = X->dims[o->n], Io = X->dims[o->m];
  ProfScope prof("slice_proj_f64", s, 2.0 * (double)X->nnz * Jm,
                 12.0 * X->nnz + 16.0 * o->F + 8.0 * (double)In * Io * Jm +
                     8.0 * X->dims[o->o] * (double)Jm);
  TK_CUDA(cudaMemsetAsync(Y, 0, sizeof(double) * (size_t)(In * Io * Jm), s));
  if (o->F == 0) return TUCKER_OK;
  const int64_t wpb = 8;
  const int64_t blocks64 = (o->F + wpb - 1) / wpb;
  const int blocks = (int)min64(blocks64, (int64_t)num_sms() * 64);
  const int np = Jm <= 32 ? 1 : (Jm <= 64 ? 2 : (Jm <= 128 ? 4 : 8));
#define TK_SP(N)                                                                              \
  if (np == N)                                                                                \
    slice_proj_f64_kernel<N><<<blocks, 256, 0, s>>>(o->F, o->fiber_root, o->fiber_idx,        \
                                                    o->fiber_ptr, o->leaf_idx, o->val, Um, Jm, \
                                                    Io, Y);
  TK_SP(1) TK_SP(2) TK_SP(4) TK_SP(8)
#undef TK_SP
  TK_LAUNCH();
  return TUCKER_OK;
}

int unfolding_gram_f64(const tucker_tensor_s* X, const Ordering* rows, const Ordering* fib,
                       double* M, cudaStream_t s) {
  // rows: ordering (n, m, o); fib: ordering (m, o, n) with its fiber map over (i_m, i_o).
  const int In = (int)X->dims[rows->n];
  const int64_t Io = X->dims[rows->o];
  int nw = 4;
  while (nw > 1 && (size_t)nw * In * sizeof(double) > 200 * 1024) nw >>= 1;
  const size_t smem = (size_t)nw * In * sizeof(double);
  if (smem > 220 * 1024) return TUCKER_EINVAL;  // rows longer than shared memory holds
  if (smem > 48 * 1024)
    TK_CUDA(cudaFuncSetAttribute(unfold_gram_f64_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  Buf st;
  TK_TRY(st.alloc(sizeof(int), s));
  TK_CUDA(cudaMemsetAsync(st.p, 0, sizeof(int), s));
  ProfScope prof("unfold_gram_f64", s, 0.0, 12.0 * 2 * X->nnz + 8.0 * In * In);
  unfold_gram_f64_kernel<<<In, nw * 32, smem, s>>>(
      rows->root_ptr, rows->fiber_idx, rows->fiber_ptr, rows->leaf_idx, rows->val,
      fib->fiber_map, Io, fib->fiber_ptr, fib->leaf_idx, fib->val, In, M, st.as<int>());
  TK_LAUNCH();
  int h = 0;
  TK_CUDA(cudaMemcpyAsync(&h, st.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  return h ? TUCKER_EINTERNAL : TUCKER_OK;
}

int slice_proj_f64_fibers(int64_t F, const int32_t* row, const int32_t* col,
                          const int64_t* fiber_ptr, const int32_t* leaf_idx, const double* val,
                          const double* Um, int Jm, int64_t ncol, double* Y, cudaStream_t s) {
  if (F == 0) return TUCKER_OK;
  const int64_t wpb = 8;
  const int blocks = (int)min64((F + wpb - 1) / wpb, (int64_t)num_sms() * 64);
  const int np = Jm <= 32 ? 1 : (Jm <= 64 ? 2 : (Jm <= 128 ? 4 : 8));
#define TK_SP(N)                                                                              \
  if (np == N)                                                                                \
    slice_proj_f64_kernel<N><<<blocks, 256, 0, s>>>(F, row, col, fiber_ptr, leaf_idx, val, Um, \
                                                    Jm, ncol, Y);
  TK_SP(1) TK_SP(2) TK_SP(4) TK_SP(8)
#undef TK_SP
  TK_LAUNCH();
  return TUCKER_OK;
}

int ttmc_f64_roots(int64_t nroots, const int64_t* root_ptr, const int32_t* fiber_idx,
                   const int64_t* fiber_ptr, const int32_t* leaf_idx, const double* val,
                   const double* Um, int Jm, const double* Uo, int Jo, double* Y, cudaStream_t s) {
  if (nroots == 0) return TUCKER_OK;
  const int cp = tile_code(Jm), cq = tile_code(Jo);
  dim3 grid((unsigned)nroots, 0, 0);
#define TK_TT(AP, AQ)                                                                          \
  if (cp == AP && cq == AQ) {                                                                  \
    dim3 g((unsigned)nroots, ceil_div(Jm, 16 * AP), ceil_div(Jo, 16 * AQ));                    \
    ttmc_f64_kernel<AP, AQ><<<g, 256, 0, s>>>(root_ptr, fiber_idx, fiber_ptr, leaf_idx, val,   \
                                              Um, Jm, Uo, Jo, Y);                              \
  }
  TK_TT(1, 1) TK_TT(1, 2) TK_TT(1, 4) TK_TT(2, 1) TK_TT(2, 2) TK_TT(2, 4) TK_TT(4, 1)
  TK_TT(4, 2) TK_TT(4, 4)
#undef TK_TT
  (void)grid;
  TK_LAUNCH();
  return TUCKER_OK;
}

int ttmc_fp64(const tucker_tensor_s* X, const Ordering* o, const double* Um, int Jm,
              const double* Uo, int Jo, double* Y, cudaStream_t s) {
  // The rank-J_m J_o updates of the fibers dominate; with enough of them they run as per-slice
  // products on the tensor cores (FP64-accurate), else on the CUDA cores.  A slice holds at
  // most I_m fibers; the tensor-core products take at most 2^24 per slice.
  if ((int64_t)Jm * Jo >= 2048 && o->F >= 4096 && X->dims[o->m] <= (1 << 24))
    return ttmc_f64_tc(X, o, Um, Jm, Uo, Jo, Y, s);
  return ttmc_f64(X, o, Um, Jm, Uo, Jo, Y, s);
}

}  // namespace tk
