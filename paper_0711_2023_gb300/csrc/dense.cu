// FP64 dense kernels: the Gram M = Y Y^T of the projected tensors (Figures hooi3, sp3, mp3:
// leading eigenvectors of U_(1) U_(1)^T etc.), and the small GEMMs of the eigensolver and of
// the core.  All reductions have a fixed order (split-K partials are summed in split order),
// so results are bitwise reproducible.  FP64 arithmetic on this part is ALU-bound; the tiles
// are sized for register reuse, not for bandwidth.
#include <algorithm>

#include "internal.h"

namespace tk {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

// C = alpha * A B + beta * X + gamma * Z, 64 x 64 tile per CTA, 4 x 4 per thread, products
// and sums in TC (A stored as TA, B converted to TC on load; epilogue in FP64).  With P given,
// the CTA instead writes its raw partial product over K-slice blockIdx.z (of length kchunk) to
// P[blockIdx.z] and the epilogue is applied by reduce_nn.
template <typename TA, typename TC>
__global__ void __launch_bounds__(256)
gemm_nn_kernel(int m, int n, int k, double alpha, const TA* __restrict__ A, int64_t lda,
               const double* __restrict__ B, int64_t ldb, double beta, const double* Xm,
               int64_t ldx, double gamma, const double* __restrict__ Zm, int64_t ldz, double* C,
               int64_t ldc, int kchunk, double* __restrict__ P) {
  __shared__ TC As[BK][BM + 1];
  __shared__ TC Bs[BK][BN];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  TC acc[4][4] = {};
  const int kb = blockIdx.z * kchunk;
  const int ke = min(k, kb + kchunk);
  for (int k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = threadIdx.x + 256 * e;  // 0..1023
      const int ar = idx / BK, ac = idx % BK;  // A tile: 64 rows x 16 cols
      const int gr = m0 + ar, gc = k0 + ac;
      As[ac][ar] = (gr < m && gc < ke) ? (TC)A[(int64_t)gr * lda + gc] : TC(0);
      const int br = idx / BN, bc = idx % BN;  // B tile: 16 rows x 64 cols
      const int hr = k0 + br, hc = n0 + bc;
      Bs[br][bc] = (hr < ke && hc < n) ? (TC)B[(int64_t)hr * ldb + hc] : TC(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      TC a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (P) {
    double* Pz = P + (int64_t)blockIdx.z * m * n;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = m0 + ty + 16 * i;
      if (r >= m) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = n0 + tx + 16 * j;
        if (c < n) Pz[(int64_t)r * n + c] = acc[i][j];
      }
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = m0 + ty + 16 * i;
    if (r >= m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = n0 + tx + 16 * j;
      if (c >= n) continue;
      double v = alpha * (double)acc[i][j];
      if (Xm) v = fma(beta, Xm[(int64_t)r * ldx + c], v);
      if (Zm) v = fma(gamma, Zm[(int64_t)r * ldz + c], v);
      C[(int64_t)r * ldc + c] = v;
    }
  }
}

// FP64 C = alpha * op(A) B + beta * X + gamma * Z with op(A) = A^T when TA (A: k x m) and A
// otherwise (A: m x k); a 16 x 16 output tile per CTA, one output per thread.  FP64 FMA
// throughput (about 2 per clock per SM on this part) bounds every FP64 product of the
// eigensolver, so the tile is sized to fill all SMs with little padding (75 columns pad to 80,
// not 128), not for register reuse.  With P given the CTA writes its raw partial over K-slice
// blockIdx.z to P[blockIdx.z] and reduce_nn applies the epilogue.
template <bool TA>
__global__ void __launch_bounds__(256)
gemm16_kernel(int m, int n, int64_t k, double alpha, const double* __restrict__ A, int64_t lda,
              const double* __restrict__ B, int64_t ldb, double beta, const double* Xm,
              int64_t ldx, double gamma, const double* __restrict__ Zm, int64_t ldz, double* C,
              int64_t ldc, int64_t kchunk, double* __restrict__ P) {
  __shared__ double As[16][17];  // [i][kk]
  __shared__ double Bs[16][17];  // [kk][j]
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * 16, n0 = blockIdx.x * 16;
  const int64_t kb = (int64_t)blockIdx.z * kchunk;
  const int64_t ke = min64(k, kb + kchunk);
  double acc = 0.0;
  for (int64_t k0 = kb; k0 < ke; k0 += 16) {
    if (TA) {
      const int64_t kr = k0 + ty;
      const int gi = m0 + tx;
      As[tx][ty] = (kr < ke && gi < m) ? A[kr * lda + gi] : 0.0;
    } else {
      const int gi = m0 + ty;
      const int64_t kc = k0 + tx;
      As[ty][tx] = (gi < m && kc < ke) ? A[(int64_t)gi * lda + kc] : 0.0;
    }
    {
      const int64_t kr = k0 + ty;
      const int gj = n0 + tx;
      Bs[ty][tx] = (kr < ke && gj < n) ? B[kr * ldb + gj] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) acc = fma(As[ty][kk], Bs[kk][tx], acc);
    __syncthreads();
  }
  const int r = m0 + ty, c = n0 + tx;
  if (r >= m || c >= n) return;
  if (P) {
    P[(int64_t)blockIdx.z * m * n + (int64_t)r * n + c] = acc;
    return;
  }
  double v = alpha * acc;
  if (Xm) v = fma(beta, Xm[(int64_t)r * ldx + c], v);
  if (Zm) v = fma(gamma, Zm[(int64_t)r * ldz + c], v);
  C[(int64_t)r * ldc + c] = v;
}

// C = alpha * (sum of the split partials, in split order) + beta * X + gamma * Z.
__global__ void reduce_nn(const double* __restrict__ P, int splits, int m, int n, double alpha,
                          double beta, const double* Xm, int64_t ldx, double gamma,
                          const double* __restrict__ Zm, int64_t ldz, double* C, int64_t ldc) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * n) return;
  const int64_t r = t / n, c = t % n;
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += P[(int64_t)z * m * n + t];
  double v = alpha * s;
  if (Xm) v = fma(beta, Xm[r * ldx + c], v);
  if (Zm) v = fma(gamma, Zm[r * ldz + c], v);
  C[r * ldc + c] = v;
}

// SYRK partials over lower-triangle tile pairs (ti >= tj) of rows x rows; K is the
// concatenation of Y1's K1 columns and Y2's K2 columns.
__global__ void __launch_bounds__(256)
syrk_kernel(int rows, const double* __restrict__ Y1, int64_t K1, const double* __restrict__ Y2,
            int64_t K2, int64_t kchunk, const int2* __restrict__ pairs,
            double* __restrict__ P) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BM + 1];
  const int2 pr = pairs[blockIdx.x];
  const int r0 = pr.x * BM, c0 = pr.y * BM;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t K = K1 + K2;
  const int64_t kb = (int64_t)blockIdx.y * kchunk;
  const int64_t ke = min64(K, kb + kchunk);
  double acc[4][4] = {};
  for (int64_t k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = threadIdx.x + 256 * e;
      const int rr = idx / BK, kk = idx % BK;  // 64 rows x 16 k
      const int64_t kg = k0 + kk;
      double va = 0.0, vb = 0.0;
      if (kg < ke) {
        const int ra = r0 + rr, rb = c0 + rr;
        if (kg < K1) {
          if (ra < rows) va = Y1[(int64_t)ra * K1 + kg];
          if (rb < rows) vb = Y1[(int64_t)rb * K1 + kg];
        } else {
          const int64_t k2 = kg - K1;
          if (ra < rows) va = Y2[(int64_t)ra * K2 + k2];
          if (rb < rows) vb = Y2[(int64_t)rb * K2 + k2];
        }
      }
      As[kk][rr] = va;
      Bs[kk][rr] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double* Pz = P + (int64_t)blockIdx.y * rows * rows;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + ty + 16 * i;
    if (r >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx + 16 * j;
      if (c < rows) Pz[(int64_t)r * rows + c] = acc[i][j];
    }
  }
}

// Sums the split partials of lower-triangle tiles and mirrors them into the upper triangle.
__global__ void syrk_reduce(const double* __restrict__ P, int splits, int rows,
                            double* __restrict__ M) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)rows * rows) return;
  const int r = (int)(t / rows), c = (int)(t % rows);
  if (r / BM < c / BM) return;  // upper tiles are written as mirrors
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += P[(int64_t)z * rows * rows + t];
  M[(int64_t)r * rows + c] = s;
  if (r / BM != c / BM) M[(int64_t)c * rows + r] = s;
}

__global__ void copy_cols_kernel(int rows, int cols, const double* __restrict__ src, int64_t lds,
                                 double* __restrict__ dst, int64_t ldd) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)rows * cols) return;
  const int64_t r = t / cols, c = t % cols;
  dst[r * ldd + c] = src[r * lds + c];
}

__global__ void scale_kernel(int64_t n, double alpha, double* x) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) x[t] *= alpha;
}

int choose_splits(int tiles, int64_t k) {
  const int target = 3 * num_sms();
  int splits = (target + tiles - 1) / tiles;
  const int64_t maxs = (k + 31) / 32;  // K slices of at least 32
  if (splits > maxs) splits = (int)maxs;
  if (splits < 1) splits = 1;
  return splits;
}

}  // namespace

namespace {

template <typename TA, typename TC>
int gemm_nn_impl(const char* name, int m, int n, int k, double alpha, const TA* A, int64_t lda,
                 const double* B, int64_t ldb, double beta, const double* Xm, int64_t ldx,
                 double gamma, const double* Zm, int64_t ldz, double* C, int64_t ldc,
                 cudaStream_t s) {
  if (m <= 0 || n <= 0) return TUCKER_OK;
  ProfScope prof(name, s, 2.0 * m * n * (double)k,
                 (double)sizeof(TA) * m * k + 8.0 * ((double)k * n + (double)m * n));
  const int tiles = ceil_div(n, BN) * ceil_div(m, BM);
  // Skinny products (the eigensolver's M V with few columns) get too few tiles to fill the
  // GPU: split K into slices summed in a fixed order by reduce_nn.
  int splits = 1;
  if (tiles < num_sms() && k >= 4 * BK) {
    splits = std::min((2 * num_sms() + tiles - 1) / tiles, k / (2 * BK));
    if (splits < 1) splits = 1;
  }
  if (splits == 1) {
    dim3 grid(ceil_div(n, BN), ceil_div(m, BM), 1);
    gemm_nn_kernel<TA, TC><<<grid, 256, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta, Xm, ldx,
                                                gamma, Zm, ldz, C, ldc, k, nullptr);
    TK_LAUNCH();
    return TUCKER_OK;
  }
  int kchunk = (k + splits - 1) / splits;
  kchunk = (kchunk + BK - 1) / BK * BK;
  splits = (k + kchunk - 1) / kchunk;
  Buf P;
  TK_TRY(P.alloc(sizeof(double) * (size_t)splits * m * n, s));
  dim3 grid(ceil_div(n, BN), ceil_div(m, BM), splits);
  gemm_nn_kernel<TA, TC><<<grid, 256, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta, Xm, ldx, gamma,
                                              Zm, ldz, C, ldc, kchunk, P.as<double>());
  TK_LAUNCH();
  reduce_nn<<<ceil_div((int64_t)m * n, 256), 256, 0, s>>>(P.as<double>(), splits, m, n, alpha,
                                                          beta, Xm, ldx, gamma, Zm, ldz, C, ldc);
  TK_LAUNCH();
  return TUCKER_OK;
}

template <bool TA>
int gemm16(const char* name, int m, int n, int64_t k, double alpha, const double* A, int64_t lda,
           const double* B, int64_t ldb, double beta, const double* Xm, int64_t ldx, double gamma,
           const double* Zm, int64_t ldz, double* C, int64_t ldc, cudaStream_t s) {
  if (m <= 0 || n <= 0) return TUCKER_OK;
  ProfScope prof(name, s, 2.0 * m * n * (double)k,
                 8.0 * ((double)m * k + (double)k * n + (double)m * n));
  const int tiles = ceil_div(n, 16) * ceil_div(m, 16);
  // Enough CTAs for two per SM; K slices of at least 64, summed in a fixed order.
  int64_t splits = 1;
  const int want = 2 * num_sms();
  if (tiles < want && k >= 128) splits = std::min<int64_t>((want + tiles - 1) / tiles, k / 64);
  int64_t kchunk = (k + splits - 1) / splits;
  kchunk = std::max<int64_t>(16, (kchunk + 15) / 16 * 16);
  splits = (k + kchunk - 1) / kchunk;
  if (splits <= 1) {
    dim3 grid(ceil_div(n, 16), ceil_div(m, 16), 1);
    gemm16_kernel<TA><<<grid, 256, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta, Xm, ldx, gamma,
                                           Zm, ldz, C, ldc, std::max<int64_t>(k, 1), nullptr);
    TK_LAUNCH();
    return TUCKER_OK;
  }
  Buf P;
  TK_TRY(P.alloc(sizeof(double) * (size_t)splits * m * n, s));
  dim3 grid(ceil_div(n, 16), ceil_div(m, 16), (unsigned)splits);
  gemm16_kernel<TA><<<grid, 256, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta, Xm, ldx, gamma,
                                         Zm, ldz, C, ldc, kchunk, P.as<double>());
  TK_LAUNCH();
  reduce_nn<<<ceil_div((int64_t)m * n, 256), 256, 0, s>>>(P.as<double>(), (int)splits, m, n,
                                                          alpha, beta, Xm, ldx, gamma, Zm, ldz,
                                                          C, ldc);
  TK_LAUNCH();
  return TUCKER_OK;
}

}  // namespace

int gemm_nn_f64(int m, int n, int k, double alpha, const double* A, int64_t lda, const double* B,
                int64_t ldb, double beta, const double* Xm, int64_t ldx, double gamma,
                const double* Zm, int64_t ldz, double* C, int64_t ldc, cudaStream_t s) {
  return gemm16<false>("gemm_nn_f64", m, n, k, alpha, A, lda, B, ldb, beta, Xm, ldx, gamma, Zm,
                       ldz, C, ldc, s);
}

int gemm_nn_f32a(int m, int n, int k, double alpha, const float* A, int64_t lda, const double* B,
                 int64_t ldb, double beta, const double* Xm, int64_t ldx, double gamma,
                 const double* Zm, int64_t ldz, double* C, int64_t ldc, cudaStream_t s) {
  return gemm_nn_impl<float, float>("gemm_nn_f32", m, n, k, alpha, A, lda, B, ldb, beta, Xm, ldx,
                                    gamma, Zm, ldz, C, ldc, s);
}

int gemm_tn_f64(int m, int n, int64_t k, const double* A, int64_t lda, const double* B,
                int64_t ldb, double* C, int64_t ldc, cudaStream_t s) {
  return gemm16<true>("gemm_tn_f64", m, n, k, 1.0, A, lda, B, ldb, 0.0, nullptr, 0, 0.0, nullptr,
                      0, C, ldc, s);
}

int syrk_f64(int rows, const double* Y1, int64_t K1, const double* Y2, int64_t K2, double* M,
             cudaStream_t s) {
  if (rows <= 0) return TUCKER_OK;
  if (!Y2) K2 = 0;
  ProfScope prof("syrk_f64", s, (double)rows * (rows + 1) * (double)(K1 + K2),
                 8.0 * rows * (double)(K1 + K2) + 8.0 * rows * rows);
  const int nt = ceil_div(rows, BM);
  const int npairs = nt * (nt + 1) / 2;
  const int64_t K = K1 + K2;
  const int splits = choose_splits(npairs, K);
  int64_t kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + BK - 1) / BK * BK;
  if (kchunk == 0) kchunk = BK;
  const int nsplit = (int)((K + kchunk - 1) / kchunk > 0 ? (K + kchunk - 1) / kchunk : 1);
  Buf pairs, P;
  TK_TRY(pairs.alloc(sizeof(int2) * npairs, s));
  TK_TRY(P.alloc(sizeof(double) * (size_t)nsplit * rows * rows, s));
  int2* hp = (int2*)malloc(sizeof(int2) * npairs);
  if (!hp) return TUCKER_ENOMEM;
  int q = 0;
  for (int i = 0; i < nt; ++i)
    for (int j = 0; j <= i; ++j) hp[q++] = make_int2(i, j);
  cudaError_t e = cudaMemcpyAsync(pairs.p, hp, sizeof(int2) * npairs, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  free(hp);
  TK_CUDA(e);
  if (K == 0) {
    TK_CUDA(cudaMemsetAsync(P.p, 0, sizeof(double) * (size_t)nsplit * rows * rows, s));
  } else {
    dim3 grid(npairs, nsplit);
    syrk_kernel<<<grid, 256, 0, s>>>(rows, Y1, K1, Y2, K2, kchunk, pairs.as<int2>(),
                                     P.as<double>());
    TK_LAUNCH();
  }
  syrk_reduce<<<ceil_div((int64_t)rows * rows, 256), 256, 0, s>>>(P.as<double>(), nsplit, rows,
                                                                  M);
  TK_LAUNCH();
  return TUCKER_OK;
}

int copy_cols_f64(int rows, int cols, const double* src, int64_t lds, double* dst, int64_t ldd,
                  cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return TUCKER_OK;
  copy_cols_kernel<<<ceil_div((int64_t)rows * cols, 256), 256, 0, s>>>(rows, cols, src, lds, dst,
                                                                       ldd);
  TK_LAUNCH();
  return TUCKER_OK;
}

int scale_f64(int64_t n, double alpha, double* x, cudaStream_t s) {
  if (n <= 0) return TUCKER_OK;
  scale_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, alpha, x);
  TK_LAUNCH();
  return TUCKER_OK;
}

}  // namespace tk
