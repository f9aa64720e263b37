// Mixed-precision projections for the tensor-core Gram:
//   ttmc_mixed        HOOI's Y = X x_m U_m^T x_o U_o^T (Figure hooi3) with FP32 factors and
//                     FP32 accumulation;
//   slice_proj_mixed  SP/MP's Y = X x_m U_m^T (Figures sp3, mp3), FP32.
// Both write Y_(n) split into two BF16 matrices, Y = hi + lo (hi = bf16(y), lo = bf16(y - hi)),
// row-major with rows padded to a multiple of 64 columns (zeros), the layout the BF16x3 Gram
// reads with TMA.  HOOI's projection can also be written in FP32 for the core.
// As in the FP64 kernels, every output element has one writer and a fixed summation order.
#include <cuda_bf16.h>
#include <math.h>

#include <functional>

#include "internal.h"

namespace tk {

namespace {

__device__ __forceinline__ void split_store(float y, __nv_bfloat16* hi, __nv_bfloat16* lo,
                                            int64_t off) {
  const __nv_bfloat16 h = __float2bfloat16_rn(y);
  hi[off] = h;
  lo[off] = __float2bfloat16_rn(y - __bfloat162float(h));
}

__global__ void f64_to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = (float)a[t];
}

// b (rows x ldb) = FP32 of a (rows x cols, dense), zeros in columns cols..ldb-1.
__global__ void f64_to_f32_rows_kernel(const double* __restrict__ a, int64_t rows, int cols,
                                       float* __restrict__ b, int64_t ldb) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * ldb) return;
  const int64_t r = t / ldb, c = t - r * ldb;
  b[t] = c < cols ? (float)a[r * cols + c] : 0.f;
}

__global__ void f32_to_f64_kernel(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = (double)a[t];
}

template <int AP, int AQ, bool VEC>
__global__ void __launch_bounds__(256)
ttmc_mixed_kernel(const int64_t* __restrict__ root_ptr, const int32_t* __restrict__ fiber_idx,
                  const int64_t* __restrict__ fiber_ptr, const int32_t* __restrict__ leaf_idx,
                  const float* __restrict__ val, const float* __restrict__ Um, int64_t ldm,
                  int Jm, const float* __restrict__ Uo, int64_t ldo, int Jo,
                  __nv_bfloat16* __restrict__ Yh, __nv_bfloat16* __restrict__ Yl, int64_t ldY,
                  float* __restrict__ Y32) {
  constexpr int TP = 16 * AP, TQ = 16 * AQ, FC = 64, RQ = (TQ + 31) / 32;
  __shared__ float su[FC][TP];
  __shared__ __align__(16) float st[FC][TQ];
  const int i = blockIdx.x;
  const int p0 = blockIdx.y * TP, q0 = blockIdx.z * TQ;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[AP][AQ];
#pragma unroll
  for (int a = 0; a < AP; ++a)
#pragma unroll
    for (int b = 0; b < AQ; ++b) acc[a][b] = 0.f;
  const int64_t fb = root_ptr[i], fe = root_ptr[i + 1];
  for (int64_t fc = fb; fc < fe; fc += FC) {
    const int nc = (int)min64(FC, fe - fc);
    if constexpr (VEC) {
      // Factor rows padded to a multiple of 4 floats and TQ = 64: a group of 8 lanes owns one
      // fiber (four per warp at once) and loads each leaf's 64-column row segment of U_o with
      // two float4 loads per lane; the leaves' indices and values come 8 at a time.
      const int gid = lane >> 3, gl = lane & 7;
      const bool in0 = q0 + 4 * gl < ldo, in1 = q0 + 4 * (gl + 8) < ldo;
      for (int c0 = warp * 4; c0 < nc; c0 += 32) {
        const int c = c0 + gid;
        const bool active = c < nc;
        int64_t l0 = 0;
        int len = 0;
        if (active) {
          const int64_t f = fc + c;
          l0 = fiber_ptr[f];
          len = (int)(fiber_ptr[f + 1] - l0);
          const int64_t im = fiber_idx[f];
          for (int tp = gl; tp < TP; tp += 8)
            su[c][tp] = (p0 + tp < Jm) ? Um[im * ldm + p0 + tp] : 0.f;
        }
        const int maxlen = __reduce_max_sync(0xffffffffu, len);
        float r[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) r[q] = 0.f;
        for (int lb = 0; lb < maxlen; lb += 8) {
          const bool have = lb + gl < len;
          const int my_idx = have ? leaf_idx[l0 + lb + gl] : 0;
          const float my_val = have ? val[l0 + lb + gl] : 0.f;
          const int cnt = min(8, maxlen - lb);
#pragma unroll 4
          for (int j = 0; j < cnt; ++j) {
            const int idx = __shfl_sync(0xffffffffu, my_idx, j, 8);
            const float x = __shfl_sync(0xffffffffu, my_val, j, 8);
            if (lb + j < len) {
              const float4* row = reinterpret_cast<const float4*>(Uo + (int64_t)idx * ldo + q0);
              const float4 u0 = in0 ? row[gl] : make_float4(0.f, 0.f, 0.f, 0.f);
              const float4 u1 = in1 ? row[gl + 8] : make_float4(0.f, 0.f, 0.f, 0.f);
              r[0] = fmaf(x, u0.x, r[0]); r[1] = fmaf(x, u0.y, r[1]);
              r[2] = fmaf(x, u0.z, r[2]); r[3] = fmaf(x, u0.w, r[3]);
              r[4] = fmaf(x, u1.x, r[4]); r[5] = fmaf(x, u1.y, r[5]);
              r[6] = fmaf(x, u1.z, r[6]); r[7] = fmaf(x, u1.w, r[7]);
            }
          }
        }
        if (active) {
          *reinterpret_cast<float4*>(&st[c][4 * gl]) = make_float4(r[0], r[1], r[2], r[3]);
          *reinterpret_cast<float4*>(&st[c][4 * (gl + 8)]) = make_float4(r[4], r[5], r[6], r[7]);
        }
      }
    } else {
      for (int c = warp; c < nc; c += 8) {
        const int64_t f = fc + c;
        const int64_t l0 = fiber_ptr[f], l1 = fiber_ptr[f + 1];
        const int64_t im = fiber_idx[f];
        for (int tp = lane; tp < TP; tp += 32)
          su[c][tp] = (p0 + tp < Jm) ? Um[im * ldm + p0 + tp] : 0.f;
        float t[RQ];
#pragma unroll
        for (int r = 0; r < RQ; ++r) t[r] = 0.f;
        for (int64_t l = l0; l < l1; ++l) {
          const float x = val[l];
          const float* row = Uo + (int64_t)leaf_idx[l] * ldo + q0;
#pragma unroll
          for (int r = 0; r < RQ; ++r) {
            const int q = lane + 32 * r;
            if (q < TQ && q0 + q < Jo) t[r] = fmaf(x, row[q], t[r]);
          }
        }
#pragma unroll
        for (int r = 0; r < RQ; ++r) {
          const int q = lane + 32 * r;
          if (q < TQ) st[c][q] = t[r];
        }
      }
    }
    __syncthreads();
    for (int c = 0; c < nc; ++c) {
      float uu[AP], tt[AQ];
#pragma unroll
      for (int a = 0; a < AP; ++a) uu[a] = su[c][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < AQ; ++b) tt[b] = st[c][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < AP; ++a)
#pragma unroll
        for (int b = 0; b < AQ; ++b) acc[a][b] = fmaf(uu[a], tt[b], acc[a][b]);
    }
    __syncthreads();
  }
  const int64_t K = (int64_t)Jm * Jo;
#pragma unroll
  for (int a = 0; a < AP; ++a) {
    const int p = p0 + ty + 16 * a;
    if (p >= Jm) continue;
#pragma unroll
    for (int b = 0; b < AQ; ++b) {
      const int q = q0 + tx + 16 * b;
      if (q >= Jo) continue;
      const int64_t col = (int64_t)p * Jo + q;
      if (Yh) split_store(acc[a][b], Yh, Yl, (int64_t)i * ldY + col);
      if (Y32) Y32[(int64_t)i * K + col] = acc[a][b];
    }
  }
  if (Yh && blockIdx.y == 0 && blockIdx.z == 0) {
    for (int64_t c = K + threadIdx.x; c < ldY; c += blockDim.x) {
      Yh[(int64_t)i * ldY + c] = __float2bfloat16_rn(0.f);
      Yl[(int64_t)i * ldY + c] = __float2bfloat16_rn(0.f);
    }
  }
}

// Row i of an SP/MP projection when slice i has no nonzeros: all zeros (one CTA).
__device__ __forceinline__ void zero_row(__nv_bfloat16* rh, __nv_bfloat16* rl, int64_t ldY) {
  const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
  for (int64_t c = threadIdx.x; c < ldY; c += blockDim.x) {
    rh[c] = z;
    rl[c] = z;
  }
}

// The columns that belong to no fiber, written as zeros by the warp of the next fiber: those of
// the i_o values between fiber f - 1 and fiber f, and after the slice's last fiber those up to
// the padded row length.
__device__ __forceinline__ void zero_gaps(const int32_t* __restrict__ fiber_idx, int64_t f,
                                          int64_t fb, int64_t fe, int64_t io, int Jm,
                                          __nv_bfloat16* rh, __nv_bfloat16* rl, int64_t ldY,
                                          int lane) {
  const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
  const int64_t gap0 = (f == fb) ? 0 : (int64_t)(fiber_idx[f - 1] + 1) * Jm;
  for (int64_t c = gap0 + lane; c < io * Jm; c += 32) {
    rh[c] = z;
    rl[c] = z;
  }
  if (f == fe - 1) {
    for (int64_t c = (io + 1) * Jm + lane; c < ldY; c += 32) {
      rh[c] = z;
      rl[c] = z;
    }
  }
}

// One CTA per root slice i_n of ordering (n, o, m); warps take the slice's fibers (i_n, i_o) in
// turn, summing each fiber's leaves in index order.  Each warp also zero-fills the columns of
// the i_o values between its fiber and the previous one, so every element of row i_n
// (including the padding) is written exactly once.
template <int NP>
__global__ void __launch_bounds__(256)
slice_proj_mixed_kernel(const int64_t* __restrict__ root_ptr, const int32_t* __restrict__ fiber_idx,
                        const int64_t* __restrict__ fiber_ptr, const int32_t* __restrict__ leaf_idx,
                        const float* __restrict__ val, const float* __restrict__ Um, int64_t ldm,
                        int Jm, __nv_bfloat16* __restrict__ Yh, __nv_bfloat16* __restrict__ Yl,
                        int64_t ldY) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t i = blockIdx.x;
  __nv_bfloat16* rh = Yh + i * ldY;
  __nv_bfloat16* rl = Yl + i * ldY;
  const int64_t fb = root_ptr[i], fe = root_ptr[i + 1];
  if (fb == fe) {
    zero_row(rh, rl, ldY);
    return;
  }
  for (int64_t f = fb + warp; f < fe; f += nw) {
    const int64_t io = fiber_idx[f];
    zero_gaps(fiber_idx, f, fb, fe, io, Jm, rh, rl, ldY, lane);
    const int64_t l0 = fiber_ptr[f], l1 = fiber_ptr[f + 1];
    for (int pc = 0; pc < Jm; pc += 32 * NP) {
      float acc[NP];
#pragma unroll
      for (int r = 0; r < NP; ++r) acc[r] = 0.f;
      // Up to 32 leaves at a time: one coalesced load of their indices and values, then the
      // row gathers, which are independent of one another and so overlap.
      for (int64_t lb = l0; lb < l1; lb += 32) {
        const int cnt = (int)min64(32, l1 - lb);
        const int my_idx = lane < cnt ? leaf_idx[lb + lane] : 0;
        const float my_val = lane < cnt ? val[lb + lane] : 0.f;
#pragma unroll 2
        for (int j = 0; j < cnt; ++j) {
          const float x = __shfl_sync(0xffffffffu, my_val, j);
          const float* row = Um + (int64_t)__shfl_sync(0xffffffffu, my_idx, j) * ldm + pc;
#pragma unroll
          for (int r = 0; r < NP; ++r) {
            const int p = lane + 32 * r;
            if (pc + p < Jm) acc[r] = fmaf(x, row[p], acc[r]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < NP; ++r) {
        const int p = lane + 32 * r;
        if (pc + p < Jm) split_store(acc[r], rh, rl, io * Jm + pc + p);
      }
    }
  }
}


// The same projection for factor rows padded to a multiple of 4 floats (16-byte aligned) and
// J_m <= 8 G = 64 (G = 8) or 128 (G = 16).  A group of G lanes owns one fiber (a warp takes
// 32 / G fibers at once): its lanes hold the fiber's sum for columns 4 l .. 4 l + 3 and
// 4 (l + G) .. + 3, load each leaf's factor row with two float4 loads, and take the fiber's leaf
// indices and values G at a time with one coalesced load.  The per-fiber work (pointers, gap
// zeroing, the BF16 split stores) is spread over the warp's fibers; leaves are summed in index
// order, so the result is reproducible.
template <int G>
__global__ void __launch_bounds__(256)
slice_proj_mixed_vec_kernel(const int64_t* __restrict__ root_ptr,
                            const int32_t* __restrict__ fiber_idx,
                            const int64_t* __restrict__ fiber_ptr,
                            const int32_t* __restrict__ leaf_idx, const float* __restrict__ val,
                            const float* __restrict__ Um, int64_t ldm, int Jm,
                            __nv_bfloat16* __restrict__ Yh, __nv_bfloat16* __restrict__ Yl,
                            int64_t ldY) {
  constexpr int NF = 32 / G;  // fibers per warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int gid = lane / G, gl = lane % G;
  const int64_t i = blockIdx.x;
  __nv_bfloat16* rh = Yh + i * ldY;
  __nv_bfloat16* rl = Yl + i * ldY;
  const int64_t fb = root_ptr[i], fe = root_ptr[i + 1];
  if (fb == fe) {
    zero_row(rh, rl, ldY);
    return;
  }
  const bool in0 = 4 * gl < ldm, in1 = 4 * (gl + G) < ldm;
  const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
  for (int64_t f0 = fb + (int64_t)warp * NF; f0 < fe; f0 += (int64_t)nw * NF) {
    const int64_t f = f0 + gid;
    const bool active = f < fe;
    int64_t io = 0, l0 = 0;
    int len = 0;
    if (active) {
      io = fiber_idx[f];
      l0 = fiber_ptr[f];
      len = (int)(fiber_ptr[f + 1] - l0);
      // columns of the i_o values between the previous fiber and this one, and after the last
      const int64_t gap0 = (f == fb) ? 0 : (int64_t)(fiber_idx[f - 1] + 1) * Jm;
      for (int64_t c = gap0 + gl; c < io * Jm; c += G) {
        rh[c] = z;
        rl[c] = z;
      }
      if (f == fe - 1)
        for (int64_t c = (io + 1) * Jm + gl; c < ldY; c += G) {
          rh[c] = z;
          rl[c] = z;
        }
    }
    const int maxlen = __reduce_max_sync(0xffffffffu, len);
    float r[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) r[q] = 0.f;
    for (int lb = 0; lb < maxlen; lb += G) {
      const bool have = lb + gl < len;
      const int my_idx = have ? leaf_idx[l0 + lb + gl] : 0;
      const float my_val = have ? val[l0 + lb + gl] : 0.f;
      const int cnt = min(G, maxlen - lb);
#pragma unroll 4
      for (int j = 0; j < cnt; ++j) {
        const int idx = __shfl_sync(0xffffffffu, my_idx, j, G);
        const float x = __shfl_sync(0xffffffffu, my_val, j, G);
        if (lb + j < len) {
          const float4* row = reinterpret_cast<const float4*>(Um + (int64_t)idx * ldm);
          const float4 u0 = in0 ? row[gl] : make_float4(0.f, 0.f, 0.f, 0.f);
          const float4 u1 = in1 ? row[gl + G] : make_float4(0.f, 0.f, 0.f, 0.f);
          r[0] = fmaf(x, u0.x, r[0]); r[1] = fmaf(x, u0.y, r[1]);
          r[2] = fmaf(x, u0.z, r[2]); r[3] = fmaf(x, u0.w, r[3]);
          r[4] = fmaf(x, u1.x, r[4]); r[5] = fmaf(x, u1.y, r[5]);
          r[6] = fmaf(x, u1.z, r[6]); r[7] = fmaf(x, u1.w, r[7]);
        }
      }
    }
    if (!active) continue;
    const int64_t o = io * Jm;
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int c = 4 * (gl + G * v);
#pragma unroll
      for (int t = 0; t < 4; t += 2) {
        if (c + t >= Jm) break;
        const float y0 = r[4 * v + t], y1 = r[4 * v + t + 1];
        if ((Jm & 1) == 0) {  // o + c + t even: a 4-byte BF16 pair
          const __nv_bfloat16 h0 = __float2bfloat16_rn(y0), h1 = __float2bfloat16_rn(y1);
          __nv_bfloat162 hh, ll;
          hh.x = h0;
          hh.y = h1;
          ll.x = __float2bfloat16_rn(y0 - __bfloat162float(h0));
          ll.y = __float2bfloat16_rn(y1 - __bfloat162float(h1));
          *reinterpret_cast<__nv_bfloat162*>(rh + o + c + t) = hh;
          *reinterpret_cast<__nv_bfloat162*>(rl + o + c + t) = ll;
        } else {
          split_store(y0, rh, rl, o + c + t);
          if (c + t + 1 < Jm) split_store(y1, rh, rl, o + c + t + 1);
        }
      }
    }
  }
}

template <int AP, int AQ>
void launch_ttmc_mixed(const tucker_tensor_s* X, const Ordering* o, const float* Um,
                       int64_t ldm, int Jm, const float* Uo, int64_t ldo, int Jo,
                       __nv_bfloat16* Yh, __nv_bfloat16* Yl, int64_t ldY, float* Y32, bool vec,
                       cudaStream_t s) {
  dim3 grid((unsigned)X->dims[o->n], ceil_div(Jm, 16 * AP), ceil_div(Jo, 16 * AQ));
  if (vec)
    ttmc_mixed_kernel<AP, AQ, true><<<grid, 256, 0, s>>>(o->root_ptr, o->fiber_idx, o->fiber_ptr,
                                                         o->leaf_idx, o->val_f32, Um, ldm, Jm, Uo,
                                                         ldo, Jo, Yh, Yl, ldY, Y32);
  else
    ttmc_mixed_kernel<AP, AQ, false><<<grid, 256, 0, s>>>(o->root_ptr, o->fiber_idx,
                                                          o->fiber_ptr, o->leaf_idx, o->val_f32,
                                                          Um, ldm, Jm, Uo, ldo, Jo, Yh, Yl, ldY,
                                                          Y32);
}

int tcode(int J) { return J <= 16 ? 1 : (J <= 32 ? 2 : 4); }

// Shape class of a projection for the autotuner: round(log2(mean fiber length)).
int fiber_class(int64_t nnz, int64_t F) {
  if (F <= 0 || nnz <= F) return 0;
  const int c = (int)lround(log2((double)nnz / (double)F));
  return c < 0 ? 0 : (c > 16 ? 16 : c);
}

bool rows16(const float* U, int64_t ld) {
  return ld % 4 == 0 && (reinterpret_cast<uintptr_t>(U) & 15) == 0;
}

}  // namespace

int f64_to_f32(const double* a, float* b, int64_t n, cudaStream_t s) {
  if (n <= 0) return TUCKER_OK;
  f64_to_f32_kernel<<<ceil_div(n, 256), 256, 0, s>>>(a, b, n);
  TK_LAUNCH();
  return TUCKER_OK;
}

int f32_to_f64(const float* a, double* b, int64_t n, cudaStream_t s) {
  if (n <= 0) return TUCKER_OK;
  f32_to_f64_kernel<<<ceil_div(n, 256), 256, 0, s>>>(a, b, n);
  TK_LAUNCH();
  return TUCKER_OK;
}

int ensure_val_f32(tucker_tensor_s* X, Ordering* ord, cudaStream_t s) {
  if (ord->val_f32) return TUCKER_OK;
  TK_CUDA(cudaMalloc(&ord->val_f32, sizeof(float) * (size_t)(X->nnz ? X->nnz : 1)));
  return f64_to_f32(ord->val, ord->val_f32, X->nnz, s);
}

int ttmc_mixed(const tucker_tensor_s* X, const Ordering* o, const float* Um, int64_t ldm, int Jm,
               const float* Uo, int64_t ldo, int Jo, __nv_bfloat16* Yh, __nv_bfloat16* Yl,
               int64_t ldY, float* Y32, cudaStream_t s) {
  if (X->dims[o->n] == 0) return TUCKER_OK;
  const double nnz = (double)X->nnz, F = (double)o->F;
  ProfScope prof("ttmc_mixed", s, 2.0 * (nnz * Jo + F * Jm * Jo),
                 8.0 * nnz + 12.0 * F + (Yh ? 4.0 : 0.0) * X->dims[o->n] * (double)Jm * Jo +
                     (Y32 ? 4.0 : 0.0) * X->dims[o->n] * (double)Jm * Jo +
                     4.0 * (X->dims[o->m] * (double)Jm + X->dims[o->o] * (double)Jo));
  const int cp = tcode(Jm), cq = tcode(Jo);
  // Variant 0: the leaf phase with lane groups and float4 rows of U_o (64-column tiles, rows
  // padded to 16 bytes); variant 1: one warp per fiber.  The autotuner picks per shape class.
  const bool vec_ok = cq == 4 && rows16(Uo, ldo);
  auto run = [&](int variant) -> int {
    const bool vec = vec_ok && variant == 0;
#define TK_TM(A, B)                                                                  \
  if (cp == A && cq == B)                                                            \
    launch_ttmc_mixed<A, B>(X, o, Um, ldm, Jm, Uo, ldo, Jo, Yh, Yl, ldY, Y32, vec, s);
    TK_TM(1, 1) TK_TM(1, 2) TK_TM(1, 4) TK_TM(2, 1) TK_TM(2, 2) TK_TM(2, 4) TK_TM(4, 1)
    TK_TM(4, 2) TK_TM(4, 4)
#undef TK_TM
    TK_LAUNCH();
    return TUCKER_OK;
  };
  if (!vec_ok) return run(1);
  return autotune_run(TUNE_TTMC_MIXED, Jm, Jo, fiber_class(X->nnz, o->F), run, s);
}

int slice_proj_mixed(const tucker_tensor_s* X, const Ordering* o, const float* Um, int64_t ldm,
                     int Jm, __nv_bfloat16* Yh, __nv_bfloat16* Yl, int64_t ldY, cudaStream_t s) {
  // ordering (n, o, m): fibers (i_n, i_o), leaves i_m.
  const int64_t In = X->dims[o->n], Io = X->dims[o->m];
  if (In == 0) return TUCKER_OK;
  ProfScope prof("slice_proj_mixed", s, 2.0 * (double)X->nnz * Jm,
                 8.0 * X->nnz + 16.0 * o->F + 4.0 * (double)In * Io * Jm +
                     4.0 * X->dims[o->o] * (double)Jm);
  // Variant 0: a lane group per fiber with float4 rows of U_m (J_m <= 128, rows padded to 16
  // bytes); variant 1: one warp per fiber.  The autotuner picks per shape class.
  const bool vec_ok = rows16(Um, ldm) && Jm <= 128;
  auto run = [&](int variant) -> int {
    if (vec_ok && variant == 0) {
      if (Jm <= 64)
        slice_proj_mixed_vec_kernel<8><<<(unsigned)In, 256, 0, s>>>(
            o->root_ptr, o->fiber_idx, o->fiber_ptr, o->leaf_idx, o->val_f32, Um, ldm, Jm, Yh,
            Yl, ldY);
      else
        slice_proj_mixed_vec_kernel<16><<<(unsigned)In, 256, 0, s>>>(
            o->root_ptr, o->fiber_idx, o->fiber_ptr, o->leaf_idx, o->val_f32, Um, ldm, Jm, Yh,
            Yl, ldY);
      TK_LAUNCH();
      return TUCKER_OK;
    }
    const int np = Jm <= 32 ? 1 : (Jm <= 64 ? 2 : (Jm <= 128 ? 4 : 8));
#define TK_SPM(N)                                                                           \
  if (np == N)                                                                              \
    slice_proj_mixed_kernel<N><<<(unsigned)In, 256, 0, s>>>(o->root_ptr, o->fiber_idx,      \
                                                            o->fiber_ptr, o->leaf_idx,      \
                                                            o->val_f32, Um, ldm, Jm, Yh, Yl, \
                                                            ldY);
    TK_SPM(1) TK_SPM(2) TK_SPM(4) TK_SPM(8)
#undef TK_SPM
    TK_LAUNCH();
    return TUCKER_OK;
  };
  if (!vec_ok) return run(1);
  return autotune_run(TUNE_SLICE_MIXED, Jm, 0, fiber_class(X->nnz, o->F), run, s);
}

int f64_to_f32_rows(const double* a, int64_t rows, int cols, float* b, int64_t ldb,
                    cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return TUCKER_OK;
  f64_to_f32_rows_kernel<<<ceil_div(rows * ldb, 256), 256, 0, s>>>(a, rows, cols, b, ldb);
  TK_LAUNCH();
  return TUCKER_OK;
}

}  // namespace tk
