// CSF/COO build-and-sort: the GPU counterpart of the paper's sort + slice step (Section 3,
// "Slice Projection": the input file is sorted on one mode so that each slice's nonzeros are
// consecutive; appendix functions sort_index and slice).  Instead of files, each ordering
// (n, m, o) is a compressed sorted form: root pointers per i_n, fibers (runs of equal
// (i_n, i_m)), leaf indices i_o and values.  Sorting is a stable LSD radix sort of 64-bit
// linearised keys, so the result is bit-exact against any stable sort of the same keys.
#include "internal.h"

namespace tk {

namespace {

constexpr int THREADS = 256;
constexpr int ITEMS = 8;
constexpr int TILE = THREADS * ITEMS;

// ---- block-wide exclusive scan of THREADS values (one per thread) ---------------------------
template <class T>
__device__ T block_exclusive_scan(T v, T* total) {
  __shared__ T warp_tot[THREADS / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    T t = lane < THREADS / 32 ? warp_tot[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < THREADS / 32) warp_tot[lane] = t;  // inclusive warp prefix
  }
  __syncthreads();
  T before = (w > 0 ? warp_tot[w - 1] : T(0)) + x - v;
  if (total) *total = warp_tot[THREADS / 32 - 1];
  __syncthreads();
  return before;
}

template <class T>
__global__ void scan_tile_sums(const T* __restrict__ in, int64_t n, T* __restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * TILE + (int64_t)threadIdx.x * ITEMS;
  T s = 0;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i)
    if (base + i < n) s += in[base + i];
  T tot;
  block_exclusive_scan<T>(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Single block: exclusive scan of `n` tile sums in place; writes the grand total to *total.
template <class T>
__global__ void scan_sums_inplace(T* sums, int64_t n, T* total) {
  __shared__ T carry_s;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int64_t c = 0; c < n; c += TILE) {
    const int64_t base = c + (int64_t)threadIdx.x * ITEMS;
    T loc[ITEMS];
    T s = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      loc[i] = base + i < n ? sums[base + i] : T(0);
      s += loc[i];
    }
    T tot;
    T pre = block_exclusive_scan<T>(s, &tot) + carry_s;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      if (base + i < n) sums[base + i] = pre;
      pre += loc[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) carry_s += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry_s;
}

template <class T>
__global__ void scan_apply(const T* in, int64_t n, const T* __restrict__ offs, T* out) {
  const int64_t base = (int64_t)blockIdx.x * TILE + (int64_t)threadIdx.x * ITEMS;
  T loc[ITEMS];
  T s = 0;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    loc[i] = base + i < n ? in[base + i] : T(0);
    s += loc[i];
  }
  T pre = block_exclusive_scan<T>(s, nullptr) + offs[blockIdx.x];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    if (base + i < n) out[base + i] = pre;
    pre += loc[i];
  }
}

// Exclusive scan of n values; *d_total (device, may be null) receives the sum.  in may equal out.
template <class T>
int exclusive_scan(const T* in, T* out, int64_t n, T* d_total, cudaStream_t s) {
  if (n <= 0) {
    if (d_total) TK_CUDA(cudaMemsetAsync(d_total, 0, sizeof(T), s));
    return TUCKER_OK;
  }
  const int64_t nb = (n + TILE - 1) / TILE;
  Buf sums;
  TK_TRY(sums.alloc(sizeof(T) * nb, s));
  scan_tile_sums<T><<<(unsigned)nb, THREADS, 0, s>>>(in, n, sums.as<T>());
  TK_LAUNCH();
  scan_sums_inplace<T><<<1, THREADS, 0, s>>>(sums.as<T>(), nb, d_total);
  TK_LAUNCH();
  scan_apply<T><<<(unsigned)nb, THREADS, 0, s>>>(in, n, sums.as<T>(), out);
  TK_LAUNCH();
  return TUCKER_OK;
}

// ---- stable LSD radix sort of (64-bit key, 32-bit value) pairs ------------------------------
// Digits of RB bits: 8 per pass, except that a key whose width leaves 9 bits for the last pass
// takes them in one 9-bit pass (33-bit keys of 2000^3 tensors: 4 passes instead of 5).
template <int RB>
__global__ void rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                        unsigned* __restrict__ counts, int nblocks) {
  constexpr int B = 1 << RB;
  __shared__ unsigned h[B];
  for (int d = threadIdx.x; d < B; d += THREADS) h[d] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * TILE;
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const int64_t i = base + r * THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & (B - 1u)], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < B; d += THREADS) counts[(int64_t)d * nblocks + blockIdx.x] = h[d];
}

// Scatter one tile.  An element's destination is the global offset of its digit for this tile
// plus its rank among equal digits earlier in the tile, so equal digits keep their order.  The
// tile is first placed in shared memory grouped by digit (tile-local offsets from its own
// histogram), then written out in that order: each digit's elements leave as one contiguous run
// instead of one scattered store per element.
template <int RB>
__global__ void __launch_bounds__(THREADS)
rs_scatter(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin, int64_t n,
           int shift, const unsigned* __restrict__ offsets, int nblocks,
           uint64_t* __restrict__ kout, uint32_t* __restrict__ vout) {
  constexpr int B = 1 << RB;
  constexpr int DPT = B / THREADS;  // digits per thread in the tile-local scan
  static_assert(B % THREADS == 0, "digit count must be a multiple of the block size");
  __shared__ unsigned run[B];   // the tile's histogram, then elements of each digit placed so far
  __shared__ unsigned loc[B];   // tile-local start of each digit's run
  __shared__ unsigned wcnt[THREADS / 32][B];
  __shared__ uint64_t sk[TILE];
  __shared__ uint32_t sv[TILE];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * TILE;
  for (int d = threadIdx.x; d < B; d += THREADS) run[d] = 0;
  __syncthreads();
  uint64_t kr[ITEMS];
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const int64_t i = base + r * THREADS + threadIdx.x;
    kr[r] = i < n ? kin[i] : 0ull;
    if (i < n) atomicAdd(&run[(unsigned)(kr[r] >> shift) & (B - 1u)], 1u);
  }
  __syncthreads();
  {
    unsigned c[DPT], t = 0;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      c[q] = run[threadIdx.x * DPT + q];
      t += c[q];
    }
    unsigned ex = block_exclusive_scan<unsigned>(t, nullptr);
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      loc[threadIdx.x * DPT + q] = ex;
      ex += c[q];
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < B; d += THREADS) run[d] = 0;
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
#pragma unroll
    for (int j = 0; j < THREADS / 32; ++j)
      for (int d = threadIdx.x; d < B; d += THREADS) wcnt[j][d] = 0;
    __syncthreads();
    const int64_t i = base + r * THREADS + threadIdx.x;
    const bool valid = i < n;
    const uint64_t k = kr[r];
    const unsigned d = valid ? ((unsigned)(k >> shift) & (B - 1u)) : (unsigned)B;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int leader = __ffs(peers) - 1;
    const unsigned rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && lane == leader) wcnt[w][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      unsigned pos = run[d] + rank;
      for (int j = 0; j < w; ++j) pos += wcnt[j][d];
      sk[loc[d] + pos] = k;
      sv[loc[d] + pos] = vin[i];
    }
    __syncthreads();
    for (int dd = threadIdx.x; dd < B; dd += THREADS) {
      unsigned tot = 0;
#pragma unroll
      for (int j = 0; j < THREADS / 32; ++j) tot += wcnt[j][dd];
      run[dd] += tot;
    }
    __syncthreads();
  }
  const int cnt = (int)(n - base < (int64_t)TILE ? n - base : (int64_t)TILE);
  for (int j = threadIdx.x; j < cnt; j += THREADS) {
    const uint64_t k = sk[j];
    const unsigned d = (unsigned)(k >> shift) & (B - 1u);
    const unsigned dest = offsets[(int64_t)d * nblocks + blockIdx.x] + (unsigned)j - loc[d];
    kout[dest] = k;
    vout[dest] = sv[j];
  }
}

template <int RB>
int radix_pass(const uint64_t* ki, const uint32_t* vi, uint64_t* ko, uint32_t* vo, int64_t n,
               int shift, unsigned* counts, int nb, cudaStream_t s) {
  rs_hist<RB><<<nb, THREADS, 0, s>>>(ki, n, shift, counts, nb);
  TK_LAUNCH();
  TK_TRY(exclusive_scan<unsigned>(counts, counts, (int64_t)(1 << RB) * nb, nullptr, s));
  rs_scatter<RB><<<nb, THREADS, 0, s>>>(ki, vi, n, shift, counts, nb, ko, vo);
  TK_LAUNCH();
  return TUCKER_OK;
}

// Sorts (keys, vals) by the low `bits` bits of the keys.  On return *out_keys/*out_vals point
// at whichever of the two buffer pairs holds the result.
int radix_sort_pairs(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int64_t n, int bits,
                     uint64_t** out_keys, uint32_t** out_vals, cudaStream_t s) {
  *out_keys = k0;
  *out_vals = v0;
  if (n <= 1) return TUCKER_OK;
  const int nb = ceil_div(n, TILE);
  Buf counts;
  TK_TRY(counts.alloc(sizeof(unsigned) * 512 * (size_t)nb, s));
  uint64_t *ki = k0, *ko = k1;
  uint32_t *vi = v0, *vo = v1;
  for (int shift = 0; shift < bits;) {
    const int rb = bits - shift == 9 ? 9 : 8;
    if (rb == 9)
      TK_TRY(radix_pass<9>(ki, vi, ko, vo, n, shift, counts.as<unsigned>(), nb, s));
    else
      TK_TRY(radix_pass<8>(ki, vi, ko, vo, n, shift, counts.as<unsigned>(), nb, s));
    shift += rb;
    uint64_t* tk_ = ki; ki = ko; ko = tk_;
    uint32_t* tv_ = vi; vi = vo; vo = tv_;
  }
  *out_keys = ki;
  *out_vals = vi;
  return TUCKER_OK;
}

int key_bits(uint64_t maxkey) {
  int b = 0;
  while (b < 64 && (maxkey >> b) != 0) ++b;
  return b;
}

// ---- canonical COO -------------------------------------------------------------------------
__global__ void make_keys_checked(const int32_t* __restrict__ i0, const int32_t* __restrict__ i1,
                                  const int32_t* __restrict__ i2, int64_t n, int64_t d0,
                                  int64_t d1, int64_t d2, uint64_t* __restrict__ keys,
                                  uint32_t* __restrict__ vals, int* status) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int64_t a = i0[t], b = i1[t], c = i2[t];
  if (a < 0 || a >= d0 || b < 0 || b >= d1 || c < 0 || c >= d2) {
    atomicOr(status, DEV_BAD_INDEX);
    a = 0; b = 0; c = 0;
  }
  keys[t] = ((uint64_t)a * (uint64_t)d1 + (uint64_t)b) * (uint64_t)d2 + (uint64_t)c;
  vals[t] = (uint32_t)t;
}

__global__ void key_heads(const uint64_t* __restrict__ keys, int64_t n, uint64_t div,
                          unsigned* __restrict__ head) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  head[t] = (t == 0 || keys[t] / div != keys[t - 1] / div) ? 1u : 0u;
}

// Sums each run of equal keys in sorted (= input) order, exactly as a sequential loop would.
__global__ void dedup_runs(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ perm,
                           const unsigned* __restrict__ uid, const double* __restrict__ vin,
                           int64_t n, int64_t d1, int64_t d2, int32_t* __restrict__ o0,
                           int32_t* __restrict__ o1, int32_t* __restrict__ o2,
                           double* __restrict__ vout) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const uint64_t k = keys[t];
  if (t > 0 && keys[t - 1] == k) return;
  double sum = 0.0;
  for (int64_t j = t; j < n && keys[j] == k; ++j) sum += vin[perm[j]];
  const unsigned u = uid[t];
  o2[u] = (int32_t)(k % (uint64_t)d2);
  o1[u] = (int32_t)((k / (uint64_t)d2) % (uint64_t)d1);
  o0[u] = (int32_t)(k / ((uint64_t)d2 * (uint64_t)d1));
  vout[u] = sum;
}

// ---- orderings -----------------------------------------------------------------------------
__global__ void make_keys(const int32_t* __restrict__ a, const int32_t* __restrict__ b,
                          const int32_t* __restrict__ c, int64_t n, int64_t db, int64_t dc,
                          uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  keys[t] = ((uint64_t)a[t] * (uint64_t)db + (uint64_t)b[t]) * (uint64_t)dc + (uint64_t)c[t];
  vals[t] = (uint32_t)t;
}

__global__ void gather_leaves(const uint32_t* __restrict__ perm, const int32_t* __restrict__ io,
                              const double* __restrict__ v, int64_t n,
                              int32_t* __restrict__ leaf, double* __restrict__ vout) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const uint32_t p = perm[t];
  leaf[t] = io[p];
  vout[t] = v[p];
}

__global__ void fill_fibers(const unsigned* __restrict__ head, const unsigned* __restrict__ fid,
                            const uint32_t* __restrict__ perm, const int32_t* __restrict__ in_,
                            const int32_t* __restrict__ im, int64_t n,
                            int64_t* __restrict__ fiber_ptr, int32_t* __restrict__ fiber_idx,
                            int32_t* __restrict__ fiber_root) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n || !head[t]) return;
  const unsigned f = fid[t];
  const uint32_t p = perm[t];
  fiber_ptr[f] = t;
  fiber_idx[f] = im[p];
  fiber_root[f] = in_[p];
}

__global__ void fill_root_ptr(const int32_t* __restrict__ fiber_root, int64_t F, int64_t In,
                              int64_t nnz, int64_t* __restrict__ root_ptr,
                              int64_t* __restrict__ fiber_ptr) {
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f > F) return;
  const int64_t cur = f < F ? fiber_root[f] : In;
  const int64_t prev = f > 0 ? fiber_root[f - 1] : -1;
  const int64_t last = (f == F) ? In : cur;
  for (int64_t i = prev + 1; i <= last; ++i) root_ptr[i] = f;
  if (f == F) fiber_ptr[F] = nnz;
}

__global__ void scatter_fiber_map(const int32_t* __restrict__ fiber_root,
                                  const int32_t* __restrict__ fiber_idx, int64_t F, int64_t Im,
                                  int32_t* __restrict__ map) {
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  map[(int64_t)fiber_root[f] * Im + fiber_idx[f]] = (int32_t)f;
}

// ---- deterministic FP64 sum of squares -----------------------------------------------------
__global__ void sumsq_partial(const double* __restrict__ v, int64_t n, double* __restrict__ part) {
  __shared__ double ws[THREADS / 32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * THREADS + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * THREADS)
    s = fma(v[i], v[i], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int j = 0; j < THREADS / 32; ++j) t += ws[j];
    part[blockIdx.x] = t;
  }
}

__global__ void sum_partials(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int j = 0; j < n; ++j) t += part[j];
    *out = t;
  }
}

}  // namespace

int exclusive_scan_u32(const unsigned* in, unsigned* out, int64_t n, unsigned* d_total,
                       cudaStream_t s) {
  return exclusive_scan<unsigned>(in, out, n, d_total, s);
}

int sum_squares(const double* d_v, int64_t n, double* d_out, cudaStream_t s) {
  const int nb = 1024;
  Buf part;
  TK_TRY(part.alloc(sizeof(double) * nb, s));
  sumsq_partial<<<nb, THREADS, 0, s>>>(d_v, n, part.as<double>());
  TK_LAUNCH();
  sum_partials<<<1, 32, 0, s>>>(part.as<double>(), nb, d_out);
  TK_LAUNCH();
  return TUCKER_OK;
}

int build_canonical(tucker_tensor_s* X, const int32_t* d_i0, const int32_t* d_i1,
                    const int32_t* d_i2, const double* d_v, int64_t n, cudaStream_t s) {
  const int64_t d0 = X->dims[0], d1 = X->dims[1], d2 = X->dims[2];
  ProfScope prof("csf_build", s, 0.0, 20.0 * n + 20.0 * n);
  Buf k0, k1, v0, v1, head, uid, stat, tot;
  TK_TRY(k0.alloc(8 * (size_t)n, s));
  TK_TRY(k1.alloc(8 * (size_t)n, s));
  TK_TRY(v0.alloc(4 * (size_t)n, s));
  TK_TRY(v1.alloc(4 * (size_t)n, s));
  TK_TRY(head.alloc(4 * (size_t)n, s));
  TK_TRY(uid.alloc(4 * (size_t)n, s));
  TK_TRY(stat.alloc(sizeof(int), s));
  TK_TRY(tot.alloc(sizeof(unsigned), s));
  TK_CUDA(cudaMemsetAsync(stat.p, 0, sizeof(int), s));
  const int nbk = ceil_div(n, 256);
  if (n > 0) {
    make_keys_checked<<<nbk, 256, 0, s>>>(d_i0, d_i1, d_i2, n, d0, d1, d2, k0.as<uint64_t>(),
                                          v0.as<uint32_t>(), stat.as<int>());
    TK_LAUNCH();
  }
  int hstat = 0;
  TK_CUDA(cudaMemcpyAsync(&hstat, stat.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  if (hstat & DEV_BAD_INDEX) return TUCKER_EINVAL;
  uint64_t *keys;
  uint32_t *perm;
  TK_TRY(radix_sort_pairs(k0.as<uint64_t>(), v0.as<uint32_t>(), k1.as<uint64_t>(),
                          v1.as<uint32_t>(), n, key_bits((uint64_t)d0 * d1 * d2 - 1), &keys,
                          &perm, s));
  unsigned nu = 0;
  if (n > 0) {
    key_heads<<<nbk, 256, 0, s>>>(keys, n, 1ull, head.as<unsigned>());
    TK_LAUNCH();
    TK_TRY(exclusive_scan<unsigned>(head.as<unsigned>(), uid.as<unsigned>(), n,
                                    tot.as<unsigned>(), s));
    TK_CUDA(cudaMemcpyAsync(&nu, tot.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    TK_CUDA(cudaStreamSynchronize(s));
  }
  X->nnz = nu;
  for (int a = 0; a < 3; ++a) TK_CUDA(cudaMalloc(&X->idx[a], sizeof(int32_t) * (nu ? nu : 1)));
  TK_CUDA(cudaMalloc(&X->val, sizeof(double) * (nu ? nu : 1)));
  if (n > 0) {
    dedup_runs<<<nbk, 256, 0, s>>>(keys, perm, uid.as<unsigned>(), d_v, n, d1, d2, X->idx[0],
                                   X->idx[1], X->idx[2], X->val);
    TK_LAUNCH();
  }
  Buf n2;
  TK_TRY(n2.alloc(sizeof(double), s));
  TK_TRY(sum_squares(X->val, X->nnz, n2.as<double>(), s));
  TK_CUDA(cudaMemcpyAsync(&X->norm2, n2.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  TK_CUDA(cudaStreamSynchronize(s));
  return TUCKER_OK;
}

int build_ordering(tucker_tensor_s* X, Ordering* ord, cudaStream_t s) {
  const int n = ord->n, m = ord->m, o = ord->o;
  const int64_t nnz = X->nnz;
  const int64_t dn = X->dims[n], dm = X->dims[m], dd = X->dims[o];
  ProfScope prof("csf_build", s, 0.0, 20.0 * nnz + 12.0 * nnz);
  // The canonical COO is sorted by (i_0, i_1, i_2) with distinct keys (build_canonical), so
  // ordering (0, 1, 2) is already in key order: its stable sort is the identity permutation
  // that make_keys writes, and no radix pass runs.
  const bool presorted = n == 0 && m == 1 && o == 2;
  Buf k0, k1, v0, v1, head, fid, tot;
  const size_t nn = (size_t)(nnz ? nnz : 1);
  TK_TRY(k0.alloc(8 * nn, s));
  TK_TRY(v0.alloc(4 * nn, s));
  if (!presorted) {
    TK_TRY(k1.alloc(8 * nn, s));
    TK_TRY(v1.alloc(4 * nn, s));
  }
  TK_TRY(head.alloc(4 * nn, s));
  TK_TRY(fid.alloc(4 * nn, s));
  TK_TRY(tot.alloc(sizeof(unsigned), s));
  const int nbk = ceil_div(nnz, 256);
  if (nnz > 0) {
    make_keys<<<nbk, 256, 0, s>>>(X->idx[n], X->idx[m], X->idx[o], nnz, dm, dd,
                                  k0.as<uint64_t>(), v0.as<uint32_t>());
    TK_LAUNCH();
  }
  uint64_t* keys = k0.as<uint64_t>();
  uint32_t* perm = v0.as<uint32_t>();
  if (!presorted)
    TK_TRY(radix_sort_pairs(k0.as<uint64_t>(), v0.as<uint32_t>(), k1.as<uint64_t>(),
                            v1.as<uint32_t>(), nnz, key_bits((uint64_t)dn * dm * dd - 1), &keys,
                            &perm, s));
  TK_CUDA(cudaMalloc(&ord->leaf_idx, sizeof(int32_t) * nn));
  TK_CUDA(cudaMalloc(&ord->val, sizeof(double) * nn));
  unsigned F = 0;
  if (nnz > 0) {
    gather_leaves<<<nbk, 256, 0, s>>>(perm, X->idx[o], X->val, nnz, ord->leaf_idx, ord->val);
    TK_LAUNCH();
    key_heads<<<nbk, 256, 0, s>>>(keys, nnz, (uint64_t)dd, head.as<unsigned>());
    TK_LAUNCH();
    TK_TRY(exclusive_scan<unsigned>(head.as<unsigned>(), fid.as<unsigned>(), nnz,
                                    tot.as<unsigned>(), s));
    TK_CUDA(cudaMemcpyAsync(&F, tot.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    TK_CUDA(cudaStreamSynchronize(s));
  }
  ord->F = F;
  TK_CUDA(cudaMalloc(&ord->fiber_ptr, sizeof(int64_t) * (F + 1)));
  TK_CUDA(cudaMalloc(&ord->fiber_idx, sizeof(int32_t) * (F ? F : 1)));
  TK_CUDA(cudaMalloc(&ord->fiber_root, sizeof(int32_t) * (F ? F : 1)));
  TK_CUDA(cudaMalloc(&ord->root_ptr, sizeof(int64_t) * (dn + 1)));
  if (nnz > 0) {
    fill_fibers<<<nbk, 256, 0, s>>>(head.as<unsigned>(), fid.as<unsigned>(), perm, X->idx[n],
                                    X->idx[m], nnz, ord->fiber_ptr, ord->fiber_idx,
                                    ord->fiber_root);
    TK_LAUNCH();
  }
  fill_root_ptr<<<ceil_div((int64_t)F + 1, 256), 256, 0, s>>>(ord->fiber_root, F, dn, nnz,
                                                               ord->root_ptr, ord->fiber_ptr);
  TK_LAUNCH();
  TK_CUDA(cudaStreamSynchronize(s));
  ord->built = true;
  return TUCKER_OK;
}

int build_fiber_map(tucker_tensor_s* X, Ordering* ord, cudaStream_t s) {
  const int64_t dn = X->dims[ord->n], dm = X->dims[ord->m];
  TK_CUDA(cudaMalloc(&ord->fiber_map, sizeof(int32_t) * (size_t)(dn * dm)));
  TK_CUDA(cudaMemsetAsync(ord->fiber_map, 0xFF, sizeof(int32_t) * (size_t)(dn * dm), s));
  if (ord->F > 0) {
    scatter_fiber_map<<<ceil_div(ord->F, 256), 256, 0, s>>>(ord->fiber_root, ord->fiber_idx,
                                                            ord->F, dm, ord->fiber_map);
    TK_LAUNCH();
  }
  return TUCKER_OK;
}

}  // namespace tk
