// Out-of-core form of Slice Projection and Multislice Projection (Figures sp3 and mp3) for
// tensors whose orderings do not fit in device memory.  The paper's motivation for SP and MP is
// exactly this: every matrix they build is a sum over slices, sum_k X_k U U^T X_k^T, so the
// tensor can be read one slice after another (it sorted the input file by slice and streamed
// the slices from disk, Section 3 "Slice Projection").  Here the slices live in pinned host
// memory and travel to the GPU over NVLink-C2C in chunks:
//
//   * build: the COO tensor is partitioned by slice on the host (counting sort, stable), and
//     each chunk of slices is sorted on the GPU (csf.cu: duplicates summed, the two orderings
//     of the chunk built) and copied back into the host orderings; only one chunk is on the
//     device at a time.  Slice-major orderings (o, n, m) exist for the three slice modes o;
//   * methods: for output mode n and projecting mode m, the chunks of ordering (o, n, m)
//     (o the third mode) are copied to the device on a copy stream (two buffers, copies of
//     chunk c+1 overlap the work on chunk c); each chunk's projection Y_c = (X_c x_m U_m^T)_(n)
//     (I_n x chunk slices * J_m) runs on the FP64 kernel of sparse.cu, and its Gram is added to
//     M on the tensor cores (gram_ozaki.cu: error-free slicing, exact integer sums) with the
//     product's epilogue M <- M + Y_c Y_c^T;
//   * MP's pseudo HO-SVD start sums the slices' own Grams X_k X_k^T (densified chunk by chunk),
//     doubled; the core is G = sum_k C[k,:]^T (x) (A^T X_k B) from the slices of mode 3.
// FP64 form only.  Device memory in use is bounded by the budget given at creation.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace tk {

// One slice-major ordering (o, n, m) in pinned host memory: roots are the slices of mode o,
// fibers (i_o, i_n), leaves i_m.
struct HostOrdering {
  int o = 0, n = 0, m = 0;
  int64_t F = 0;
  int64_t* root_ptr = nullptr;   // [I_o + 1]
  int32_t* fiber_idx = nullptr;  // [F] i_n
  int32_t* fiber_root = nullptr; // [F] i_o
  int64_t* fiber_ptr = nullptr;  // [F + 1]
  int32_t* leaf_idx = nullptr;   // [nnz] i_m
  double* val = nullptr;         // [nnz]
};

}  // namespace tk

struct tucker_stream_s {
  int64_t dims[3] = {0, 0, 0};
  int64_t nnz = 0;
  double norm2 = 0.0;
  int64_t budget = 0;
  std::vector<int64_t> chunks[3];   // slice boundaries of each slice mode (k0 = chunks[o][c])
  int64_t max_chunk_nnz = 0, max_chunk_fibers = 0, max_chunk_slices = 0;
  tk::HostOrdering ord[6];          // slot ordering_slot(o, n, m)
};

namespace tk {

namespace {

void free_host_ordering(HostOrdering& h) {
  cudaFreeHost(h.root_ptr);
  cudaFreeHost(h.fiber_idx);
  cudaFreeHost(h.fiber_root);
  cudaFreeHost(h.fiber_ptr);
  cudaFreeHost(h.leaf_idx);
  cudaFreeHost(h.val);
  h = HostOrdering();
}

void free_chunk_tensor(tucker_tensor_s* T) {
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

// Device bytes a chunk of `nnz` nonzeros needs while it is sorted (keys, permutations, the
// canonical COO and two orderings), with margin.
int64_t build_bytes_per_nnz() { return 112; }

}  // namespace

}  // namespace tk

using namespace tk;

extern "C" int tucker_stream_destroy(tucker_stream_tensor X);

extern "C" int tucker_stream_create(const tucker_coo* X, int64_t budget, void* stream,
                                    tucker_stream_tensor* out) {
  if (!X || !out) return TUCKER_EINVAL;
  *out = nullptr;
  for (int a = 0; a < 3; ++a)
    if (X->dims[a] < 1 || X->dims[a] > 2147483647ll) return TUCKER_EINVAL;
  if ((double)X->dims[0] * (double)X->dims[1] * (double)X->dims[2] >= 4.6e18) return TUCKER_EINVAL;
  if (X->nnz < 0 || X->nnz > 2147483647ll) return TUCKER_EINVAL;
  if (X->where != TUCKER_HOST && X->where != TUCKER_DEVICE) return TUCKER_EINVAL;
  if (X->nnz > 0 && (!X->idx[0] || !X->idx[1] || !X->idx[2] || !X->val)) return TUCKER_EINVAL;
  if (budget < (int64_t)1 << 16) return TUCKER_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  tucker_stream_s* T = new (std::nothrow) tucker_stream_s();
  if (!T) return TUCKER_ENOMEM;
  for (int a = 0; a < 3; ++a) T->dims[a] = X->dims[a];
  T->budget = budget;
  const int64_t n = X->nnz;
  // The COO on the host (copied back when it came from the device).
  std::vector<int32_t> hidx[3];
  std::vector<double> hval;
  const int32_t* ci[3] = {X->idx[0], X->idx[1], X->idx[2]};
  const double* cv = X->val;
  if (X->where == TUCKER_DEVICE && n > 0) {
    for (int a = 0; a < 3; ++a) {
      hidx[a].resize(n);
      TK_CUDA(cudaMemcpy(hidx[a].data(), X->idx[a], sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
      ci[a] = hidx[a].data();
    }
    hval.resize(n);
    TK_CUDA(cudaMemcpy(hval.data(), X->val, sizeof(double) * n, cudaMemcpyDeviceToHost));
    cv = hval.data();
  }
  for (int64_t t = 0; t < n; ++t)
    for (int a = 0; a < 3; ++a)
      if (ci[a][t] < 0 || ci[a][t] >= X->dims[a]) {
        tucker_stream_destroy(T);
        return TUCKER_EINVAL;
      }
  const int64_t cap = std::max<int64_t>(1, budget / build_bytes_per_nnz());
  int st = TUCKER_OK;
  for (int o = 0; o < 3 && st == TUCKER_OK; ++o) {
    const int a = o == 0 ? 1 : 0, b = o == 2 ? 1 : 2;   // the other modes, a < b
    const int64_t Io = X->dims[o];
    // Stable counting sort of the nonzeros by their slice index i_o.
    std::vector<int64_t> cnt(Io + 1, 0);
    for (int64_t t = 0; t < n; ++t) ++cnt[ci[o][t] + 1];
    for (int64_t k = 0; k < Io; ++k) cnt[k + 1] += cnt[k];
    std::vector<int64_t> perm(n);
    {
      std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
      for (int64_t t = 0; t < n; ++t) perm[pos[ci[o][t]]++] = t;
    }
    // Chunks of whole slices, each at most `cap` nonzeros (a larger single slice is a chunk).
    std::vector<int64_t>& ch = T->chunks[o];
    ch.assign(1, 0);
    while (ch.back() < Io) {
      int64_t k1 = ch.back() + 1;
      while (k1 < Io && cnt[k1 + 1] - cnt[ch.back()] <= cap) ++k1;
      ch.push_back(k1);
    }
    // Host orderings (o, a, b) and (o, b, a), capacity for every nonzero.
    HostOrdering* H[2] = {&T->ord[ordering_slot(o, a, b)], &T->ord[ordering_slot(o, b, a)]};
    const int sec[2][2] = {{a, b}, {b, a}};
    for (int h = 0; h < 2 && st == TUCKER_OK; ++h) {
      HostOrdering& ho = *H[h];
      ho.o = o;
      ho.n = sec[h][0];
      ho.m = sec[h][1];
      const size_t nn = (size_t)std::max<int64_t>(n, 1);
      if (cudaMallocHost(&ho.root_ptr, sizeof(int64_t) * (Io + 1)) != cudaSuccess ||
          cudaMallocHost(&ho.fiber_idx, sizeof(int32_t) * nn) != cudaSuccess ||
          cudaMallocHost(&ho.fiber_root, sizeof(int32_t) * nn) != cudaSuccess ||
          cudaMallocHost(&ho.fiber_ptr, sizeof(int64_t) * (nn + 1)) != cudaSuccess ||
          cudaMallocHost(&ho.leaf_idx, sizeof(int32_t) * nn) != cudaSuccess ||
          cudaMallocHost(&ho.val, sizeof(double) * nn) != cudaSuccess)
        st = TUCKER_ENOMEM;
      if (st == TUCKER_OK) ho.root_ptr[0] = 0;
    }
    int64_t Foff[2] = {0, 0}, Loff = 0;
    double norm2 = 0.0;
    std::vector<int32_t> ck[3];
    std::vector<double> cvv;
    for (size_t c = 0; c + 1 < ch.size() && st == TUCKER_OK; ++c) {
      const int64_t k0 = ch[c], k1 = ch[c + 1], t0 = cnt[k0], t1 = cnt[k1], cn = t1 - t0;
      T->max_chunk_slices = std::max(T->max_chunk_slices, k1 - k0);
      // The chunk as a small third-order tensor (i_o - k0, i_a, i_b).
      for (int q = 0; q < 3; ++q) ck[q].resize(cn);
      cvv.resize(cn);
      for (int64_t t = 0; t < cn; ++t) {
        const int64_t src = perm[t0 + t];
        ck[0][t] = (int32_t)(ci[o][src] - k0);
        ck[1][t] = ci[a][src];
        ck[2][t] = ci[b][src];
        cvv[t] = cv[src];
      }
      tucker_tensor_s* C = new (std::nothrow) tucker_tensor_s();
      if (!C) {
        st = TUCKER_ENOMEM;
        break;
      }
      C->dims[0] = k1 - k0;
      C->dims[1] = X->dims[a];
      C->dims[2] = X->dims[b];
      cudaGetDevice(&C->device);
      {
        Buf di[3], dv;
        for (int q = 0; q < 3 && st == TUCKER_OK; ++q) {
          st = di[q].alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(cn, 1), s);
          if (st == TUCKER_OK && cn > 0 &&
              cudaMemcpyAsync(di[q].p, ck[q].data(), sizeof(int32_t) * cn, cudaMemcpyHostToDevice,
                              s) != cudaSuccess)
            st = TUCKER_ECUDA;
        }
        if (st == TUCKER_OK) st = dv.alloc(sizeof(double) * (size_t)std::max<int64_t>(cn, 1), s);
        if (st == TUCKER_OK && cn > 0 &&
            cudaMemcpyAsync(dv.p, cvv.data(), sizeof(double) * cn, cudaMemcpyHostToDevice, s) !=
                cudaSuccess)
          st = TUCKER_ECUDA;
        if (st == TUCKER_OK)
          st = build_canonical(C, di[0].as<int32_t>(), di[1].as<int32_t>(), di[2].as<int32_t>(),
                               dv.as<double>(), cn, s);
      }
      for (int h = 0; h < 2 && st == TUCKER_OK; ++h) {
        Ordering* ord = nullptr;
        st = ensure_ordering(C, 0, h == 0 ? 1 : 2, h == 0 ? 2 : 1, s, &ord);
        if (st != TUCKER_OK) break;
        HostOrdering& ho = *H[h];
        const int64_t F = ord->F, L = C->nnz;
        std::vector<int64_t> rp(k1 - k0 + 1), fp(F + 1);
        if (cudaMemcpyAsync(rp.data(), ord->root_ptr, sizeof(int64_t) * (k1 - k0 + 1),
                            cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(fp.data(), ord->fiber_ptr, sizeof(int64_t) * (F + 1),
                            cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            (F > 0 && (cudaMemcpyAsync(ho.fiber_idx + Foff[h], ord->fiber_idx,
                                       sizeof(int32_t) * F, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                       cudaMemcpyAsync(ho.fiber_root + Foff[h], ord->fiber_root,
                                       sizeof(int32_t) * F, cudaMemcpyDeviceToHost, s) != cudaSuccess)) ||
            (L > 0 && (cudaMemcpyAsync(ho.leaf_idx + Loff, ord->leaf_idx, sizeof(int32_t) * L,
                                       cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                       cudaMemcpyAsync(ho.val + Loff, ord->val, sizeof(double) * L,
                                       cudaMemcpyDeviceToHost, s) != cudaSuccess)) ||
            cudaStreamSynchronize(s) != cudaSuccess) {
          st = TUCKER_ECUDA;
          break;
        }
        for (int64_t k = 1; k <= k1 - k0; ++k) ho.root_ptr[k0 + k] = rp[k] + Foff[h];
        for (int64_t f = 0; f < F; ++f) {
          ho.fiber_root[Foff[h] + f] += (int32_t)k0;
          ho.fiber_ptr[Foff[h] + f] = fp[f] + Loff;
        }
        ho.fiber_ptr[Foff[h] + F] = fp[F] + Loff;
        T->max_chunk_fibers = std::max(T->max_chunk_fibers, F);
        Foff[h] += F;
      }
      if (st == TUCKER_OK) {
        T->max_chunk_nnz = std::max(T->max_chunk_nnz, C->nnz);
        Loff += C->nnz;
        norm2 += C->norm2;
      }
      free_chunk_tensor(C);
    }
    if (st == TUCKER_OK) {
      H[0]->F = Foff[0];
      H[1]->F = Foff[1];
      if (o == 0) {
        T->nnz = Loff;
        T->norm2 = norm2;
      }
    }
  }
  if (st != TUCKER_OK) {
    tucker_stream_destroy(T);
    return st;
  }
  *out = T;
  return TUCKER_OK;
}

extern "C" int tucker_stream_destroy(tucker_stream_tensor T) {
  if (!T) return TUCKER_OK;
  cudaDeviceSynchronize();
  for (auto& h : T->ord) free_host_ordering(h);
  delete T;
  return TUCKER_OK;
}

extern "C" int tucker_stream_info(tucker_stream_tensor X, int64_t* nnz, double* norm2,
                                  int64_t* chunks) {
  if (!X) return TUCKER_EINVAL;
  if (nnz) *nnz = X->nnz;
  if (norm2) *norm2 = X->norm2;
  if (chunks) *chunks = (int64_t)X->chunks[0].size() - 1;
  return TUCKER_OK;
}

namespace tk {
namespace {

// Rebases a chunk's pointers to its own arrays: fiber_ptr -= L0, fiber_root -= k0, root_ptr -= F0.
__global__ void rebase_chunk(int64_t* __restrict__ fiber_ptr, int32_t* __restrict__ fiber_root,
                             int64_t F, int64_t L0, int32_t k0, int64_t* __restrict__ root_ptr,
                             int64_t nk, int64_t F0) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t <= F) fiber_ptr[t] -= L0;
  if (t < F) fiber_root[t] -= k0;
  if (t <= nk) root_ptr[t] -= F0;
}

// Y[i_n, (i_o - k0) I_m + i_m] = x for the chunk's nonzeros (one warp per fiber): the slices
// themselves, side by side, for the slice Gram sums of MP's start.
__global__ void densify_fibers(int64_t F, const int32_t* __restrict__ row,
                               const int32_t* __restrict__ slice, const int64_t* __restrict__ fp,
                               const int32_t* __restrict__ leaf, const double* __restrict__ val,
                               int64_t Im, int64_t ldY, double* __restrict__ Y) {
  const int64_t f = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (f >= F) return;
  double* out = Y + (int64_t)row[f] * ldY + (int64_t)slice[f] * Im;
  for (int64_t l = fp[f] + lane; l < fp[f + 1]; l += 32) out[leaf[l]] = val[l];
}

__global__ void add_into(double* __restrict__ y, const double* __restrict__ x, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) y[t] += x[t];
}

// Device copy of one chunk of a host ordering (two of these alternate).
struct ChunkBuf {
  Buf root_ptr, fiber_idx, fiber_root, fiber_ptr, leaf_idx, val;
  cudaEvent_t copied = nullptr, used = nullptr;
  int64_t nk = 0, F = 0, L = 0;
};

class Streamer {
 public:
  Streamer(tucker_stream_s* X, cudaStream_t compute) : X_(X), cs_(compute) {}
  ~Streamer() {
    for (auto& b : buf_) {
      if (b.copied) cudaEventDestroy(b.copied);
      if (b.used) cudaEventDestroy(b.used);
    }
    if (copy_stream_) cudaStreamDestroy(copy_stream_);
  }
  int init() {
    TK_CUDA(cudaStreamCreateWithFlags(&copy_stream_, cudaStreamNonBlocking));
    const size_t nk = (size_t)X_->max_chunk_slices + 1, F = (size_t)X_->max_chunk_fibers + 1,
                 L = (size_t)std::max<int64_t>(X_->max_chunk_nnz, 1);
    for (auto& b : buf_) {
      TK_TRY(b.root_ptr.alloc(sizeof(int64_t) * nk, cs_));
      TK_TRY(b.fiber_idx.alloc(sizeof(int32_t) * F, cs_));
      TK_TRY(b.fiber_root.alloc(sizeof(int32_t) * F, cs_));
      TK_TRY(b.fiber_ptr.alloc(sizeof(int64_t) * (F + 1), cs_));
      TK_TRY(b.leaf_idx.alloc(sizeof(int32_t) * L, cs_));
      TK_TRY(b.val.alloc(sizeof(double) * L, cs_));
      TK_CUDA(cudaEventCreateWithFlags(&b.copied, cudaEventDisableTiming));
      TK_CUDA(cudaEventCreateWithFlags(&b.used, cudaEventDisableTiming));
      TK_CUDA(cudaEventRecord(b.used, cs_));
    }
    TK_CUDA(cudaStreamSynchronize(cs_));   // buffers allocated before the copy stream uses them
    return TUCKER_OK;
  }
  // Runs body(chunk buffer, k0, nk) on the compute stream for every chunk of ordering (o, n, m),
  // the copy of chunk c + 1 overlapping the work on chunk c.
  template <class Body>
  int for_chunks(int o, int n, int m, Body body) {
    const HostOrdering& h = X_->ord[ordering_slot(o, n, m)];
    const std::vector<int64_t>& ch = X_->chunks[o];
    const int nc = (int)ch.size() - 1;
    auto issue = [&](int c) -> int {
      ChunkBuf& b = buf_[c & 1];
      const int64_t k0 = ch[c], k1 = ch[c + 1];
      const int64_t F0 = h.root_ptr[k0], F1 = h.root_ptr[k1];
      const int64_t L0 = h.fiber_ptr[F0], L1 = h.fiber_ptr[F1];
      b.nk = k1 - k0;
      b.F = F1 - F0;
      b.L = L1 - L0;
      TK_CUDA(cudaStreamWaitEvent(copy_stream_, b.used, 0));
      TK_CUDA(cudaMemcpyAsync(b.root_ptr.p, h.root_ptr + k0, sizeof(int64_t) * (b.nk + 1),
                              cudaMemcpyHostToDevice, copy_stream_));
      TK_CUDA(cudaMemcpyAsync(b.fiber_ptr.p, h.fiber_ptr + F0, sizeof(int64_t) * (b.F + 1),
                              cudaMemcpyHostToDevice, copy_stream_));
      if (b.F > 0) {
        TK_CUDA(cudaMemcpyAsync(b.fiber_idx.p, h.fiber_idx + F0, sizeof(int32_t) * b.F,
                                cudaMemcpyHostToDevice, copy_stream_));
        TK_CUDA(cudaMemcpyAsync(b.fiber_root.p, h.fiber_root + F0, sizeof(int32_t) * b.F,
                                cudaMemcpyHostToDevice, copy_stream_));
      }
      if (b.L > 0) {
        TK_CUDA(cudaMemcpyAsync(b.leaf_idx.p, h.leaf_idx + L0, sizeof(int32_t) * b.L,
                                cudaMemcpyHostToDevice, copy_stream_));
        TK_CUDA(cudaMemcpyAsync(b.val.p, h.val + L0, sizeof(double) * b.L, cudaMemcpyHostToDevice,
                                copy_stream_));
      }
      rebase_chunk<<<ceil_div(std::max(b.F, b.nk) + 1, 256), 256, 0, copy_stream_>>>(
          b.fiber_ptr.as<int64_t>(), b.fiber_root.as<int32_t>(), b.F, L0, (int32_t)k0,
          b.root_ptr.as<int64_t>(), b.nk, F0);
      TK_LAUNCH();
      TK_CUDA(cudaEventRecord(b.copied, copy_stream_));
      bytecs_ += 8.0 * (b.nk + 1) + 16.0 * b.F + 8.0 + 12.0 * b.L;
      return TUCKER_OK;
    };
    if (nc > 0) TK_TRY(issue(0));
    for (int c = 0; c < nc; ++c) {
      if (c + 1 < nc) TK_TRY(issue(c + 1));
      ChunkBuf& b = buf_[c & 1];
      TK_CUDA(cudaStreamWaitEvent(cs_, b.copied, 0));
      TK_TRY(body(b, ch[c]));
      TK_CUDA(cudaEventRecord(b.used, cs_));
    }
    return TUCKER_OK;
  }
  double bytes() const { return bytecs_; }

 private:
  tucker_stream_s* X_;
  cudaStream_t cs_;
  cudaStream_t copy_stream_ = nullptr;
  ChunkBuf buf_[2];
  double bytecs_ = 0.0;
};

// M <- (accumulate ? M : 0) + Y Y^T, Y rows x K, FP64-accurate on the tensor cores.
int gram_accumulate(int rows, const double* Y, int64_t K, bool accumulate, double* M, int* status,
                    cudaStream_t s) {
  OzSlices S;
  TK_TRY(oz_split_rows(Y, K, rows, K, nullptr, 0, 0, OZ_GRAM_SLICES, &S, s));
  return oz_gemm_nt(S, S, true, 1.0, accumulate ? 1.0 : 0.0, accumulate ? M : nullptr, rows, 0.0,
                    nullptr, 0, M, rows, status, s, "gram_ozaki");
}

enum class SMethod { SP, MP };
const int SP_PAIRS_S[3][2] = {{0, 2}, {1, 0}, {2, 1}};   // Figure sp3

struct SRun {
  tucker_stream_s* X = nullptr;
  int J[3] = {0, 0, 0};
  cudaStream_t s = 0;
  Buf U[3], M, G, Gt, W, Y, sc, st;
  std::vector<double> fits;
  int rank_def = 0;
  int64_t dim(int a) const { return X->dims[a]; }
};

// The third mode o of a term (n, m).
int third(int n, int m) { return 3 - n - m; }

// M (+)= sum over the chunks of ordering (o, n, m) of Gram((X_c x_m U_m^T)_(n)).
int stream_term(SRun& r, Streamer& S, int n, int m, bool accumulate) {
  const int o = third(n, m);
  const int Jm = r.J[m];
  bool acc = accumulate;
  return S.for_chunks(o, n, m, [&](ChunkBuf& b, int64_t) -> int {
    const int64_t K = b.nk * Jm;
    TK_CUDA(cudaMemsetAsync(r.Y.p, 0, sizeof(double) * (size_t)(r.dim(n) * K), r.s));
    TK_TRY(slice_proj_f64_fibers(b.F, b.fiber_idx.as<int32_t>(), b.fiber_root.as<int32_t>(),
                                 b.fiber_ptr.as<int64_t>(), b.leaf_idx.as<int32_t>(),
                                 b.val.as<double>(), r.U[m].as<double>(), Jm, b.nk,
                                 r.Y.as<double>(), r.s));
    TK_TRY(gram_accumulate((int)r.dim(n), r.Y.as<double>(), K, acc, r.M.as<double>(),
                           r.st.as<int>(), r.s));
    acc = true;
    return TUCKER_OK;
  });
}

// M = X_(n) X_(n)^T = sum over the slices of mode o of X_k X_k^T (chunks densified).
int stream_unfolding_gram(SRun& r, Streamer& S, int n) {
  const int o = n == 0 ? 1 : 0, m = third(n, o);
  const int64_t Im = r.dim(m);
  bool acc = false;
  return S.for_chunks(o, n, m, [&](ChunkBuf& b, int64_t) -> int {
    const int64_t K = b.nk * Im;
    TK_CUDA(cudaMemsetAsync(r.Y.p, 0, sizeof(double) * (size_t)(r.dim(n) * K), r.s));
    if (b.F > 0) {
      densify_fibers<<<ceil_div(b.F * 32, 256), 256, 0, r.s>>>(
          b.F, b.fiber_idx.as<int32_t>(), b.fiber_root.as<int32_t>(), b.fiber_ptr.as<int64_t>(),
          b.leaf_idx.as<int32_t>(), b.val.as<double>(), Im, K, r.Y.as<double>());
      TK_LAUNCH();
    }
    TK_TRY(gram_accumulate((int)r.dim(n), r.Y.as<double>(), K, acc, r.M.as<double>(),
                           r.st.as<int>(), r.s));
    acc = true;
    return TUCKER_OK;
  });
}

// G = sum over the slices k of mode 3 of C[k, :]^T (x) W_k with W_k = A^T X_k B (ordering
// (2, 0, 1)), then |G|^2 and the fit.
int stream_core_fit(SRun& r, Streamer& S, double* fit, double* g2) {
  const int J1 = r.J[0], J2 = r.J[1], J3 = r.J[2];
  const int64_t nG = (int64_t)J1 * J2 * J3;
  TK_CUDA(cudaMemsetAsync(r.G.p, 0, sizeof(double) * nG, r.s));
  TK_TRY(S.for_chunks(2, 0, 1, [&](ChunkBuf& b, int64_t k0) -> int {
    TK_TRY(ttmc_f64_roots(b.nk, b.root_ptr.as<int64_t>(), b.fiber_idx.as<int32_t>(),
                          b.fiber_ptr.as<int64_t>(), b.leaf_idx.as<int32_t>(), b.val.as<double>(),
                          r.U[0].as<double>(), J1, r.U[1].as<double>(), J2, r.W.as<double>(),
                          r.s));
    TK_TRY(gemm_tn_f64(J1 * J2, J3, b.nk, r.W.as<double>(), (int64_t)J1 * J2,
                       r.U[2].as<double>() + k0 * J3, J3, r.Gt.as<double>(), J3, r.s));
    add_into<<<ceil_div(nG, 256), 256, 0, r.s>>>(r.G.as<double>(), r.Gt.as<double>(), nG);
    TK_LAUNCH();
    return TUCKER_OK;
  }));
  TK_TRY(sum_squares(r.G.as<double>(), nG, r.sc.as<double>(), r.s));
  TK_TRY(fit_on_device(r.X->norm2, r.sc.as<double>(), r.sc.as<double>() + 1, r.s));
  double h[2];
  int hs = 0;
  TK_CUDA(cudaMemcpyAsync(h, r.sc.p, sizeof(h), cudaMemcpyDeviceToHost, r.s));
  TK_CUDA(cudaMemcpyAsync(&hs, r.st.p, sizeof(int), cudaMemcpyDeviceToHost, r.s));
  TK_CUDA(cudaStreamSynchronize(r.s));
  if (hs & DEV_TIMEOUT) {
    set_error_detail("streamed Gram: a bounded wait in a tensor-core product gave up");
    return TUCKER_ETIMEOUT;
  }
  *g2 = h[0];
  *fit = h[1];
  return TUCKER_OK;
}

int eig_s(SRun& r, int n, bool warm) {
  EigStats es;
  TK_TRY(eig_topk_f64(r.M.as<double>(), (int)r.dim(n), r.J[n],
                      warm ? r.U[n].as<double>() : nullptr, r.U[n].as<double>(), nullptr, r.s,
                      &es));
  if (es.rank_deficient) r.rank_def |= 1 << n;
  return TUCKER_OK;
}

int run_streamed(SMethod method, tucker_stream_s* X, const int32_t J[3], const tucker_opts* opts,
                 tucker_result* out, double* bytes_streamed) {
  if (!X || !J || !out || !out->G || !out->U[0] || !out->U[1] || !out->U[2]) return TUCKER_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (J[a] < 1 || J[a] > X->dims[a]) return TUCKER_EINVAL;
  if (out->where != TUCKER_HOST && out->where != TUCKER_DEVICE) return TUCKER_EINVAL;
  tucker_opts o;
  if (opts) {
    o = *opts;
  } else {
    memset(&o, 0, sizeof(o));
    o.precision = TUCKER_FP64;
    o.tol = 1e-4;
    o.max_iter = 50;
  }
  if (o.precision != TUCKER_FP64) {
    set_error_detail("the streamed methods run in the FP64 form only");
    return TUCKER_EINVAL;
  }
  if (o.max_iter < 1 || isnan(o.tol) || o.tol == INFINITY || o.flags != 0) return TUCKER_EINVAL;
  if (o.init_where != TUCKER_HOST && o.init_where != TUCKER_DEVICE) return TUCKER_EINVAL;
  if (method == SMethod::SP && !o.init[2]) return TUCKER_EINVAL;
  if (X->nnz == 0 || !(X->norm2 > 0.0)) return TUCKER_EEMPTY;
  SRun r;
  r.X = X;
  r.s = (cudaStream_t)o.stream;
  for (int a = 0; a < 3; ++a) r.J[a] = J[a];
  const cudaMemcpyKind to_dev =
      o.init_where == TUCKER_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  int64_t maxI = 0, ymax = 0;
  for (int a = 0; a < 3; ++a) {
    TK_TRY(r.U[a].alloc(sizeof(double) * r.dim(a) * J[a], r.s));
    maxI = std::max(maxI, r.dim(a));
  }
  // The chunk projection: I_n x (slices of the chunk x J_m), or x I_m for MP's start.
  for (int n = 0; n < 3; ++n)
    for (int m = 0; m < 3; ++m) {
      if (m == n) continue;
      const int64_t w = method == SMethod::MP ? std::max<int64_t>(r.J[m], r.dim(m)) : r.J[m];
      ymax = std::max(ymax, r.dim(n) * X->max_chunk_slices * w);
    }
  TK_TRY(r.Y.alloc(sizeof(double) * (size_t)ymax, r.s));
  TK_TRY(r.M.alloc(sizeof(double) * maxI * maxI, r.s));
  const int64_t nG = (int64_t)J[0] * J[1] * J[2];
  TK_TRY(r.G.alloc(sizeof(double) * nG, r.s));
  TK_TRY(r.Gt.alloc(sizeof(double) * nG, r.s));
  TK_TRY(r.W.alloc(sizeof(double) * X->max_chunk_slices * J[0] * J[1], r.s));
  TK_TRY(r.sc.alloc(sizeof(double) * 2, r.s));
  TK_TRY(r.st.alloc(sizeof(int), r.s));
  TK_CUDA(cudaMemsetAsync(r.st.p, 0, sizeof(int), r.s));
  Streamer S(X, r.s);
  TK_TRY(S.init());
  bool have[3] = {false, false, false};
  if (method == SMethod::SP) {
    Buf raw;
    TK_TRY(raw.alloc(sizeof(double) * r.dim(2) * J[2], r.s));
    TK_CUDA(cudaMemcpyAsync(raw.p, o.init[2], sizeof(double) * r.dim(2) * J[2], to_dev, r.s));
    TK_TRY(normalize_columns(raw.as<double>(), (int)r.dim(2), J[2], r.U[2].as<double>(), r.s));
  } else {
    for (int n = 1; n < 3; ++n) {
      if (o.init[n]) {
        TK_CUDA(cudaMemcpyAsync(r.U[n].p, o.init[n], sizeof(double) * r.dim(n) * J[n], to_dev, r.s));
      } else {
        TK_TRY(stream_unfolding_gram(r, S, n));
        TK_TRY(scale_f64(r.dim(n) * r.dim(n), 2.0, r.M.as<double>(), r.s));   // pseudo HO-SVD
        TK_TRY(eig_s(r, n, false));
      }
      have[n] = true;
    }
  }
  double old = 0.0, gprev = 0.0;
  for (int it = 0; it < o.max_iter; ++it) {
    for (int step = 0; step < 3; ++step) {
      int n = step;
      if (method == SMethod::SP) {
        n = SP_PAIRS_S[step][0];
        TK_TRY(stream_term(r, S, n, SP_PAIRS_S[step][1], false));
      } else {
        const int m1 = n == 0 ? 1 : 0, m2 = n == 2 ? 1 : 2;
        TK_TRY(stream_term(r, S, n, m1, false));
        TK_TRY(stream_term(r, S, n, m2, true));
      }
      TK_TRY(eig_s(r, n, have[n]));
      have[n] = true;
    }
    double fit, g2;
    TK_TRY(stream_core_fit(r, S, &fit, &g2));
    r.fits.push_back(fit);
    if (method == SMethod::SP) {
      const double gn = sqrt(g2);
      if (it >= 1 && (1.0 - gprev / gn) < o.tol) break;
      gprev = gn;
    } else {
      if (fit - old < o.tol) break;
      old = fit;
    }
  }
  const cudaMemcpyKind from_dev =
      out->where == TUCKER_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  TK_CUDA(cudaMemcpyAsync(out->G, r.G.p, sizeof(double) * nG, from_dev, r.s));
  for (int a = 0; a < 3; ++a)
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
  if (bytes_streamed) *bytes_streamed = S.bytes();
  return TUCKER_OK;
}

}  // namespace
}  // namespace tk

extern "C" int tucker_sp_streamed(tucker_stream_tensor X, const int32_t J[3],
                                  const tucker_opts* opts, tucker_result* out,
                                  double* bytes_streamed) {
  return run_streamed(SMethod::SP, X, J, opts, out, bytes_streamed);
}

extern "C" int tucker_mp_streamed(tucker_stream_tensor X, const int32_t J[3],
                                  const tucker_opts* opts, tucker_result* out,
                                  double* bytes_streamed) {
  return run_streamed(SMethod::MP, X, J, opts, out, bytes_streamed);
}
