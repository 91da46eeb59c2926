// Batched products C_i = A_i * B_i (many independent SpGEMMs in shared
// launches).  The operands are packed into one block-diagonal problem
//   A = diag(A_1, ..., A_n),  B = [B_1; ...; B_n]  (rows stacked)
// where A_i's columns are shifted by the first packed row of B_i and B_i
// keeps its own column numbers.  Row r of A_i then multiplies exactly the
// rows of B_i, so row r of the packed product is row r of C_i with C_i's
// own columns, and every stage of the single-product path (binning, the
// per-bin persistent launches, the coarse and fine levels) runs once over
// the rows of all products: each bin's row list is the device work queue
// that the products share.  Packing is one gather per array; values are
// re-gathered by every numeric call, so the caller may change them in place
// between calls (plan reuse with new values).
#include <algorithm>
#include <new>
#include <vector>

#include "internal.h"

using namespace magnus;

namespace {

#define CUDA_TRY(x)                                              \
  do {                                                           \
    cudaError_t _e = (x);                                        \
    if (_e != cudaSuccess) return magnus::api_cuda_fail(_e, #x); \
  } while (0)

#define MAG_TRY(x)                  \
  do {                              \
    int _s = (x);                   \
    if (_s != MAGNUS_OK) return _s; \
  } while (0)

struct PackSrc {
  const int64_t* rp;
  const int32_t* col;
  const double* val;
};

__device__ __forceinline__ int find_part(const int64_t* __restrict__ off, int count, int64_t x) {
  // last p in [0, count) with off[p] <= x (off is nondecreasing, off[0] = 0)
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void k_pack_rowptr(const PackSrc* __restrict__ src, const int64_t* __restrict__ row_off,
                              const int64_t* __restrict__ nnz_off, int count, int64_t total_rows,
                              int64_t* __restrict__ out) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= total_rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    if (r == total_rows) {
      out[r] = nnz_off[count];
      continue;
    }
    const int p = find_part(row_off, count, r);
    out[r] = src[p].rp[r - row_off[p]] + nnz_off[p];
  }
}

constexpr int PACK_NT = 256;
constexpr int PACK_PER = 16;

// out[e] = src[p](e - nnz_off[p]) (+ col_add[p] for columns) for the product
// p holding packed entry e.  A block takes a tile of PACK_NT * PACK_PER
// entries; one search finds the tile's first product and each thread walks
// forward from it.
template <bool COL, bool VAL>
__global__ void k_pack_nz(const PackSrc* __restrict__ src, const int64_t* __restrict__ nnz_off,
                          const int32_t* __restrict__ col_add, int count, int64_t total,
                          int32_t* __restrict__ out_col, double* __restrict__ out_val) {
  __shared__ int s_p;
  constexpr int64_t TILE = (int64_t)PACK_NT * PACK_PER;
  for (int64_t e0 = (int64_t)blockIdx.x * TILE; e0 < total; e0 += (int64_t)gridDim.x * TILE) {
    __syncthreads();
    if (threadIdx.x == 0) s_p = find_part(nnz_off, count, e0);
    __syncthreads();
    int p = s_p;
#pragma unroll 4
    for (int k = 0; k < PACK_PER; ++k) {
      const int64_t e = e0 + (int64_t)k * PACK_NT + threadIdx.x;
      if (e >= total) break;
      while (nnz_off[p + 1] <= e) ++p;
      const int64_t l = e - nnz_off[p];
      if (COL) out_col[e] = src[p].col[l] + (col_add ? col_add[p] : 0);
      if (VAL) out_val[e] = src[p].val[l];
    }
  }
}

__global__ void k_gather_offsets(const int64_t* __restrict__ c_rp, const int64_t* __restrict__ row_off,
                                 int n, int64_t* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = c_rp[row_off[i]];
}

unsigned grid_for(int64_t work, int64_t per_block, int num_sms) {
  int64_t b = (work + per_block - 1) / per_block;
  const int64_t cap = (int64_t)num_sms * 16;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

struct magnus_batch_s {
  int count = 0;
  int device = 0;
  int num_sms = 1;
  std::vector<magnus_csr_t> A, B;
  std::vector<int64_t> a_row_off, a_nnz_off, b_row_off, b_nnz_off;
  std::vector<int32_t> col_add;
  std::vector<PackSrc> src_a_h, src_b_h;
  // device
  PackSrc* src_a = nullptr;
  PackSrc* src_b = nullptr;
  int64_t* d_a_row_off = nullptr;
  int64_t* d_a_nnz_off = nullptr;
  int64_t* d_b_row_off = nullptr;
  int64_t* d_b_nnz_off = nullptr;
  int32_t* d_col_add = nullptr;
  int64_t* c_off_d = nullptr;
  magnus_csr_t pa{}, pb{};   // packed descriptors
  int64_t* pa_rp = nullptr;
  int32_t* pa_col = nullptr;
  double* pa_val = nullptr;
  int64_t* pb_rp = nullptr;
  int32_t* pb_col = nullptr;
  double* pb_val = nullptr;
  std::vector<void*> owned;
  magnus_plan_t inner = nullptr;
  bool use_graph = false;
  bool symbolic_done = false;
  GraphSlot graph;
  cudaStream_t last_stream = nullptr;
};

namespace {

template <typename T>
int batch_alloc(magnus_batch_t b, T** p, size_t count, cudaStream_t s) {
  void* v = nullptr;
  cudaError_t e = cudaMallocAsync(&v, std::max<size_t>(count, 1) * sizeof(T), s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return api_cuda_fail(e, "cudaMallocAsync");
  }
  b->owned.push_back(v);
  *p = reinterpret_cast<T*>(v);
  return MAGNUS_OK;
}

int pack_values(magnus_batch_t b, cudaStream_t s) {
  const int64_t na = b->a_nnz_off[b->count], nb = b->b_nnz_off[b->count];
  const int64_t tile = (int64_t)PACK_NT * PACK_PER;
  if (na > 0) {
    k_pack_nz<false, true><<<grid_for(na, tile, b->num_sms), PACK_NT, 0, s>>>(
        b->src_a, b->d_a_nnz_off, nullptr, b->count, na, nullptr, b->pa_val);
    count_launch();
  }
  if (nb > 0) {
    k_pack_nz<false, true><<<grid_for(nb, tile, b->num_sms), PACK_NT, 0, s>>>(
        b->src_b, b->d_b_nnz_off, nullptr, b->count, nb, nullptr, b->pb_val);
    count_launch();
  }
  CUDA_TRY(cudaGetLastError());
  return MAGNUS_OK;
}

int plan_batched_impl(magnus_batch_t b, int32_t count, const magnus_csr_t* A,
                      const magnus_csr_t* B, const magnus_params_t* params, cudaStream_t s) {
  CUDA_TRY(cudaGetDevice(&b->device));
  CUDA_TRY(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device));
  b->count = count;
  b->A.assign(A, A + count);
  b->B.assign(B, B + count);
  b->a_row_off.assign(count + 1, 0);
  b->a_nnz_off.assign(count + 1, 0);
  b->b_row_off.assign(count + 1, 0);
  b->b_nnz_off.assign(count + 1, 0);
  b->col_add.assign(count, 0);
  int64_t max_cols = 0;
  for (int i = 0; i < count; ++i) {
    const magnus_csr_t& a = A[i];
    const magnus_csr_t& bb = B[i];
    if (a.n_rows < 0 || a.n_cols < 0 || a.nnz < 0 || bb.n_rows < 0 || bb.n_cols < 0 ||
        bb.nnz < 0 || !a.row_ptr || !bb.row_ptr || (a.nnz > 0 && !a.col) ||
        (bb.nnz > 0 && !bb.col) || a.n_cols != bb.n_rows || (a.nnz > 0 && bb.n_rows == 0))
      return MAGNUS_INVALID_ARG;
    b->a_row_off[i + 1] = b->a_row_off[i] + a.n_rows;
    b->a_nnz_off[i + 1] = b->a_nnz_off[i] + a.nnz;
    b->b_row_off[i + 1] = b->b_row_off[i] + bb.n_rows;
    b->b_nnz_off[i + 1] = b->b_nnz_off[i] + bb.nnz;
    b->col_add[i] = (int32_t)std::min<int64_t>(b->b_row_off[i], INT32_MAX);
    max_cols = std::max(max_cols, bb.n_cols);
  }
  const int64_t lim = ((int64_t)1 << 31) - 1;
  if (b->a_row_off[count] >= lim || b->b_row_off[count] >= lim || max_cols > lim)
    return MAGNUS_INDEX_OVERFLOW;
  b->src_a_h.resize(count);
  b->src_b_h.resize(count);
  for (int i = 0; i < count; ++i) {
    b->src_a_h[i] = PackSrc{A[i].row_ptr, A[i].col, A[i].val};
    b->src_b_h[i] = PackSrc{B[i].row_ptr, B[i].col, B[i].val};
  }
  const int64_t ra = b->a_row_off[count], rb = b->b_row_off[count];
  const int64_t na = b->a_nnz_off[count], nb = b->b_nnz_off[count];
  MAG_TRY(batch_alloc(b, &b->src_a, count, s));
  MAG_TRY(batch_alloc(b, &b->src_b, count, s));
  MAG_TRY(batch_alloc(b, &b->d_a_row_off, count + 1, s));
  MAG_TRY(batch_alloc(b, &b->d_a_nnz_off, count + 1, s));
  MAG_TRY(batch_alloc(b, &b->d_b_row_off, count + 1, s));
  MAG_TRY(batch_alloc(b, &b->d_b_nnz_off, count + 1, s));
  MAG_TRY(batch_alloc(b, &b->d_col_add, count, s));
  MAG_TRY(batch_alloc(b, &b->c_off_d, count + 1, s));
  MAG_TRY(batch_alloc(b, &b->pa_rp, ra + 1, s));
  MAG_TRY(batch_alloc(b, &b->pa_col, na, s));
  MAG_TRY(batch_alloc(b, &b->pa_val, na, s));
  MAG_TRY(batch_alloc(b, &b->pb_rp, rb + 1, s));
  MAG_TRY(batch_alloc(b, &b->pb_col, nb, s));
  MAG_TRY(batch_alloc(b, &b->pb_val, nb, s));
  CUDA_TRY(cudaMemcpyAsync(b->src_a, b->src_a_h.data(), count * sizeof(PackSrc), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(b->src_b, b->src_b_h.data(), count * sizeof(PackSrc), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(b->d_a_row_off, b->a_row_off.data(), (count + 1) * 8, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(b->d_a_nnz_off, b->a_nnz_off.data(), (count + 1) * 8, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(b->d_b_row_off, b->b_row_off.data(), (count + 1) * 8, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(b->d_b_nnz_off, b->b_nnz_off.data(), (count + 1) * 8, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(b->d_col_add, b->col_add.data(), count * 4, cudaMemcpyHostToDevice, s));
  const int64_t tile = (int64_t)PACK_NT * PACK_PER;
  k_pack_rowptr<<<grid_for(ra + 1, 256, b->num_sms), 256, 0, s>>>(b->src_a, b->d_a_row_off,
                                                                  b->d_a_nnz_off, count, ra, b->pa_rp);
  k_pack_rowptr<<<grid_for(rb + 1, 256, b->num_sms), 256, 0, s>>>(b->src_b, b->d_b_row_off,
                                                                  b->d_b_nnz_off, count, rb, b->pb_rp);
  count_launch(2);
  if (na > 0) {
    k_pack_nz<true, false><<<grid_for(na, tile, b->num_sms), PACK_NT, 0, s>>>(
        b->src_a, b->d_a_nnz_off, b->d_col_add, count, na, b->pa_col, nullptr);
    count_launch();
  }
  if (nb > 0) {
    k_pack_nz<true, false><<<grid_for(nb, tile, b->num_sms), PACK_NT, 0, s>>>(
        b->src_b, b->d_b_nnz_off, nullptr, count, nb, b->pb_col, nullptr);
    count_launch();
  }
  CUDA_TRY(cudaGetLastError());
  b->pa = magnus_csr_t{ra, rb, na, b->pa_rp, b->pa_col, b->pa_val};
  b->pb = magnus_csr_t{rb, std::max<int64_t>(max_cols, 1), nb, b->pb_rp, b->pb_col, b->pb_val};
  magnus_params_t p;
  magnus_params_default(&p);
  if (params) p = *params;
  b->use_graph = p.numeric_graph == 1;
  p.numeric_graph = 0;  // the batch captures the value packing with the numeric phase
  MAG_TRY(magnus_plan(&b->inner, &b->pa, &b->pb, &p, s));
  CUDA_TRY(cudaStreamSynchronize(s));  // host offset arrays are read by the copies above
  return MAGNUS_OK;
}

}  // namespace

extern "C" {

int magnus_plan_batched(magnus_batch_t* batch, int32_t count, const magnus_csr_t* A,
                        const magnus_csr_t* B, const magnus_params_t* params, void* stream) {
  if (!batch) return MAGNUS_INVALID_ARG;
  *batch = nullptr;
  if (count < 1 || !A || !B) return MAGNUS_INVALID_ARG;
  magnus_batch_t b = new (std::nothrow) magnus_batch_s();
  if (!b) return MAGNUS_OUT_OF_MEMORY;
  cudaStream_t s = (cudaStream_t)stream;
  b->last_stream = s;
  const int st = plan_batched_impl(b, count, A, B, params, s);
  if (st != MAGNUS_OK) {
    magnus_free_batched(b);
    return st;
  }
  *batch = b;
  return MAGNUS_OK;
}

int magnus_batch_layout(magnus_batch_t b, int64_t* row_offsets, int64_t* total_rows) {
  if (!b) return MAGNUS_INVALID_ARG;
  if (row_offsets) std::copy(b->a_row_off.begin(), b->a_row_off.end(), row_offsets);
  if (total_rows) *total_rows = b->a_row_off[b->count];
  return MAGNUS_OK;
}

int magnus_symbolic_batched(magnus_batch_t b, int64_t* c_row_ptr, int64_t* c_offsets,
                            void* stream) {
  if (!b || !c_row_ptr || !c_offsets) return MAGNUS_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  b->last_stream = s;
  b->symbolic_done = false;
  int64_t total = 0;
  MAG_TRY(magnus_symbolic(b->inner, c_row_ptr, &total, s));
  k_gather_offsets<<<grid_for(b->count + 1, 256, b->num_sms), 256, 0, s>>>(
      c_row_ptr, b->d_a_row_off, b->count + 1, b->c_off_d);
  count_launch();
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(c_offsets, b->c_off_d, (b->count + 1) * sizeof(int64_t),
                           cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  b->symbolic_done = true;
  return MAGNUS_OK;
}

int magnus_numeric_batched(magnus_batch_t b, const int64_t* c_row_ptr, int32_t* c_col,
                           double* c_val, void* stream) {
  if (!b || !c_row_ptr) return MAGNUS_INVALID_ARG;
  if (!b->symbolic_done) return MAGNUS_NOT_SYMBOLIC;
  cudaStream_t s = (cudaStream_t)stream;
  b->last_stream = s;
  auto body = [&]() -> int {
    MAG_TRY(pack_values(b, s));
    return magnus_numeric(b->inner, b->pa_val, b->pb_val, c_row_ptr, c_col, c_val, s);
  };
  if (b->use_graph && s != nullptr) {
    const void* key[3] = {c_row_ptr, c_col, c_val};
    return b->graph.run(key, 3, s, body);
  }
  return body();
}

magnus_plan_t magnus_batch_inner_plan(magnus_batch_t b) { return b ? b->inner : nullptr; }

int magnus_autotune_batched(magnus_batch_t b, const magnus_params_t* base, int64_t sample_products,
                            int32_t max_trials, magnus_params_t* best,
                            magnus_tune_report_t* report, void* stream) {
  if (!b || !best) return MAGNUS_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  b->last_stream = s;
  MAG_TRY(pack_values(b, s));  // the trials read the packed values
  return magnus_autotune(&b->pa, &b->pb, base, sample_products, max_trials, best, report, stream);
}

int magnus_batch_info(magnus_batch_t b, magnus_plan_info_t* info) {
  if (!b || !info) return MAGNUS_INVALID_ARG;
  return magnus_plan_info(b->inner, info);
}

void magnus_free_batched(magnus_batch_t b) {
  if (!b) return;
  cudaStream_t s = b->last_stream;
  b->graph.reset();
  if (b->inner) magnus_free(b->inner);
  for (void* v : b->owned) cudaFreeAsync(v, s);
  delete b;
}

}  // extern "C"
