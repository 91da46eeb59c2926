// Autotuner: measures plan + symbolic + numeric for candidate parameter sets
// on the caller's operands (or on a row sample of A) and keeps the fastest.
//
// The paper fixes the dense-versus-sort threshold and derives the chunk
// lengths from a cache model (Section 3.5, Section 4.1.1).  On the GPU those
// model values are starting points: the search is coordinate descent from the
// automatic parameters over the sort threshold, the wide-row sort limit, the
// coarse and fine chunk lengths and the fine-level hybrid threshold, each
// dimension tried only when the rows it governs exist; then the fine
// level's chunk accumulator (dense array or hash map), the coarse level's
// staging form (outer product or row-wise runs) and the block shape of the
// warp-sort kernels (2, 4 or 8 warps per block).  Every candidate
// computes the same C (parameters never change results beyond FP64 summation
// order), so C is allocated once.  Results are cached per operand shape and
// base parameters.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
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

// device, operand shapes, sample size and the base parameters (as bytes: a
// search from other base parameters, e.g. a forced category, is another entry)
using Key = std::tuple<int, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t,
                       std::string>;
std::mutex g_tune_mu;
std::map<Key, magnus_params_t> g_tune_cache;

__global__ void k_rebase(const int64_t* __restrict__ rp, int64_t r0, int64_t n, int64_t base,
                         int64_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = rp[r0 + i] - rp[r0] + base;
}

struct DevBuf {
  std::vector<void*> p;
  cudaStream_t s;
  explicit DevBuf(cudaStream_t st) : s(st) {}
  ~DevBuf() {
    for (void* v : p) cudaFreeAsync(v, s);
  }
  template <typename T>
  int get(T** out, size_t n) {
    void* v = nullptr;
    cudaError_t e = cudaMallocAsync(&v, std::max<size_t>(n, 1) * sizeof(T), s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return api_cuda_fail(e, "cudaMallocAsync");
    }
    p.push_back(v);
    *out = reinterpret_cast<T*>(v);
    return MAGNUS_OK;
  }
};

// One measured run of the whole step (plan, symbolic, numeric) in ms.
int trial(const magnus_csr_t* A, const magnus_csr_t* B, const magnus_params_t& p,
          int64_t* c_rp, int32_t* c_col, double* c_val, int64_t nnz_expect, cudaStream_t s,
          cudaEvent_t e0, cudaEvent_t e1, float* ms, magnus_plan_info_t* info) {
  CUDA_TRY(cudaEventRecord(e0, s));
  magnus_plan_t pl = nullptr;
  MAG_TRY(magnus_plan(&pl, A, B, &p, s));
  int64_t nnz = 0;
  int st = magnus_symbolic(pl, c_rp, &nnz, s);
  if (st == MAGNUS_OK && nnz_expect >= 0 && nnz != nnz_expect) st = MAGNUS_BAD_STATE;
  if (st == MAGNUS_OK) st = magnus_numeric(pl, A->val, B->val, c_rp, c_col, c_val, s);
  if (st == MAGNUS_OK && info) st = magnus_plan_info(pl, info);
  magnus_free(pl);
  MAG_TRY(st);
  CUDA_TRY(cudaEventRecord(e1, s));
  CUDA_TRY(cudaEventSynchronize(e1));
  CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
  return MAGNUS_OK;
}

}  // namespace

extern "C" {

int magnus_autotune(const magnus_csr_t* A, const magnus_csr_t* B, const magnus_params_t* base,
                    int64_t sample_products, int32_t max_trials, magnus_params_t* best,
                    magnus_tune_report_t* rep, void* stream) {
  if (!A || !B || !best || A->n_cols != B->n_rows || max_trials < 1) return MAGNUS_INVALID_ARG;
  if (A->nnz > 0 && (!A->val || !B->val)) return MAGNUS_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  magnus_params_t p0;
  magnus_params_default(&p0);
  if (base) p0 = *base;
  magnus_tune_report_t r;
  memset(&r, 0, sizeof(r));
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  const Key key{dev,       A->n_rows, A->n_cols, A->nnz,          B->n_rows,
                B->n_cols, B->nnz,    sample_products,
                std::string(reinterpret_cast<const char*>(&p0), sizeof(p0))};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      *best = it->second;
      r.from_cache = 1;
      if (rep) *rep = r;
      return MAGNUS_OK;
    }
  }
  DevBuf buf(s);
  // the operand tuned on: A itself, or evenly spaced row blocks of A
  magnus_csr_t At = *A;
  {
    magnus_plan_t pl = nullptr;
    MAG_TRY(magnus_plan(&pl, A, B, &p0, s));
    magnus_plan_info_t info;
    int st = magnus_plan_info(pl, &info);
    magnus_free(pl);
    MAG_TRY(st);
    r.products_full = info.n_interprod;
    if (sample_products > 0 && info.n_interprod > sample_products && A->n_rows > 64) {
      const int nblk = 16;
      const double frac = (double)sample_products / (double)info.n_interprod;
      int64_t rows_blk = std::max<int64_t>(1, (int64_t)(frac * A->n_rows / nblk));
      std::vector<int64_t> hrp(A->n_rows + 1);
      CUDA_TRY(cudaMemcpyAsync(hrp.data(), A->row_ptr, hrp.size() * 8, cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaStreamSynchronize(s));
      std::vector<int64_t> r0s;
      int64_t rows = 0, nz = 0;
      for (int b = 0; b < nblk; ++b) {
        const int64_t r0 = (int64_t)((double)b * A->n_rows / nblk);
        const int64_t r1 = std::min<int64_t>(A->n_rows, r0 + rows_blk);
        if (r1 <= r0 || (!r0s.empty() && r0 < r0s.back())) continue;
        r0s.push_back(r0);
        r0s.push_back(r1);
        rows += r1 - r0;
        nz += hrp[r1] - hrp[r0];
      }
      int64_t* rp;
      int32_t* col;
      double* val;
      MAG_TRY(buf.get(&rp, rows + 1));
      MAG_TRY(buf.get(&col, nz));
      MAG_TRY(buf.get(&val, nz));
      int64_t ro = 0, zo = 0;
      for (size_t i = 0; i < r0s.size(); i += 2) {
        const int64_t r0 = r0s[i], r1 = r0s[i + 1];
        const int64_t z0 = hrp[r0], z1 = hrp[r1];
        k_rebase<<<(unsigned)std::min<int64_t>(1024, (r1 - r0 + 256) / 256), 256, 0, s>>>(
            A->row_ptr, r0, r1 - r0, zo, rp + ro);
        CUDA_TRY(cudaGetLastError());
        if (z1 > z0) {
          CUDA_TRY(cudaMemcpyAsync(col + zo, A->col + z0, (z1 - z0) * 4, cudaMemcpyDeviceToDevice, s));
          CUDA_TRY(cudaMemcpyAsync(val + zo, A->val + z0, (z1 - z0) * 8, cudaMemcpyDeviceToDevice, s));
        }
        ro += r1 - r0;
        zo += z1 - z0;
      }
      At = magnus_csr_t{rows, A->n_cols, nz, rp, col, val};
      r.sampled_rows = rows;
    }
  }
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  int64_t* c_rp = nullptr;
  int32_t* c_col = nullptr;
  double* c_val = nullptr;
  int st = buf.get(&c_rp, At.n_rows + 1);
  int64_t nnz = 0;
  if (st == MAGNUS_OK) {
    magnus_plan_t pl = nullptr;
    st = magnus_plan(&pl, &At, B, &p0, s);
    if (st == MAGNUS_OK) {
      st = magnus_symbolic(pl, c_rp, &nnz, s);
      magnus_free(pl);
    }
  }
  if (st == MAGNUS_OK) st = buf.get(&c_col, nnz);
  if (st == MAGNUS_OK) st = buf.get(&c_val, nnz);
  magnus_params_t cur = p0;
  float best_ms = 0.f;
  magnus_plan_info_t info{};
  if (st == MAGNUS_OK) {
    // warm-up, then the base measurement
    float ms = 0.f;
    st = trial(&At, B, cur, c_rp, c_col, c_val, nnz, s, e0, e1, &ms, nullptr);
    if (st == MAGNUS_OK) st = trial(&At, B, cur, c_rp, c_col, c_val, nnz, s, e0, e1, &best_ms, &info);
    r.base_ms = best_ms;
    r.trials = 1;
  }
  // coordinate descent
  struct Dim { int32_t magnus_params_t::*field; std::vector<int32_t> vals; bool active; };
  const bool has_coarse = info.rows_per_category[MAGNUS_CAT_COARSE] > 0;
  const bool has_fine = info.rows_per_category[MAGNUS_CAT_FINE] > 0;
  std::vector<Dim> dims = {
      {&magnus_params_t::sort_threshold, {64, 128, 256, 512, 1025}, true},
      {&magnus_params_t::wide_sort_max, {-1, 256, 512, 1024}, p0.force_category < 0},
      {&magnus_params_t::chunk_len_coarse_log2, {11, 12, 13}, has_coarse},
      {&magnus_params_t::chunk_len_fine_log2, {7, 8, 9, 10}, has_fine || has_coarse},
      {&magnus_params_t::dense_chunk_threshold, {1, 32, 128, 257}, has_fine || has_coarse},
      {&magnus_params_t::chunk_accumulator, {0, 1}, has_fine || has_coarse},
      {&magnus_params_t::coarse_reorder, {1, 2}, has_coarse},
      {&magnus_params_t::coarse_bucket_sort, {-1, 1}, has_coarse},
      {&magnus_params_t::sort_block_warps, {2, 4, 8},
       info.rows_per_category[MAGNUS_CAT_SORT] > 0},
  };
  for (const Dim& d : dims) {
    if (st != MAGNUS_OK || !d.active) continue;
    for (int32_t v : d.vals) {
      if (r.trials >= max_trials) break;
      if (cur.*(d.field) == v) continue;
      magnus_params_t cand = cur;
      cand.*(d.field) = v;
      float ms = 0.f;
      const int ts = trial(&At, B, cand, c_rp, c_col, c_val, nnz, s, e0, e1, &ms, nullptr);
      ++r.trials;
      if (ts != MAGNUS_OK) {
        if (ts == MAGNUS_INVALID_ARG) continue;  // a value this operand does not admit
        st = ts;
        break;
      }
      if (ms < best_ms) {
        best_ms = ms;
        cur = cand;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  MAG_TRY(st);
  r.best_ms = best_ms;
  *best = cur;
  if (rep) *rep = r;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = cur;
  return MAGNUS_OK;
}

}  // extern "C"
