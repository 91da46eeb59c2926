// C ABI of the MAGNUS SpGEMM library: parameter model, setup (plan),
// symbolic and numeric phases.  Host orchestration only; every step of the
// computation runs in the kernels of the other translation units.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "internal.h"

using namespace magnus;

namespace magnus {
uint64_t launches_total();
size_t fine_smem_for(bool numeric, int shift, bool hybrid);
}

static thread_local std::string g_cuda_err;

static int cuda_fail(cudaError_t e, const char* where) {
  g_cuda_err = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return MAGNUS_OUT_OF_MEMORY;
  return MAGNUS_CUDA_ERROR;
}

namespace magnus {
int api_cuda_fail(cudaError_t e, const char* where) { return cuda_fail(e, where); }
}

#define CUDA_TRY(x)                                   \
  do {                                                \
    cudaError_t _e = (x);                             \
    if (_e != cudaSuccess) return cuda_fail(_e, #x);  \
  } while (0)

#define MAG_TRY(x)             \
  do {                         \
    int _s = (x);              \
    if (_s != MAGNUS_OK) return _s; \
  } while (0)

static int ceil_log2_i64(int64_t x) {
  int b = 0;
  while (((int64_t)1 << b) < x) ++b;
  return b;
}

// ---------------------------------------------------------------------------
// Chunk model: Eq. 2 of Section 3.5 evaluated with GPU storage terms.
//   s_denseAccum  numeric 8 + 1/8 bytes per column (FP64 value + bitmap bit),
//                 symbolic 1/8 byte (bitmap bit only)
//   s_chunkFine   8 bytes in shared memory (count + offset, int32 each);
//                 the active write lines of the reorder (two 128-byte lines per
//                 chunk, col and val streams) live in L2, shared by all
//                 resident blocks, so they bound the chunk count separately.
// Among chunk lengths that satisfy both budgets, the one minimising Eq. 2
// is taken.  When none does, the coarse level is needed: the widest column
// range with a feasible fine level is m_CmaxSMEM (the analogue of Eq. 5).
int magnus_chunk_model(int64_t m_c, int64_t smem_bytes, int64_t l2_bytes, int32_t resident_blocks,
                       magnus_chunk_model_t* out) {
  if (!out || m_c <= 0 || smem_bytes <= 0 || l2_bytes <= 0 || resident_blocks <= 0)
    return MAGNUS_INVALID_ARG;
  const int M = ceil_log2_i64(m_c);
  const double s_da_num = 8.0 + 1.0 / 8.0;
  const double s_da_sym = 1.0 / 8.0;
  const double s_cf = 8.0;
  const double line_bytes = 256.0;
  double nmax = (double)l2_bytes / 2.0 / ((double)resident_blocks * line_bytes);
  int nmax_log2 = 0;
  while (std::ldexp(1.0, nmax_log2 + 1) <= nmax) ++nmax_log2;
  if (nmax_log2 > 12) nmax_log2 = 12;  // shared-memory bookkeeping limit
  auto feasible = [&](int m, int c, double s_da) {
    const double acc = std::ldexp(1.0, c) * s_da;
    const double book = std::ldexp(1.0, m - c) * s_cf;
    return (m - c) <= nmax_log2 && acc + book <= (double)smem_bytes;
  };
  auto best_c = [&](int m, double s_da) {
    int best = -1;
    double bests = 0.0;
    for (int c = 5; c <= m; ++c) {
      if (!feasible(m, c, s_da)) continue;
      const double s = std::ldexp(1.0, c) * s_da + std::ldexp(1.0, m - c) * s_cf;
      if (best < 0 || s < bests) {
        best = c;
        bests = s;
      }
    }
    return best;
  };
  memset(out, 0, sizeof(*out));
  out->m_c_log2 = M;
  out->n_chunks_fine_max_log2 = nmax_log2;
  int m = M < 5 ? 5 : M;
  int c = best_c(m, s_da_num);
  while (c < 0 && m > 5) {
    --m;
    c = best_c(m, s_da_num);
  }
  if (c < 0) c = 5;
  out->m_c_max_log2 = m;
  out->chunk_len_fine_log2 = c;
  out->n_chunks_coarse = (M > m) ? (int32_t)(1 << (M - m)) : 1;
  out->fine_smem_bytes = (int64_t)(std::ldexp(1.0, c) * s_da_num + std::ldexp(1.0, m - c) * s_cf);
  // Symbolic: bitmap only.  A single chunk over the whole range when the
  // bitmap fits (no reorder at all); otherwise the Eq. 2 minimiser.
  const int msym = M < 5 ? 5 : M;
  if (std::ldexp(1.0, msym) * s_da_sym <= (double)smem_bytes) {
    out->chunk_len_fine_sym_log2 = msym;
  } else {
    int cs = best_c(msym, s_da_sym);
    out->chunk_len_fine_sym_log2 = cs < 0 ? c : cs;
  }
  return MAGNUS_OK;
}

// ---------------------------------------------------------------------------
struct magnus_plan_s {
  int device = 0;
  int num_sms = 0;
  int smem_optin = 0;
  int64_t l2_bytes = 0;
  Csr A{}, B{};
  magnus_params_t params{};
  int sort_T = 256;
  int dense_cols = 8192;
  int shift_fine = 13;
  int shift_fine_sym = 20;
  int shift_coarse = 24;
  int n_chunks_coarse = 1;
  int dthr = 256;
  int hash = 0;     // numeric fine chunks: hash-map accumulator
  int col_bits = 0;
  int64_t scratch_cap = 0;  // bytes
  // device arrays owned by the plan
  std::vector<void*> owned;
  int64_t owned_bytes = 0;
  int64_t* P = nullptr;
  uint8_t* bin = nullptr;
  int32_t* lo = nullptr;
  int32_t* hi = nullptr;
  int32_t* rows_sorted = nullptr;
  RowDesc* desc = nullptr;       // per listed row (bin order)
  uint64_t* seg = nullptr;       // per nonzero of A (seg_pack)
  int64_t bin_off[NUM_BINS + 1] = {0};
  // fine rows (heaviest first), batches as list index ranges
  std::vector<int32_t> fine_rows;
  std::vector<int64_t> fine_P;
  std::vector<int32_t> fine_lo, fine_hi;
  int32_t* fine_rows_d = nullptr;
  int64_t* fine_P_d = nullptr;
  int64_t fine_slab = 0;      // staging capacity (products) of one fine block
  int fine_grid_num = 0;      // resident blocks of the numeric fine kernel
  int fine_grid_sym = 0;      // resident blocks of the symbolic fine kernel
  // coarse rows
  std::vector<int32_t> coarse_rows;
  std::vector<int64_t> coarse_P;
  std::vector<int64_t> coarse_nnz;
  std::vector<int64_t> coarse_batches;
  int32_t* coarse_rows_d = nullptr;
  int32_t* bucket_cnt = nullptr;
  unsigned long long* big_stats = nullptr;  // [3] of the last numeric call (coarse large buckets)
  int64_t* coarse_offs = nullptr;  // bucket offsets of every coarse batch (symbolic -> numeric)
  std::vector<int64_t> coarse_offs_at;  // start of each batch's offsets in coarse_offs
  bool coarse_rowwise = false;          // row-wise staged reorder (else the outer product)
  CoarseItem* coarse_items_d = nullptr;  // its work items, in coarse list order
  std::vector<int64_t> coarse_item_first;  // first item of each coarse list row (+ total)
  // sorted slot order of the sort rows (symbolic -> numeric)
  uint8_t* perm = nullptr;
  int64_t perm_off[NUM_BINS + 1] = {0};
  uint16_t* perm2 = nullptr;         // block sort bins: sorted slot order
  int64_t* perm2_off = nullptr;      // per block-bin row (both bins), + total
  // state and statistics
  bool symbolic_done = false;
  int64_t nnz_c = -1;
  int64_t n_interprod = 0, max_P = 0;
  int64_t rows_cat[4] = {0}, prods_cat[4] = {0};
  int64_t staged_numeric = 0, scratch_used = 0;
  int key32[NUM_BINS] = {0};
  // timing
  bool timing = false;
  cudaEvent_t ev[2 * MAGNUS_STAGE_COUNT] = {};
  bool ev_used[MAGNUS_STAGE_COUNT] = {};
  bool use_graph = false;
  GraphSlot graph;                     // numeric phase (numeric_graph = 1)
  std::vector<cudaEvent_t> big_ev[2];  // per phase: event pairs around each batch's large-bucket kernel
  int big_ev_used[2] = {0, 0};
  cudaStream_t last_stream = nullptr;
};

namespace magnus {
// kernels_coarse.cu: reads and clears the flag of a bounded device wait that
// gave up (synchronises the stream)
cudaError_t wait_timeout_take(int* timed_out, cudaStream_t s);
// kernels_coarse.cu: a bounded wait that nothing completes
cudaError_t launch_wait_selftest(long long limit_cycles, cudaStream_t s);
}  // namespace magnus

namespace {

int dev_alloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return cuda_fail(e, "cudaMallocAsync");
  }
  return MAGNUS_OK;
}

template <typename T>
int plan_alloc(magnus_plan_t pl, T** p, size_t count, cudaStream_t s) {
  void* v;
  MAG_TRY(dev_alloc(&v, count * sizeof(T), s));
  pl->owned.push_back(v);
  pl->owned_bytes += (int64_t)(count * sizeof(T));
  *p = reinterpret_cast<T*>(v);
  return MAGNUS_OK;
}

// Stream-ordered scratch freed when the guard goes out of scope.
struct Scratch {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t st) : s(st) {}
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
  template <typename T>
  int get(T** p, size_t count) {
    void* v;
    MAG_TRY(dev_alloc(&v, count * sizeof(T), s));
    ptrs.push_back(v);
    *p = reinterpret_cast<T*>(v);
    return MAGNUS_OK;
  }
};

void ensure_pool_retains(int dev) {
  static bool done[64] = {false};
  if (dev < 0 || dev >= 64 || done[dev]) return;
  // Keep up to 16 GB of freed scratch for reuse by later calls (a plan's
  // arrays and staging are freed and reallocated every product); larger
  // transient staging goes back to the device at the next synchronisation.
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = (uint64_t)16 << 30;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done[dev] = true;
}

struct StageTimer {
  magnus_plan_t p;
  int stage;
  cudaStream_t s;
  StageTimer(magnus_plan_t pl, int st, cudaStream_t str) : p(pl), stage(st), s(str) {
    if (p->timing) {
      cudaEventRecord(p->ev[2 * stage], s);
      p->ev_used[stage] = true;
    }
  }
  ~StageTimer() {
    if (p->timing) cudaEventRecord(p->ev[2 * stage + 1], s);
  }
};

int check_csr(const magnus_csr_t* M) {
  if (!M) return MAGNUS_INVALID_ARG;
  if (M->n_rows < 0 || M->n_cols < 0 || M->nnz < 0) return MAGNUS_INVALID_ARG;
  if (M->n_rows >= ((int64_t)1 << 31) - 1 || M->n_cols > ((int64_t)1 << 31) - 1)
    return MAGNUS_INDEX_OVERFLOW;
  if (!M->row_ptr) return MAGNUS_INVALID_ARG;
  if (M->nnz > 0 && !M->col) return MAGNUS_INVALID_ARG;
  return MAGNUS_OK;
}

// Batches of consecutive list entries with sum(P) <= cap (a single entry
// above the cap forms its own batch).  Returns boundaries.
std::vector<int64_t> make_batches(const std::vector<int64_t>& P, int64_t cap_products,
                                  int64_t max_rows) {
  std::vector<int64_t> b{0};
  int64_t acc = 0, rows = 0;
  for (size_t i = 0; i < P.size(); ++i) {
    if (rows > 0 && (acc + P[i] > cap_products || rows >= max_rows)) {
      b.push_back((int64_t)i);
      acc = 0;
      rows = 0;
    }
    acc += P[i];
    ++rows;
  }
  if (b.back() != (int64_t)P.size()) b.push_back((int64_t)P.size());
  return b;
}

}  // namespace

extern "C" {

int magnus_params_default(magnus_params_t* p) {
  if (!p) return MAGNUS_INVALID_ARG;
  memset(p, 0, sizeof(*p));
  p->force_category = MAGNUS_CAT_AUTO;
  return MAGNUS_OK;
}

const char* magnus_strerror(int s) {
  switch (s) {
    case MAGNUS_OK: return "ok";
    case MAGNUS_INVALID_ARG: return "invalid argument";
    case MAGNUS_UNSORTED_OR_DUP: return "input CSR has unsorted, duplicate or out-of-range columns";
    case MAGNUS_INDEX_OVERFLOW: return "size exceeds the index types";
    case MAGNUS_OUT_OF_MEMORY: return "out of device memory";
    case MAGNUS_CUDA_ERROR: return "CUDA error";
    case MAGNUS_TIMEOUT: return "device wait timed out";
    case MAGNUS_NOT_SYMBOLIC: return "numeric called before symbolic";
    case MAGNUS_BAD_STATE: return "plan in a bad state";
    case MAGNUS_SCRATCH_LIMIT:
      return "the allocation-free numeric entry point needs more staging than its fixed buffer "
             "(MAGNUS_NOALLOC_SCRATCH_BYTES) holds, or the plan has coarse rows";
    case MAGNUS_WORKSPACE_TOO_SMALL:
      return "the caller's workspace is smaller than magnus_workspace_size";
    default: return "unknown status";
  }
}

const char* magnus_last_cuda_error(void) { return g_cuda_err.c_str(); }

uint64_t magnus_launch_count(void) { return launches_total(); }

int magnus_device_memory(size_t* free_bytes, size_t* pool_idle_bytes) {
  size_t fr = 0, tot = 0;
  CUDA_TRY(cudaMemGetInfo(&fr, &tot));
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  cudaMemPool_t pool;
  CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t reserved = 0, used = 0;
  CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved));
  CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
  if (free_bytes) *free_bytes = fr;
  if (pool_idle_bytes) *pool_idle_bytes = (size_t)(reserved > used ? reserved - used : 0);
  return MAGNUS_OK;
}

void magnus_free(magnus_plan_t p) {
  if (!p) return;
  cudaStream_t s = p->last_stream;
  for (void* v : p->owned) cudaFreeAsync(v, s);
  for (int i = 0; i < 2 * MAGNUS_STAGE_COUNT; ++i)
    if (p->ev[i]) cudaEventDestroy(p->ev[i]);
  for (int ph = 0; ph < 2; ++ph)
    for (cudaEvent_t e : p->big_ev[ph]) cudaEventDestroy(e);
  p->graph.reset();
  delete p;
}

static int plan_impl(magnus_plan_t pl, const magnus_csr_t* A, const magnus_csr_t* B,
                     const magnus_params_t* params, cudaStream_t s) {
  CUDA_TRY(cudaGetDevice(&pl->device));
  ensure_pool_retains(pl->device);
  CUDA_TRY(cudaDeviceGetAttribute(&pl->num_sms, cudaDevAttrMultiProcessorCount, pl->device));
  CUDA_TRY(cudaDeviceGetAttribute(&pl->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                  pl->device));
  int l2 = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, pl->device));
  pl->l2_bytes = l2;
  pl->A = Csr{A->n_rows, A->n_cols, A->nnz, A->row_ptr, A->col, A->val};
  pl->B = Csr{B->n_rows, B->n_cols, B->nnz, B->row_ptr, B->col, B->val};
  if (params) pl->params = *params; else magnus_params_default(&pl->params);
  const magnus_params_t& P = pl->params;
  if (P.force_category < -1 || P.force_category > 3) return MAGNUS_INVALID_ARG;
  if (P.numeric_graph != 0 && P.numeric_graph != 1) return MAGNUS_INVALID_ARG;
  pl->use_graph = P.numeric_graph == 1;
  if (P.l2_fetch_bytes != 0 && P.l2_fetch_bytes != 32 && P.l2_fetch_bytes != 64 &&
      P.l2_fetch_bytes != 128)
    return MAGNUS_INVALID_ARG;
  if (P.l2_fetch_bytes > 0) {
    size_t cur = 0;
    CUDA_TRY(cudaDeviceGetLimit(&cur, cudaLimitMaxL2FetchGranularity));
    if (cur != (size_t)P.l2_fetch_bytes)
      CUDA_TRY(cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)P.l2_fetch_bytes));
  }
  if (P.sort_threshold < 0 || P.sort_threshold > SORT_BLOCK_MAX + 1) return MAGNUS_INVALID_ARG;
  if (P.wide_sort_max < -1 || P.wide_sort_max > SORT_BLOCK_MAX) return MAGNUS_INVALID_ARG;
  if (P.chunk_accumulator != 0 && P.chunk_accumulator != 1) return MAGNUS_INVALID_ARG;
  if (P.coarse_reorder < 0 || P.coarse_reorder > 2) return MAGNUS_INVALID_ARG;
  if (P.sort_block_warps != 0 && P.sort_block_warps != 2 && P.sort_block_warps != 4 &&
      P.sort_block_warps != 8)
    return MAGNUS_INVALID_ARG;
  if (P.coarse_bucket_sort < -1 || P.coarse_bucket_sort > 1) return MAGNUS_INVALID_ARG;
  pl->sort_T = P.sort_threshold > 0 ? P.sort_threshold : 256;
  const int64_t m_c = B->n_cols > 0 ? B->n_cols : 1;
  pl->col_bits = ceil_log2_i64(m_c);
  // chunk model with a 64 KB accumulator budget per block (two fine blocks
  // per SM) and a 128 KB bitmap budget for the symbolic phase
  magnus_chunk_model_t cm, cms;
  MAG_TRY(magnus_chunk_model(m_c, 64 * 1024, pl->l2_bytes, pl->num_sms * 2, &cm));
  MAG_TRY(magnus_chunk_model(m_c, 128 * 1024, pl->l2_bytes, pl->num_sms, &cms));
  pl->dense_cols = 8192;
  // Fine chunks are accumulated by one warp each: a numeric chunk is at most
  // 2^10 columns (8 KB of FP64 per warp), a symbolic chunk 2^13 columns (a
  // 1 KB bitmap per warp).
  pl->shift_fine = P.chunk_len_fine_log2 > 0 ? P.chunk_len_fine_log2 : cm.chunk_len_fine_log2;
  if (pl->shift_fine > 10) pl->shift_fine = 10;
  if (pl->shift_fine < 5) pl->shift_fine = 5;
  pl->shift_fine_sym = std::min(13, pl->shift_fine + 3);
  (void)cms;
  // Coarse chunks of 2^13 columns split a heavy row into independent
  // (row, chunk) work items of eight warp chunks each.
  int sc = P.chunk_len_coarse_log2 > 0 ? P.chunk_len_coarse_log2 : std::min(cm.m_c_max_log2, 13);
  if (sc > pl->col_bits) sc = pl->col_bits;
  if (sc < pl->shift_fine) sc = pl->shift_fine;
  if (sc - pl->shift_fine > 12) sc = pl->shift_fine + 12;  // fine chunks per coarse chunk
  if (sc > 31) sc = 31;
  pl->shift_coarse = sc;
  pl->n_chunks_coarse = (int)((m_c + ((int64_t)1 << sc) - 1) >> sc);
  // fine-level hybrid (Section 3.4): chunks below dthr products sort in a
  // warp (at most 256), the others use a warp's dense accumulator.  The
  // paper's CPU threshold is 256; on the GPU a warp's dense accumulator
  // (1,024 FP64 columns in shared memory) beats the warp sort down to about
  // 16 products per chunk, and the sort's staging costs occupancy, so the
  // automatic value is 1 (dense only; the autotuner tries the hybrid).
  pl->dthr = P.dense_chunk_threshold > 0 ? std::min(P.dense_chunk_threshold, 257) : 1;
  pl->hash = P.chunk_accumulator;
  for (int b = BIN_SORT32; b <= BIN_SORT1024; ++b) {
    const int sb = 4 + b;  // log2 of the bin capacity: 5, 6, 7, 8, 9, 10
    pl->key32[b] = (pl->col_bits + sb <= 32) ? 1 : 0;
  }
  size_t free_b = 0, total_b = 0;
  CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  if (P.max_scratch_bytes > 0) {
    pl->scratch_cap = P.max_scratch_bytes;
  } else {
    pl->scratch_cap = std::min<int64_t>((int64_t)(free_b / 6), (int64_t)16 << 30);
    if (pl->scratch_cap < ((int64_t)64 << 20)) pl->scratch_cap = (int64_t)64 << 20;
  }

  const int64_t n = A->n_rows;
  if (P.validate) {
    int* flag;
    MAG_TRY(plan_alloc(pl, &flag, 1, s));
    CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
    CUDA_TRY(launch_validate(pl->A, flag, s));
    CUDA_TRY(launch_validate(pl->B, flag, s));
    int h = 0;
    CUDA_TRY(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (h) return MAGNUS_UNSORTED_OR_DUP;
  }
  MAG_TRY(plan_alloc(pl, &pl->P, n + 1, s));
  MAG_TRY(plan_alloc(pl, &pl->bin, n + 1, s));
  MAG_TRY(plan_alloc(pl, &pl->lo, n + 1, s));
  MAG_TRY(plan_alloc(pl, &pl->hi, n + 1, s));
  MAG_TRY(plan_alloc(pl, &pl->rows_sorted, n + 1, s));
  MAG_TRY(plan_alloc(pl, &pl->desc, n + 1, s));
  MAG_TRY(plan_alloc(pl, &pl->seg, (size_t)A->nnz + 1, s));
  CatParams cp;
  cp.sort_threshold = pl->sort_T;
  cp.force = P.force_category;
  cp.dense_cols = pl->dense_cols;
  cp.fine_shift = pl->shift_fine;
  cp.fine_max_chunks = FINE_MAX_CHUNKS;
  // A fine row is staged whole in its block's slab; the slabs of all resident
  // blocks share the staging budget.  Rows with more products than a slab
  // are split across blocks by the coarse level instead.
  pl->fine_grid_num =
      fine_rows_blocks_per_sm(true, pl->shift_fine, pl->dthr > 1 || pl->hash) * pl->num_sms;
  pl->fine_grid_sym = fine_rows_blocks_per_sm(false, pl->shift_fine_sym, pl->dthr > 1) * pl->num_sms;
  pl->fine_slab = std::min<int64_t>((int64_t)1 << 20,
                                    pl->scratch_cap / (12 * (int64_t)pl->fine_grid_num));
  if (pl->fine_slab < 256) pl->fine_slab = 256;
  cp.fine_max_products = pl->fine_slab;
  // On GB300 a fine-level row runs on one block (one SM) while the coarse
  // level spreads every row over the whole GPU in (row, chunk) work items;
  // rows wider than the dense accumulator use the coarse level unless the
  // fine level is forced.
  cp.prefer_fine = 0;
  // Rows too wide for the dense accumulator but with at most this many
  // products sort in registers (one warp) or in one block instead of taking
  // the coarse level's four passes over their products.
  cp.wide_sort_max = P.wide_sort_max == 0 ? SORT_BLOCK_MAX : (P.wide_sort_max < 0 ? 0 : P.wide_sort_max);
  CUDA_TRY(launch_rowinfo(pl->A, pl->B, cp, pl->P, pl->bin, pl->lo, pl->hi, pl->seg, s));
  int64_t* stats;
  MAG_TRY(plan_alloc(pl, &stats, 2 + NUM_BINS + 1, s));
  CUDA_TRY(launch_reduce_stats(pl->P, n, stats, s));
  const int64_t nblk = bin_partition_blocks(n);
  const int64_t m = (int64_t)NUM_BINS * nblk;
  Scratch tmp(s);
  int64_t* blk;
  MAG_TRY(tmp.get(&blk, (size_t)(m + 1 + scan_tmp_elems(m) + 1)));
  CUDA_TRY(launch_bin_partition(pl->bin, n, pl->rows_sorted, stats + 2, blk, nblk, s));
  CUDA_TRY(launch_row_desc(pl->rows_sorted, n, pl->A.rp, pl->desc, s));
  int64_t hstats[2 + NUM_BINS + 1];
  CUDA_TRY(cudaMemcpyAsync(hstats, stats, sizeof(hstats), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  pl->n_interprod = hstats[0];
  pl->max_P = hstats[1];
  for (int b = 0; b <= NUM_BINS; ++b) pl->bin_off[b] = hstats[2 + b];

  auto copy_bin = [&](int b, std::vector<int32_t>& rows, std::vector<int64_t>& Pv,
                      std::vector<int32_t>* lo, std::vector<int32_t>* hi) -> int {
    const int64_t cnt = pl->bin_off[b + 1] - pl->bin_off[b];
    rows.resize(cnt);
    Pv.resize(cnt);
    if (cnt == 0) return MAGNUS_OK;
    CUDA_TRY(cudaMemcpyAsync(rows.data(), pl->rows_sorted + pl->bin_off[b], cnt * 4,
                             cudaMemcpyDeviceToHost, s));
    int64_t* pg;
    MAG_TRY(tmp.get(&pg, (size_t)cnt));
    CUDA_TRY(launch_gather_i64(pl->P, pl->rows_sorted + pl->bin_off[b], cnt, pg, s));
    CUDA_TRY(cudaMemcpyAsync(Pv.data(), pg, cnt * 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (lo && hi) {
      lo->resize(cnt);
      hi->resize(cnt);
      std::vector<int32_t> lo_all(pl->A.n_rows), hi_all(pl->A.n_rows);
      CUDA_TRY(cudaMemcpyAsync(lo_all.data(), pl->lo, pl->A.n_rows * 4, cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaMemcpyAsync(hi_all.data(), pl->hi, pl->A.n_rows * 4, cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaStreamSynchronize(s));
      for (int64_t i = 0; i < cnt; ++i) {
        (*lo)[i] = lo_all[rows[i]];
        (*hi)[i] = hi_all[rows[i]];
      }
    }
    return MAGNUS_OK;
  };

  // sorted slot order of the sort rows: 32*E bytes per row of each sort bin
  {
    int64_t o = 0;
    for (int b = 0; b <= NUM_BINS; ++b) {
      pl->perm_off[b] = o;
      if (b >= BIN_SORT32 && b <= BIN_SORT256)
        o += (pl->bin_off[b + 1] - pl->bin_off[b]) * ((int64_t)32 << (b - BIN_SORT32));
    }
    MAG_TRY(plan_alloc(pl, &pl->perm, (size_t)o + 16, s));
    // block sort bins: P_i two-byte slots per row, at the prefix sum of P
    const int64_t nblk = pl->bin_off[BIN_SORT1024 + 1] - pl->bin_off[BIN_SORT512];
    int64_t tot = 0;
    if (nblk > 0) {
      MAG_TRY(plan_alloc(pl, &pl->perm2_off, (size_t)nblk + 1, s));
      CUDA_TRY(launch_gather_i64(pl->P, pl->rows_sorted + pl->bin_off[BIN_SORT512], nblk,
                                 pl->perm2_off, s));
      int64_t* stmp;
      MAG_TRY(tmp.get(&stmp, (size_t)scan_tmp_elems(nblk) + 2));
      CUDA_TRY(launch_exclusive_scan_i64(pl->perm2_off, nblk, stmp, s));
      CUDA_TRY(cudaMemcpyAsync(&tot, pl->perm2_off + nblk, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaStreamSynchronize(s));
    }
    MAG_TRY(plan_alloc(pl, &pl->perm2, (size_t)tot + 8, s));
  }
  // per-category statistics and the dense row count
  std::vector<int32_t> drows;
  std::vector<int64_t> dP;
  MAG_TRY(copy_bin(BIN_DENSE, drows, dP, nullptr, nullptr));
  MAG_TRY(copy_bin(BIN_FINE, pl->fine_rows, pl->fine_P, &pl->fine_lo, &pl->fine_hi));
  MAG_TRY(copy_bin(BIN_COARSE, pl->coarse_rows, pl->coarse_P, nullptr, nullptr));
  for (int b = BIN_SORT32; b <= BIN_SORT1024; ++b)
    pl->rows_cat[MAGNUS_CAT_SORT] += pl->bin_off[b + 1] - pl->bin_off[b];
  pl->rows_cat[MAGNUS_CAT_DENSE] = (int64_t)drows.size();
  pl->rows_cat[MAGNUS_CAT_FINE] = (int64_t)pl->fine_rows.size();
  pl->rows_cat[MAGNUS_CAT_COARSE] = (int64_t)pl->coarse_rows.size();
  auto sum = [](const std::vector<int64_t>& v) { return std::accumulate(v.begin(), v.end(), (int64_t)0); };
  pl->prods_cat[MAGNUS_CAT_DENSE] = sum(dP);
  pl->prods_cat[MAGNUS_CAT_FINE] = sum(pl->fine_P);
  pl->prods_cat[MAGNUS_CAT_COARSE] = sum(pl->coarse_P);
  pl->prods_cat[MAGNUS_CAT_SORT] = pl->n_interprod - pl->prods_cat[1] - pl->prods_cat[2] - pl->prods_cat[3];

  // fine rows: heaviest first (taken in this order by the persistent fine kernel)
  if (!pl->fine_rows.empty()) {
    const size_t nf = pl->fine_rows.size();
    std::vector<size_t> order(nf);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t a, size_t b) { return pl->fine_P[a] > pl->fine_P[b]; });
    std::vector<int32_t> r2(nf), l2(nf), h2(nf);
    std::vector<int64_t> p2(nf);
    for (size_t i = 0; i < nf; ++i) {
      r2[i] = pl->fine_rows[order[i]];
      p2[i] = pl->fine_P[order[i]];
      l2[i] = pl->fine_lo[order[i]];
      h2[i] = pl->fine_hi[order[i]];
    }
    pl->fine_rows.swap(r2);
    pl->fine_P.swap(p2);
    pl->fine_lo.swap(l2);
    pl->fine_hi.swap(h2);
    MAG_TRY(plan_alloc(pl, &pl->fine_rows_d, nf, s));
    MAG_TRY(plan_alloc(pl, &pl->fine_P_d, nf, s));
    CUDA_TRY(cudaMemcpyAsync(pl->fine_rows_d, pl->fine_rows.data(), nf * 4, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(pl->fine_P_d, pl->fine_P.data(), nf * 8, cudaMemcpyHostToDevice, s));
  }
  // Sparse wide coarse rows.  d = products per column of the row that a
  // typical product belongs to (rows weighted by their products, so a few
  // heavy rows of a power-law matrix dominate).  Dense rows (R-MAT: a 2^13
  // chunk receives >= 1024 products) keep the chunks of the block dense
  // accumulator.  Sparser rows widen the chunks: to about 2048 products per
  // (row, chunk) bucket when the fine level inside still sees >= 8 products
  // per 2^10-column chunk, else to about 128 (a warp sort per bucket), so the
  // per-bucket bookkeeping does not outgrow the products.
  if (!pl->coarse_rows.empty() && P.chunk_len_coarse_log2 <= 0) {
    double sp = 0.0, sp2 = 0.0;
    for (int64_t p : pl->coarse_P) {
      sp += (double)p;
      sp2 += (double)p * (double)p;
    }
    const double m_cd = (double)(B->n_cols > 0 ? B->n_cols : 1);
    const double d = sp > 0.0 ? sp2 / sp / m_cd : 0.0;
    int sc = pl->shift_coarse;
    if (d * 8192.0 < 1024.0) {
      const double target = d * 1024.0 >= 8.0 ? 2048.0 : 128.0;
      while (sc < pl->col_bits && sc < 31 && sc - pl->shift_fine < 12 &&
             d * std::ldexp(1.0, sc) < target)
        ++sc;
    }
    if (sc != pl->shift_coarse) {
      pl->shift_coarse = sc;
      pl->n_chunks_coarse = (int)((B->n_cols + ((int64_t)1 << sc) - 1) >> sc);
      if (pl->n_chunks_coarse < 1) pl->n_chunks_coarse = 1;
    }
  }
  // coarse rows: batched by staging capacity (two 12 B/product buffers) and
  // by the size of the (row, chunk) bookkeeping
  if (!pl->coarse_rows.empty()) {
    const size_t nc = pl->coarse_rows.size();
    // coarse staging: 12 B per product, plus 12 B for the fine level inside
    // coarse chunks wider than one block's dense accumulator
    const int64_t per = pl->shift_coarse <= 13 ? 12 : 24;
    const int64_t cap = std::max<int64_t>(pl->scratch_cap / per, pl->max_P);
    const int64_t max_rows = std::max<int64_t>(1, ((int64_t)1 << 28) / pl->n_chunks_coarse);
    pl->coarse_batches = make_batches(pl->coarse_P, cap, max_rows);
    MAG_TRY(plan_alloc(pl, &pl->coarse_rows_d, nc, s));
    CUDA_TRY(cudaMemcpyAsync(pl->coarse_rows_d, pl->coarse_rows.data(), nc * 4,
                             cudaMemcpyHostToDevice, s));
    // nnz of A per coarse row, for sizing the CSC buffers
    std::vector<int64_t> rp(pl->A.n_rows + 1);
    CUDA_TRY(cudaMemcpyAsync(rp.data(), pl->A.rp, (pl->A.n_rows + 1) * 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    pl->coarse_nnz.resize(nc);
    for (size_t i = 0; i < nc; ++i) pl->coarse_nnz[i] = rp[pl->coarse_rows[i] + 1] - rp[pl->coarse_rows[i]];
    // work items of the row-wise staged reorder: runs of CS_NJ nonzeros of A
    // automatic: row-wise when B rows are barely shared (the coarse rows'
    // nonzeros of A reference each B row about once, so the outer product's
    // one read per batch saves nothing); the outer product otherwise
    int64_t coarse_nnz_total = 0;
    for (int64_t z : pl->coarse_nnz) coarse_nnz_total += z;
    const bool low_reuse = coarse_nnz_total <= 2 * pl->B.n_rows;
    pl->coarse_rowwise = P.coarse_reorder == 2 ||
                         (P.coarse_reorder == 0 && low_reuse &&
                          pl->n_chunks_coarse <= CS_MAX_CHUNKS);
    if (pl->coarse_rowwise && pl->n_chunks_coarse > CS_MAX_CHUNKS) return MAGNUS_INVALID_ARG;
    if (pl->coarse_rowwise) {
      std::vector<CoarseItem> items;
      pl->coarse_item_first.assign(nc + 1, 0);
      for (size_t i = 0; i < nc; ++i) {
        pl->coarse_item_first[i] = (int64_t)items.size();
        const int64_t a0 = rp[pl->coarse_rows[i]], a1 = rp[pl->coarse_rows[i] + 1];
        for (int64_t j0 = a0; j0 < a1; j0 += CS_NJ)
          items.push_back(CoarseItem{j0, (int32_t)i, (int32_t)std::min<int64_t>(CS_NJ, a1 - j0)});
      }
      pl->coarse_item_first[nc] = (int64_t)items.size();
      MAG_TRY(plan_alloc(pl, &pl->coarse_items_d, items.size(), s));
      // pageable source: the copy has left the vector when the call returns
      CUDA_TRY(cudaMemcpyAsync(pl->coarse_items_d, items.data(), items.size() * sizeof(CoarseItem),
                               cudaMemcpyHostToDevice, s));
    }
    MAG_TRY(plan_alloc(pl, &pl->bucket_cnt, nc * (size_t)pl->n_chunks_coarse, s));
    MAG_TRY(plan_alloc(pl, &pl->big_stats, 3, s));
    // the bucket offsets of each batch, kept from the symbolic pass for the
    // numeric pass (the outer-product histogram is the same in both)
    pl->coarse_offs_at.assign(1, 0);
    for (size_t bi = 0; bi + 1 < pl->coarse_batches.size(); ++bi) {
      const int64_t rows = pl->coarse_batches[bi + 1] - pl->coarse_batches[bi];
      pl->coarse_offs_at.push_back(pl->coarse_offs_at.back() + rows * pl->n_chunks_coarse + 1);
    }
    MAG_TRY(plan_alloc(pl, &pl->coarse_offs, (size_t)pl->coarse_offs_at.back() + 1, s));
    CUDA_TRY(cudaMemsetAsync(pl->big_stats, 0, 3 * sizeof(unsigned long long), s));
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  return MAGNUS_OK;
}

int magnus_plan(magnus_plan_t* plan, const magnus_csr_t* A, const magnus_csr_t* B,
                const magnus_params_t* params, void* stream) {
  if (!plan) return MAGNUS_INVALID_ARG;
  *plan = nullptr;
  MAG_TRY(check_csr(A));
  MAG_TRY(check_csr(B));
  if (A->n_cols != B->n_rows) return MAGNUS_INVALID_ARG;
  if (A->nnz > 0 && B->n_rows == 0) return MAGNUS_INVALID_ARG;
  // the segment table keeps B row starts in SEG_BS_BITS bits
  if (B->nnz >= ((int64_t)1 << SEG_BS_BITS)) return MAGNUS_INDEX_OVERFLOW;
  cudaStream_t s = (cudaStream_t)stream;
  magnus_plan_t pl = new (std::nothrow) magnus_plan_s();
  if (!pl) return MAGNUS_OUT_OF_MEMORY;
  pl->last_stream = s;
  int st = plan_impl(pl, A, B, params, s);
  if (st != MAGNUS_OK) {
    magnus_free(pl);
    return st;
  }
  *plan = pl;
  return MAGNUS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Scratch of one phase call.  Every device buffer a symbolic or numeric call
// needs beyond the plan's own arrays is carved from one region: either the
// caller's workspace or one stream-ordered allocation freed at the end of
// the call.  The same carving, run without a base, measures the region
// (magnus_workspace_size).  The categories run one after another on the
// call's stream, so the fine level, the coarse level and the C.rowPtr scan
// reuse the same bytes.
namespace {

struct Arena {
  unsigned char* base = nullptr;  // NULL: measure only
  size_t cap = 0, off = 0, peak = 0;
  bool overflow = false;
  template <typename T>
  T* get(size_t count) {
    const size_t a = (off + 255) & ~(size_t)255;
    off = a + (count ? count : 1) * sizeof(T);
    if (off > peak) peak = off;
    if (!base) return nullptr;
    if (off > cap) {
      overflow = true;
      return nullptr;
    }
    return reinterpret_cast<T*>(base + a);
  }
};

// Coarse batches [b0, b1) of the coarse list, with the staging maxima.
struct CoarseSizes {
  int64_t maxP = 0, maxNnz = 0, maxRows = 0;
};

CoarseSizes coarse_sizes(magnus_plan_t pl) {
  CoarseSizes z;
  const size_t nbat = pl->coarse_batches.empty() ? 0 : pl->coarse_batches.size() - 1;
  for (size_t bi = 0; bi < nbat; ++bi) {
    int64_t p = 0, q = 0;
    for (int64_t i = pl->coarse_batches[bi]; i < pl->coarse_batches[bi + 1]; ++i) {
      p += pl->coarse_P[i];
      q += pl->coarse_nnz[i];
    }
    z.maxP = std::max(z.maxP, p);
    z.maxNnz = std::max(z.maxNnz, q);
    z.maxRows = std::max(z.maxRows, pl->coarse_batches[bi + 1] - pl->coarse_batches[bi]);
  }
  return z;
}

// The fine rows of a phase stage their products unless the symbolic pass
// counts them directly (one bitmap over a small, dense enough column range;
// k_fine_rows applies the same test).
bool fine_needs_staging(magnus_plan_t pl, bool numeric) {
  if (numeric) return !pl->fine_rows.empty();
  for (size_t i = 0; i < pl->fine_rows.size(); ++i) {
    const int64_t range = (int64_t)pl->fine_hi[i] - pl->fine_lo[i] + 1;
    if (!(range <= ((int64_t)1 << 19) && ((range + 31) >> 5) <= 4 * pl->fine_P[i])) return true;
  }
  return false;
}

struct PhaseScratch {
  int64_t* bounds = nullptr;      // row range: per bin [begin, end) of the range's rows
  int32_t* fine_sub = nullptr;    // row range: the range's fine rows (heaviest first)
  int64_t* fine_sub_P = nullptr;
  int32_t* queue = nullptr;       // fine: row counter
  int32_t* scol = nullptr;        // fine: staging slabs
  double* sval = nullptr;
  CoarseArgs co{};                // coarse: scratch pointers
  int64_t* scan_tmp = nullptr;    // symbolic: C.rowPtr scan
};

// Carves (or, with ar.base == NULL, measures) the scratch of one phase call.
void carve_phase(magnus_plan_t pl, bool numeric, bool rows_mode, Arena& ar, PhaseScratch& ps) {
  const int64_t nfine = (int64_t)pl->fine_rows.size();
  if (rows_mode) {
    ps.bounds = ar.get<int64_t>(2 * NUM_BINS);
    if (nfine > 0) {
      ps.fine_sub = ar.get<int32_t>((size_t)nfine);
      ps.fine_sub_P = ar.get<int64_t>((size_t)nfine);
    }
  }
  const size_t shared_start = ar.off;
  // fine level
  if (nfine > 0) {
    ps.queue = ar.get<int32_t>(1);
    if (fine_needs_staging(pl, numeric)) {
      const size_t grid = (size_t)(numeric ? pl->fine_grid_num : pl->fine_grid_sym);
      ps.scol = ar.get<int32_t>(grid * (size_t)pl->fine_slab);
      if (numeric) ps.sval = ar.get<double>(grid * (size_t)pl->fine_slab);
    }
  }
  // coarse level (reuses the fine level's bytes)
  ar.off = shared_start;
  if (!pl->coarse_batches.empty()) {
    const CoarseSizes z = coarse_sizes(pl);
    const int64_t nB = pl->B.n_rows;
    const int64_t nbk = z.maxRows * pl->n_chunks_coarse;
    CoarseArgs& a = ps.co;
    if (!pl->coarse_rowwise) {  // the outer product's A^CSC and work offsets
      a.col_cnt = ar.get<int32_t>((size_t)nB + 1);
      a.col_ptr = ar.get<int64_t>((size_t)nB + 1);
      a.csc_row = ar.get<int32_t>((size_t)z.maxNnz);
      if (numeric) a.csc_val = ar.get<double>((size_t)z.maxNnz);
      a.rows_b = ar.get<int32_t>((size_t)nB + 1);
      a.item_off = ar.get<int64_t>((size_t)nB + 1);
    }
    a.n_rows_b = ar.get<int32_t>(2);
    a.counts = ar.get<int64_t>((size_t)nbk + 1);
    a.cursor = ar.get<unsigned long long>((size_t)nbk);
    const bool fine_inside = pl->shift_coarse > 13;
    // staging, padded so that the bucket sort's bulk copies may round a
    // bucket's window out to 16-byte boundaries
    a.chunk_col = ar.get<int32_t>((size_t)z.maxP + 8);
    if (fine_inside) a.fine_col = ar.get<int32_t>((size_t)z.maxP);
    if (numeric) {
      a.chunk_val = ar.get<double>((size_t)z.maxP + 4);
      if (fine_inside) a.fine_val = ar.get<double>((size_t)z.maxP);
      a.bucket_out = ar.get<int64_t>((size_t)nbk);
    }
    a.scan_tmp = ar.get<int64_t>((size_t)scan_tmp_elems(std::max<int64_t>(nB, nbk)) + 2);
    a.big_list = ar.get<BigBucket>((size_t)nbk);
    a.n_big = ar.get<int32_t>(2);
  }
  // the symbolic pass's C.rowPtr scan (after every category)
  ar.off = shared_start;
  if (!numeric) ps.scan_tmp = ar.get<int64_t>((size_t)scan_tmp_elems(pl->A.n_rows) + 2);
  ar.off = ar.peak;
}

size_t phase_bytes(magnus_plan_t pl, bool numeric, bool rows_mode) {
  Arena ar;
  PhaseScratch ps;
  carve_phase(pl, numeric, rows_mode, ar, ps);
  return ar.peak;
}

// The region of one call: the caller's workspace, or one stream-ordered
// allocation released (stream-ordered) when the call returns.
struct PhaseRegion {
  cudaStream_t s = nullptr;
  void* owned = nullptr;
  ~PhaseRegion() {
    if (owned) cudaFreeAsync(owned, s);
  }
};

int open_region(magnus_plan_t pl, bool numeric, bool rows_mode, void* ws, size_t ws_bytes,
                cudaStream_t s, PhaseRegion& reg, PhaseScratch& ps) {
  const size_t need = phase_bytes(pl, numeric, rows_mode);
  Arena ar;
  if (ws) {
    if (ws_bytes < need) return MAGNUS_WORKSPACE_TOO_SMALL;
    if (((uintptr_t)ws & 255) != 0) return MAGNUS_INVALID_ARG;
    ar.base = static_cast<unsigned char*>(ws);
    ar.cap = ws_bytes;
  } else {
    reg.s = s;
    MAG_TRY(dev_alloc(&reg.owned, need, s));
    ar.base = static_cast<unsigned char*>(reg.owned);
    ar.cap = need;
  }
  carve_phase(pl, numeric, rows_mode, ar, ps);
  return ar.overflow ? MAGNUS_WORKSPACE_TOO_SMALL : MAGNUS_OK;
}

}  // namespace


// Runs one phase (symbolic or numeric) over every category.  With a row
// range (numeric only) just the rows [r0, r1) are computed, and their
// entries are written from c_col / c_val[0] on (offsets less
// C.rowPtr[r0]).
struct RowRange {
  bool on = false;
  int64_t r0 = 0, r1 = 0;
};

static int run_phase(magnus_plan_t pl, bool numeric, const RowRange& rr, int64_t* out_cnt,
                     const int64_t* c_rp, int32_t* c_col, double* c_val, const PhaseScratch& ps,
                     cudaStream_t s) {
  Csr A = pl->A, B = pl->B;
  const int st_base = numeric ? MAGNUS_STAGE_NUM_SORT : MAGNUS_STAGE_SYM_SORT;
  const int64_t* c_base = rr.on ? c_rp + rr.r0 : nullptr;
  if (rr.on) {
    BinOffsets bo;
    for (int b = 0; b <= NUM_BINS; ++b) bo.v[b] = pl->bin_off[b];
    CUDA_TRY(launch_bin_bounds(pl->rows_sorted, bo, rr.r0, rr.r1, ps.bounds, s));
  }
  // sort rows
  {
    StageTimer tm(pl, st_base + 0, s);
    for (int b = BIN_SORT32; b <= BIN_SORT1024; ++b) {
      SortArgs a{};
      a.A = A;
      a.B = B;
      a.desc = pl->desc + pl->bin_off[b];
      a.seg = pl->seg;
      a.n_rows = pl->bin_off[b + 1] - pl->bin_off[b];
      a.key32 = pl->key32[b];
      a.perm = pl->perm + pl->perm_off[b];
      a.perm2 = pl->perm2;
      a.perm2_off = (pl->perm2_off && b >= BIN_SORT512) ? pl->perm2_off + (pl->bin_off[b] - pl->bin_off[BIN_SORT512]) : nullptr;
      a.out_cnt = out_cnt;
      a.c_rp = c_rp;
      a.c_col = c_col;
      a.c_val = c_val;
      a.range = rr.on ? ps.bounds + 2 * b : nullptr;
      a.c_base = c_base;
      a.block_warps = pl->params.sort_block_warps;
      if (b <= BIN_SORT256) CUDA_TRY(launch_sort_rows(b, numeric, a, pl->num_sms, s));
      else CUDA_TRY(launch_sort_rows_block(b, numeric, a, pl->num_sms, s));
    }
  }
  // dense rows
  {
    StageTimer tm(pl, st_base + 1, s);
    DenseArgs a{};
    a.A = A;
    a.B = B;
    a.rows = pl->rows_sorted + pl->bin_off[BIN_DENSE];
    a.n_rows = pl->bin_off[BIN_DENSE + 1] - pl->bin_off[BIN_DENSE];
    a.lo = pl->lo;
    a.hi = pl->hi;
    a.dense_cols = pl->dense_cols;
    a.out_cnt = out_cnt;
    a.c_rp = c_rp;
    a.c_col = c_col;
    a.c_val = c_val;
    a.range = rr.on ? ps.bounds + 2 * BIN_DENSE : nullptr;
    a.c_base = c_base;
    CUDA_TRY(launch_dense_rows(numeric, a, pl->num_sms, s));
  }
  int64_t staged = 0;
  // fine rows: one persistent launch; each block stages its row in its slab
  if (!pl->fine_rows.empty()) {
    StageTimer tm(pl, st_base + 2, s);
    const int32_t* rows = pl->fine_rows_d;
    const int64_t* rows_P = pl->fine_P_d;
    int64_t nf = (int64_t)pl->fine_rows.size();
    if (rr.on) {
      // the range's fine rows, still heaviest first
      std::vector<int32_t> sub;
      std::vector<int64_t> subP;
      for (size_t i = 0; i < pl->fine_rows.size(); ++i) {
        if (pl->fine_rows[i] >= rr.r0 && pl->fine_rows[i] < rr.r1) {
          sub.push_back(pl->fine_rows[i]);
          subP.push_back(pl->fine_P[i]);
        }
      }
      nf = (int64_t)sub.size();
      if (nf > 0) {
        CUDA_TRY(cudaMemcpyAsync(ps.fine_sub, sub.data(), sub.size() * 4, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(ps.fine_sub_P, subP.data(), subP.size() * 8,
                                 cudaMemcpyHostToDevice, s));
        // pageable sources: the copies have left the vectors when the calls return
      }
      rows = ps.fine_sub;
      rows_P = ps.fine_sub_P;
      for (int64_t p : subP) staged += p;
    } else if (numeric) {
      for (int64_t p : pl->fine_P) staged += p;
    }
    if (nf > 0) {
      const int shift = numeric ? pl->shift_fine : pl->shift_fine_sym;
      const int grid = numeric ? pl->fine_grid_num : pl->fine_grid_sym;
      CUDA_TRY(cudaMemsetAsync(ps.queue, 0, sizeof(int32_t), s));
      if (ps.scol)
        pl->scratch_used = std::max<int64_t>(pl->scratch_used,
                                             (int64_t)grid * pl->fine_slab * (numeric ? 12 : 4));
      FineArgs a{};
      a.A = A;
      a.B = B;
      a.rows = rows;
      a.n_rows = nf;
      a.slab_elems = pl->fine_slab;
      a.queue = ps.queue;
      a.row_products = rows_P;
      a.lo = pl->lo;
      a.hi = pl->hi;
      a.shift = shift;
      a.dense_chunk_threshold = pl->dthr;
      a.hash = numeric ? pl->hash : 0;
      a.stage_col = ps.scol;
      a.stage_val = ps.sval;
      a.out_cnt = out_cnt;
      a.c_rp = c_rp;
      a.c_col = c_col;
      a.c_val = c_val;
      a.c_base = c_base;
      CUDA_TRY(launch_fine_rows(numeric, a, grid, s));
    }
  }
  // coarse rows, batch by batch (a row range runs the part of each batch
  // inside it)
  {
    StageTimer tm(pl, st_base + 3, s);
    const size_t nbat = pl->coarse_batches.empty() ? 0 : pl->coarse_batches.size() - 1;
    if (nbat > 0) {
      int64_t i0 = 0, i1 = (int64_t)pl->coarse_rows.size();
      if (rr.on) {
        // the coarse list is ascending by row (bin order); rows fit int32
        i0 = std::lower_bound(pl->coarse_rows.begin(), pl->coarse_rows.end(), (int32_t)rr.r0) -
             pl->coarse_rows.begin();
        i1 = std::lower_bound(pl->coarse_rows.begin(), pl->coarse_rows.end(), (int32_t)rr.r1) -
             pl->coarse_rows.begin();
      }
      CoarseArgs a = ps.co;
      a.A = A;
      a.B = B;
      a.shift_coarse = pl->shift_coarse;
      a.n_chunks = pl->n_chunks_coarse;
      a.shift_fine = pl->shift_fine;
      a.dense_chunk_threshold = pl->dthr;
      a.hash = numeric ? pl->hash : 0;
      a.num_sms = pl->num_sms;
      const CoarseSizes z = coarse_sizes(pl);
      const bool fine_inside = pl->shift_coarse > 13;
      pl->scratch_used = std::max<int64_t>(pl->scratch_used,
                                           z.maxP * (numeric ? 12 : 4) * (fine_inside ? 2 : 1));
      a.bucket_cnt = pl->bucket_cnt;
      if (numeric) {
        a.big_stats = pl->big_stats;
        CUDA_TRY(cudaMemsetAsync(pl->big_stats, 0, 3 * sizeof(unsigned long long), s));
      }
      const int ph = numeric ? 1 : 0;
      pl->big_ev_used[ph] = 0;
      if (pl->timing) {
        while (pl->big_ev[ph].size() < 2 * nbat) {
          cudaEvent_t e;
          CUDA_TRY(cudaEventCreate(&e));
          pl->big_ev[ph].push_back(e);
        }
      }
      a.out_cnt = out_cnt;
      a.c_rp = c_rp;
      a.c_col = c_col;
      a.c_val = c_val;
      a.c_base = c_base;
      int used = 0;
      for (size_t bi = 0; bi < nbat; ++bi) {
        const int64_t b0 = pl->coarse_batches[bi], b1 = pl->coarse_batches[bi + 1];
        const int64_t r0 = std::max(b0, i0), r1 = std::min(b1, i1);
        if (r0 >= r1) continue;
        a.rows = pl->coarse_rows_d + r0;
        a.n_rows = r1 - r0;
        a.list_base = r0;
        int64_t nz = 0;
        for (int64_t i = r0; i < r1; ++i) {
          nz += pl->coarse_nnz[i];
          if (numeric) staged += pl->coarse_P[i];
        }
        a.nnz_batch = nz;
        a.seg = pl->seg;
        // automatic: the block sort for buckets of chunks wider than the block
        // dense accumulator (sparse buckets, e.g. the massive nonsquare
        // workload); the dense accumulator for narrower, denser chunks (its
        // bitmap is cheap there, and the sort would pad small buckets)
        a.bucket_sort = pl->params.coarse_bucket_sort > 0 ||
                        (pl->params.coarse_bucket_sort == 0 && pl->shift_coarse > 13);
        if (pl->coarse_rowwise) {
          a.items = pl->coarse_items_d + pl->coarse_item_first[r0];
          a.n_items = (int32_t)(pl->coarse_item_first[r1] - pl->coarse_item_first[r0]);
          a.item_ctr = a.n_rows_b;
        }
        // the bucket offsets kept by the symbolic pass cover whole batches
        const bool whole = r0 == b0 && r1 == b1;
        a.saved_offs = (pl->coarse_offs && whole) ? pl->coarse_offs + pl->coarse_offs_at[bi] : nullptr;
        if (pl->timing) {
          a.big_ev0 = pl->big_ev[ph][2 * used];
          a.big_ev1 = pl->big_ev[ph][2 * used + 1];
          pl->big_ev_used[ph] = ++used;
        }
        CUDA_TRY(run_coarse_batch(numeric, a, s));
      }
    }
  }
  if (numeric) pl->staged_numeric = staged;
  return MAGNUS_OK;
}

static int symbolic_impl(magnus_plan_t pl, int64_t* c_row_ptr, int64_t* nnz_c, void* ws,
                         size_t ws_bytes, cudaStream_t s) {
  pl->last_stream = s;
  pl->symbolic_done = false;
  for (int i = 0; i < MAGNUS_STAGE_COUNT; ++i) pl->ev_used[i] = false;
  pl->big_ev_used[0] = pl->big_ev_used[1] = 0;
  const int64_t n = pl->A.n_rows;
  PhaseRegion reg;
  PhaseScratch ps;
  MAG_TRY(open_region(pl, false, false, ws, ws_bytes, s, reg, ps));
  CUDA_TRY(cudaMemsetAsync(c_row_ptr, 0, (size_t)(n + 1) * sizeof(int64_t), s));
  MAG_TRY(run_phase(pl, false, RowRange{}, c_row_ptr, nullptr, nullptr, nullptr, ps, s));
  {
    StageTimer tm(pl, MAGNUS_STAGE_SYM_SCAN, s);
    CUDA_TRY(launch_exclusive_scan_i64(c_row_ptr, n, ps.scan_tmp, s));
  }
  int64_t h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, c_row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  int timed_out = 0;
  CUDA_TRY(wait_timeout_take(&timed_out, s));  // synchronises the stream
  if (timed_out) return MAGNUS_TIMEOUT;
  *nnz_c = h;
  pl->nnz_c = h;
  pl->symbolic_done = true;
  return MAGNUS_OK;
}

static int numeric_impl(magnus_plan_t pl, const RowRange& rr, const double* a_val,
                        const double* b_val, const int64_t* c_row_ptr, int32_t* c_col,
                        double* c_val, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (!pl || !c_row_ptr) return MAGNUS_INVALID_ARG;
  if (!pl->symbolic_done) return MAGNUS_NOT_SYMBOLIC;
  if ((pl->A.nnz > 0 && !a_val) || (pl->B.nnz > 0 && !b_val)) return MAGNUS_INVALID_ARG;
  if (pl->nnz_c > 0 && (!c_col || !c_val)) return MAGNUS_INVALID_ARG;
  pl->last_stream = s;
  for (int i = MAGNUS_STAGE_NUM_SORT; i <= MAGNUS_STAGE_NUM_COARSE; ++i) pl->ev_used[i] = false;
  pl->big_ev_used[1] = 0;
  pl->A.val = a_val;
  pl->B.val = b_val;
  auto body = [&]() -> int {
    PhaseRegion reg;
    PhaseScratch ps;
    MAG_TRY(open_region(pl, true, rr.on, ws, ws_bytes, s, reg, ps));
    return run_phase(pl, true, rr, nullptr, c_row_ptr, c_col, c_val, ps, s);
  };
  if (!rr.on && pl->use_graph && !pl->timing && s != nullptr) {
    const void* key[6] = {a_val, b_val, c_row_ptr, c_col, c_val, ws};
    return pl->graph.run(key, 6, s, body);
  }
  return body();
}

extern "C" {

int magnus_symbolic(magnus_plan_t pl, int64_t* c_row_ptr, int64_t* nnz_c, void* stream) {
  if (!pl || !c_row_ptr || !nnz_c) return MAGNUS_INVALID_ARG;
  return symbolic_impl(pl, c_row_ptr, nnz_c, nullptr, 0, (cudaStream_t)stream);
}

int magnus_symbolic_ws(magnus_plan_t pl, int64_t* c_row_ptr, int64_t* nnz_c, void* workspace,
                       size_t workspace_bytes, void* stream) {
  if (!pl || !c_row_ptr || !nnz_c || !workspace) return MAGNUS_INVALID_ARG;
  return symbolic_impl(pl, c_row_ptr, nnz_c, workspace, workspace_bytes, (cudaStream_t)stream);
}

int magnus_numeric(magnus_plan_t pl, const double* a_val, const double* b_val,
                   const int64_t* c_row_ptr, int32_t* c_col, double* c_val, void* stream) {
  return numeric_impl(pl, RowRange{}, a_val, b_val, c_row_ptr, c_col, c_val, nullptr, 0,
                      (cudaStream_t)stream);
}

int magnus_numeric_ws(magnus_plan_t pl, const double* a_val, const double* b_val,
                      const int64_t* c_row_ptr, int32_t* c_col, double* c_val, void* workspace,
                      size_t workspace_bytes, void* stream) {
  if (!workspace) return MAGNUS_INVALID_ARG;
  return numeric_impl(pl, RowRange{}, a_val, b_val, c_row_ptr, c_col, c_val, workspace,
                      workspace_bytes, (cudaStream_t)stream);
}

int magnus_numeric_rows(magnus_plan_t pl, int64_t row_begin, int64_t row_end, const double* a_val,
                        const double* b_val, const int64_t* c_row_ptr, int32_t* c_col,
                        double* c_val, void* workspace, size_t workspace_bytes, void* stream) {
  if (!pl) return MAGNUS_INVALID_ARG;
  if (row_begin < 0 || row_end < row_begin || row_end > pl->A.n_rows) return MAGNUS_INVALID_ARG;
  if (!pl->symbolic_done) return MAGNUS_NOT_SYMBOLIC;
  if (row_begin == row_end) return MAGNUS_OK;
  RowRange rr;
  rr.on = true;
  rr.r0 = row_begin;
  rr.r1 = row_end;
  // the slab's entries may be fewer than nnz(C): only NULL outputs of an
  // empty C are accepted, as for magnus_numeric
  return numeric_impl(pl, rr, a_val, b_val, c_row_ptr, c_col, c_val, workspace, workspace_bytes,
                      (cudaStream_t)stream);
}

int magnus_wait_selftest(int64_t limit_cycles, void* stream) {
  if (limit_cycles <= 0 || limit_cycles > ((int64_t)1 << 31)) return MAGNUS_INVALID_ARG;
  CUDA_TRY(launch_wait_selftest((long long)limit_cycles, (cudaStream_t)stream));
  return MAGNUS_OK;
}

int magnus_device_status(void* stream) {
  int timed_out = 0;
  CUDA_TRY(wait_timeout_take(&timed_out, (cudaStream_t)stream));
  return timed_out ? MAGNUS_TIMEOUT : MAGNUS_OK;
}

int magnus_workspace_size(magnus_plan_t pl, size_t* bytes) {
  if (!pl || !bytes) return MAGNUS_INVALID_ARG;
  size_t b = phase_bytes(pl, false, false);
  b = std::max(b, phase_bytes(pl, true, false));
  b = std::max(b, phase_bytes(pl, true, true));
  *bytes = b;
  return MAGNUS_OK;
}

}  // extern "C"


extern "C" {

// ---------------------------------------------------------------------------
// Allocation-free numeric phase: the fine-level staging lives in this static
// device array instead of the stream-ordered pool.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MAGNUS_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch on the current device (host code may
// not use the symbol itself as a device pointer).  Looked up on every call:
// the lookup allocates nothing, and a cached address would dangle after the
// device's context is destroyed and created again.
static int noalloc_scratch_address(unsigned char** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                     "cudaGetSymbolAddress(g_noalloc_scratch)");
  *out = reinterpret_cast<unsigned char*>(p);
  return MAGNUS_OK;
}

// Fine blocks of the allocation-free numeric phase: as many staging slabs as
// fit the fixed array (after its 512-byte counter area), at most one resident
// wave; 0 without fine rows, -1 when the plan is refused.
static int noalloc_fine_grid(magnus_plan_t pl) {
  if (!pl->coarse_rows.empty()) return -1;
  if (pl->fine_rows.empty()) return 0;
  const size_t slab_bytes = (((size_t)pl->fine_slab * 12) + 255) & ~(size_t)255;
  const size_t avail = MAGNUS_NOALLOC_SCRATCH_BYTES - 512;
  if (slab_bytes > avail) return -1;
  return (int)std::min<size_t>((size_t)pl->fine_grid_num, avail / slab_bytes);
}

int magnus_numeric_noalloc(magnus_plan_t pl, const double* a_val, const double* b_val,
                           const int64_t* c_row_ptr, int32_t* c_col, double* c_val, void* stream) {
  if (!pl || !c_row_ptr) return MAGNUS_INVALID_ARG;
  if (!pl->symbolic_done) return MAGNUS_NOT_SYMBOLIC;
  if ((pl->A.nnz > 0 && !a_val) || (pl->B.nnz > 0 && !b_val)) return MAGNUS_INVALID_ARG;
  if (pl->nnz_c > 0 && (!c_col || !c_val)) return MAGNUS_INVALID_ARG;
  // The fine kernel stages one row per block in a slab of fine_slab products;
  // the fixed buffer holds the row counter and as many slabs as fit, and the
  // persistent grid is limited to that many blocks.
  const int grid = noalloc_fine_grid(pl);
  if (grid < 0) return MAGNUS_SCRATCH_LIMIT;
  const int shift = pl->shift_fine;
  unsigned char* scratch = nullptr;
  MAG_TRY(noalloc_scratch_address(&scratch));
  cudaStream_t s = (cudaStream_t)stream;
  pl->last_stream = s;
  Csr A = pl->A, B = pl->B;
  A.val = a_val;
  B.val = b_val;
  for (int b = BIN_SORT32; b <= BIN_SORT1024; ++b) {
    SortArgs a{};
    a.A = A;
    a.B = B;
    a.desc = pl->desc + pl->bin_off[b];
    a.seg = pl->seg;
    a.n_rows = pl->bin_off[b + 1] - pl->bin_off[b];
    a.key32 = pl->key32[b];
    a.perm = pl->perm + pl->perm_off[b];
    a.perm2 = pl->perm2;
    a.perm2_off = (pl->perm2_off && b >= BIN_SORT512) ? pl->perm2_off + (pl->bin_off[b] - pl->bin_off[BIN_SORT512]) : nullptr;
    a.c_rp = c_row_ptr;
    a.c_col = c_col;
    a.c_val = c_val;
    a.block_warps = pl->params.sort_block_warps;
    if (b <= BIN_SORT256) CUDA_TRY(launch_sort_rows(b, true, a, pl->num_sms, s));
    else CUDA_TRY(launch_sort_rows_block(b, true, a, pl->num_sms, s));
  }
  {
    DenseArgs a{};
    a.A = A;
    a.B = B;
    a.rows = pl->rows_sorted + pl->bin_off[BIN_DENSE];
    a.n_rows = pl->bin_off[BIN_DENSE + 1] - pl->bin_off[BIN_DENSE];
    a.lo = pl->lo;
    a.hi = pl->hi;
    a.dense_cols = pl->dense_cols;
    a.c_rp = c_row_ptr;
    a.c_col = c_col;
    a.c_val = c_val;
    CUDA_TRY(launch_dense_rows(true, a, pl->num_sms, s));
  }
  if (!pl->fine_rows.empty()) {
    // byte 0..255: row counter (cleared here: every call starts from row 0);
    // then grid slabs, columns of all slabs first, values after them
    int32_t* queue = reinterpret_cast<int32_t*>(scratch);
    CUDA_TRY(cudaMemsetAsync(queue, 0, sizeof(int32_t), s));
    unsigned char* base = scratch + 256;
    const size_t col_bytes = (((size_t)grid * pl->fine_slab * 4) + 255) & ~(size_t)255;
    FineArgs a{};
    a.A = A;
    a.B = B;
    a.rows = pl->fine_rows_d;
    a.n_rows = (int64_t)pl->fine_rows.size();
    a.slab_elems = pl->fine_slab;
    a.queue = queue;
    a.row_products = pl->fine_P_d;
    a.lo = pl->lo;
    a.hi = pl->hi;
    a.shift = shift;
    a.dense_chunk_threshold = pl->dthr;
    a.hash = pl->hash;
    a.stage_col = reinterpret_cast<int32_t*>(base);
    a.stage_val = reinterpret_cast<double*>(base + col_bytes);
    a.c_rp = c_row_ptr;
    a.c_col = c_col;
    a.c_val = c_val;
    CUDA_TRY(launch_fine_rows(true, a, grid, s));
  }
  return MAGNUS_OK;
}

int magnus_plan_info(magnus_plan_t pl, magnus_plan_info_t* info) {
  if (!pl || !info) return MAGNUS_INVALID_ARG;
  memset(info, 0, sizeof(*info));
  info->n_rows = pl->A.n_rows;
  info->n_cols = pl->B.n_cols;
  info->n_interprod = pl->n_interprod;
  info->max_row_products = pl->max_P;
  info->nnz_c = pl->symbolic_done ? pl->nnz_c : -1;
  info->rows_empty = pl->bin_off[BIN_EMPTY + 1] - pl->bin_off[BIN_EMPTY];
  for (int c = 0; c < 4; ++c) {
    info->rows_per_category[c] = pl->rows_cat[c];
    info->products_per_category[c] = pl->prods_cat[c];
  }
  info->staged_products_numeric = pl->staged_numeric;
  info->scratch_bytes = pl->scratch_used;
  info->sort_threshold = pl->sort_T;
  info->chunk_len_fine_log2 = pl->shift_fine;
  info->chunk_len_fine_sym_log2 = pl->shift_fine_sym;
  info->chunk_len_coarse_log2 = pl->shift_coarse;
  info->n_chunks_coarse = pl->n_chunks_coarse;
  info->dense_cols = pl->dense_cols;
  info->dense_chunk_threshold = pl->dthr;
  info->key_bits32 = pl->key32[BIN_SORT256];
  info->n_batches_fine = pl->fine_rows.empty() ? 0 : 1;
  info->n_batches_coarse = pl->coarse_batches.empty() ? 0 : (int)pl->coarse_batches.size() - 1;
  info->plan_bytes = pl->owned_bytes;
  {
    size_t ws = 0;
    magnus_workspace_size(pl, &ws);
    info->workspace_bytes = (int64_t)ws;
  }
  info->noalloc_fine_blocks = noalloc_fine_grid(pl);
  if (pl->big_stats) {
    unsigned long long h[3] = {0, 0, 0};
    CUDA_TRY(cudaMemcpy(h, pl->big_stats, sizeof(h), cudaMemcpyDeviceToHost));
    info->coarse_dense_products = (int64_t)h[0];
    info->coarse_dense_nnz = (int64_t)h[1];
    info->coarse_dense_buckets = (int64_t)h[2];
  }
  return MAGNUS_OK;
}

int magnus_enable_timing(magnus_plan_t pl, int enable) {
  if (!pl) return MAGNUS_INVALID_ARG;
  if (enable && !pl->ev[0]) {
    for (int i = 0; i < 2 * MAGNUS_STAGE_COUNT; ++i) CUDA_TRY(cudaEventCreate(&pl->ev[i]));
  }
  pl->timing = enable != 0;
  return MAGNUS_OK;
}

int magnus_stage_times(magnus_plan_t pl, double* ms, int n) {
  if (!pl || !ms || n < 0) return MAGNUS_INVALID_ARG;
  for (int i = 0; i < n && i < MAGNUS_STAGE_COUNT; ++i) {
    ms[i] = 0.0;
    if (i == MAGNUS_STAGE_SYM_COARSE_BIG || i == MAGNUS_STAGE_NUM_COARSE_BIG) {
      const int ph = i == MAGNUS_STAGE_NUM_COARSE_BIG ? 1 : 0;
      if (!pl->timing) continue;
      for (int b = 0; b < pl->big_ev_used[ph]; ++b) {
        CUDA_TRY(cudaEventSynchronize(pl->big_ev[ph][2 * b + 1]));
        float f = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&f, pl->big_ev[ph][2 * b], pl->big_ev[ph][2 * b + 1]));
        ms[i] += f;
      }
      continue;
    }
    if (pl->timing && pl->ev_used[i]) {
      CUDA_TRY(cudaEventSynchronize(pl->ev[2 * i + 1]));
      float f = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&f, pl->ev[2 * i], pl->ev[2 * i + 1]));
      ms[i] = f;
    }
  }
  return MAGNUS_OK;
}

}  // extern "C"
