// Internal declarations shared by the host orchestration (magnus_api.cu) and
// the kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/magnus.h"

namespace magnus {

// Row bins.  Sort rows are split by capacity (32 * E products, E = 1,2,4,8)
// so each warp kernel sorts in registers with a fixed network size; rows of
// 257..1024 products (bins SORT512, SORT1024) sort in one warp and replay in
// one warp (SORT512) or one thread block (SORT1024).
enum Bin : int {
  BIN_EMPTY = 0,
  BIN_SORT32 = 1,
  BIN_SORT64 = 2,
  BIN_SORT128 = 3,
  BIN_SORT256 = 4,
  BIN_SORT512 = 5,
  BIN_SORT1024 = 6,
  BIN_DENSE = 7,
  BIN_FINE = 8,
  BIN_COARSE = 9,
  NUM_BINS = 10
};

constexpr int SORT_MAX = 256;        // largest warp sort-row capacity
constexpr int SORT_BLOCK_MAX = 1024; // largest block sort-row capacity
constexpr int DENSE_NT = 256;        // threads of the dense/fine block kernels
constexpr int FINE_MAX_CHUNKS = 4096;  // fine chunks one block can bookkeep in smem

// Parameters a kernel needs to categorise a row (Section 3.1).
struct CatParams {
  int32_t sort_threshold;     // sort iff P < sort_threshold
  int32_t force;              // -1 or a magnus_category
  int32_t dense_cols;         // dense iff column range <= dense_cols
  int32_t fine_shift;         // fine chunk = col >> fine_shift (numeric)
  int32_t fine_max_chunks;    // fine iff the row spans <= this many fine chunks
  int64_t fine_max_products;  // ... and its products fit one block's staging slab
  int32_t prefer_fine;        // automatic mode: fine level (1) or coarse level (0) for
                              // rows wider than the dense accumulator
  int32_t wide_sort_max;      // automatic mode: rows wider than the dense accumulator
                              // with at most this many products use the sort bins
};

struct Csr {
  int64_t n_rows, n_cols, nnz;
  const int64_t* rp;
  const int32_t* col;
  const double* val;
};

// Kernel launchers (defined in the kernel translation units).  All return
// cudaGetLastError() of the launch.
cudaError_t launch_validate(const Csr& M, int* d_flag, cudaStream_t s);
cudaError_t launch_rowinfo(const Csr& A, const Csr& B, CatParams cp, int64_t* P, uint8_t* bin,
                           int32_t* lo, int32_t* hi, uint64_t* seg,
                           cudaStream_t s);

// A range and id of a listed row (16 bytes, one vector load).
struct __align__(16) RowDesc {
  int64_t as;   // A.rowPtr[row]
  int32_t na;   // nonzeros of the row of A
  int32_t row;  // row id
};
cudaError_t launch_row_desc(const int32_t* rows, int64_t n, const int64_t* a_rp, RowDesc* desc,
                            cudaStream_t s);
cudaError_t launch_bin_partition(const uint8_t* bin, int64_t n, int32_t* rows_out,
                                 int64_t* bin_counts_dev, int64_t* blk_scratch, int64_t nblk_cap,
                                 cudaStream_t s);
int64_t bin_partition_blocks(int64_t n);
// For a row range [r0, r1): per bin b, the positions [begin, end) of the
// range's rows in the bin's list, relative to the bin's first entry
// (rows_sorted is ascending within each bin).
// out: 2 * NUM_BINS int64 (device).
struct BinOffsets { int64_t v[NUM_BINS + 1]; };
cudaError_t launch_bin_bounds(const int32_t* rows_sorted, BinOffsets off, int64_t r0, int64_t r1,
                              int64_t* out, cudaStream_t s);
cudaError_t launch_gather_i64(const int64_t* src, const int32_t* idx, int64_t n, int64_t* dst,
                              cudaStream_t s);
cudaError_t launch_reduce_stats(const int64_t* P, int64_t n, int64_t* out2 /*sum,max*/,
                                cudaStream_t s);

// Device-wide exclusive scan of int64 in place: a[0..n) -> exclusive prefix,
// a[n] = total (a must hold n+1 elements).  `tmp` needs scan_tmp_elems(n).
int64_t scan_tmp_elems(int64_t n);
cudaError_t launch_exclusive_scan_i64(int64_t* a, int64_t n, int64_t* tmp, cudaStream_t s);
cudaError_t launch_scan_i32_to_i64(const int32_t* in, int64_t n, int64_t* out, int64_t* tmp,
                                   cudaStream_t s);

// Segment table entry of a nonzero of A: the start of the B row it selects
// (B.rowPtr[A.col[j]], low SEG_BS_BITS bits; B has fewer than 2^40
// nonzeros, checked by magnus_plan) and the row's length (high bits,
// saturated at 2^24 - 1: only rows of at most 1,024 products read the table,
// and their B rows are that short).
constexpr int SEG_BS_BITS = 40;
__host__ __device__ __forceinline__ uint64_t seg_pack(int64_t bs, int64_t len) {
  const int64_t l = len < ((int64_t)1 << (64 - SEG_BS_BITS)) - 1 ? len
                                                                  : ((int64_t)1 << (64 - SEG_BS_BITS)) - 1;
  return (uint64_t)bs | ((uint64_t)l << SEG_BS_BITS);
}
__host__ __device__ __forceinline__ int64_t seg_start(uint64_t x) {
  return (int64_t)(x & ((1ull << SEG_BS_BITS) - 1));
}
__host__ __device__ __forceinline__ int seg_length(uint64_t x) { return (int)(x >> SEG_BS_BITS); }

// Sort rows (warp per row).  cnt_out: per-row count (symbolic) written at
// c_row_ptr-like array position row (count stored in out_cnt[row]).
struct SortArgs {
  Csr A, B;
  const RowDesc* desc;  // descriptors of the bin's rows
  const uint64_t* seg;    // per nonzero of A: its B row (seg_pack)
  int64_t n_rows;
  int key32;            // 1: (col << slot_bits | slot) fits 32 bits
  uint8_t* perm;        // sorted slot order, 32*E bytes per listed row
                        // (written by the symbolic pass, replayed by the numeric pass)
  uint16_t* perm2;      // bins SORT512/1024: sorted slot order, P_i entries per row at
  const int64_t* perm2_off;  // perm2 + perm2_off[k] for the bin's k-th row
  // symbolic
  int64_t* out_cnt;     // indexed by row
  // numeric
  const int64_t* c_rp;
  int32_t* c_col;
  double* c_val;
  // numeric on a row range (magnus_numeric_rows); both NULL for the whole
  // matrix.  range: device [begin, end) of the bin's list; c_base: device
  // int64 subtracted from every output offset (C.rowPtr[row_begin]).
  const int64_t* range;
  const int64_t* c_base;
  int32_t block_warps;  // warps per block of the warp-sort kernels (0 = per phase default)
};
cudaError_t launch_sort_rows(int bin, bool numeric, const SortArgs& a, int num_sms, cudaStream_t s);
cudaError_t launch_sort_rows_block(int bin, bool numeric, const SortArgs& a, int num_sms,
                                   cudaStream_t s);

// Dense rows (block per row).
struct DenseArgs {
  Csr A, B;
  const int32_t* rows;
  int64_t n_rows;
  const int32_t* lo;   // per row (indexed by row id)
  const int32_t* hi;
  int32_t dense_cols;
  int64_t* out_cnt;
  const int64_t* c_rp;
  int32_t* c_col;
  double* c_val;
  const int64_t* range;   // as in SortArgs
  const int64_t* c_base;
};
cudaError_t launch_dense_rows(bool numeric, const DenseArgs& a, int num_sms, cudaStream_t s);

// Fine rows: a persistent grid whose blocks take rows (heaviest first) from
// a device counter; each block stages its current row in its own slab of
// slab_elems products (stage_col/stage_val + blockIdx.x * slab_elems).
struct FineArgs {
  Csr A, B;
  const int32_t* rows;      // fine rows, heaviest first
  int64_t n_rows;
  int64_t slab_elems;       // staging capacity per block (products)
  int32_t* queue;           // zeroed counter of taken rows
  const int64_t* row_products;  // P of each listed row
  const int32_t* lo;
  const int32_t* hi;
  int32_t shift;            // fine chunk shift for this phase
  int32_t dense_chunk_threshold;
  int32_t hash;             // numeric: hash-map accumulator for chunks <= 128 products
  int32_t* stage_col;
  double* stage_val;
  int64_t* out_cnt;
  const int64_t* c_rp;
  int32_t* c_col;
  double* c_val;
  const int64_t* c_base;  // as in SortArgs (the row list is already the range's)
};
cudaError_t launch_fine_rows(bool numeric, const FineArgs& a, int grid, cudaStream_t s);
// Resident blocks per SM of the fine-row kernel for a phase and chunk shift.
int fine_rows_blocks_per_sm(bool numeric, int shift, bool hybrid);

// A coarse (row, chunk) bucket too large for a warp sort, as listed by
// k_bucket_small for the large-bucket accumulators: its staged products
// [p0, p0 + n), its coarse chunk c, and `out` = its first entry in C
// (numeric; C.rowPtr of the row less the output base plus the bucket's
// offset in the row) or its index in the symbolic per-(row, chunk) counts.
struct BigBucket {
  int64_t p0;
  int64_t out;
  int32_t n;
  int32_t c;
};

// A work item of the row-wise staged coarse reorder: nonzeros
// [j0, j0 + nj) of A (nj <= CS_NJ) of the coarse row at position li of the
// coarse row list.
constexpr int CS_NJ = 256;
struct CoarseItem {
  int64_t j0;
  int32_t li;
  int32_t nj;
};
// The row-wise staged reorder keeps per-chunk counters in shared memory and
// is used up to this many coarse chunks; beyond it, the outer product.
constexpr int CS_MAX_CHUNKS = 512;

// Coarse level (Algorithm 4) for one batch of coarse rows.
struct CoarseArgs {
  Csr A, B;
  const int32_t* rows;       // batch rows (global row ids)
  int64_t n_rows;            // rows in batch
  int64_t list_base;         // index of the batch's first row in the coarse list
  int32_t shift_coarse;      // coarse chunk = col >> shift_coarse
  int32_t n_chunks;          // coarse chunks (m_C >> shift_coarse, rounded up)
  int32_t shift_fine;        // fine chunk shift inside a coarse chunk
  int32_t dense_chunk_threshold;
  int32_t hash;               // numeric: hash-map accumulator for fine chunks <= 128 products
  // scratch (device)
  int32_t* col_cnt;          // n_B + 1   (A^CSC column counts / pointers)
  int64_t* col_ptr;          // n_B + 1
  int32_t* csc_row;          // nnz of the batch rows
  double* csc_val;
  int64_t* item_off;         // n_B + 1: outer-product work items per B row, then offsets
  int32_t* rows_b;           // coarseRowsB list
  int32_t* n_rows_b;         // device counter
  int64_t* counts;           // n_rows * n_chunks + 1 (becomes offsetsCoarse)
  unsigned long long* cursor; // n_rows * n_chunks: reorder position per bucket
  int32_t* chunk_col;        // staged products
  double* chunk_val;
  int32_t* fine_col;         // second staging buffer for the fine level
  double* fine_val;
  int64_t* scan_tmp;
  BigBucket* big_list;       // buckets too large for a warp: block-sort ones from the
                             // front, larger ones from the back (nbk entries)
  int32_t* n_big;
  // results
  int32_t* bucket_cnt;       // symbolic: per (coarse list row, chunk) nnz; numeric: read
  int64_t* bucket_out;       // numeric: output offset per (batch row, chunk)
  int64_t* out_cnt;          // symbolic: per row nnz (indexed by row)
  const int64_t* c_rp;
  int32_t* c_col;
  double* c_val;
  const int64_t* c_base;     // as in SortArgs
  int num_sms;
  int64_t nnz_batch;         // nnz of A over the batch rows
  unsigned long long* big_stats;  // optional [3]: products, C entries, count of large buckets
  int64_t* saved_offs;       // optional [n_rows * n_chunks + 1]: the batch's bucket offsets,
                             // written by the symbolic pass, reused by the numeric pass
  cudaEvent_t big_ev0, big_ev1;   // optional: recorded around the large-bucket kernel
  // row-wise staged reorder (used when items != NULL): the batch's work items
  const uint64_t* seg;       // segment table of A (B row start and length per nonzero)
  const CoarseItem* items;
  int32_t n_items;
  int32_t* item_ctr;         // device counter, zeroed by each launch
  int32_t bucket_sort;       // 1: buckets of 257..2048 products take the block sort
};
cudaError_t run_coarse_batch(bool numeric, CoarseArgs& a, cudaStream_t s);
cudaError_t launch_coarse_stage(bool reorder, bool numeric, const CoarseArgs& a, cudaStream_t s);

// Process-wide kernel launch counter.
void count_launch(int n = 1);

// Records a CUDA error for magnus_last_cuda_error and maps it to a status.
int api_cuda_fail(cudaError_t e, const char* where);

// A CUDA graph of a stream-ordered sequence, captured on first use and
// replayed while the pointers it was captured with (its key) stay the same.
struct GraphSlot {
  cudaGraphExec_t exec = nullptr;
  const void* key[8] = {};
  int nkey = 0;
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    nkey = 0;
  }
  // body() enqueues the work on s and returns a magnus status.
  template <class F>
  int run(const void* const* k, int nk, cudaStream_t s, F&& body) {
    bool same = exec != nullptr && nk == nkey;
    for (int i = 0; same && i < nk; ++i) same = key[i] == k[i];
    if (!same) {
      reset();
      cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
      if (e != cudaSuccess) return api_cuda_fail(e, "cudaStreamBeginCapture");
      int st = body();
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(s, &g);
      if (st != 0) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (e != cudaSuccess) return api_cuda_fail(e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        exec = nullptr;
        return api_cuda_fail(e, "cudaGraphInstantiate");
      }
      for (int i = 0; i < nk; ++i) key[i] = k[i];
      nkey = nk;
    }
    cudaError_t e = cudaGraphLaunch(exec, s);
    if (e != cudaSuccess) return api_cuda_fail(e, "cudaGraphLaunch");
    return 0;
  }
};

}  // namespace magnus
