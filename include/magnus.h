/*
 * magnus.h - C ABI of the GB300 (sm_103a) MAGNUS SpGEMM library.
 *
 * Computes C = A * B for sparse matrices in CSR form with FP64 values,
 * int32 column indices and int64 row pointers, following MAGNUS
 * (Wolfson-Pou, Laukemann, Petrini, ICS'25, arXiv 2501.07056):
 *
 *   setup     (Section 3.1)   per-row intermediate-product count P_i and row
 *                             categorisation into sort / dense / fine / coarse;
 *   symbolic  (Section 2.1)   exact nnz of every row of C ("precise
 *                             prediction") and the prefix sum into C.rowPtr;
 *   numeric   (Algorithms 1-4) coarse reorder (Algorithm 4), fine reorder
 *                             (Algorithm 3), per-chunk hybrid accumulation
 *                             (sort or dense, Section 3.4) and CSR output.
 *
 * Conventions shared by every entry point:
 *   - Matrix and output pointers are DEVICE pointers (cudaMalloc'ed or any
 *     memory the current device can address).  They are owned by the caller
 *     and must stay valid until the call's work on `stream` has finished.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All device work is ordered on it.  The current device must be
 *     the device that owns the pointers.
 *   - Every function returns a magnus status (0 = MAGNUS_OK).  No C++
 *     exception crosses this boundary.  After MAGNUS_CUDA_ERROR the CUDA
 *     error string is available from magnus_last_cuda_error().
 *   - Input CSR rows must hold strictly ascending column indices in
 *     [0, n_cols) (the paper does not fix an order; this library requires
 *     it, and checks it when magnus_params_t.validate is set).
 *   - Output rows of C hold strictly ascending column indices.  An entry is
 *     present whenever some product reaches it, even if its value sums to 0.
 */
#ifndef MAGNUS_H
#define MAGNUS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
enum magnus_status {
  MAGNUS_OK = 0,
  MAGNUS_INVALID_ARG = 1,        /* NULL pointer, negative size, A.n_cols != B.n_rows */
  MAGNUS_UNSORTED_OR_DUP = 2,    /* validate=1 found an unsorted/duplicate/out-of-range column */
  MAGNUS_INDEX_OVERFLOW = 3,     /* a size does not fit the index types (cols >= 2^31, rows >= 2^31,
                                    nnz of B >= 2^40) */
  MAGNUS_OUT_OF_MEMORY = 4,      /* device allocation failed or the request exceeds the memory cap */
  MAGNUS_CUDA_ERROR = 5,         /* a CUDA runtime call failed; see magnus_last_cuda_error() */
  MAGNUS_TIMEOUT = 6,            /* a bounded device-side wait expired (see magnus_device_status) */
  MAGNUS_NOT_SYMBOLIC = 7,       /* magnus_numeric called before magnus_symbolic on this plan */
  MAGNUS_BAD_STATE = 8,          /* the plan was built for other inputs or is unusable */
  MAGNUS_SCRATCH_LIMIT = 9,      /* magnus_numeric_noalloc: the fixed staging buffer is too small */
  MAGNUS_WORKSPACE_TOO_SMALL = 10 /* a caller workspace smaller than magnus_workspace_size */
};

/* ---- row categories (Section 3.1) ------------------------------------- */
enum magnus_category {
  MAGNUS_CAT_AUTO = -1,   /* categorise each row by the rules of Section 3.1 */
  MAGNUS_CAT_SORT = 0,    /* sort-based accumulator over the whole row (Algorithm 2) */
  MAGNUS_CAT_DENSE = 1,   /* dense accumulator over the row's column range (Algorithm 1) */
  MAGNUS_CAT_FINE = 2,    /* fine-level reorder then per-chunk accumulation (Algorithm 3) */
  MAGNUS_CAT_COARSE = 3   /* coarse-level reorder (Algorithm 4), then the fine level */
};

/* ---- CSR operand -------------------------------------------------------
 * row_ptr: n_rows+1 int64, row_ptr[0] = 0, nondecreasing, row_ptr[n_rows] = nnz.
 * col:     nnz int32, per row strictly ascending, in [0, n_cols).
 * val:     nnz float64; may be NULL where only the structure is needed
 *          (magnus_plan, magnus_symbolic).  All three are device pointers.  */
typedef struct {
  int64_t n_rows;
  int64_t n_cols;
  int64_t nnz;
  const int64_t* row_ptr;
  const int32_t* col;
  const double* val;
} magnus_csr_t;

/* ---- tuning parameters ---------------------------------------------------
 * Every field has an "automatic" value (0, or -1 for force_category) that the
 * planner replaces by a value derived from the device (Section 3.5 model
 * re-derived for shared memory and L2; see magnus_chunk_model).
 *
 * sort_threshold      rows with P_i < sort_threshold use the sort accumulator
 *                     (Section 3.1, category 1).  Range 1..1025; 0 = 256
 *                     (the threshold of Section 4.1.1).  Rows of up to 256
 *                     products sort in a group of lanes, rows of 257..1024 in
 *                     one warp (symbolic, and numeric up to 512 products) or
 *                     one thread block (numeric, 513..1024 products).
 * force_category      -1 = automatic; otherwise every non-empty row is put in
 *                     that category (used to exercise each stage).
 * chunk_len_fine_log2 log2 of the fine chunk length (columns) for the numeric
 *                     phase; 0 = from the model.
 * chunk_len_coarse_log2 log2 of the coarse chunk length (columns); 0 = from
 *                     the model (m_CmaxSMEM).  A coarse chunk length below
 *                     the fine one is raised to it.
 * dense_chunk_threshold per-chunk hybrid threshold (Section 3.4): a fine chunk
 *                     with at least this many products uses the dense
 *                     accumulator, otherwise the sort accumulator (a warp
 *                     bitonic sort; values above 257 act as 257); 0 = 1
 *                     (dense only: on GB300 a warp's dense accumulator
 *                     beats the warp sort down to about 16 products per
 *                     chunk; the autotuner tries the hybrid).
 * validate            1 = check the input CSR structure on the device in
 *                     magnus_plan (returns MAGNUS_UNSORTED_OR_DUP on failure).
 * max_scratch_bytes   upper bound on the reorder staging buffer of one batch
 *                     (Section 3.3 batching); 0 = automatic (1/6 of the free
 *                     device memory at plan time, at most 16 GB).
 * l2_fetch_bytes      L2 fetch granularity (cudaLimitMaxL2FetchGranularity,
 *                     32, 64 or 128 bytes) set once by magnus_plan for the
 *                     calling process and left in place (the limit is a
 *                     property of the CUDA context, not of the GPU).  32 stops
 *                     the gathers of short B rows from pulling whole 128-byte
 *                     lines; 0 = leave the process setting alone.
 * numeric_graph       1 = magnus_numeric (and magnus_numeric_batched)
 *                     captures its launches in a CUDA graph on the first call
 *                     and replays the graph on later calls with the same
 *                     value and output pointers (plan reuse with new values
 *                     costs one graph launch instead of one launch per
 *                     kernel).  Needs a stream other than the legacy default
 *                     stream (NULL), else the launches run uncaptured; stage
 *                     timing (magnus_enable_timing) also runs uncaptured.
 *                     0 = no graph.
 * wide_sort_max       automatic categorisation only: a row with at least
 *                     sort_threshold and at most wide_sort_max products uses
 *                     the sort accumulator when its column range is too wide
 *                     for the dense accumulator (instead of the fine/coarse
 *                     levels, where the paper sends such rows) or more than
 *                     twice its product count (a sparse row, which the block
 *                     dense accumulator would spend its time zeroing and
 *                     scanning).  GPU rules.  Range 1..1024; 0 = 1024;
 *                     -1 = off (such rows take the dense accumulator when
 *                     their range fits it, else the reorder levels).
 * chunk_accumulator   accumulator of the fine level's non-sort chunks:
 *                     0 = dense array and bitmap (Algorithm 1); 1 = hash map
 *                     (the extension of Algorithm 1 named in Section 2.1,
 *                     storage per Section 3.5's closing remark): a numeric
 *                     chunk of at most 128 products accumulates in its warp's
 *                     open-addressing table of 256 columns (linear probing),
 *                     then the distinct columns are sorted by the warp;
 *                     larger chunks keep the dense accumulator.  The
 *                     symbolic phase counts with the bitmap either way (the
 *                     counts do not depend on the accumulator).  0 or 1.
 * coarse_reorder      how the coarse level stages the products of a batch
 *                     into its (row, coarse chunk) buckets (Algorithm 4):
 *                     1 = outer product over the batch's A^CSC (each needed
 *                     B row read once per batch, products appended one by
 *                     one); 2 = row-wise in work items of 256 nonzeros of A,
 *                     each sub-tile of 2,048 products counting-sorted by
 *                     chunk in shared memory and written to the buckets as
 *                     whole runs (at most 512 coarse chunks); 0 = automatic
 *                     (2 when the chunks allow it, else 1).
 * sort_block_warps    warps per thread block of the warp-sort kernels (rows of
 *                     at most 256 products; every warp works on its own rows,
 *                     so the block shape only changes occupancy and the
 *                     resident wave): 2, 4 or 8 for both phases; 0 = 4 for
 *                     the numeric phase and 8 for the symbolic phase.
 * coarse_bucket_sort  coarse (row, chunk) buckets of 257..2048 products are
 *                     accumulated by a block-wide bitonic sort (Algorithm 2;
 *                     the hybrid of Section 3.4 choosing sort for the smaller
 *                     chunks) instead of the dense accumulator or the fine
 *                     level: 1 = on, -1 = off, 0 = automatic (on when the
 *                     coarse chunks are wider than the 2^13-column block
 *                     dense accumulator: sparse buckets; off otherwise, where
 *                     the dense accumulator wins).  Buckets of at most 256
 *                     products always take a warp sort.  */
typedef struct {
  int32_t sort_threshold;
  int32_t force_category;
  int32_t chunk_len_fine_log2;
  int32_t chunk_len_coarse_log2;
  int32_t dense_chunk_threshold;
  int32_t validate;
  int64_t max_scratch_bytes;
  int32_t l2_fetch_bytes;
  int32_t numeric_graph;
  int32_t wide_sort_max;
  int32_t chunk_accumulator;
  int32_t coarse_reorder;
  int32_t sort_block_warps;
  int32_t coarse_bucket_sort;
} magnus_params_t;

/* Fill *p with the automatic values.  Returns MAGNUS_INVALID_ARG on NULL. */
int magnus_params_default(magnus_params_t* p);

typedef struct magnus_plan_s* magnus_plan_t;

/* magnus_plan - setup phase (Section 3.1).
 * Computes P_i = sum_{j in S(A_i)} nnz(B_j) (Section 5, n_interProd per row),
 * each row's intermediate column range, and the category of every row; sorts
 * rows into per-category lists.  Reads A and B structure (values unused);
 * A->n_cols must equal B->n_rows.  The plan keeps copies of the two
 * descriptors (not of the data): A and B must stay unchanged and alive until
 * magnus_free.  `params` may be NULL (all automatic).  Synchronises `stream`
 * (category counts and per-category row lists are read back).  On success
 * *plan owns device memory released by magnus_free.  On failure *plan is set
 * to NULL. */
int magnus_plan(magnus_plan_t* plan, const magnus_csr_t* A, const magnus_csr_t* B,
                const magnus_params_t* params, void* stream);

/* magnus_symbolic - exact nnz of every row of C (Section 2.1, precise
 * prediction) and C.rowPtr by prefix sum.
 * c_row_ptr: device, A.n_rows+1 int64, written (c_row_ptr[0] = 0).
 * nnz_c:     host, receives c_row_ptr[A.n_rows].  The call synchronises
 *            `stream` to read it (the caller needs it to allocate C).
 * Per-(row, coarse chunk) counts of coarse rows are kept in the plan for
 * magnus_numeric.  MAGNUS_TIMEOUT if a bounded device wait gave up (see
 * magnus_device_status); the counts are then incomplete. */
int magnus_symbolic(magnus_plan_t plan, int64_t* c_row_ptr, int64_t* nnz_c, void* stream);

/* magnus_numeric - Algorithms 1-4: fills C.col and C.val.
 * a_val, b_val: device values of A and B (same structure as at plan time;
 *               they may differ from the values seen earlier, so a plan can
 *               be reused for new values).
 * c_row_ptr:    the array written by magnus_symbolic on this plan.
 * c_col, c_val: device, nnz_c entries each, written.
 * Does not synchronise the stream.  Returns MAGNUS_NOT_SYMBOLIC if
 * magnus_symbolic has not completed on this plan. */
int magnus_numeric(magnus_plan_t plan, const double* a_val, const double* b_val,
                   const int64_t* c_row_ptr, int32_t* c_col, double* c_val, void* stream);

/* ---- caller-owned workspace and row slabs -------------------------------
 * The symbolic and numeric phases need device scratch beyond the plan's own
 * arrays: the fine level's staging slabs (Algorithm 3), the coarse level's
 * CSC copy of A, bucket counts and 12-byte-per-product staging (Algorithm 4;
 * its batches are cut by the staging limit of Section 3.3), and the scan
 * temporaries of C.rowPtr.  magnus_symbolic / magnus_numeric take it from
 * the stream-ordered memory pool for the duration of the call.  The _ws
 * variants take it from a caller-owned device region instead and allocate
 * nothing.
 *
 * magnus_workspace_size  *bytes receives a size sufficient for every
 *                        magnus_symbolic_ws, magnus_numeric_ws and
 *                        magnus_numeric_rows call on this plan (host only, no
 *                        device work).
 * workspace              device pointer, 256-byte aligned, workspace_bytes
 *                        long, owned by the caller; it must not be used by
 *                        anything else until the call's work on `stream` has
 *                        finished.  Too small: MAGNUS_WORKSPACE_TOO_SMALL
 *                        before any work is enqueued.  Misaligned:
 *                        MAGNUS_INVALID_ARG.
 *
 * magnus_numeric_rows - the numeric phase for rows [row_begin, row_end) of C
 * only, on a plan of the whole product: the phase split of Section 2.1
 * (C.rowPtr from the symbolic phase is an input of the numeric phase) makes
 * every row's place in C known, so C can be produced slab by slab when it
 * does not fit the device (the memory-bounded batching of rows of Section
 * 3.3, applied to the output).
 *   c_row_ptr   the whole C.rowPtr written by magnus_symbolic (device,
 *               A.n_rows + 1 int64); it is read, not written.
 *   c_col/c_val device, at least c_row_ptr[row_end] - c_row_ptr[row_begin]
 *               entries: entry e of C (c_row_ptr[row_begin] <= e <
 *               c_row_ptr[row_end]) is written at index e -
 *               c_row_ptr[row_begin].  The slab's own row pointers are
 *               c_row_ptr[row_begin..row_end] - c_row_ptr[row_begin].
 *   workspace   NULL (scratch from the pool) or a caller region as above.
 * 0 <= row_begin <= row_end <= A.n_rows, else MAGNUS_INVALID_ARG; an empty
 * range returns MAGNUS_OK without work.  Results equal the same rows of
 * magnus_numeric (within the value tolerance; structure identical).  Does
 * not synchronise the stream; never captured in the plan's numeric graph.
 * Rows of the coarse level are computed in the part of each coarse batch
 * that lies in the range (the batch's histogram is recomputed unless the
 * range covers the whole batch). */
int magnus_workspace_size(magnus_plan_t plan, size_t* bytes);
int magnus_symbolic_ws(magnus_plan_t plan, int64_t* c_row_ptr, int64_t* nnz_c, void* workspace,
                       size_t workspace_bytes, void* stream);
int magnus_numeric_ws(magnus_plan_t plan, const double* a_val, const double* b_val,
                      const int64_t* c_row_ptr, int32_t* c_col, double* c_val, void* workspace,
                      size_t workspace_bytes, void* stream);
int magnus_numeric_rows(magnus_plan_t plan, int64_t row_begin, int64_t row_end,
                        const double* a_val, const double* b_val, const int64_t* c_row_ptr,
                        int32_t* c_col, double* c_val, void* workspace, size_t workspace_bytes,
                        void* stream);

/* magnus_numeric_noalloc - the numeric phase without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory once they are running, for example a solver that
 * multiplies the same structure with new values every iteration inside a
 * framework whose allocator owns the whole device (a cudaMalloc from a library
 * would exceed its budget or fragment its pool), or a loop that must not let
 * cudaMalloc/cudaFree synchronise the device.  magnus_plan and magnus_symbolic
 * still allocate; run them during set-up.
 *
 * Arguments, results and tolerance are those of magnus_numeric.  The fine
 * level stages one row per thread block in a slab of 12 bytes per product;
 * here the slabs, and the counter through which blocks take rows, come from
 * one static device array of MAGNUS_NOALLOC_SCRATCH_BYTES, which every GPU
 * that loads this library holds until the process exits, and the fine kernel
 * runs with as many blocks as slabs fit in it.  Plans that contain coarse
 * rows (force_category, very wide C, or rows with more products than a
 * slab), or whose slab alone exceeds the array, are rejected with
 * MAGNUS_SCRATCH_LIMIT before any work is enqueued.
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, no allocation); the first call on a device may load
 * the library's device code, so make that first call before any stream
 * capture.  The fine rows run on magnus_plan_info().noalloc_fine_blocks
 * blocks, one per staging slab that fits the array: a plan meant for this
 * entry point should set max_scratch_bytes so that its slab (12 B per
 * product of its heaviest fine row, at most 2^20 products) leaves room for
 * about one slab per SM (e.g. max_scratch_bytes = 16 MB gives slabs of a
 * few thousand products and the full resident wave), else the fine level
 * runs on fewer blocks than the GPU has SMs.
 * All calls share the one array: calls that may overlap on the GPU (other
 * streams, other host threads) race on it and must be serialised by the
 * caller.  The row counter is cleared by every call (stream-ordered
 * cudaMemsetAsync, no allocation); the slabs need no clearing (every staged
 * entry is written before it is read). */
#define MAGNUS_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
int magnus_numeric_noalloc(magnus_plan_t plan, const double* a_val, const double* b_val,
                           const int64_t* c_row_ptr, int32_t* c_col, double* c_val,
                           void* stream);

/* Release the plan and all device memory it owns.  Safe on NULL.  Work the
 * plan enqueued must be complete or ordered before any reuse of that memory
 * (frees are stream-ordered on the plan's last stream). */
void magnus_free(magnus_plan_t plan);

/* Static message for a status code. */
const char* magnus_strerror(int status);

/* Text of the last CUDA error seen by this library in the calling thread
 * (empty string if none). */
const char* magnus_last_cuda_error(void);

/* ---- batched products ----------------------------------------------------
 * Many independent products C_i = A_i * B_i (i < count) planned and run
 * together, so that every launch serves the rows of all products.  The paper
 * computes one product at a time; the batch is a packing of the inputs, not a
 * change of the arithmetic: the operands are gathered into one block-diagonal
 * problem (A_i's columns shifted past the rows of B_1..B_{i-1}, B_i's columns
 * unchanged), whose row r of product i is row r of C_i in C_i's own columns.
 *
 * Layout of C: one packed CSR over the rows of all products in order.
 * Product i owns packed rows [row_offsets[i], row_offsets[i+1]) and packed
 * entries [c_offsets[i], c_offsets[i+1]); its own row pointers are
 * c_row_ptr[row_offsets[i] .. row_offsets[i+1]] - c_offsets[i].
 *
 * magnus_plan_batched  A, B: host arrays of `count` descriptors of device CSR
 *                      operands (A[i].n_cols == B[i].n_rows).  The operands
 *                      must stay alive and unchanged in structure until
 *                      magnus_free_batched; values are read by every
 *                      magnus_numeric_batched call.  The batch holds a packed
 *                      copy of both operands (16 B per row and 12 B per
 *                      nonzero) and the inner plan.  Totals of rows must stay
 *                      below 2^31.  Synchronises `stream`.
 * magnus_batch_layout  row_offsets (host, count+1) and the total number of
 *                      rows of C; either pointer may be NULL.
 * magnus_symbolic_batched
 *                      c_row_ptr: device, total_rows+1 int64 (written);
 *                      c_offsets: host, count+1 int64 (written; c_offsets[count]
 *                      is nnz of all products).  Synchronises `stream`.
 * magnus_numeric_batched
 *                      c_col / c_val: device, c_offsets[count] entries each.
 *                      With params.numeric_graph = 1 the value packing and the
 *                      numeric phase are captured in one CUDA graph and
 *                      replayed on later calls with the same output pointers.
 * magnus_batch_info    the inner plan's magnus_plan_info.
 * Status codes as for the single-product calls. */
typedef struct magnus_batch_s* magnus_batch_t;
int magnus_plan_batched(magnus_batch_t* batch, int32_t count, const magnus_csr_t* A,
                        const magnus_csr_t* B, const magnus_params_t* params, void* stream);
int magnus_batch_layout(magnus_batch_t batch, int64_t* row_offsets, int64_t* total_rows);
int magnus_symbolic_batched(magnus_batch_t batch, int64_t* c_row_ptr, int64_t* c_offsets,
                            void* stream);
int magnus_numeric_batched(magnus_batch_t batch, const int64_t* c_row_ptr, int32_t* c_col,
                           double* c_val, void* stream);
void magnus_free_batched(magnus_batch_t batch);
/* The inner plan of the packed problem (owned by the batch; valid until
 * magnus_free_batched), for magnus_enable_timing / magnus_stage_times /
 * magnus_plan_info.  NULL for a NULL batch. */
magnus_plan_t magnus_batch_inner_plan(magnus_batch_t batch);

/* ---- autotuner -----------------------------------------------------------
 * magnus_autotune measures the whole step (magnus_plan + magnus_symbolic +
 * magnus_numeric, CUDA events on `stream`) for candidate parameter sets and
 * returns the fastest in *best.  The search starts from *base (NULL = the
 * automatic parameters) and does coordinate descent over sort_threshold
 * (64..1025), wide_sort_max, chunk_len_coarse_log2 (11..13, when coarse rows
 * exist), chunk_len_fine_log2 (7..10), dense_chunk_threshold and
 * chunk_accumulator (when fine or coarse rows exist), coarse_reorder (when
 * coarse rows exist) and sort_block_warps (2, 4, 8; when sort rows exist);
 * at most max_trials measured runs.  The paper fixes the
 * threshold and derives the chunk lengths from its cache model (Section 3.5,
 * Section 4.1.1); on the GPU those values are the starting point.
 * sample_products > 0 and a product with more intermediate products than
 * that: the runs use 16 evenly spaced row blocks of A holding about
 * sample_products products (a device copy of those rows).
 * A and B need values.  Results are cached per (device, shapes, nnz,
 * sample_products, base parameters): a repeated call returns the cached set with
 * report->from_cache = 1.  The device memory of the trials (one C of the
 * tuned operand and the plans' scratch) is released before returning.
 * Synchronises `stream`.  Status codes as for magnus_plan. */
typedef struct {
  int32_t trials;          /* measured runs (the base run counts as one) */
  int32_t from_cache;      /* 1 if *best came from the cache (no runs) */
  int64_t sampled_rows;    /* rows of A used, 0 = all */
  int64_t products_full;   /* n_interProd of the full product */
  float base_ms;           /* step time with *base */
  float best_ms;           /* step time with *best */
} magnus_tune_report_t;

int magnus_autotune(const magnus_csr_t* A, const magnus_csr_t* B, const magnus_params_t* base,
                    int64_t sample_products, int32_t max_trials, magnus_params_t* best,
                    magnus_tune_report_t* report, void* stream);

/* magnus_autotune_batched - magnus_autotune on a batch's packed
 * block-diagonal operands (the products' rows sampled together), so that
 * later batches of the same kind of products can be planned with *best
 * (magnus_plan_batched's params).  Packs the current values first (they are
 * read by the trials); the batch itself is left as it was planned.  Status
 * codes as for magnus_autotune. */
int magnus_autotune_batched(magnus_batch_t batch, const magnus_params_t* base,
                            int64_t sample_products, int32_t max_trials, magnus_params_t* best,
                            magnus_tune_report_t* report, void* stream);

/* ---- building-block microbenchmark ---------------------------------------
 * The steps of one reorder level (Section 4.1, Figures 5-6) on a stream of
 * `length` (index, value) pairs with indices in [0, m): histogram per chunk
 * (index >> shift, 2^n_chunks_log2 chunks), prefix sum, reorder into chunk
 * order (element by element, and staged through shared memory), and
 * per-chunk dense accumulation (one block's shared-memory
 * accumulator; only when the chunk length 2^shift is at most 2^13), each
 * timed with CUDA events on `stream`; beside them a copy of the stream and a
 * dense accumulator over all of [0, m) in global memory (FP64 atomics, no
 * locality generation).  col/val: device input (caller-owned).
 * out_col/out_val: device, `length` entries: chunk c's unique indices
 * (ascending, global numbering) with their sums start at the chunk's first
 * element in chunk order; chunk_nnz (device, n_chunks entries, may be NULL
 * when no accumulation runs) gets their counts.  m <= 2^31, n_chunks_log2 in
 * 0..14.  Allocates and frees its scratch; synchronises `stream`.  The paper
 * has no counterpart as an API: it is its microbenchmark. */
typedef struct {
  float copy_ms;
  float histogram_ms;
  float scan_ms;
  float reorder_ms;
  float accumulate_ms;          /* -1 when the chunks exceed 2^13 indices */
  float global_accumulate_ms;
  int32_t n_chunks;
  int32_t chunk_len_log2;
  float reorder_staged_ms;      /* tile sorted by chunk in shared memory, then
                                   written as runs; -1 above 4096 chunks */
  int32_t reserved;
} magnus_microbench_t;

int magnus_microbench_chunks(const int32_t* col, const double* val, int64_t length, int64_t m,
                             int32_t n_chunks_log2, int32_t* out_col, double* out_val,
                             int64_t* chunk_nnz, magnus_microbench_t* result, void* stream);

/* ---- rates of the device's building operations ---------------------------
 * magnus_microbench_rates measures, on the current device, the rates that
 * bound the SpGEMM kernels (the paper has no counterpart: its bounds are a
 * CPU's streaming bandwidth).  Gathers: chunks per second of random chunks of
 * 16..256 bytes at chunk-aligned offsets of a 2 GB array, and of CSR B rows
 * of 8 entries (32 bytes of columns and 64 bytes of values from two arrays).
 * Shared memory: updates per second device-wide of an 8,192-entry FP64 array
 * per block (3 blocks of 256 threads per SM) by atomicAdd at distinct
 * addresses, random addresses, and 8 lanes per address, by a plain add, and
 * by u32 atomicAdd at random addresses.  Allocates (about 2 GB) and frees
 * its buffers; synchronises `stream`. */
typedef struct {
  double gather_16;                      /* chunks/s, 16-byte chunks */
  double gather_32;
  double gather_64;
  double gather_128;
  double gather_256;
  double gather_csr_row8;                /* B rows/s, 32 B columns + 64 B values */
  double smem_f64_atomic_distinct;       /* updates/s */
  double smem_f64_atomic_random;
  double smem_f64_atomic_8_per_address;
  double smem_f64_add_plain;
  double smem_u32_atomic_random;
  int32_t sms;                           /* multiprocessors of the device */
  int32_t reserved;
} magnus_rates_t;
int magnus_microbench_rates(magnus_rates_t* rates, void* stream);

/* ---- plan introspection ------------------------------------------------ */
typedef struct {
  int64_t n_rows;               /* rows of A (= rows of C) */
  int64_t n_cols;               /* columns of B (= m_C) */
  int64_t n_interprod;          /* sum of P_i (Section 5) */
  int64_t max_row_products;     /* max P_i */
  int64_t nnz_c;                /* after magnus_symbolic, else -1 */
  int64_t rows_empty;           /* rows with P_i = 0 */
  int64_t rows_per_category[4]; /* indexed by magnus_category */
  int64_t products_per_category[4];
  int64_t staged_products_numeric; /* products written to and re-read from
                                      global staging by the last numeric call */
  int64_t scratch_bytes;        /* largest staging buffer used */
  int32_t sort_threshold;
  int32_t chunk_len_fine_log2;
  int32_t chunk_len_fine_sym_log2;
  int32_t chunk_len_coarse_log2;
  int32_t n_chunks_coarse;
  int32_t dense_cols;           /* max column range of a dense row */
  int32_t dense_chunk_threshold;
  int32_t key_bits32;           /* 1 if sort keys fit in 32 bits */
  int32_t n_batches_fine;
  int32_t n_batches_coarse;
  int64_t coarse_dense_products; /* last numeric call: products of the coarse
                                    (row, chunk) buckets too large for a warp
                                    sort, accumulated by the block-wide dense
                                    (or fine-level) kernel */
  int64_t coarse_dense_nnz;      /* last numeric call: entries of C those
                                    buckets produced */
  int64_t coarse_dense_buckets;  /* last numeric call: number of such buckets */
  int64_t plan_bytes;            /* device memory owned by the plan */
  int64_t workspace_bytes;       /* magnus_workspace_size of the plan */
  int32_t noalloc_fine_blocks;   /* thread blocks magnus_numeric_noalloc runs the fine
                                    rows on (its fixed buffer holds that many staging
                                    slabs of 12 B x the plan's slab products; the
                                    numeric pool path runs one resident wave); 0 when
                                    the plan has no fine rows; -1 when that entry
                                    point refuses the plan */
  int32_t reserved;
} magnus_plan_info_t;

int magnus_plan_info(magnus_plan_t plan, magnus_plan_info_t* info);
int magnus_batch_info(magnus_batch_t batch, magnus_plan_info_t* info);

/* ---- device timing of the stages --------------------------------------
 * When enabled on a plan, every later magnus_symbolic / magnus_numeric call
 * records CUDA events on its stream around each stage; magnus_stage_times
 * returns the elapsed milliseconds of the last call (synchronising on the
 * events).  Stage indices: see MAGNUS_STAGE_*.  Disabled by default. */
enum magnus_stage {
  MAGNUS_STAGE_SYM_SORT = 0, MAGNUS_STAGE_SYM_DENSE = 1, MAGNUS_STAGE_SYM_FINE = 2,
  MAGNUS_STAGE_SYM_COARSE = 3, MAGNUS_STAGE_SYM_SCAN = 4,
  MAGNUS_STAGE_NUM_SORT = 5, MAGNUS_STAGE_NUM_DENSE = 6, MAGNUS_STAGE_NUM_FINE = 7,
  MAGNUS_STAGE_NUM_COARSE = 8,
  /* subsets of the coarse stages: the accumulation of the large (row, chunk)
   * buckets (block-wide dense accumulator), summed over the coarse batches */
  MAGNUS_STAGE_SYM_COARSE_BIG = 9, MAGNUS_STAGE_NUM_COARSE_BIG = 10,
  MAGNUS_STAGE_COUNT = 11
};
int magnus_enable_timing(magnus_plan_t plan, int enable);
int magnus_stage_times(magnus_plan_t plan, double* ms, int n);

/* Device memory on the current device that new work may still use:
 * *free_bytes is cudaMemGetInfo's free memory and *pool_idle_bytes the
 * memory the device's default stream-ordered pool holds without using it
 * (this library's scratch comes from that pool and reuses it first).
 * A serving loop admits requests against their sum (the symbolic phase gives
 * each C's exact size before it is allocated, Section 2.1).  Either pointer
 * may be NULL. */
int magnus_device_memory(size_t* free_bytes, size_t* pool_idle_bytes);

/* ---- page-locked host buffers ------------------------------------------
 * For callers that move operands and results across the host link (the
 * paper has no counterpart; it runs on the host).  magnus_host_alloc maps
 * `bytes` of anonymous host memory advised to use transparent huge pages,
 * touches every page and registers the range with the CUDA driver as
 * page-locked, so device copies to and from it run at the link's rate even
 * when host memory is fragmented (page-locked memory in small pages copies
 * several times slower then).  *ptr is the host address, usable as a
 * cudaMemcpyAsync source or destination.  Release it with magnus_host_free
 * and the same size; no device work may still use it.  Errors:
 * MAGNUS_INVALID_ARG (NULL ptr or zero size), MAGNUS_OUT_OF_MEMORY (the
 * mapping failed), MAGNUS_CUDA_ERROR (registration failed; nothing is kept).
 * The mapping starts on a huge-page boundary and is rounded up to whole huge
 * pages, so a buffer may hold up to one huge page (512 MB with 64 KB base
 * pages) more than asked.  Allocation touches the whole range (about 0.2 s
 * for 8 GB): do it once and reuse the buffer. */
int magnus_host_alloc(size_t bytes, void** ptr);
int magnus_host_free(void* ptr, size_t bytes);

/* Number of kernels this library has launched in this process. */
uint64_t magnus_launch_count(void);

/* magnus_device_status - synchronises `stream` and reports whether a bounded
 * device-side wait of this library gave up since the last report (then
 * MAGNUS_TIMEOUT; the flag is cleared), else MAGNUS_OK.  The waits are those
 * of the coarse level's bucket sort on its bulk copies (one-dimensional TMA
 * copies of a bucket's staged products into shared memory, Section 3.3's
 * chunk staging): each gives up after about a second of SM clock, lets the
 * block's copies in flight land and ends the block, leaving its buckets
 * unwritten.  magnus_symbolic reports such a timeout itself (it
 * synchronises anyway); a numeric call does not synchronise, so a caller
 * that wants the check calls this after it.  MAGNUS_CUDA_ERROR when the
 * synchronisation fails. */
int magnus_device_status(void* stream);

/* magnus_wait_selftest - exercises the bounded wait: one block announces a
 * copy on an mbarrier and issues none, waits `limit_cycles` SM clocks
 * (1..2^31), gives up and raises the flag that magnus_device_status reports
 * (so the next magnus_device_status returns MAGNUS_TIMEOUT).  No copy is in
 * flight at any time.  MAGNUS_INVALID_ARG for a limit out of range. */
int magnus_wait_selftest(int64_t limit_cycles, void* stream);

/* ---- chunk model (host only; no GPU needed) -----------------------------
 * The paper sizes chunks so that the accumulator and the reorder bookkeeping
 * of one thread fit its private L2 (Section 3.5, Eq. 2-7).  On the GPU the
 * private store is a thread block's shared memory and the active write lines
 * of the reorder live in the shared L2, so Eq. 2 is evaluated with two
 * budgets (shared memory per block, L2 share per resident block).
 * Inputs: m_c (columns of C), smem_bytes (accumulator budget per block),
 * l2_bytes (device L2), resident_blocks (blocks resident device-wide).
 * Output fields are log2 chunk lengths in columns.  Returns MAGNUS_INVALID_ARG
 * for non-positive inputs. */
typedef struct {
  int32_t m_c_log2;             /* ceil(log2(m_c)) */
  int32_t chunk_len_fine_log2;  /* numeric: FP64 value + 1 bitmap bit per column */
  int32_t chunk_len_fine_sym_log2; /* symbolic: 1 bitmap bit per column */
  int32_t n_chunks_fine_max_log2;  /* max fine chunks one row may use (L2 bound) */
  int32_t m_c_max_log2;         /* widest column range handled by the fine level alone */
  int32_t n_chunks_coarse;      /* m_C / 2^m_c_max_log2 (1 = fine level suffices) */
  int64_t fine_smem_bytes;      /* shared memory of the fine accumulator + bookkeeping */
} magnus_chunk_model_t;

int magnus_chunk_model(int64_t m_c, int64_t smem_bytes, int64_t l2_bytes,
                       int32_t resident_blocks, magnus_chunk_model_t* out);

#ifdef __cplusplus
}
#endif

#endif /* MAGNUS_H */
