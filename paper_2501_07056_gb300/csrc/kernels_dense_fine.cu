// Dense-category rows (Algorithm 1 over the row's column range) and
// fine-level rows (Algorithm 3): one thread block per row.
#include "fine_level.cuh"

namespace magnus {

constexpr int NT = DENSE_NT;

// ---------------------------------------------------------------------------
// Dense rows: the accumulator covers [lo, hi], the row's intermediate column
// range, which the setup guarantees is at most dense_cols wide.  FP64 adds go
// to shared memory; a bitmap marks touched columns, and the bitmap scan
// emits them in ascending order.
template <bool NUMERIC>
__global__ void __launch_bounds__(NT) k_dense_rows(DenseArgs a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  double* acc = reinterpret_cast<double*>(dsm);
  uint32_t* bits = reinterpret_cast<uint32_t*>(dsm + (NUMERIC ? (size_t)a.dense_cols * 8 : 0));
  __shared__ TileSmem<NT> ts;
  // rows [first, n) of the bin's list: all of them, or a row range's
  const int64_t first = (NUMERIC && a.range) ? a.range[0] : 0;
  const int64_t n_end = (NUMERIC && a.range) ? a.range[1] : a.n_rows;
  const int64_t cbase = (NUMERIC && a.c_base) ? *a.c_base : 0;
  for (int64_t t = first + blockIdx.x; t < n_end; t += gridDim.x) {
    const int32_t row = a.rows[t];
    const int32_t lo = a.lo[row], hi = a.hi[row];
    const int range = hi - lo + 1;
    const int nwords = (range + 31) >> 5;
    for (int i = threadIdx.x; i < nwords; i += NT) bits[i] = 0u;
    if (NUMERIC)
      for (int i = threadIdx.x; i < range; i += NT) acc[i] = 0.0;
    __syncthreads();
    block_for_each_product<NT, NUMERIC>(a.A, a.B, a.A.rp[row], a.A.rp[row + 1], ts,
                                        [&](int32_t col, double v, int64_t) {
                                          const int idx = col - lo;
                                          atomicOr(&bits[idx >> 5], 1u << (idx & 31));
                                          if (NUMERIC) atomicAdd(&acc[idx], v);
                                        });
    const int64_t outp = NUMERIC ? a.c_rp[row] - cbase : 0;
    const int64_t n = block_emit_bitmap<NT, NUMERIC>(bits, nwords, acc, lo, a.c_col, a.c_val,
                                                     outp, ts.ws);
    if (!NUMERIC && threadIdx.x == 0) a.out_cnt[row] = n;
    __syncthreads();
  }
}

cudaError_t launch_dense_rows(bool numeric, const DenseArgs& a, int num_sms, cudaStream_t s) {
  if (a.n_rows == 0) return cudaSuccess;
  const size_t smem = (numeric ? (size_t)a.dense_cols * 8 : 0) + (size_t)(a.dense_cols / 32 + 1) * 4;
  int64_t blocks = a.n_rows;
  const int64_t cap = (int64_t)num_sms * 8;
  if (blocks > cap) blocks = cap;
  cudaError_t e;
  if (numeric) {
    e = cudaFuncSetAttribute(k_dense_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_dense_rows<true><<<(unsigned)blocks, NT, smem, s>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_dense_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_dense_rows<false><<<(unsigned)blocks, NT, smem, s>>>(a);
  }
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fine level (Algorithm 3), one row per block at a time; a persistent grid
// whose blocks take rows (heaviest first) from a device counter.
//   histogram:   products per fine chunk (col >> shift), in shared memory
//   prefix sum:  chunk offsets (n_chunks + 1 entries)
//   reorder:     products written to the block's staging slab at
//                offset[chunk] + running count; columns are kept relative to
//                the row's first chunk (chunk << shift | column in chunk)
//   accumulate:  one chunk per warp, by the hybrid of Section 3.4: a warp
//                sort for chunks below the threshold, a warp-private dense
//                accumulator otherwise (warp_chunks_accumulate); chunks are
//                emitted in column order.
// Symbolic phase: a row dense enough for one block bitmap over its whole
// column range (range <= 2^19, range / 32 <= 4 * P) is counted directly from
// A and B without a reorder; other rows take the chunked path with bitmaps
// only.
template <bool NUMERIC, bool HYBRID>
__global__ void __launch_bounds__(NT) k_fine_rows(FineArgs a) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const FineSmem f = fine_carve(fsm, NUMERIC, a.shift, HYBRID);
  __shared__ TileSmem<NT> ts;
  __shared__ int64_t s_next;
  int32_t* const slab_col = a.stage_col ? a.stage_col + (int64_t)blockIdx.x * a.slab_elems : nullptr;
  double* const slab_val = a.stage_val ? a.stage_val + (int64_t)blockIdx.x * a.slab_elems : nullptr;
  fine_clear<NUMERIC>(f, a.shift);
  for (;;) {
    // rows are listed heaviest first; blocks take the next one when free
    if (threadIdx.x == 0) s_next = atomicAdd(a.queue, 1);
    __syncthreads();
    const int64_t t = s_next;
    __syncthreads();
    if (t >= a.n_rows) break;
    const int32_t row = a.rows[t];
    const int32_t lo = a.lo[row], hi = a.hi[row];
    const int64_t as = a.A.rp[row], ae = a.A.rp[row + 1];
    if (!NUMERIC) {
      const int64_t range = (int64_t)hi - lo + 1;
      const int64_t words = (range + 31) >> 5;
      if (range <= ((int64_t)1 << DIRECT_BITS_LOG2) && words <= 4 * a.row_products[t]) {
        // direct count: one bitmap over [lo, hi], then the bitmap is cleared
        // again so the chunked path finds its warp bitmaps zero
        for (int64_t i = threadIdx.x; i < words; i += NT) f.direct[i] = 0u;
        __syncthreads();
        block_for_each_product<NT, false>(a.A, a.B, as, ae, ts, [&](int32_t col, double, int64_t) {
          const int idx = col - lo;
          atomicOr(&f.direct[idx >> 5], 1u << (idx & 31));
        });
        int64_t c = 0;
        for (int64_t i = threadIdx.x; i < words; i += NT) c += __popc(f.direct[i]);
        c = block_sum<NT>(c, ts.ws);
        if (threadIdx.x == 0) a.out_cnt[row] = c;
        for (int64_t i = threadIdx.x; i < words; i += NT) f.direct[i] = 0u;
        fine_clear<false>(f, a.shift);
        continue;
      }
    }
    const int32_t c0 = lo >> a.shift;
    const int nch = (hi >> a.shift) - c0 + 1;
    const int64_t col_base = (int64_t)c0 << a.shift;
    for (int i = threadIdx.x; i < nch; i += NT) f.cnt[i] = 0;
    __syncthreads();
    // histogram
    block_for_each_product<NT, false>(a.A, a.B, as, ae, ts, [&](int32_t col, double, int64_t) {
      atomicAdd(&f.cnt[(col >> a.shift) - c0], 1);
    });
    // prefix sum -> offsets; counts become the reorder cursors
    int32_t run = 0;
    for (int i0 = 0; i0 < nch; i0 += NT) {
      const int i = i0 + threadIdx.x;
      const int64_t c = (i < nch) ? f.cnt[i] : 0;
      int64_t tot;
      const int64_t ex = block_exclusive_scan<NT>(c, ts.ws, &tot);
      if (i < nch) {
        f.off[i] = run + (int32_t)ex;
        f.cnt[i] = 0;
      }
      run += (int32_t)tot;
    }
    if (threadIdx.x == 0) f.off[nch] = run;
    __syncthreads();
    // reorder into the block's slab
    block_for_each_product<NT, NUMERIC>(a.A, a.B, as, ae, ts, [&](int32_t col, double v, int64_t) {
      const int ch = (col >> a.shift) - c0;
      const int pos = f.off[ch] + atomicAdd(&f.cnt[ch], 1);
      st_stream(&slab_col[pos], (int32_t)(col - col_base));
      if (NUMERIC) st_stream(&slab_val[pos], v);
    });
    const int64_t outp = NUMERIC ? a.c_rp[row] - (a.c_base ? *a.c_base : 0) : 0;
    int32_t* oc = NUMERIC ? a.c_col + outp : nullptr;
    double* ov = NUMERIC ? a.c_val + outp : nullptr;
    const int64_t count = warp_chunks_accumulate<NUMERIC, HYBRID>(
        f, nch, a.shift, slab_col, slab_val, col_base, oc, ov, a.dense_chunk_threshold, a.hash);
    if (!NUMERIC && threadIdx.x == 0) a.out_cnt[row] = count;
    __syncthreads();
  }
}

template <bool NUMERIC, bool HYBRID>
static int fine_rows_occupancy(size_t smem) {
  int n = 0;
  cudaError_t e = cudaFuncSetAttribute(k_fine_rows<NUMERIC, HYBRID>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fine_rows<NUMERIC, HYBRID>, NT, smem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n < 1 ? 1 : n;
}

int fine_rows_blocks_per_sm(bool numeric, int shift, bool hybrid) {
  const size_t smem = fine_smem_bytes(numeric, shift, hybrid);
  if (numeric) return hybrid ? fine_rows_occupancy<true, true>(smem) : fine_rows_occupancy<true, false>(smem);
  return hybrid ? fine_rows_occupancy<false, true>(smem) : fine_rows_occupancy<false, false>(smem);
}

template <bool NUMERIC, bool HYBRID>
static cudaError_t launch_fine_rows_t(const FineArgs& a, unsigned blocks, size_t smem,
                                      cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_fine_rows<NUMERIC, HYBRID>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_fine_rows<NUMERIC, HYBRID><<<blocks, NT, smem, s>>>(a);
  return cudaSuccess;
}

cudaError_t launch_fine_rows(bool numeric, const FineArgs& a, int grid, cudaStream_t s) {
  if (a.n_rows == 0) return cudaSuccess;
  // the sort and hash accumulators share the per-warp staging
  const bool hybrid = a.dense_chunk_threshold > 1 || (numeric && a.hash);
  const size_t smem = fine_smem_bytes(numeric, a.shift, hybrid);
  int64_t blocks = grid;
  if (blocks > a.n_rows) blocks = a.n_rows;
  if (blocks < 1) blocks = 1;
  const unsigned b = (unsigned)blocks;
  cudaError_t e;
  if (numeric)
    e = hybrid ? launch_fine_rows_t<true, true>(a, b, smem, s) : launch_fine_rows_t<true, false>(a, b, smem, s);
  else
    e = hybrid ? launch_fine_rows_t<false, true>(a, b, smem, s) : launch_fine_rows_t<false, false>(a, b, smem, s);
  if (e != cudaSuccess) return e;
  count_launch();
  return cudaGetLastError();
}

size_t fine_smem_for(bool numeric, int shift, bool hybrid) {
  return fine_smem_bytes(numeric, shift, hybrid);
}

}  // namespace magnus
