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
  for (int64_t t = blockIdx.x; t < a.n_rows; t += gridDim.x) {
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
    const int64_t outp = NUMERIC ? a.c_rp[row] : 0;
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
// Fine level (Algorithm 3) for one row per block.
//   histogram:   counts of products per fine chunk (col >> shift)
//   prefix sum:  chunk offsets (offsetsFine, n_chunks + 1 entries)
//   reorder:     products written to the staging buffers at
//                offset[chunk] + running count, with the column made
//                relative to the row's first chunk (chunk-local column plus
//                chunk index << shift, so merged chunks sort without a search)
//   accumulate:  chunks in ascending order; a chunk with at least
//                dense_chunk_threshold products uses the dense accumulator
//                over its 2^shift columns, otherwise consecutive small chunks
//                are merged (up to GROUP_SORT_CAP products) and sorted
//                together (Section 3.4 hybrid; Section 4.1.1 chunk merging).
// A row spanning a single chunk is accumulated directly, without reorder.
template <bool NUMERIC>
__global__ void __launch_bounds__(NT) k_fine_rows(FineArgs a) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const FineSmem f = fine_carve(fsm, NUMERIC, a.shift, FINE_MAX_CHUNKS);
  __shared__ TileSmem<NT> ts;
  const int cl = 1 << a.shift;
  for (int64_t t = blockIdx.x; t < a.n_rows; t += gridDim.x) {
    const int32_t row = a.rows[t];
    const int32_t lo = a.lo[row], hi = a.hi[row];
    const int32_t c0 = lo >> a.shift;
    const int nch = (hi >> a.shift) - c0 + 1;
    const int64_t col_base = (int64_t)c0 << a.shift;
    const int64_t as = a.A.rp[row], ae = a.A.rp[row + 1];
    int32_t* oc = NUMERIC ? a.c_col + a.c_rp[row] : nullptr;
    double* ov = NUMERIC ? a.c_val + a.c_rp[row] : nullptr;
    int64_t count;
    if (nch == 1) {
      // single chunk: accumulate straight from A and B
      const int range = hi - (int32_t)col_base + 1;
      const int nwords = (range + 31) >> 5;
      for (int i = threadIdx.x; i < nwords; i += NT) f.bits[i] = 0u;
      if (NUMERIC)
        for (int i = threadIdx.x; i < range; i += NT) f.acc[i] = 0.0;
      __syncthreads();
      block_for_each_product<NT, NUMERIC>(a.A, a.B, as, ae, ts, [&](int32_t col, double v, int64_t) {
        const int idx = col - (int32_t)col_base;
        atomicOr(&f.bits[idx >> 5], 1u << (idx & 31));
        if (NUMERIC) atomicAdd(&f.acc[idx], v);
      });
      count = block_emit_bitmap<NT, NUMERIC>(f.bits, nwords, f.acc, col_base, oc, ov, 0, ts.ws);
    } else {
      int32_t* scol = a.stage_col + a.stage_off[t];
      double* sval = NUMERIC ? a.stage_val + a.stage_off[t] : nullptr;
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
      // reorder
      block_for_each_product<NT, NUMERIC>(a.A, a.B, as, ae, ts, [&](int32_t col, double v, int64_t) {
        const int ch = (col >> a.shift) - c0;
        const int pos = f.off[ch] + atomicAdd(&f.cnt[ch], 1);
        st_stream(&scol[pos], (int32_t)(col - col_base));
        if (NUMERIC) st_stream(&sval[pos], v);
      });
      count = fine_accumulate_chunks<NUMERIC>(f, nch, a.shift, a.dense_chunk_threshold, scol, sval,
                                              col_base, oc, ov, ts.ws);
    }
    if (!NUMERIC && threadIdx.x == 0) a.out_cnt[row] = count;
    __syncthreads();
    (void)cl;
  }
}

cudaError_t launch_fine_rows(bool numeric, const FineArgs& a, cudaStream_t s) {
  if (a.n_rows == 0) return cudaSuccess;
  const size_t smem = fine_smem_bytes(numeric, a.shift, FINE_MAX_CHUNKS);
  int64_t blocks = a.n_rows;
  if (blocks > (1 << 20)) blocks = 1 << 20;
  cudaError_t e;
  if (numeric) {
    e = cudaFuncSetAttribute(k_fine_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fine_rows<true><<<(unsigned)blocks, NT, smem, s>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_fine_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fine_rows<false><<<(unsigned)blocks, NT, smem, s>>>(a);
  }
  count_launch();
  return cudaGetLastError();
}

size_t fine_smem_for(bool numeric, int shift) { return fine_smem_bytes(numeric, shift, FINE_MAX_CHUNKS); }

}  // namespace magnus
