// Row-wise staged coarse reorder (the reorder step of Algorithm 4, Section
// 3.3, in a GPU form that writes whole runs).
//
// Algorithm 4 walks the batch's submatrix of A column by column (an outer
// product) so that every needed B row is read once per batch, and appends
// each product to the staging area of its (row, coarse chunk) bucket.  On a
// GPU those appends are scattered 4- and 8-byte stores, one bucket per lane.
// Here persistent blocks take work items instead, each a coarse row's run of
// at most CS_NJ nonzeros of A, and generate that run's products row-wise
// (consecutive threads take consecutive entries of a B row, so B rows are
// read with coalesced loads; B rows that many coarse rows share stay in L2).
// Every sub-tile of CS_ST products is counting-sorted by coarse chunk in
// shared memory; one atomic per (sub-tile, chunk) reserves a run in the
// bucket, and the run is written contiguously, so the staging area receives
// whole lines, the GPU counterpart of the paper's write-combining buffers
// for non-temporal stores.  The histogram pass (the bucket sizes, before the
// row-chained prefix sum) counts per item in shared memory and adds each
// chunk's count to its bucket once.
#include "common.cuh"

namespace magnus {

constexpr int CS_NT = 256;                 // threads per block
constexpr int CS_PER = 8;                  // products per thread per sub-tile
constexpr int CS_ST = CS_NT * CS_PER;      // products per sub-tile

// Shared memory: per-chunk counters, offsets and reserved run starts, then
// the staged sub-tile (local column, value, chunk).
__host__ __device__ inline size_t coarse_stage_smem(int nc, bool reorder, bool numeric) {
  size_t b = (size_t)nc * 4;                                  // h
  if (reorder) {
    b += (size_t)(nc + 1) * 4;                                // hoff
    b = (b + 7) & ~(size_t)7;
    b += (size_t)nc * 8;                                      // gbase
    b += (size_t)CS_ST * 4;                                   // scol
    if (numeric) b += (size_t)CS_ST * 8;                      // sval
    b += (size_t)CS_ST * 2;                                   // chunk of each staged entry
  }
  return b;
}

template <bool REORDER, bool NUMERIC>
__global__ void __launch_bounds__(CS_NT)
    k_coarse_stage(Csr A, Csr B, const uint64_t* __restrict__ seg,
                   const CoarseItem* __restrict__ items, int32_t n_items,
                   int32_t* __restrict__ item_ctr, int64_t list_base, int sc, int nc,
                   int64_t* __restrict__ counts, unsigned long long* __restrict__ cursor,
                   int32_t* __restrict__ chunk_col, double* __restrict__ chunk_val) {
  extern __shared__ __align__(16) unsigned char csm[];
  int32_t* h = reinterpret_cast<int32_t*>(csm);
  int32_t* hoff = h + nc;
  int64_t* gbase = nullptr;
  int32_t* scol = nullptr;
  double* sval = nullptr;
  uint16_t* sch = nullptr;
  if (REORDER) {
    size_t o = ((size_t)nc * 4 + (size_t)(nc + 1) * 4 + 7) & ~(size_t)7;
    gbase = reinterpret_cast<int64_t*>(csm + o);
    o += (size_t)nc * 8;
    if (NUMERIC) {
      sval = reinterpret_cast<double*>(csm + o);
      o += (size_t)CS_ST * 8;
    }
    scol = reinterpret_cast<int32_t*>(csm + o);
    o += (size_t)CS_ST * 4;
    sch = reinterpret_cast<uint16_t*>(csm + o);
  }
  __shared__ int64_t s_off[CS_NJ + 1];
  __shared__ int64_t s_bs[CS_NJ];
  __shared__ double s_av[NUMERIC ? CS_NJ : 1];
  __shared__ int64_t ws[CS_NT / 32 + 1];
  __shared__ int s_item;
  const int tid = threadIdx.x;
  for (int i = tid; i < nc; i += CS_NT) h[i] = 0;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(item_ctr, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const CoarseItem ci = items[it];
    const int64_t t = ci.li - list_base;  // the row's index in the batch
    // the item's B rows: start, length (prefix sum) and A value
    int64_t L = 0, bs = 0;
    double av = 0.0;
    if (tid < ci.nj) {
      const int64_t j = ci.j0 + tid;
      const uint64_t sg = seg[j];
      bs = seg_start(sg);
      L = seg_length(sg);
      if (L == ((1 << (64 - SEG_BS_BITS)) - 1)) {  // saturated length: read it from B
        const int32_t c = A.col[j];
        L = B.rp[c + 1] - B.rp[c];
      }
      if (NUMERIC) av = A.val[j];
    }
    int64_t tot;
    const int64_t off = block_exclusive_scan<CS_NT>(L, ws, &tot);
    if (tid < CS_NJ) {
      s_off[tid] = off;
      s_bs[tid] = bs;
      if (NUMERIC) s_av[tid] = av;
    }
    __syncthreads();
    for (int64_t p0 = 0; p0 < tot; p0 += CS_ST) {
      const int n_st = (int)((tot - p0) < CS_ST ? (tot - p0) : CS_ST);
      int32_t col[CS_PER];
      double val[CS_PER];
      int rank[CS_PER];
#pragma unroll
      for (int k = 0; k < CS_PER; ++k) {
        const int q = k * CS_NT + tid;
        col[k] = -1;
        val[k] = 0.0;
        rank[k] = 0;
        if (q < n_st) {
          const int64_t p = p0 + q;
          const int g = upper_bound_i64(s_off, ci.nj, p) - 1;
          const int64_t kk = s_bs[g] + (p - s_off[g]);
          col[k] = __ldg(B.col + kk);
          if (NUMERIC) val[k] = s_av[g] * __ldg(B.val + kk);
        }
      }
#pragma unroll
      for (int k = 0; k < CS_PER; ++k)
        if (col[k] >= 0) rank[k] = atomicAdd(&h[col[k] >> sc], 1);
      if (!REORDER) continue;  // histogram: the counts accumulate over the item
      __syncthreads();
      // chunk offsets inside the sub-tile, and one reserved run per chunk
      int32_t run = 0;
      for (int i0 = 0; i0 < nc; i0 += CS_NT) {
        const int i = i0 + tid;
        const int64_t v = (i < nc) ? h[i] : 0;
        int64_t tsum;
        const int64_t ex = block_exclusive_scan<CS_NT>(v, ws, &tsum);
        if (i < nc) {
          hoff[i] = run + (int32_t)ex;
          if (v > 0) gbase[i] = (int64_t)atomicAdd(&cursor[t * nc + i], (unsigned long long)v);
        }
        run += (int32_t)tsum;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < CS_PER; ++k) {
        if (col[k] >= 0) {
          const int ch = col[k] >> sc;
          const int pos = hoff[ch] + rank[k];
          scol[pos] = col[k] - (ch << sc);
          if (NUMERIC) sval[pos] = val[k];
          sch[pos] = (uint16_t)ch;
        }
      }
      __syncthreads();
      for (int i = tid; i < n_st; i += CS_NT) {
        const int ch = sch[i];
        const int64_t gp = gbase[ch] + (i - hoff[ch]);
        st_stream(&chunk_col[gp], scol[i]);
        if (NUMERIC) st_stream(&chunk_val[gp], sval[i]);
      }
      for (int i = tid; i < nc; i += CS_NT) h[i] = 0;
      __syncthreads();
    }
    if (!REORDER) {
      __syncthreads();
      for (int i = tid; i < nc; i += CS_NT) {
        const int v = h[i];
        if (v > 0) {
          atomicAdd(reinterpret_cast<unsigned long long*>(&counts[t * nc + i]),
                    (unsigned long long)v);
          h[i] = 0;
        }
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_coarse_stage(bool reorder, bool numeric, const CoarseArgs& a,
                                cudaStream_t s) {
  if (a.n_items == 0) return cudaSuccess;
  const size_t smem = coarse_stage_smem(a.n_chunks, reorder, numeric);
  auto kern = reorder ? (numeric ? k_coarse_stage<true, true> : k_coarse_stage<true, false>)
                      : k_coarse_stage<false, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CS_NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (int64_t)a.num_sms * per_sm;
  if (blocks > a.n_items) blocks = a.n_items;
  e = cudaMemsetAsync(a.item_ctr, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)blocks, CS_NT, smem, s>>>(a.A, a.B, a.seg, a.items, a.n_items, a.item_ctr,
                                            a.list_base, a.shift_coarse, a.n_chunks, a.counts,
                                            a.cursor, a.chunk_col, a.chunk_val);
  count_launch();
  return cudaGetLastError();
}

}  // namespace magnus
