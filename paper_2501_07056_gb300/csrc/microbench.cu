// Building-block microbenchmark (Section 4.1, Figures 5-6): the steps of
// one reorder level applied to a stream of (index, value) pairs, each timed
// on the device, beside a copy of the stream (the streaming bound) and a
// dense accumulator over the whole index range in global memory (no
// locality generation).
//
//   histogram  count of the stream's elements per chunk (index >> shift),
//              one shared-memory histogram per block over a contiguous tile
//   scan       exclusive prefix over the (chunk, block) counts, chunk-major,
//              so every block knows where its part of each chunk starts
//   reorder    second pass over each tile writing (index - chunk base,
//              value) at the block's offset for the chunk, element by element,
//              and a staged variant that sorts each tile by chunk in shared
//              memory first and writes runs (<= 4096 chunks)
//   accumulate one block per chunk: shared-memory dense accumulator of the
//              chunk's 2^shift indices, emitted in index order (Algorithm 1)
//
// The accumulate step needs 2^shift <= 2^13 (one block's accumulator).
#include <algorithm>

#include "common.cuh"
#include "internal.h"

using namespace magnus;

namespace {

constexpr int MB_NT = 256;
constexpr int MB_MAX_CHUNKS_LOG2 = 14;
constexpr int MB_ACC_LOG2 = 13;

__global__ void k_mb_copy(const int32_t* __restrict__ col, const double* __restrict__ val,
                          int64_t n, int32_t* __restrict__ oc, double* __restrict__ ov) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    oc[i] = col[i];
    ov[i] = val[i];
  }
}

__global__ void k_mb_hist(const int32_t* __restrict__ col, int64_t n, int64_t tile, int shift,
                          int nch, int64_t* __restrict__ counts) {
  extern __shared__ int32_t sh_cnt[];
  for (int c = threadIdx.x; c < nch; c += blockDim.x) sh_cnt[c] = 0;
  __syncthreads();
  const int64_t b0 = (int64_t)blockIdx.x * tile;
  const int64_t b1 = std::min<int64_t>(n, b0 + tile);
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) atomicAdd(&sh_cnt[col[i] >> shift], 1);
  __syncthreads();
  for (int c = threadIdx.x; c < nch; c += blockDim.x)
    counts[(int64_t)c * gridDim.x + blockIdx.x] = sh_cnt[c];
}

__global__ void k_mb_reorder(const int32_t* __restrict__ col, const double* __restrict__ val,
                             int64_t n, int64_t tile, int shift, int nch,
                             const int64_t* __restrict__ offs, int32_t* __restrict__ oc,
                             double* __restrict__ ov) {
  extern __shared__ int32_t sh_cur[];
  for (int c = threadIdx.x; c < nch; c += blockDim.x) sh_cur[c] = 0;
  __syncthreads();
  const int64_t b0 = (int64_t)blockIdx.x * tile;
  const int64_t b1 = std::min<int64_t>(n, b0 + tile);
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    const int32_t c = col[i];
    const int ch = c >> shift;
    const int64_t pos = offs[(int64_t)ch * gridDim.x + blockIdx.x] + atomicAdd(&sh_cur[ch], 1);
    st_stream(&oc[pos], c - (ch << shift));
    st_stream(&ov[pos], val[i]);
  }
}

// Staged reorder (the GPU form of the paper's write-combining buffers for the
// reorder's streaming stores): a block loads a tile of MB_TILE elements,
// sorts it by chunk in shared memory (histogram, scan, scatter), and writes
// each chunk's run of the tile to consecutive global positions, so the
// stores coalesce instead of scattering element by element.  Per-chunk
// cursors carry the block's position in each chunk across its tiles.
constexpr int MB_TILE = 2048;
constexpr int MB_STAGED_MAX_CHUNKS = 4096;

__global__ void __launch_bounds__(MB_NT)
    k_mb_reorder_staged(const int32_t* __restrict__ col, const double* __restrict__ val,
                        int64_t n, int64_t tile, int shift, int nch,
                        const int64_t* __restrict__ offs, int32_t* __restrict__ oc,
                        double* __restrict__ ov) {
  extern __shared__ __align__(16) unsigned char sm[];
  int32_t* cur = reinterpret_cast<int32_t*>(sm);          // [nch] block's position per chunk
  int32_t* cnt = cur + nch;                               // [nch] tile histogram, then cursor
  int32_t* loff = cnt + nch;                              // [nch + 1] tile offsets
  int32_t* scol = loff + nch + 1;                         // [MB_TILE]
  double* sval = reinterpret_cast<double*>(sm + (((size_t)(3 * nch + 1 + MB_TILE) * 4 + 15) & ~(size_t)15));
  __shared__ int64_t ws[MB_NT / 32 + 1];
  for (int c = threadIdx.x; c < nch; c += MB_NT) cur[c] = 0;
  const int64_t b0 = (int64_t)blockIdx.x * tile;
  const int64_t b1 = std::min<int64_t>(n, b0 + tile);
  constexpr int PER = MB_TILE / MB_NT;
  for (int64_t t0 = b0; t0 < b1; t0 += MB_TILE) {
    for (int c = threadIdx.x; c < nch; c += MB_NT) cnt[c] = 0;
    __syncthreads();
    int32_t cl[PER];
    double vl[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int64_t i = t0 + k * MB_NT + threadIdx.x;
      cl[k] = i < b1 ? col[i] : -1;
      vl[k] = i < b1 ? val[i] : 0.0;
      if (cl[k] >= 0) atomicAdd(&cnt[cl[k] >> shift], 1);
    }
    __syncthreads();
    // exclusive scan of the tile histogram (chunks striped over threads)
    int32_t run = 0;
    for (int c0 = 0; c0 < nch; c0 += MB_NT) {
      const int c = c0 + threadIdx.x;
      const int64_t v = c < nch ? cnt[c] : 0;
      int64_t tot;
      const int64_t ex = block_exclusive_scan<MB_NT>(v, ws, &tot);
      if (c < nch) {
        loff[c] = run + (int32_t)ex;
        cnt[c] = 0;
      }
      run += (int32_t)tot;
    }
    if (threadIdx.x == 0) loff[nch] = run;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      if (cl[k] >= 0) {
        const int ch = cl[k] >> shift;
        const int p = loff[ch] + atomicAdd(&cnt[ch], 1);
        scol[p] = cl[k];
        sval[p] = vl[k];
      }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < run; p += MB_NT) {
      const int32_t c = scol[p];
      const int ch = c >> shift;
      const int64_t pos = offs[(int64_t)ch * gridDim.x + blockIdx.x] + cur[ch] + (p - loff[ch]);
      st_stream(&oc[pos], c - (ch << shift));
      st_stream(&ov[pos], sval[p]);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < nch; c += MB_NT) cur[c] += cnt[c];
    __syncthreads();
  }
}

// One block per chunk (persistent): dense accumulation, then the chunk's
// unique indices in order with their sums, written from the chunk's first
// element; nnz per chunk recorded.
__global__ void __launch_bounds__(MB_NT)
    k_mb_accum(const int32_t* __restrict__ ic, const double* __restrict__ iv,
               const int64_t* __restrict__ offs, int nblk, int nch, int shift,
               int32_t* __restrict__ oc, double* __restrict__ ov, int64_t* __restrict__ nnz) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int cl = 1 << shift;
  const int words = cl >= 32 ? cl >> 5 : 1;
  double* acc = reinterpret_cast<double*>(sm);
  uint32_t* bits = reinterpret_cast<uint32_t*>(sm + (size_t)cl * 8);
  __shared__ int64_t ws[MB_NT / 32 + 1];
  for (int i = threadIdx.x; i < cl; i += MB_NT) acc[i] = 0.0;
  for (int i = threadIdx.x; i < words; i += MB_NT) bits[i] = 0u;
  __syncthreads();
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const int64_t p0 = offs[(int64_t)c * nblk];
    const int64_t p1 = offs[(int64_t)(c + 1) * nblk];
    for (int64_t p = p0 + threadIdx.x; p < p1; p += MB_NT) {
      const int idx = ic[p];
      atomicOr(&bits[idx >> 5], 1u << (idx & 31));
      atomicAdd(&acc[idx], iv[p]);
    }
    __syncthreads();
    int64_t total = 0;
    for (int w0 = 0; w0 < words; w0 += MB_NT) {
      const int wd = w0 + threadIdx.x;
      uint32_t m = wd < words ? bits[wd] : 0u;
      int64_t tot;
      int64_t o = p0 + total + block_exclusive_scan<MB_NT>((int64_t)__popc(m), ws, &tot);
      if (wd < words) bits[wd] = 0u;
      while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        const int idx = wd * 32 + b;
        oc[o] = (c << shift) + idx;
        ov[o] = acc[idx];
        acc[idx] = 0.0;
        ++o;
      }
      total += tot;
    }
    if (threadIdx.x == 0) nnz[c] = total;
    __syncthreads();
  }
}

__global__ void k_mb_global(const int32_t* __restrict__ col, const double* __restrict__ val,
                            int64_t n, double* __restrict__ gacc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&gacc[col[i]], val[i]);
}

}  // namespace

extern "C" {

int magnus_microbench_chunks(const int32_t* col, const double* val, int64_t length, int64_t m,
                             int32_t n_chunks_log2, int32_t* out_col, double* out_val,
                             int64_t* chunk_nnz, magnus_microbench_t* res, void* stream) {
  if (!col || !val || !out_col || !out_val || !res || length < 1 || m < 1 ||
      m > ((int64_t)1 << 31) || n_chunks_log2 < 0 || n_chunks_log2 > MB_MAX_CHUNKS_LOG2)
    return MAGNUS_INVALID_ARG;
  int mbits = 0;
  while (((int64_t)1 << mbits) < m) ++mbits;
  const int shift = std::max(0, mbits - n_chunks_log2);
  const int nch = (int)((m + ((int64_t)1 << shift) - 1) >> shift);
  const bool accum = shift <= MB_ACC_LOG2;
  if (accum && !chunk_nnz) return MAGNUS_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int nblk = sms * 4;
  const int64_t tile = (length + nblk - 1) / nblk;
  const int64_t ncnt = (int64_t)nch * nblk;
  int64_t* offs = nullptr;
  int64_t* tmp = nullptr;
  double* gacc = nullptr;
  int32_t* scol = nullptr;
  double* sval = nullptr;
  cudaEvent_t ev[12];
  for (auto& e : ev) cudaEventCreate(&e);
  int st = MAGNUS_OK;
  auto fail = [&](cudaError_t e, const char* w) { st = api_cuda_fail(e, w); };
  cudaError_t e;
  if ((e = cudaMallocAsync(&offs, (size_t)(ncnt + 1) * 8, s)) != cudaSuccess) fail(e, "cudaMallocAsync");
  if (st == 0 && (e = cudaMallocAsync(&tmp, (size_t)(scan_tmp_elems(ncnt) + 2) * 8, s)) != cudaSuccess)
    fail(e, "cudaMallocAsync");
  if (st == 0 && (e = cudaMallocAsync(&gacc, (size_t)m * 8, s)) != cudaSuccess) fail(e, "cudaMallocAsync");
  if (st == 0 && (e = cudaMallocAsync(&scol, (size_t)length * 4, s)) != cudaSuccess) fail(e, "cudaMallocAsync");
  if (st == 0 && (e = cudaMallocAsync(&sval, (size_t)length * 8, s)) != cudaSuccess) fail(e, "cudaMallocAsync");
  const size_t hsm = (size_t)nch * 4;
  if (st == 0) {
    cudaFuncSetAttribute(k_mb_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm);
    cudaFuncSetAttribute(k_mb_reorder, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm);
    const unsigned g = (unsigned)sms * 8;
    cudaEventRecord(ev[0], s);
    k_mb_copy<<<g, MB_NT, 0, s>>>(col, val, length, out_col, out_val);
    cudaEventRecord(ev[1], s);
    k_mb_hist<<<nblk, MB_NT, hsm, s>>>(col, length, tile, shift, nch, offs);
    cudaEventRecord(ev[2], s);
    e = launch_exclusive_scan_i64(offs, ncnt, tmp, s);
    if (e != cudaSuccess) fail(e, "scan");
    cudaEventRecord(ev[3], s);
    k_mb_reorder<<<nblk, MB_NT, hsm, s>>>(col, val, length, tile, shift, nch, offs, scol, sval);
    cudaEventRecord(ev[4], s);
    if (nch <= MB_STAGED_MAX_CHUNKS) {
      // staged reorder into the same buffers (same positions per chunk)
      const size_t ssm = (((size_t)(3 * nch + 1 + MB_TILE) * 4 + 15) & ~(size_t)15) + (size_t)MB_TILE * 8;
      cudaFuncSetAttribute(k_mb_reorder_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm);
      cudaEventRecord(ev[8], s);
      k_mb_reorder_staged<<<nblk, MB_NT, ssm, s>>>(col, val, length, tile, shift, nch, offs, scol,
                                                   sval);
      cudaEventRecord(ev[9], s);
      count_launch();
    }
    cudaEventRecord(ev[10], s);
    if (accum) {
      const size_t asm_ = ((size_t)8 << shift) + (((size_t)1 << shift) >= 32 ? ((size_t)1 << shift) / 8 : 4);
      cudaFuncSetAttribute(k_mb_accum, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)asm_);
      int per = 1;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mb_accum, MB_NT, asm_);
      const int ga = std::min(nch, std::max(1, per) * sms);
      k_mb_accum<<<ga, MB_NT, asm_, s>>>(scol, sval, offs, nblk, nch, shift, out_col, out_val,
                                         chunk_nnz);
    }
    cudaEventRecord(ev[5], s);
    cudaMemsetAsync(gacc, 0, (size_t)m * 8, s);
    cudaEventRecord(ev[6], s);
    k_mb_global<<<g, MB_NT, 0, s>>>(col, val, length, gacc);
    cudaEventRecord(ev[7], s);
    count_launch(accum ? 5 : 4);
    e = cudaGetLastError();
    if (e != cudaSuccess) fail(e, "microbench launch");
    e = cudaEventSynchronize(ev[7]);
    if (st == 0 && e != cudaSuccess) fail(e, "cudaEventSynchronize");
  }
  if (st == 0) {
    float t[8] = {0};
    for (int i = 0; i < 4; ++i) cudaEventElapsedTime(&t[i], ev[i], ev[i + 1]);
    cudaEventElapsedTime(&t[4], ev[10], ev[5]);
    cudaEventElapsedTime(&t[5], ev[6], ev[7]);
    res->copy_ms = t[0];
    res->histogram_ms = t[1];
    res->scan_ms = t[2];
    res->reorder_ms = t[3];
    res->accumulate_ms = accum ? t[4] : -1.0f;
    res->global_accumulate_ms = t[5];
    res->reorder_staged_ms = -1.0f;
    if (nch <= MB_STAGED_MAX_CHUNKS) cudaEventElapsedTime(&res->reorder_staged_ms, ev[8], ev[9]);
    res->n_chunks = nch;
    res->chunk_len_log2 = shift;
  }
  for (void* p : {(void*)offs, (void*)tmp, (void*)gacc, (void*)scol, (void*)sval})
    if (p) cudaFreeAsync(p, s);
  for (auto& x : ev) cudaEventDestroy(x);
  return st;
}

}  // extern "C"
