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
#include <cstring>

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

// ---------------------------------------------------------------------------
// Rates of the GB300 operations the SpGEMM kernels are built from (no
// counterpart in the paper; these bound the kernels' rooflines):
//  * random gathers of chunks of 16..256 bytes at chunk-aligned offsets of a
//    large array (a B row is such a chunk; the sort kernels gather one per
//    nonzero of A), one chunk per chunk/16 lanes with 16-byte loads, and the
//    CSR form of a B row of 8 entries: 32 bytes of columns and 64 bytes of
//    values from two arrays;
//  * shared-memory accumulation: FP64 atomicAdd at distinct and at random
//    addresses and with 8 lanes per address, a plain FP64 add, and u32
//    atomicAdd, each thread updating an 8,192-entry block-private array.

__device__ __forceinline__ uint64_t mb_mix(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

template <int LP>  // lanes per chunk (chunk bytes / 16)
__global__ void k_mb_gather(const uint4* __restrict__ a, uint64_t nchunks, uint64_t work,
                            uint4* __restrict__ out) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
  uint4 acc = make_uint4(0, 0, 0, 0);
  for (uint64_t t = tid; t < work * LP; t += nthr) {
    const uint64_t c = mb_mix(t / LP) % nchunks;
    const uint4 v = __ldg(a + c * LP + (t % LP));
    acc.x ^= v.x;
    acc.y ^= v.y;
    acc.z ^= v.z;
    acc.w ^= v.w;
  }
  if ((acc.x ^ acc.y ^ acc.z ^ acc.w) == 0x9e3779b9u) out[tid & 1023] = acc;
}

// rows of 8 entries: 32 B of columns (2 lanes) and 64 B of values (4 lanes)
__global__ void k_mb_gather_csr(const uint4* __restrict__ cols, const uint4* __restrict__ vals,
                                uint64_t nrows, uint64_t work, uint4* __restrict__ out) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
  uint4 acc = make_uint4(0, 0, 0, 0);
  for (uint64_t t = tid; t < work * 4; t += nthr) {
    const uint64_t r = mb_mix(t / 4) % nrows;
    const int q = (int)(t % 4);
    uint4 v = __ldg(vals + r * 4 + q);
    if (q < 2) {
      const uint4 w = __ldg(cols + r * 2 + q);
      v.x ^= w.x;
      v.y ^= w.y;
    }
    acc.x ^= v.x;
    acc.y ^= v.y;
    acc.z ^= v.z;
    acc.w ^= v.w;
  }
  if ((acc.x ^ acc.y ^ acc.z ^ acc.w) == 0x9e3779b9u) out[tid & 1023] = acc;
}

constexpr int MB_ACC_N = 8192;

__device__ __forceinline__ uint32_t mb_hash(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

// MODE 0 f64 atomic distinct, 1 f64 atomic random, 2 f64 atomic 8 lanes per
// address, 3 plain f64 add (distinct), 4 u32 atomic random
template <int MODE>
__global__ void __launch_bounds__(MB_NT) k_mb_atomics(int iters, double* __restrict__ out) {
  extern __shared__ double acc_s[];
  for (int i = threadIdx.x; i < MB_ACC_N; i += blockDim.x) acc_s[i] = 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const double v = 1.0 + threadIdx.x * 1e-3;
  for (int it = 0; it < iters; ++it) {
    int idx;
    if (MODE == 0 || MODE == 3) idx = (w * 1024 + it * 32 + lane) & (MB_ACC_N - 1);
    else if (MODE == 2) idx = (int)(mb_hash(it * 64 + w * 4 + (lane >> 3)) & (MB_ACC_N - 1));
    else idx = (int)(mb_hash(it * 256 + threadIdx.x + blockIdx.x * 7919) & (MB_ACC_N - 1));
    if (MODE <= 2) atomicAdd(&acc_s[idx], v);
    else if (MODE == 3) acc_s[idx] += v;
    else atomicAdd(reinterpret_cast<unsigned*>(acc_s) + 2 * idx, 1u);
  }
  __syncthreads();
  double t = 0.0;
  for (int i = threadIdx.x; i < MB_ACC_N; i += blockDim.x) t += acc_s[i];
  if (t == -1.0) out[blockIdx.x] = t;
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

/* magnus_microbench_rates: see magnus.h. */
int magnus_microbench_rates(magnus_rates_t* r, void* stream) {
  if (!r) return MAGNUS_INVALID_ARG;
  memset(r, 0, sizeof(*r));
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return api_cuda_fail(cudaGetLastError(), "cudaDeviceGetAttribute");
  const size_t bytes = (size_t)2 << 30;
  uint4* a = nullptr;
  uint4* o = nullptr;
  double* od = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&a), bytes, s);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&o), 1024 * sizeof(uint4), s);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&od), 4096 * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(a, 1, bytes, s);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const uint64_t work = (uint64_t)64 << 20;  // chunks per gather launch
  const unsigned gb = (unsigned)sms * 8;
  auto timed = [&](auto launch, float* out_ms) {
    if (e != cudaSuccess) return;
    launch();
    e = cudaEventRecord(e0, s);
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    *out_ms = ms / 3.f;
    count_launch(4);
  };
  const double gch = (double)work;
  float ms = 0.f;
  timed([&] { k_mb_gather<1><<<gb, MB_NT, 0, s>>>(a, bytes / 16, work, o); }, &ms);
  r->gather_16 = gch / (ms * 1e-3);
  timed([&] { k_mb_gather<2><<<gb, MB_NT, 0, s>>>(a, bytes / 32, work, o); }, &ms);
  r->gather_32 = gch / (ms * 1e-3);
  timed([&] { k_mb_gather<4><<<gb, MB_NT, 0, s>>>(a, bytes / 64, work, o); }, &ms);
  r->gather_64 = gch / (ms * 1e-3);
  timed([&] { k_mb_gather<8><<<gb, MB_NT, 0, s>>>(a, bytes / 128, work, o); }, &ms);
  r->gather_128 = gch / (ms * 1e-3);
  timed([&] { k_mb_gather<16><<<gb, MB_NT, 0, s>>>(a, bytes / 256, work, o); }, &ms);
  r->gather_256 = gch / (ms * 1e-3);
  {
    const uint64_t nrows = (bytes / 3) / 32;  // 32 B of columns + 64 B of values each
    timed([&] { k_mb_gather_csr<<<gb, MB_NT, 0, s>>>(a, a + nrows * 2, nrows, work, o); }, &ms);
    r->gather_csr_row8 = gch / (ms * 1e-3);
  }
  // shared-memory accumulation: 3 blocks of 64 KB per SM
  const unsigned ga = (unsigned)sms * 3;
  const size_t smem = MB_ACC_N * sizeof(double);
  auto atom = [&](auto kern, int iters, double* out_rate) {
    if (e != cudaSuccess) return;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    timed([&] { kern<<<ga, MB_NT, smem, s>>>(iters, od); }, &ms);
    *out_rate = (double)ga * MB_NT * iters / (ms * 1e-3);
  };
  atom(k_mb_atomics<0>, 2048, &r->smem_f64_atomic_distinct);
  atom(k_mb_atomics<1>, 2048, &r->smem_f64_atomic_random);
  atom(k_mb_atomics<2>, 512, &r->smem_f64_atomic_8_per_address);
  atom(k_mb_atomics<3>, 2048, &r->smem_f64_add_plain);
  atom(k_mb_atomics<4>, 2048, &r->smem_u32_atomic_random);
  r->sms = sms;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(a, s);
  cudaFreeAsync(o, s);
  cudaFreeAsync(od, s);
  const cudaError_t fin = e == cudaSuccess ? cudaStreamSynchronize(s) : e;
  return fin == cudaSuccess ? MAGNUS_OK : api_cuda_fail(fin, "magnus_microbench_rates");
}

}  // extern "C"
