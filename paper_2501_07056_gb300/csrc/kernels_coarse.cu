// Coarse level (Algorithm 4) for one batch of coarse rows (Section 3.3):
//   1. coarseRowsB and the CSC form of the batch's submatrix of A
//      (histogram, prefix sum, scatter);
//   2. outer-product histogram: for each needed B row and each batch row i
//      that references it, countsCoarse[i][B.col >> shiftCoarse] += 1;
//   3. row-chained prefix sum (one exclusive scan of the row-major
//      countsCoarse matrix gives every row's chunk offsets after the previous
//      row's);
//   4. outer-product reorder: the products A.val * B.val with their
//      chunk-local columns are written at offsetsCoarse + running count;
//   5. the fine level on every (row, coarse chunk): a warp sort for small
//      chunks, a thread block running Algorithm 3 for large ones.
// Each B row is loaded once per batch and reused for every batch row that
// references it (the reason Algorithm 4 uses the outer product).
#include <type_traits>

#include "fine_level.cuh"
#include "sort_accum.cuh"

namespace magnus {

static inline unsigned grid_cap_c(int64_t blocks, int64_t cap) {
  return (unsigned)(blocks < cap ? (blocks < 1 ? 1 : blocks) : cap);
}

__global__ void k_csc_count(Csr A, const int32_t* __restrict__ rows, int64_t nb,
                            int32_t* __restrict__ col_cnt, int32_t* __restrict__ rows_b,
                            int32_t* __restrict__ n_rows_b) {
  const int lane = lane_id();
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nb; t += nw) {
    const int32_t row = rows[t];
    for (int64_t j = A.rp[row] + lane; j < A.rp[row + 1]; j += 32) {
      const int32_t b = A.col[j];
      if (atomicAdd(&col_cnt[b], 1) == 0) rows_b[atomicAdd(n_rows_b, 1)] = b;
    }
  }
}

template <bool NUMERIC>
__global__ void k_csc_fill(Csr A, const int32_t* __restrict__ rows, int64_t nb,
                           const int64_t* __restrict__ col_ptr, int32_t* __restrict__ cursor,
                           int32_t* __restrict__ csc_row, double* __restrict__ csc_val) {
  const int lane = lane_id();
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nb; t += nw) {
    const int32_t row = rows[t];
    for (int64_t j = A.rp[row] + lane; j < A.rp[row + 1]; j += 32) {
      const int32_t b = A.col[j];
      const int64_t pos = col_ptr[b] + atomicAdd(&cursor[b], 1);
      csc_row[pos] = (int32_t)t;
      if (NUMERIC) csc_val[pos] = A.val[j];
    }
  }
}

// Outer-product traversal, load balanced.  The work of B row b is
// nnz(B_b) x nnz(column b of A^CSC) products; it is cut into items of
// 32 consecutive entries of the B row times outer_et(L) consecutive entries
// of the A^CSC column (at most 1024 products), and every warp takes an equal
// contiguous range of items.  Lanes hold one entry of the B row each and
// reuse it for every A^CSC entry of the item.  A B row of L < 32 entries
// takes Lp = next power of two >= L lanes, so 32 / Lp A^CSC entries share
// one warp step, and its items are 32 / Lp times longer.  Lanes hitting the
// same (row, chunk) are combined with match_any so one atomic serves them.
constexpr int OUTER_ET = 32;

__device__ __forceinline__ int outer_lanes(int64_t L) {
  int lp = 1;
  while (lp < L && lp < 32) lp <<= 1;
  return lp;
}

__device__ __forceinline__ int64_t outer_et(int64_t L) {
  return (int64_t)OUTER_ET * (32 / outer_lanes(L));
}

__global__ void k_outer_items(const int64_t* __restrict__ b_rp, const int64_t* __restrict__ col_ptr,
                              int64_t nB, int64_t* __restrict__ items) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nB;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t L = b_rp[b + 1] - b_rp[b];
    const int64_t C = col_ptr[b + 1] - col_ptr[b];
    const int64_t et = outer_et(L);
    items[b] = (L > 0 && C > 0) ? ((L + 31) / 32) * ((C + et - 1) / et) : 0;
  }
}

template <bool REORDER, bool NUMERIC>
__global__ void k_coarse_outer(Csr B, const int64_t* __restrict__ item_off, int64_t nB,
                               const int64_t* __restrict__ col_ptr,
                               const int32_t* __restrict__ csc_row,
                               const double* __restrict__ csc_val, int sc, int nc,
                               int64_t* __restrict__ counts,
                               unsigned long long* __restrict__ cursor,
                               int32_t* __restrict__ chunk_col, double* __restrict__ chunk_val) {
  const int lane = lane_id();
  const int64_t total = item_off[nB];
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t per = (total + nwarps - 1) / nwarps;
  int64_t it = wid * per;
  const int64_t it_end = (it + per < total) ? it + per : total;
  if (it >= it_end) return;
  int64_t b = upper_bound_i64(item_off, (int)(nB + 1), it) - 1;
  while (it < it_end) {
    if (item_off[b + 1] <= it) b = upper_bound_i64(item_off, (int)(nB + 1), it) - 1;
    const int64_t bs = B.rp[b];
    const int64_t L = B.rp[b + 1] - bs;
    const int64_t cs = col_ptr[b], C = col_ptr[b + 1] - cs;
    const int64_t EB = (L + 31) / 32;
    const int64_t li = it - item_off[b];
    const int64_t et = li / EB, eb = li - et * EB;
    const int Lt = (int)((L - eb * 32) < 32 ? (L - eb * 32) : 32);
    const int Lp = outer_lanes(Lt);
    const int G = 32 / Lp;
    const int64_t ET = outer_et(L);
    const int sub = lane / Lp, kk = lane & (Lp - 1);
    const bool valid = kk < Lt;
    const int64_t k = eb * 32 + kk;
    const int32_t col = valid ? B.col[bs + k] : 0;
    const double bv = (NUMERIC && valid) ? B.val[bs + k] : 0.0;
    const int chunk = col >> sc;
    const int64_t e0 = cs + et * ET;
    const int64_t e1 = (e0 + ET < cs + C) ? e0 + ET : cs + C;
    // the A^CSC entry of the next step is loaded one step ahead
    int32_t t_nx = (valid && e0 + sub < e1) ? csc_row[e0 + sub] : 0;
    double av_nx = (NUMERIC && valid && e0 + sub < e1) ? csc_val[e0 + sub] : 0.0;
    for (int64_t eg = e0; eg < e1; eg += G) {
      const int64_t e = eg + sub;
      const bool on = valid && e < e1;
      const int32_t t = t_nx;
      const double av = av_nx;
      const int64_t en = e + G;
      if (valid && en < e1) {
        t_nx = csc_row[en];
        if (NUMERIC) av_nx = csc_val[en];
      }
      const unsigned active = __ballot_sync(FULL, on);
      if (on) {
        const int64_t slot = (int64_t)t * nc + chunk;
        const unsigned m = __match_any_sync(active, (unsigned long long)slot);
        const int leader = __ffs(m) - 1;
        if (!REORDER) {
          if (lane == leader)
            atomicAdd(reinterpret_cast<unsigned long long*>(&counts[slot]),
                      (unsigned long long)__popc(m));
        } else {
          // the cursor starts at the bucket's offset: one atomic gives the
          // group's absolute position
          unsigned long long base = 0;
          if (lane == leader) base = atomicAdd(&cursor[slot], (unsigned long long)__popc(m));
          base = __shfl_sync(m, base, leader);
          const int64_t pos = (int64_t)base + __popc(m & ((1u << lane) - 1));
          st_stream(&chunk_col[pos], col - (chunk << sc));
          if (NUMERIC) st_stream(&chunk_val[pos], av * bv);
        }
      }
    }
    ++it;
  }
}

// Output offset of every (batch row, coarse chunk) inside its row of C:
// exclusive prefix over the chunks of the row's symbolic chunk counts.
__global__ void k_bucket_offsets(const int32_t* __restrict__ bucket_cnt, int64_t nb, int nc,
                                 int64_t list_base, int64_t* __restrict__ bucket_out) {
  const int lane = lane_id();
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nb; t += nw) {
    int64_t run = 0;
    for (int c0 = 0; c0 < nc; c0 += 32) {
      const int c = c0 + lane;
      const int64_t v = (c < nc) ? bucket_cnt[(list_base + t) * nc + c] : 0;
      const int64_t inc = warp_inclusive_scan(v);
      if (c < nc) bucket_out[t * nc + c] = run + inc - v;
      run += __shfl_sync(FULL, inc, 31);
    }
  }
}

__global__ void k_row_totals(const int32_t* __restrict__ bucket_cnt, const int32_t* __restrict__ rows,
                             int64_t nb, int nc, int64_t list_base, int64_t* __restrict__ out_cnt) {
  const int lane = lane_id();
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nb; t += nw) {
    int64_t s = 0;
    for (int c = lane; c < nc; c += 32) s += bucket_cnt[(list_base + t) * nc + c];
    s = warp_sum(s);
    if (lane == 0) out_cnt[rows[t]] = s;
  }
}

// Small coarse chunks (at most 256 products): one warp sorts and merges.
template <int E, typename K, bool NUMERIC>
__device__ __forceinline__ int bucket_warp(const int32_t* __restrict__ ccol,
                                           const double* __restrict__ cval, int n, double* vals,
                                           K* skeys, int32_t col_add, int32_t* out_col,
                                           double* out_val) {
  using KT = KeyTraits<K>;
  constexpr int SB = Log2Cap<E>::v;
  const int lane = lane_id();
  K key[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int s = e * 32 + lane;
    if (s < n) {
      key[e] = KT::template make<SB>(ccol[s], s);
      if (NUMERIC) vals[s] = cval[s];
    } else {
      key[e] = ~K(0);
    }
  }
  warp_bitonic_sort<E>(key);
  __syncwarp();
  return warp_merge_emit<E, K, NUMERIC>(key, n, vals, skeys, col_add, out_col, out_val);
}

constexpr int BK_NW = 4;

template <typename K, bool NUMERIC>
__global__ void __launch_bounds__(BK_NW * 32)
    k_bucket_small(const int64_t* __restrict__ offs, int64_t nbk, const int32_t* __restrict__ chunk_col,
                   const double* __restrict__ chunk_val, int sc, int nc, int64_t list_base,
                   const int32_t* __restrict__ rows, int32_t* __restrict__ bucket_cnt,
                   const int64_t* __restrict__ bucket_out, const int64_t* __restrict__ c_rp, const int64_t* __restrict__ c_base,
                   int32_t* __restrict__ c_col, double* __restrict__ c_val,
                   BigBucket* __restrict__ big_list, int32_t* __restrict__ n_big,
                   unsigned long long* __restrict__ big_stats, int mid_max) {
  __shared__ double s_vals[BK_NW][NUMERIC ? SORT_MAX : 1];
  __shared__ K s_keys[BK_NW][NUMERIC ? SORT_MAX : 1];
  const int lane = lane_id(), w = warp_id();
  const int64_t nw = (int64_t)gridDim.x * BK_NW;
  unsigned long long big_p = 0, big_z = 0, big_n = 0;  // lane 0's tallies
  for (int64_t id = (int64_t)blockIdx.x * BK_NW + w; id < nbk; id += nw) {
    const int64_t p0 = offs[id];
    const int n = (int)(offs[id + 1] - p0);
    const int64_t t = id / nc;
    const int c = (int)(id - t * nc);
    if (n > SORT_MAX) {
      if (lane == 0) {
        // the whole record of the bucket, so the large-bucket kernels start
        // each bucket from one load instead of a chain of dependent ones
        BigBucket bb;
        bb.p0 = p0;
        bb.n = n;
        bb.c = c;
        bb.out = NUMERIC ? c_rp[rows[t]] - (c_base ? *c_base : 0) + bucket_out[id]
                         : (list_base + t) * nc + c;
        // buckets of at most mid_max products from the front of the list
        // (the block sort, n_big[1] of them), larger ones from the back (the
        // block dense accumulator or the fine level, n_big[0] of them)
        if (n <= mid_max) big_list[atomicAdd(&n_big[1], 1)] = bb;
        else big_list[nbk - 1 - atomicAdd(&n_big[0], 1)] = bb;
        big_p += (unsigned long long)n;
        big_n += 1;
        if (NUMERIC) big_z += (unsigned long long)bucket_cnt[(list_base + t) * nc + c];
      }
      continue;
    }
    int32_t* oc = nullptr;
    double* ov = nullptr;
    if (NUMERIC) {
      if (n == 0) continue;
      const int64_t o = c_rp[rows[t]] - (c_base ? *c_base : 0) + bucket_out[id];
      oc = c_col + o;
      ov = c_val + o;
    }
    int cnt = 0;
    if (n > 0) {
      const int32_t col_add = c << sc;
      const int32_t* cc = chunk_col + p0;
      const double* cv = NUMERIC ? chunk_val + p0 : nullptr;
      if (n <= 32) cnt = bucket_warp<1, K, NUMERIC>(cc, cv, n, s_vals[w], s_keys[w], col_add, oc, ov);
      else if (n <= 64) cnt = bucket_warp<2, K, NUMERIC>(cc, cv, n, s_vals[w], s_keys[w], col_add, oc, ov);
      else if (n <= 128) cnt = bucket_warp<4, K, NUMERIC>(cc, cv, n, s_vals[w], s_keys[w], col_add, oc, ov);
      else cnt = bucket_warp<8, K, NUMERIC>(cc, cv, n, s_vals[w], s_keys[w], col_add, oc, ov);
    }
    if (!NUMERIC && lane == 0) bucket_cnt[(list_base + t) * nc + c] = cnt;
    __syncwarp();
  }
  if (big_stats && lane == 0 && big_n > 0) {
    atomicAdd(&big_stats[0], big_p);
    atomicAdd(&big_stats[1], big_z);
    atomicAdd(&big_stats[2], big_n);
  }
}

// Large coarse chunks: one block runs the fine level (Algorithm 3) on the
// chunk's staged products: histogram and reorder into the second staging
// buffer by fine chunk, then warp-private dense accumulation.  The fine
// shift is min(sc, sf) (the launch sizes shared memory with it).
template <bool NUMERIC, bool HYBRID>
__global__ void __launch_bounds__(FNT)
    k_bucket_big(const BigBucket* __restrict__ big_end,
                 const int32_t* __restrict__ n_big, const int32_t* __restrict__ chunk_col,
                 const double* __restrict__ chunk_val, int32_t* __restrict__ fine_col,
                 double* __restrict__ fine_val, int sc, int sf,
                 int32_t* __restrict__ bucket_cnt, int32_t* __restrict__ c_col,
                 double* __restrict__ c_val, int dthr, int hash) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const int shift = sf < sc ? sf : sc;
  const FineSmem f = fine_carve(fsm, NUMERIC, shift, HYBRID);
  __shared__ int64_t ws[FNT / 32 + 1];
  const int nbig = *n_big;
  const int nch = 1 << (sc - shift);
  fine_clear<NUMERIC>(f, shift);
  BigBucket nxt{};
  if (blockIdx.x < nbig) nxt = big_end[-1 - (int64_t)blockIdx.x];
  for (int q = blockIdx.x; q < nbig; q += gridDim.x) {
    const BigBucket bb = nxt;
    if (q + gridDim.x < nbig) nxt = big_end[-1 - (int64_t)(q + gridDim.x)];  // in flight
    const int64_t p0 = bb.p0;
    const int n = bb.n;
    const int c = bb.c;
    const int64_t col_base = (int64_t)c << sc;
    int32_t* oc = nullptr;
    double* ov = nullptr;
    if (NUMERIC) {
      oc = c_col + bb.out;
      ov = c_val + bb.out;
    }
    const int32_t* cc = chunk_col + p0;
    const double* cv = NUMERIC ? chunk_val + p0 : nullptr;
    int64_t cnt;
    if (nch == 1) {
      if (threadIdx.x == 0) {
        f.off[0] = 0;
        f.off[1] = n;
      }
      __syncthreads();
      cnt = warp_chunks_accumulate<NUMERIC, HYBRID>(f, 1, shift, cc, cv, col_base, oc, ov, dthr, hash);
    } else {
      // histogram over the fine chunks of the coarse chunk
      for (int i = threadIdx.x; i < nch; i += FNT) f.cnt[i] = 0;
      __syncthreads();
      for (int p = threadIdx.x; p < n; p += FNT) atomicAdd(&f.cnt[cc[p] >> shift], 1);
      __syncthreads();
      int32_t run = 0;
      for (int i0 = 0; i0 < nch; i0 += FNT) {
        const int i = i0 + threadIdx.x;
        const int64_t v = (i < nch) ? f.cnt[i] : 0;
        int64_t tot;
        const int64_t ex = block_exclusive_scan<FNT>(v, ws, &tot);
        if (i < nch) {
          f.off[i] = run + (int32_t)ex;
          f.cnt[i] = 0;
        }
        run += (int32_t)tot;
      }
      if (threadIdx.x == 0) f.off[nch] = run;
      __syncthreads();
      int32_t* fc = fine_col + p0;
      double* fv = NUMERIC ? fine_val + p0 : nullptr;
      for (int p = threadIdx.x; p < n; p += FNT) {
        const int32_t col = cc[p];
        const int ch = col >> shift;
        const int pos = f.off[ch] + atomicAdd(&f.cnt[ch], 1);
        st_stream(&fc[pos], col);
        if (NUMERIC) st_stream(&fv[pos], cv[p]);
      }
      __syncthreads();
      cnt = warp_chunks_accumulate<NUMERIC, HYBRID>(f, nch, shift, fc, fv, col_base, oc, ov, dthr, hash);
    }
    if (!NUMERIC && threadIdx.x == 0) bucket_cnt[bb.out] = (int32_t)cnt;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// One-dimensional bulk copies (the TMA engine's cp.async.bulk) from global
// to shared memory, completed on an mbarrier with a transaction count.
// Every wait is bounded by the SM clock (about a second); a wait that gives
// up sets g_wait_timeout, which the host reads and clears
// (wait_timeout_take, behind magnus_symbolic and magnus_device_status).
__device__ int g_wait_timeout;

constexpr long long WAIT_CYCLES = 1ll << 31;  // about one second at 2 GHz

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one arrival that also announces `bytes` of copies to come
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_to_shared(void* dst, const void* src, unsigned bytes,
                                               uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// shared-memory reads of the generic proxy are ordered before the next bulk
// copy into the same buffer
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// true when the barrier's phase of this parity completed within the bound
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity,
                                          long long limit = WAIT_CYCLES) {
  const unsigned a = smem_addr(bar);
  const long long t0 = clock64();
  for (;;) {
    unsigned done;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

// Self-test of the bounded wait: one thread announces 16 bytes on an
// mbarrier and issues no copy, so the phase never completes; the wait gives
// up after `limit` SM clocks and raises g_wait_timeout.  No copy is ever in
// flight, so the block may end at once.
__global__ void k_wait_selftest(long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
    mbar_arrive_expect(&bar, 16u);
    if (!mbar_wait(&bar, 0u, limit)) atomicExch(&g_wait_timeout, 1);
  }
}

cudaError_t launch_wait_selftest(long long limit, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(limit);
  count_launch();
  return cudaGetLastError();
}

// Reads and clears the bounded-wait flag (synchronises the stream).
cudaError_t wait_timeout_take(int* timed_out, cudaStream_t s) {
  int h = 0;
  const int zero = 0;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&h, g_wait_timeout, sizeof(int));
  if (e == cudaSuccess && h) e = cudaMemcpyToSymbol(g_wait_timeout, &zero, sizeof(int));
  *timed_out = h;
  return e;
}

// Coarse buckets of 257..BS_CAP products: the sort accumulator widened to
// a thread block (Algorithm 2; the per-chunk hybrid of Section 3.4 choosing
// sort for the smaller chunks).  A bucket's staged products are contiguous,
// so one thread stages them into shared memory with two bulk copies
// (columns, values) while the block still works on the previous bucket:
// the buffers alternate, and the next bucket's copies are issued before the
// current bucket's are awaited.  Keys (chunk-local column, position in the
// bucket) are sorted (bucket_sort_keys), and the runs of equal columns
// summed in position order, so the bucket needs no atomics at all (a dense
// accumulator's FP64 atomics contend on the hub columns of power-law rows).
// Emission is striped: thread t takes sorted positions t, t + BS_NT, ...,
// whose ranks among the run heads come from a prefix over a head bitmap, so
// consecutive threads write consecutive entries of C.
constexpr int BS_NT = 256;
constexpr int BS_CAP = BS_NT * BR;  // 2,048 products
constexpr int BS_PB = 11;           // position bits of a key
// one staging buffer: the bucket's columns from the 16-byte boundary at or
// below its first product to the one at or above its end (at most 6 more
// entries than the bucket), and its values likewise (at most 2 more)
constexpr int BS_CB = (BS_CAP + 8) * 4;
constexpr int BS_VB = (BS_CAP + 4) * 8;

inline size_t bucket_sort_smem(bool numeric) {
  return 2 * (size_t)BS_CB + (numeric ? 2 * (size_t)BS_VB : 0);
}

// Issued by one thread: the bulk copies of bucket bb into one buffer pair.
// The staging arrays are carved with 16-byte aligned starts and padded at
// the end, so the rounded windows stay inside them.
template <bool NUMERIC>
__device__ __forceinline__ void stage_bucket(const BigBucket& bb, const int32_t* chunk_col,
                                             const double* chunk_val, unsigned char* cbuf,
                                             unsigned char* vbuf, uint64_t* bar) {
  const int64_t c0 = bb.p0 & ~(int64_t)3, c1 = (bb.p0 + bb.n + 3) & ~(int64_t)3;
  const unsigned cbytes = (unsigned)(c1 - c0) * 4u;
  unsigned vbytes = 0;
  int64_t v0 = 0;
  if (NUMERIC) {
    v0 = bb.p0 & ~(int64_t)1;
    const int64_t v1 = (bb.p0 + bb.n + 1) & ~(int64_t)1;
    vbytes = (unsigned)(v1 - v0) * 8u;
  }
  fence_proxy_async();
  mbar_arrive_expect(bar, cbytes + vbytes);
  if (cbytes) bulk_to_shared(cbuf, chunk_col + c0, cbytes, bar);
  if (NUMERIC && vbytes) bulk_to_shared(vbuf, chunk_val + v0, vbytes, bar);
}

// Block sort of one bucket's keys (chunk-local column << PB | position) by
// column sub-ranges: the bucket's column range is split into 2*NT
// sub-ranges (the high word of the column's offset from the smallest column
// times a per-bucket multiplier, monotone in the column), the keys are
// counted and scattered into their sub-ranges through shared memory, and
// every thread sorts its two adjacent sub-ranges in registers (odd-even
// merge networks: each of 16 keys, or both together as 32 when some
// sub-range holds more than 16).  That is about a third of the
// compare-exchanges of the block bitonic network, with four barriers instead
// of its shared-memory stages.  A pair of more than 32 keys (a narrow or
// skewed bucket) sends the bucket to block_sort_keys.  On return
// key[e] holds sorted position t*BR + e, as block_sort_keys leaves it.
template <int NT, int PB, typename K>
__device__ __forceinline__ void bucket_sort_keys(K (&key)[BR], int n, K* s_key, int32_t* s_cnt,
                                                 int32_t* s_bst, uint32_t* s_red, int32_t* s_ws) {
  constexpr int NWB = NT / 32;
  constexpr int NS = 2 * NT;  // sub-ranges: thread t owns 2t and 2t + 1
  const int t = threadIdx.x, lane = lane_id(), w = warp_id();
  uint32_t mn = 0xffffffffu, mx = 0u;
#pragma unroll
  for (int e = 0; e < BR; ++e) {
    if (e * NT + t < n) {
      const uint32_t c = (uint32_t)(key[e] >> PB);
      mn = min(mn, c);
      mx = max(mx, c);
    }
  }
  mn = warp_min(mn);
  mx = warp_max(mx);
  if (lane == 0) {
    s_red[w] = mn;
    s_red[NWB + w] = mx;
  }
  s_cnt[2 * t] = 0;
  s_cnt[2 * t + 1] = 0;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NWB; ++i) {
    mn = min(mn, s_red[i]);
    mx = max(mx, s_red[NWB + i]);
  }
  const uint32_t range = mx - mn + 1u;
  const uint32_t mul =
      range <= (uint32_t)NS ? 0u
                            : (uint32_t)fminf((float)NS * 4294967296.0f / (float)range, 4294967040.0f);
  uint32_t br[BR];  // sub-range << 16 | rank in it
#pragma unroll
  for (int e = 0; e < BR; ++e) {
    br[e] = 0u;
    if (e * NT + t < n) {
      const uint32_t o = (uint32_t)(key[e] >> PB) - mn;
      const uint32_t b = range <= (uint32_t)NS ? o : min(__umulhi(o, mul), (uint32_t)NS - 1u);
      br[e] = (b << 16) | (uint32_t)atomicAdd(&s_cnt[b], 1);
    }
  }
  __syncthreads();
  const int c0 = s_cnt[2 * t], c1 = s_cnt[2 * t + 1];
  // each sub-range sorted alone when all hold at most 16 keys, else each
  // thread's pair together when all pairs hold at most 32
  const bool over32 = __syncthreads_or(c0 + c1 > 32) != 0;
  const bool over16 = __syncthreads_or(c0 > 16 || c1 > 16) != 0;
  int tot;
  const int st = block_exclusive_scan<NT>(c0 + c1, s_ws, &tot);
  s_bst[2 * t] = st;
  s_bst[2 * t + 1] = st + c0;
  __syncthreads();
#pragma unroll
  for (int e = 0; e < BR; ++e)
    if (e * NT + t < n) s_key[s_bst[br[e] >> 16] + (int)(br[e] & 0xffffu)] = key[e];
  __syncthreads();
  if (over32) {  // the block network, on the keys in any order
#pragma unroll
    for (int e = 0; e < BR; ++e) key[e] = e * NT + t < n ? s_key[e * NT + t] : ~K(0);
    __syncthreads();
    block_sort_keys<NT>(key, s_key);
    return;
  }
  auto sort_run = [&](auto nk, int from, int c) {
    constexpr int N = decltype(nk)::value;
    K kk[N];
#pragma unroll
    for (int i = 0; i < N; ++i) kk[i] = i < c ? s_key[from + i] : ~K(0);
    lane_oddeven_sort<N>(kk);
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i < c) s_key[from + i] = kk[i];
  };
  if (over16) {
    sort_run(std::integral_constant<int, 32>{}, st, c0 + c1);
  } else {
    sort_run(std::integral_constant<int, 16>{}, st, c0);
    sort_run(std::integral_constant<int, 16>{}, st + c0, c1);
  }
  __syncthreads();
#pragma unroll
  for (int e = 0; e < BR; ++e) {
    const int q = t * BR + e;
    key[e] = q < n ? s_key[q] : ~K(0);
  }
  __syncthreads();
}

template <typename K, bool NUMERIC>
__global__ void __launch_bounds__(BS_NT, 4)
    k_bucket_sort(const BigBucket* __restrict__ list, const int32_t* __restrict__ n_list,
                  const int32_t* __restrict__ chunk_col, const double* __restrict__ chunk_val,
                  int sc, int32_t* __restrict__ bucket_cnt, int32_t* __restrict__ c_col,
                  double* __restrict__ c_val) {
  extern __shared__ __align__(128) unsigned char bsm[];  // two column, two value buffers
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ K s_key[BS_CAP];
  __shared__ uint32_t s_head[BS_CAP / 32];
  __shared__ int32_t s_hpre[BS_CAP / 32 + 1];
  __shared__ int32_t s_cnt[2 * BS_NT];
  __shared__ int32_t s_bst[2 * BS_NT];
  __shared__ uint32_t s_red[2 * (BS_NT / 32)];
  __shared__ int32_t s_ws[BS_NT / 32 + 1];
  const int t = threadIdx.x;
  const int lane = lane_id(), w = warp_id();
  constexpr K PMASK = (K(1) << BS_PB) - 1;
  if (t == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  const int nl = *n_list;
  BigBucket nxt{};
  if (blockIdx.x < nl) {
    nxt = list[blockIdx.x];
    if (t == 0) stage_bucket<NUMERIC>(nxt, chunk_col, chunk_val, bsm, bsm + 2 * BS_CB, &s_bar[0]);
  }
  int buf = 0;
  unsigned phases = 0u;  // bit b: parity of buffer b's next completion
  for (int q = blockIdx.x; q < nl; q += gridDim.x) {
    const BigBucket bb = nxt;
    const bool more = q + gridDim.x < nl;
    if (more) {  // the next bucket's record, and its copies into the other buffers
      nxt = list[q + gridDim.x];
      if (t == 0)
        stage_bucket<NUMERIC>(nxt, chunk_col, chunk_val, bsm + (buf ^ 1) * BS_CB,
                              bsm + 2 * BS_CB + (buf ^ 1) * BS_VB, &s_bar[buf ^ 1]);
    }
    const unsigned par = (phases >> buf) & 1u;
    const bool ok = mbar_wait(&s_bar[buf], par);
    if (__syncthreads_or(!ok)) {
      // give up on the bucket list; the copies in flight land first
      if (t == 0) atomicExch(&g_wait_timeout, 1);
      if (!ok) mbar_wait(&s_bar[buf], par);
      if (more) mbar_wait(&s_bar[buf ^ 1], (phases >> (buf ^ 1)) & 1u);
      return;
    }
    phases ^= 1u << buf;
    const int32_t* cb = reinterpret_cast<const int32_t*>(bsm + buf * BS_CB) + (bb.p0 & 3);
    const double* vb =
        NUMERIC ? reinterpret_cast<const double*>(bsm + 2 * BS_CB + buf * BS_VB) + (bb.p0 & 1)
                : nullptr;
    const int n = bb.n;
    K key[BR];
#pragma unroll
    for (int e = 0; e < BR; ++e) {
      const int pos = e * BS_NT + t;
      key[e] = pos < n ? ((K)(uint32_t)cb[pos] << BS_PB) | (K)pos : ~K(0);
    }
    bucket_sort_keys<BS_NT, BS_PB>(key, n, s_key, s_cnt, s_bst, s_red, s_ws);
    // sorted positions t*BR + e: stage them, mark the run heads
#pragma unroll
    for (int e = 0; e < BR; ++e) s_key[t * BR + e] = key[e];
    __syncthreads();
    uint32_t hb = 0;
#pragma unroll
    for (int e = 0; e < BR; ++e) {
      const int qp = t * BR + e;
      const K prev = (e > 0) ? key[e - 1] : (t > 0 ? s_key[qp - 1] : ~K(0));
      const bool head = qp < n && (qp == 0 || (key[e] >> BS_PB) != (prev >> BS_PB));
      hb |= head ? (1u << e) : 0u;
    }
    // BR = 8 head bits per thread: threads 4i..4i+3 fill word i
    {
      const uint32_t mine = hb << (8 * (t & 3));
      uint32_t wd = mine;
      wd |= __shfl_xor_sync(FULL, wd, 1);
      wd |= __shfl_xor_sync(FULL, wd, 2);
      if ((t & 3) == 0) s_head[t >> 2] = wd;
    }
    __syncthreads();
    if (w == 0) {  // prefix of the head counts over the 64 words
      const int c0 = __popc(s_head[lane]), c1 = __popc(s_head[32 + lane]);
      const int i0 = warp_inclusive_scan(c0);
      const int t0 = __shfl_sync(FULL, i0, 31);
      const int i1 = warp_inclusive_scan(c1);
      s_hpre[lane] = i0 - c0;
      s_hpre[32 + lane] = t0 + i1 - c1;
      if (lane == 31) s_hpre[64] = t0 + i1;
    }
    __syncthreads();
    if (NUMERIC) {
      const int64_t col_base = (int64_t)bb.c << sc;
#pragma unroll
      for (int e = 0; e < BR; ++e) {
        const int qp = e * BS_NT + t;
        const uint32_t wd = s_head[qp >> 5];
        if (qp < n && ((wd >> (qp & 31)) & 1u)) {
          const int rank = s_hpre[qp >> 5] + __popc(wd & ((1u << (qp & 31)) - 1u));
          const K k0 = s_key[qp];
          const K c = k0 >> BS_PB;
          double acc = vb[(int)(k0 & PMASK)];
          for (int q2 = qp + 1; q2 < n; ++q2) {  // the run, in position order
            const K k2 = s_key[q2];
            if ((k2 >> BS_PB) != c) break;
            acc += vb[(int)(k2 & PMASK)];
          }
          c_col[bb.out + rank] = (int32_t)(col_base + (int64_t)c);
          c_val[bb.out + rank] = acc;
        }
      }
    } else if (t == 0) {
      bucket_cnt[bb.out] = s_hpre[64];
    }
    __syncthreads();
    buf ^= 1;
  }
}

// Large coarse chunks whose column range (2^sc <= 2^13) fits one block's
// dense accumulator: Algorithm 1 straight from the coarse staging, with no
// second reorder.  FP64 values and the bitmap live in shared memory.  The
// scatter loop issues BD_UNROLL loads per thread before its atomics.
// Emission is warp-cooperative: warp w owns a contiguous range of bitmap
// words; each word is expanded by a ballot so the warp writes its set
// columns as one coalesced run, reading (and re-zeroing) the 32 accumulator
// slots of the word together, four words per step so that their reads
// overlap.  The words are cleared after use,
// so the accumulator is clean for the next chunk.
constexpr int BUCKET_DENSE_LOG2 = 13;
constexpr int BD_UNROLL = 4;

template <bool NUMERIC>
__global__ void __launch_bounds__(FNT)
    k_bucket_dense(const BigBucket* __restrict__ big_end, const int32_t* __restrict__ n_big,
                   const int32_t* __restrict__ chunk_col, const double* __restrict__ chunk_val,
                   int sc, int32_t* __restrict__ bucket_cnt, int32_t* __restrict__ c_col,
                   double* __restrict__ c_val) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const int cl = 1 << sc;
  const int words = cl >= 32 ? cl >> 5 : 1;
  const int wpw = (words + FNW - 1) / FNW;  // words per warp (<= 32 for sc <= 13)
  const int lane = lane_id(), w = warp_id();
  double* acc = reinterpret_cast<double*>(dsm);
  uint32_t* bits = reinterpret_cast<uint32_t*>(dsm + (NUMERIC ? (size_t)cl * 8 : 0));
  __shared__ int32_t wcnt[FNW];
  if (NUMERIC)
    for (int i = threadIdx.x; i < cl; i += FNT) acc[i] = 0.0;
  for (int i = threadIdx.x; i < words; i += FNT) bits[i] = 0u;
  __syncthreads();
  const int nbig = *n_big;
  const int wd0 = w * wpw;
  const int my_wd = wd0 + lane;
  const bool own = lane < wpw && my_wd < words;
  BigBucket nxt{};
  if (blockIdx.x < nbig) nxt = big_end[-1 - (int64_t)blockIdx.x];
  for (int q = blockIdx.x; q < nbig; q += gridDim.x) {
    const BigBucket bb = nxt;
    if (q + gridDim.x < nbig) nxt = big_end[-1 - (int64_t)(q + gridDim.x)];  // in flight
    const int64_t p0 = bb.p0;
    const int n = bb.n;
    const int c = bb.c;
    const int32_t* cc = chunk_col + p0;
    const double* cv = NUMERIC ? chunk_val + p0 : nullptr;
    for (int p = threadIdx.x; p < n; p += BD_UNROLL * FNT) {
      int idx[BD_UNROLL];
      double v[BD_UNROLL];
#pragma unroll
      for (int u = 0; u < BD_UNROLL; ++u) {
        const int pu = p + u * FNT;
        idx[u] = pu < n ? cc[pu] : -1;
        if (NUMERIC) v[u] = pu < n ? cv[pu] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < BD_UNROLL; ++u) {
        if (idx[u] >= 0) {
          atomicOr(&bits[idx[u] >> 5], 1u << (idx[u] & 31));
          if (NUMERIC) atomicAdd(&acc[idx[u]], v[u]);
        }
      }
    }
    __syncthreads();
    const uint32_t mine = own ? bits[my_wd] : 0u;
    const int cnt = warp_sum(__popc(mine));
    if (lane == 0) wcnt[w] = cnt;
    __syncthreads();
    if (NUMERIC) {
      int64_t o = bb.out;
      for (int i = 0; i < w; ++i) o += wcnt[i];
      const int64_t col_base = (int64_t)c << sc;
      const unsigned below = (1u << lane) - 1u;
      // four words per step: their accumulator reads are independent
      for (int j0 = 0; j0 < wpw; j0 += 4) {
        uint32_t m[4];
        int64_t ob[4];
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          m[u] = __shfl_sync(FULL, mine, (j0 + u) & 31);
          if (j0 + u >= wpw) m[u] = 0u;
          ob[u] = o;
          o += __popc(m[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          v[u] = 0.0;
          if ((m[u] >> lane) & 1u) {
            const int idx = (wd0 + j0 + u) * 32 + lane;
            v[u] = acc[idx];
            acc[idx] = 0.0;
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if ((m[u] >> lane) & 1u) {
            const int64_t pos = ob[u] + __popc(m[u] & below);
            c_col[pos] = (int32_t)(col_base + (wd0 + j0 + u) * 32 + lane);
            c_val[pos] = v[u];
          }
        }
      }
    } else if (threadIdx.x == 0) {
      int total = 0;
      for (int i = 0; i < FNW; ++i) total += wcnt[i];
      bucket_cnt[bb.out] = total;
    }
    if (own) bits[my_wd] = 0u;
    __syncthreads();
  }
}

template <bool NUMERIC>
static cudaError_t coarse_impl(CoarseArgs& a, cudaStream_t s) {
  cudaError_t e;
  const int64_t nB = a.B.n_rows;
  const int64_t nbk = a.n_rows * a.n_chunks;
  const int nt = 256;
  const unsigned gw = grid_cap_c((a.n_rows + 7) / 8, (int64_t)a.num_sms * 32);
#define CK(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
  const unsigned go = (unsigned)a.num_sms * 16;
  if (a.items) {
    // row-wise staged reorder: histogram (unless the symbolic pass kept the
    // bucket offsets), row-chained prefix sum, then the reorder in runs
    if (NUMERIC && a.saved_offs) {
      CK(cudaMemcpyAsync(a.counts, a.saved_offs, (size_t)(nbk + 1) * sizeof(int64_t),
                         cudaMemcpyDeviceToDevice, s));
    } else {
      CK(cudaMemsetAsync(a.counts, 0, (size_t)(nbk + 1) * sizeof(int64_t), s));
      CK(launch_coarse_stage(false, false, a, s));
      CK(launch_exclusive_scan_i64(a.counts, nbk, a.scan_tmp, s));
      if (a.saved_offs)
        CK(cudaMemcpyAsync(a.saved_offs, a.counts, (size_t)(nbk + 1) * sizeof(int64_t),
                           cudaMemcpyDeviceToDevice, s));
    }
    CK(cudaMemcpyAsync(a.cursor, a.counts, (size_t)nbk * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    CK(launch_coarse_stage(true, NUMERIC, a, s));
  } else {
    // 1. A^CSC and coarseRowsB
    CK(cudaMemsetAsync(a.col_cnt, 0, (size_t)(nB + 1) * sizeof(int32_t), s));
    CK(cudaMemsetAsync(a.n_rows_b, 0, sizeof(int32_t), s));
    k_csc_count<<<gw, nt, 0, s>>>(a.A, a.rows, a.n_rows, a.col_cnt, a.rows_b, a.n_rows_b);
    count_launch();
    CK(cudaGetLastError());
    CK(launch_scan_i32_to_i64(a.col_cnt, nB, a.col_ptr, a.scan_tmp, s));
    CK(cudaMemsetAsync(a.col_cnt, 0, (size_t)(nB + 1) * sizeof(int32_t), s));
    k_csc_fill<NUMERIC><<<gw, nt, 0, s>>>(a.A, a.rows, a.n_rows, a.col_ptr, a.col_cnt, a.csc_row,
                                          a.csc_val);
    count_launch();
    CK(cudaGetLastError());
    // 2. histogram over balanced work items of the outer product
    k_outer_items<<<grid_cap_c((nB + 255) / 256, (int64_t)a.num_sms * 32), nt, 0, s>>>(
        a.B.rp, a.col_ptr, nB, a.item_off);
    count_launch();
    CK(cudaGetLastError());
    CK(launch_exclusive_scan_i64(a.item_off, nB, a.scan_tmp, s));
    if (NUMERIC && a.saved_offs) {
      // the symbolic pass over the same batch kept the bucket offsets
      CK(cudaMemcpyAsync(a.counts, a.saved_offs, (size_t)(nbk + 1) * sizeof(int64_t),
                         cudaMemcpyDeviceToDevice, s));
    } else {
      CK(cudaMemsetAsync(a.counts, 0, (size_t)(nbk + 1) * sizeof(int64_t), s));
      k_coarse_outer<false, false><<<go, nt, 0, s>>>(a.B, a.item_off, nB, a.col_ptr, a.csc_row,
                                                     a.csc_val, a.shift_coarse, a.n_chunks,
                                                     a.counts, a.cursor, a.chunk_col, a.chunk_val);
      count_launch();
      CK(cudaGetLastError());
      // 3. row-chained prefix sum
      CK(launch_exclusive_scan_i64(a.counts, nbk, a.scan_tmp, s));
      if (a.saved_offs)
        CK(cudaMemcpyAsync(a.saved_offs, a.counts, (size_t)(nbk + 1) * sizeof(int64_t),
                           cudaMemcpyDeviceToDevice, s));
    }
    // 4. reorder
    CK(cudaMemcpyAsync(a.cursor, a.counts, (size_t)nbk * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    k_coarse_outer<true, NUMERIC><<<go, nt, 0, s>>>(a.B, a.item_off, nB, a.col_ptr, a.csc_row,
                                                    a.csc_val, a.shift_coarse, a.n_chunks, a.counts,
                                                    a.cursor, a.chunk_col, a.chunk_val);
    count_launch();
    CK(cudaGetLastError());
  }
  // 5. fine level per (row, coarse chunk)
  if (NUMERIC) {
    k_bucket_offsets<<<gw, nt, 0, s>>>(a.bucket_cnt, a.n_rows, a.n_chunks, a.list_base,
                                       a.bucket_out);
    count_launch();
    CK(cudaGetLastError());
  }
  CK(cudaMemsetAsync(a.n_big, 0, 2 * sizeof(int32_t), s));
  const bool k32 = a.shift_coarse + 8 <= 32;
  const unsigned gb = grid_cap_c((nbk + BK_NW - 1) / BK_NW, (int64_t)a.num_sms * 64);
  // buckets of 257..BS_CAP products go to the block sort when enabled
  const int mid_max = a.bucket_sort ? BS_CAP : 0;
  if (k32)
    k_bucket_small<uint32_t, NUMERIC><<<gb, BK_NW * 32, 0, s>>>(
        a.counts, nbk, a.chunk_col, a.chunk_val, a.shift_coarse, a.n_chunks, a.list_base, a.rows,
        a.bucket_cnt, a.bucket_out, a.c_rp, a.c_base, a.c_col, a.c_val, a.big_list, a.n_big,
        a.big_stats, mid_max);
  else
    k_bucket_small<uint64_t, NUMERIC><<<gb, BK_NW * 32, 0, s>>>(
        a.counts, nbk, a.chunk_col, a.chunk_val, a.shift_coarse, a.n_chunks, a.list_base, a.rows,
        a.bucket_cnt, a.bucket_out, a.c_rp, a.c_base, a.c_col, a.c_val, a.big_list, a.n_big,
        a.big_stats, mid_max);
  count_launch();
  CK(cudaGetLastError());
  if (a.big_ev0) CK(cudaEventRecord(a.big_ev0, s));
  if (mid_max > 0) {
    // the grid is one resident wave; blocks beyond the list's length exit
    auto kern = (a.shift_coarse + BS_PB <= 32) ? k_bucket_sort<uint32_t, NUMERIC>
                                               : k_bucket_sort<uint64_t, NUMERIC>;
    const size_t smem = bucket_sort_smem(NUMERIC);
    CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 1;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BS_NT, smem));
    if (per_sm < 1) per_sm = 1;
    kern<<<(unsigned)(a.num_sms * per_sm), BS_NT, smem, s>>>(a.big_list, a.n_big + 1, a.chunk_col,
                                                        a.chunk_val, a.shift_coarse,
                                                        a.bucket_cnt, a.c_col, a.c_val);
    count_launch();
    CK(cudaGetLastError());
  }
  const BigBucket* big_end = a.big_list + nbk;
  if (a.shift_coarse <= BUCKET_DENSE_LOG2) {
    const size_t cl = (size_t)1 << a.shift_coarse;
    const size_t smem = (NUMERIC ? cl * 8 : 0) + (cl >= 32 ? cl / 8 : 4);
    CK(cudaFuncSetAttribute(k_bucket_dense<NUMERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)smem));
    int per_sm = 1;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bucket_dense<NUMERIC>, FNT, smem));
    if (per_sm < 1) per_sm = 1;
    k_bucket_dense<NUMERIC><<<(unsigned)(a.num_sms * per_sm), FNT, smem, s>>>(
        big_end, a.n_big, a.chunk_col, a.chunk_val, a.shift_coarse, a.bucket_cnt, a.c_col,
        a.c_val);
  } else {
    // the sort and hash accumulators share the per-warp staging
    const bool hybrid = a.dense_chunk_threshold > 1 || (NUMERIC && a.hash);
    const size_t smem = fine_smem_bytes(NUMERIC, a.shift_fine < a.shift_coarse ? a.shift_fine : a.shift_coarse,
                                        hybrid);
    auto kern = hybrid ? k_bucket_big<NUMERIC, true> : k_bucket_big<NUMERIC, false>;
    CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)a.num_sms * 2, FNT, smem, s>>>(
        big_end, a.n_big, a.chunk_col, a.chunk_val, a.fine_col, a.fine_val,
        a.shift_coarse, a.shift_fine, a.bucket_cnt, a.c_col, a.c_val, a.dense_chunk_threshold,
        a.hash);
  }
  count_launch();
  CK(cudaGetLastError());
  if (a.big_ev1) CK(cudaEventRecord(a.big_ev1, s));
  if (!NUMERIC) {
    k_row_totals<<<gw, nt, 0, s>>>(a.bucket_cnt, a.rows, a.n_rows, a.n_chunks, a.list_base,
                                   a.out_cnt);
    count_launch();
    CK(cudaGetLastError());
  }
#undef CK
  return cudaSuccess;
}

cudaError_t run_coarse_batch(bool numeric, CoarseArgs& a, cudaStream_t s) {
  if (a.n_rows == 0) return cudaSuccess;
  return numeric ? coarse_impl<true>(a, s) : coarse_impl<false>(a, s);
}

}  // namespace magnus
