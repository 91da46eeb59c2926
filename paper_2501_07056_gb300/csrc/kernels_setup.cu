// Setup phase (Section 3.1): input validation, per-row intermediate-product
// counts P_i, row column ranges and categories, the stable partition of rows
// into per-category lists, and device-wide prefix sums.
#include "common.cuh"

namespace magnus {

static uint64_t g_launches = 0;
void count_launch(int n) { __atomic_fetch_add(&g_launches, (uint64_t)n, __ATOMIC_RELAXED); }
uint64_t launches_total() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

static inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
static inline unsigned grid_cap(int64_t blocks, int64_t cap) {
  return (unsigned)(blocks < cap ? (blocks < 1 ? 1 : blocks) : cap);
}

// ---------------------------------------------------------------------------
// Validation: row pointers monotone and consistent, columns strictly
// ascending per row and inside [0, n_cols).  One warp per row.  Sets *flag
// to 1 on any violation.
__global__ void k_validate(Csr M, int* flag) {
  const int lane = lane_id();
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < M.n_rows;
       i += nwarps) {
    const int64_t s = M.rp[i], e = M.rp[i + 1];
    bool bad = false;
    if (lane == 0) {
      if (e < s || s < 0 || e > M.nnz) bad = true;
      if (i == 0 && s != 0) bad = true;
      if (i == M.n_rows - 1 && e != M.nnz) bad = true;
    }
    if (!__any_sync(FULL, bad)) {
      for (int64_t j = s + lane; j < e; j += 32) {
        const int32_t c = M.col[j];
        if (c < 0 || (int64_t)c >= M.n_cols) bad = true;
        if (j > s && M.col[j - 1] >= c) bad = true;
      }
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicExch(flag, 1);
  }
}

cudaError_t launch_validate(const Csr& M, int* d_flag, cudaStream_t s) {
  if (M.n_rows == 0) return cudaSuccess;
  const int nt = 256;
  unsigned g = grid_cap(cdiv(M.n_rows, nt / 32), 1 << 16);
  k_validate<<<g, nt, 0, s>>>(M, d_flag);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Row analysis (Section 3.1): P_i, column range [lo, hi] of the intermediate
// product (from the first and last column of each referenced B row, which is
// valid because rows are sorted), and the bin of the row.
// Also writes the segment table: for every nonzero j of A, the start and the
// length of the B row it selects (B.rowPtr[A.col[j]] and the row's nnz,
// packed into one word by seg_pack), so later passes read it as a stream
// instead of gathering B.rowPtr again.
//
// The B.rowPtr gathers are the pass's cost.  When B has fewer than 2^32
// nonzeros they read a copy of B.rowPtr narrowed to 32 bits (RP = uint32_t):
// half the bytes, and for B of up to about 2^25 rows a table that stays in
// L2 while A's columns and the segment table stream past it.

// Bin of a row from its products alone; need_range when the choice needs the
// row's column range.
__device__ __forceinline__ int rowinfo_sort_bin(int64_t q) {
  return q <= 32 ? BIN_SORT32 : q <= 64 ? BIN_SORT64 : q <= 128 ? BIN_SORT128
         : q <= 256 ? BIN_SORT256 : q <= 512 ? BIN_SORT512 : BIN_SORT1024;
}

__device__ __forceinline__ int rowinfo_first_bin(int64_t p, const CatParams& cp, bool* need_range) {
  *need_range = false;
  if (p <= 0) return BIN_EMPTY;
  const bool sort_ok = p <= SORT_BLOCK_MAX;
  const bool want_sort = (cp.force == MAGNUS_CAT_SORT) ? sort_ok
                         : (cp.force < 0 ? (p < cp.sort_threshold) : false);
  if (want_sort) return rowinfo_sort_bin(p);
  *need_range = true;
  return BIN_EMPTY;
}

// Bin of a row whose column range [lo, hi] was needed.
__device__ __forceinline__ int rowinfo_range_bin(int64_t p, int32_t lo, int32_t hi,
                                                 const CatParams& cp) {
  const int64_t range = (int64_t)hi - lo + 1;
  const int64_t nfine = (int64_t)(hi >> cp.fine_shift) - (lo >> cp.fine_shift) + 1;
  const bool dense_ok = range <= cp.dense_cols;
  const bool fine_ok = nfine <= cp.fine_max_chunks && p <= cp.fine_max_products &&
                       p < ((int64_t)1 << 31);
  if (cp.force == MAGNUS_CAT_COARSE) return BIN_COARSE;
  if (cp.force == MAGNUS_CAT_FINE) return fine_ok ? BIN_FINE : BIN_COARSE;
  // automatic: a row of at most wide_sort_max products that fills less than
  // half of its column range sorts instead (the dense accumulator's work
  // follows the range, the sort's the products)
  if (dense_ok && (cp.force >= 0 || p > cp.wide_sort_max || range <= 2 * p)) return BIN_DENSE;
  if (cp.force < 0 && p <= cp.wide_sort_max) return rowinfo_sort_bin(p);
  return (cp.prefer_fine && fine_ok) ? BIN_FINE : BIN_COARSE;
}

// V lanes per row (rows of more than about 8 nonzeros on average).
template <int V, typename RP>
__global__ void k_rowinfo(Csr A, const RP* __restrict__ brp, Csr B, CatParams cp,
                          int64_t* __restrict__ P, uint8_t* __restrict__ bin,
                          int32_t* __restrict__ lo_out, int32_t* __restrict__ hi_out,
                          uint64_t* __restrict__ seg) {
  const int sub = threadIdx.x & (V - 1);
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / V);
  const unsigned gmask = (V == 32) ? FULL : (((1u << V) - 1) << ((threadIdx.x & 31) & ~(V - 1)));
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / V;; i += groups) {
    // uniform trip count per warp: every group of the warp iterates together
    const int64_t first_row_of_warp = i - ((threadIdx.x & 31) / V);
    if (first_row_of_warp >= A.n_rows) break;
    const bool active = i < A.n_rows;
    int64_t s = 0, e = 0;
    if (active) { s = A.rp[i]; e = A.rp[i + 1]; }
    int64_t p = 0;
    // the B row bounds of a row that fits one step stay in registers for
    // the column range below
    int64_t r0 = 0, r1 = 0, r2 = 0, r3 = 0;
    // two entries per lane and step, their loads issued together
    for (int64_t j = s + sub; j < e; j += 2 * V) {
      const int64_t j2 = j + V;
      const bool two = j2 < e;
      const int32_t c = A.col[j];
      const int32_t c2 = two ? A.col[j2] : 0;
      const int64_t b0 = (int64_t)brp[c], b1 = (int64_t)brp[c + 1];
      const int64_t b2 = two ? (int64_t)brp[c2] : 0, b3 = two ? (int64_t)brp[c2 + 1] : 0;
      p += (b1 - b0) + (b3 - b2);
      seg[j] = seg_pack(b0, b1 - b0);
      if (two) seg[j2] = seg_pack(b2, b3 - b2);
      r0 = b0;
      r1 = b1;
      r2 = b2;
      r3 = b3;
    }
#pragma unroll
    for (int d = V / 2; d > 0; d >>= 1) p += __shfl_xor_sync(gmask, p, d, V);
    // need_range is uniform within a group (p is the group-reduced sum)
    bool need_range = false;
    int b = rowinfo_first_bin(p, cp, &need_range);
    int32_t lo = 0x7fffffff, hi = -1;
    if (need_range) {
      if (e - s <= 2 * V) {  // one step: the bounds are r0..r3 (empty pairs when unused)
        if (r1 > r0) {
          lo = B.col[r0];
          hi = B.col[r1 - 1];
        }
        if (r3 > r2) {
          const int32_t c0 = B.col[r2], c1 = B.col[r3 - 1];
          lo = c0 < lo ? c0 : lo;
          hi = c1 > hi ? c1 : hi;
        }
      } else {
        for (int64_t j = s + sub; j < e; j += V) {
          const int32_t c = A.col[j];
          const int64_t bs = (int64_t)brp[c], be = (int64_t)brp[c + 1];
          if (be > bs) {
            const int32_t c0 = B.col[bs], c1 = B.col[be - 1];
            lo = c0 < lo ? c0 : lo;
            hi = c1 > hi ? c1 : hi;
          }
        }
      }
#pragma unroll
      for (int d = V / 2; d > 0; d >>= 1) {
        int32_t l2 = __shfl_xor_sync(gmask, lo, d, V);
        int32_t h2 = __shfl_xor_sync(gmask, hi, d, V);
        lo = l2 < lo ? l2 : lo;
        hi = h2 > hi ? h2 : hi;
      }
      b = rowinfo_range_bin(p, lo, hi, cp);
    }
    if (active && sub == 0) {
      P[i] = p;
      bin[i] = (uint8_t)b;
      lo_out[i] = need_range ? lo : 0;
      hi_out[i] = need_range ? hi : -1;
    }
  }
}

// One lane per row (rows of at most about 8 nonzeros on average): each step
// issues the loads of U entries of the row together, so a warp keeps up to
// 32 * U column loads and then 32 * U B-row-bound gathers in flight instead
// of a few per lane.
template <int U, typename RP>
__global__ void __launch_bounds__(256) k_rowinfo_lane(Csr A, const RP* __restrict__ brp, Csr B,
                                                      CatParams cp, int64_t* __restrict__ P,
                                                      uint8_t* __restrict__ bin,
                                                      int32_t* __restrict__ lo_out,
                                                      int32_t* __restrict__ hi_out,
                                                      uint64_t* __restrict__ seg) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n_rows; i += stride) {
    const int64_t s = A.rp[i], e = A.rp[i + 1];
    int64_t p = 0;
    for (int64_t j0 = s; j0 < e; j0 += U) {
      const int64_t left = e - j0;
      int32_t c[U];
#pragma unroll
      for (int k = 0; k < U; ++k) c[k] = k < left ? __ldg(A.col + j0 + k) : 0;
      int64_t b0[U], b1[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        b0[k] = k < left ? (int64_t)__ldg(brp + c[k]) : 0;
        b1[k] = k < left ? (int64_t)__ldg(brp + c[k] + 1) : 0;
      }
#pragma unroll
      for (int k = 0; k < U; ++k) {
        if (k < left) {
          p += b1[k] - b0[k];
          seg[j0 + k] = seg_pack(b0[k], b1[k] - b0[k]);
        }
      }
    }
    bool need_range = false;
    int b = rowinfo_first_bin(p, cp, &need_range);
    int32_t lo = 0x7fffffff, hi = -1;
    if (need_range) {
      for (int64_t j0 = s; j0 < e; j0 += U) {
        const int64_t left = e - j0;
        int32_t c[U];
#pragma unroll
        for (int k = 0; k < U; ++k) c[k] = k < left ? __ldg(A.col + j0 + k) : 0;
        int64_t bs[U], be[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
          bs[k] = k < left ? (int64_t)__ldg(brp + c[k]) : 0;
          be[k] = k < left ? (int64_t)__ldg(brp + c[k] + 1) : 0;
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
          if (be[k] > bs[k]) {  // empty B rows (and the unused slots) add nothing
            const int32_t c0 = B.col[bs[k]], c1 = B.col[be[k] - 1];
            lo = c0 < lo ? c0 : lo;
            hi = c1 > hi ? c1 : hi;
          }
        }
      }
      b = rowinfo_range_bin(p, lo, hi, cp);
    }
    P[i] = p;
    bin[i] = (uint8_t)b;
    lo_out[i] = need_range ? lo : 0;
    hi_out[i] = need_range ? hi : -1;
  }
}

__global__ void k_narrow_rp(const int64_t* __restrict__ rp, int64_t n,
                            uint32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (uint32_t)rp[i];
}

template <typename RP>
static void launch_rowinfo_rp(const Csr& A, const RP* brp, const Csr& B, CatParams cp,
                              int64_t* P, uint8_t* bin, int32_t* lo, int32_t* hi, uint64_t* seg,
                              cudaStream_t s) {
  const double avg = A.n_rows ? (double)A.nnz / (double)A.n_rows : 0.0;
  const int nt = 256;
  if (avg <= 8.0) {
    const unsigned g = grid_cap(cdiv(A.n_rows, nt), 1 << 20);
    k_rowinfo_lane<8, RP><<<g, nt, 0, s>>>(A, brp, B, cp, P, bin, lo, hi, seg);
    return;
  }
  int v = 1;  // lanes per row: about half the row's nonzeros (two per lane)
  while (v < 32 && 2 * v < avg) v <<= 1;
  const unsigned g = grid_cap(cdiv(A.n_rows * v, nt), 1 << 20);
  switch (v) {
    case 8: k_rowinfo<8, RP><<<g, nt, 0, s>>>(A, brp, B, cp, P, bin, lo, hi, seg); break;
    case 16: k_rowinfo<16, RP><<<g, nt, 0, s>>>(A, brp, B, cp, P, bin, lo, hi, seg); break;
    default: k_rowinfo<32, RP><<<g, nt, 0, s>>>(A, brp, B, cp, P, bin, lo, hi, seg); break;
  }
}

cudaError_t launch_rowinfo(const Csr& A, const Csr& B, CatParams cp, int64_t* P, uint8_t* bin,
                           int32_t* lo, int32_t* hi, uint64_t* seg,
                           cudaStream_t s) {
  if (A.n_rows == 0) return cudaSuccess;
  // the 32-bit copy of B.rowPtr, stream-ordered and freed after the pass; the
  // pass reads B.rowPtr itself when B has 2^32 nonzeros or more or the copy
  // cannot be allocated
  uint32_t* brp32 = nullptr;
  if (B.nnz < ((int64_t)1 << 32) &&
      cudaMallocAsync(reinterpret_cast<void**>(&brp32), (size_t)(B.n_rows + 1) * 4, s) !=
          cudaSuccess) {
    cudaGetLastError();
    brp32 = nullptr;
  }
  if (brp32) {
    k_narrow_rp<<<grid_cap(cdiv(B.n_rows + 1, 256), 4096), 256, 0, s>>>(B.rp, B.n_rows, brp32);
    count_launch();
    launch_rowinfo_rp<uint32_t>(A, brp32, B, cp, P, bin, lo, hi, seg, s);
  } else {
    launch_rowinfo_rp<int64_t>(A, B.rp, B, cp, P, bin, lo, hi, seg, s);
  }
  count_launch();
  const cudaError_t e = cudaGetLastError();
  if (brp32) cudaFreeAsync(brp32, s);
  return e;
}

// ---------------------------------------------------------------------------
// Stable partition of rows by bin (a one-digit counting sort).
constexpr int BP_NT = 256;
constexpr int BP_ITERS = 16;
constexpr int BP_ROWS = BP_NT * BP_ITERS;

int64_t bin_partition_blocks(int64_t n) { return cdiv(n, BP_ROWS); }

__global__ void k_bin_count(const uint8_t* __restrict__ bin, int64_t n, int64_t* blkcnt,
                            int64_t nblk) {
  __shared__ int cnt[NUM_BINS];
  if (threadIdx.x < NUM_BINS) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * BP_ROWS;
  for (int it = 0; it < BP_ITERS; ++it) {
    const int64_t i = base + it * BP_NT + threadIdx.x;
    if (i < n) atomicAdd(&cnt[bin[i]], 1);
  }
  __syncthreads();
  if (threadIdx.x < NUM_BINS) blkcnt[(int64_t)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void k_bin_scatter(const uint8_t* __restrict__ bin, int64_t n,
                              const int64_t* __restrict__ blkoff, int64_t nblk,
                              int32_t* __restrict__ rows_out) {
  __shared__ int wcnt[BP_NT / 32][NUM_BINS];
  __shared__ int64_t running[NUM_BINS];
  const int lane = lane_id(), wid = warp_id();
  if (threadIdx.x < NUM_BINS) running[threadIdx.x] = blkoff[(int64_t)threadIdx.x * nblk + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * BP_ROWS;
  for (int it = 0; it < BP_ITERS; ++it) {
    const int64_t i = base + it * BP_NT + threadIdx.x;
    const int b = (i < n) ? (int)bin[i] : NUM_BINS;  // NUM_BINS = no row
    if (threadIdx.x < (BP_NT / 32) * NUM_BINS) (&wcnt[0][0])[threadIdx.x] = 0;
    __syncthreads();
    const unsigned m = __match_any_sync(FULL, b);
    const int rank = __popc(m & ((1u << lane) - 1));
    if (b < NUM_BINS && rank == 0) wcnt[wid][b] = __popc(m);
    __syncthreads();
    if (b < NUM_BINS) {
      int64_t off = running[b] + rank;
      for (int w = 0; w < wid; ++w) off += wcnt[w][b];
      rows_out[off] = (int32_t)i;
    }
    __syncthreads();
    if (threadIdx.x < NUM_BINS) {
      int t = 0;
      for (int w = 0; w < BP_NT / 32; ++w) t += wcnt[w][threadIdx.x];
      running[threadIdx.x] += t;
    }
    __syncthreads();
  }
}

// bin_counts_dev[b] = offset of bin b in rows_out (b = 0..NUM_BINS), derived
// from the scanned block counts.
__global__ void k_bin_offsets(const int64_t* blkoff, int64_t nblk, int64_t* bin_off) {
  const int b = threadIdx.x;
  if (b <= NUM_BINS) bin_off[b] = blkoff[(int64_t)b * nblk];
}

cudaError_t launch_bin_partition(const uint8_t* bin, int64_t n, int32_t* rows_out,
                                 int64_t* bin_off_dev, int64_t* blk, int64_t nblk_cap,
                                 cudaStream_t s) {
  // blk must hold NUM_BINS*nblk + 1 + scan_tmp_elems(NUM_BINS*nblk) elements
  const int64_t nblk = bin_partition_blocks(n);
  if (nblk > nblk_cap) return cudaErrorInvalidValue;
  const int64_t m = (int64_t)NUM_BINS * nblk;
  if (nblk > 0) {
    k_bin_count<<<(unsigned)nblk, BP_NT, 0, s>>>(bin, n, blk, nblk);
    count_launch();
  }
  cudaError_t err = launch_exclusive_scan_i64(blk, m, blk + m + 1, s);
  if (err != cudaSuccess) return err;
  // blk[m] = total; bin offsets read blk[b*nblk] for b <= NUM_BINS (b = NUM_BINS -> blk[m])
  k_bin_offsets<<<1, 32, 0, s>>>(blk, nblk, bin_off_dev);
  count_launch();
  if (nblk > 0) {
    k_bin_scatter<<<(unsigned)nblk, BP_NT, 0, s>>>(bin, n, blk, nblk, rows_out);
    count_launch();
  }
  return cudaGetLastError();
}

// Row descriptors of a row list: the A range and id of every listed row, so
// per-row kernels start from one coalesced 16-byte load.
__global__ void k_row_desc(const int32_t* __restrict__ rows, int64_t n,
                           const int64_t* __restrict__ a_rp, RowDesc* __restrict__ desc) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = rows[t];
    RowDesc d;
    d.as = a_rp[r];
    d.na = (int32_t)(a_rp[r + 1] - d.as);
    d.row = r;
    desc[t] = d;
  }
}

cudaError_t launch_row_desc(const int32_t* rows, int64_t n, const int64_t* a_rp, RowDesc* desc,
                            cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_row_desc<<<grid_cap(cdiv(n, 256), 1 << 16), 256, 0, s>>>(rows, n, a_rp, desc);
  count_launch();
  return cudaGetLastError();
}

// Row range [r0, r1) -> per bin, the positions of its rows in the bin's
// list, relative to the bin's first entry (lower bounds of r0 and r1; each
// bin's list is ascending by row).
__global__ void k_bin_bounds(const int32_t* __restrict__ rows, BinOffsets off, int64_t r0,
                             int64_t r1, int64_t* __restrict__ out) {
  const int b = threadIdx.x;
  if (b >= NUM_BINS) return;
  for (int k = 0; k < 2; ++k) {
    const int64_t key = k == 0 ? r0 : r1;
    int64_t lo = off.v[b], hi = off.v[b + 1];
    while (lo < hi) {
      const int64_t mid = lo + ((hi - lo) >> 1);
      if ((int64_t)rows[mid] < key) lo = mid + 1;
      else hi = mid;
    }
    out[2 * b + k] = lo - off.v[b];
  }
}

cudaError_t launch_bin_bounds(const int32_t* rows_sorted, BinOffsets off, int64_t r0, int64_t r1,
                              int64_t* out, cudaStream_t s) {
  k_bin_bounds<<<1, 32, 0, s>>>(rows_sorted, off, r0, r1, out);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_gather_i64(const int64_t* src, const int32_t* idx, int64_t n, int64_t* dst) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = src[idx[t]];
}

cudaError_t launch_gather_i64(const int64_t* src, const int32_t* idx, int64_t n, int64_t* dst,
                              cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_gather_i64<<<grid_cap(cdiv(n, 256), 1 << 16), 256, 0, s>>>(src, idx, n, dst);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_reduce_stats(const int64_t* P, int64_t n, unsigned long long* out) {
  int64_t sum = 0, mx = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = P[t];
    sum += p;
    mx = p > mx ? p : mx;
  }
  sum = warp_sum(sum);
  mx = warp_max(mx);
  if (lane_id() == 0) {
    atomicAdd(&out[0], (unsigned long long)sum);
    atomicMax(&out[1], (unsigned long long)mx);
  }
}

cudaError_t launch_reduce_stats(const int64_t* P, int64_t n, int64_t* out2, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out2, 0, 2 * sizeof(int64_t), s);
  if (e != cudaSuccess || n == 0) return e;
  k_reduce_stats<<<grid_cap(cdiv(n, 256), 2048), 256, 0, s>>>(P, n, (unsigned long long*)out2);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exclusive scan of int64 (reduce / scan partials / downsweep).
constexpr int SC_NT = 256;
constexpr int SC_ITEMS = 8;
constexpr int64_t SC_TILE = SC_NT * SC_ITEMS;

int64_t scan_tmp_elems(int64_t n) {
  if (n <= SC_TILE) return 0;
  const int64_t nb = cdiv(n, SC_TILE);
  return nb + 1 + scan_tmp_elems(nb);
}

__global__ void k_scan_reduce(const int64_t* __restrict__ a, int64_t n, int64_t* __restrict__ part) {
  __shared__ int64_t ws[SC_NT / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * SC_TILE;
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k) {
    const int64_t i = base + k * SC_NT + threadIdx.x;
    if (i < n) s += a[i];
  }
  s = block_sum<SC_NT>(s, ws);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Scans one tile per block in place and adds part[blockIdx.x] (if part).
// Block 0 of a single-tile scan writes a[n] = total.
__global__ void k_scan_tile(int64_t* __restrict__ a, int64_t n, const int64_t* __restrict__ part,
                            int write_total) {
  __shared__ int64_t ws[SC_NT / 32 + 1];
  __shared__ int64_t tile[SC_TILE];
  const int64_t base = (int64_t)blockIdx.x * SC_TILE;
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k) {
    const int64_t i = base + k * SC_NT + threadIdx.x;
    tile[k * SC_NT + threadIdx.x] = (i < n) ? a[i] : 0;
  }
  __syncthreads();
  int64_t v[SC_ITEMS];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k) {
    v[k] = tile[threadIdx.x * SC_ITEMS + k];
    s += v[k];
  }
  int64_t tot;
  int64_t ex = block_exclusive_scan<SC_NT>(s, ws, &tot);
  if (part) ex += part[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k) {
    tile[threadIdx.x * SC_ITEMS + k] = ex;
    ex += v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k) {
    const int64_t i = base + k * SC_NT + threadIdx.x;
    if (i < n) a[i] = tile[k * SC_NT + threadIdx.x];
  }
  if (write_total && threadIdx.x == 0) {
    if (part) a[n] = part[gridDim.x];  // total of all tiles
    else a[n] = tot;
  }
}

cudaError_t launch_exclusive_scan_i64(int64_t* a, int64_t n, int64_t* tmp, cudaStream_t s) {
  if (n <= SC_TILE) {
    k_scan_tile<<<1, SC_NT, 0, s>>>(a, n, nullptr, 1);
    count_launch();
    return cudaGetLastError();
  }
  const int64_t nb = cdiv(n, SC_TILE);
  k_scan_reduce<<<(unsigned)nb, SC_NT, 0, s>>>(a, n, tmp);
  count_launch();
  cudaError_t e = launch_exclusive_scan_i64(tmp, nb, tmp + nb + 1, s);
  if (e != cudaSuccess) return e;
  // tmp[0..nb) = exclusive partials, tmp[nb] = total
  k_scan_tile<<<(unsigned)nb, SC_NT, 0, s>>>(a, n, tmp, 0);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(a + n, tmp + nb, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
}

__global__ void k_i32_to_i64(const int32_t* in, int64_t n, int64_t* out) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = in[t];
}

cudaError_t launch_scan_i32_to_i64(const int32_t* in, int64_t n, int64_t* out, int64_t* tmp,
                                   cudaStream_t s) {
  if (n > 0) {
    k_i32_to_i64<<<grid_cap(cdiv(n, 256), 1 << 16), 256, 0, s>>>(in, n, out);
    count_launch();
  }
  return launch_exclusive_scan_i64(out, n, tmp, s);
}

}  // namespace magnus
