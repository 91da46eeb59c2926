// Device-side building blocks shared by the MAGNUS kernels: warp/block
// scans, warp and block bitonic sorting networks, and launch bookkeeping.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace magnus {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }

// Inclusive warp scan (Hillis-Steele over shuffles).
template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T x) {
  const int lane = lane_id();
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T y = __shfl_up_sync(FULL, x, d);
    if (lane >= d) x += y;
  }
  return x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(FULL, x, d);
  return x;
}

template <typename T>
__device__ __forceinline__ T warp_max(T x) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    T y = __shfl_xor_sync(FULL, x, d);
    x = y > x ? y : x;
  }
  return x;
}

template <typename T>
__device__ __forceinline__ T warp_min(T x) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    T y = __shfl_xor_sync(FULL, x, d);
    x = y < x ? y : x;
  }
  return x;
}

// Exclusive block scan over NT threads (one value per thread).  `ws` must hold
// NT/32 + 1 elements of shared memory.  Returns the exclusive prefix; *total
// receives the block sum.  Contains __syncthreads (all threads must call).
template <int NT, typename T>
__device__ __forceinline__ T block_exclusive_scan(T x, T* ws, T* total) {
  const int lane = lane_id(), wid = warp_id();
  T inc = warp_inclusive_scan(x);
  if (lane == 31) ws[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T w = (lane < NT / 32) ? ws[lane] : T(0);
    T wi = warp_inclusive_scan(w);
    if (lane < NT / 32) ws[lane] = wi - w;
    if (lane == NT / 32 - 1) ws[NT / 32] = wi;
  }
  __syncthreads();
  T res = ws[wid] + inc - x;
  if (total) *total = ws[NT / 32];
  __syncthreads();
  return res;
}

template <int NT, typename T>
__device__ __forceinline__ T block_sum(T x, T* ws) {
  T tot;
  block_exclusive_scan<NT, T>(x, ws, &tot);
  return tot;
}

// ---------------------------------------------------------------------------
// Warp bitonic sort, E keys per lane.  Logical position of (lane, e) is
// q = lane * E + e ("blocked" layout), so the partner of a compare-exchange at
// distance j < E is in the same lane and at distance j >= E it is lane ^ (j/E).
// On return the keys are ascending in q.
//
// The direction of a compare-exchange depends only on bit `size` of q.  For
// size >= E that bit comes from the lane alone, for size < E from e alone, so
// each stage needs one lane predicate (or none) and one min/max per key.
__device__ __forceinline__ uint32_t kmin(uint32_t a, uint32_t b) { return min(a, b); }
__device__ __forceinline__ uint32_t kmax(uint32_t a, uint32_t b) { return max(a, b); }
__device__ __forceinline__ uint64_t kmin(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint64_t kmax(uint64_t a, uint64_t b) { return a < b ? b : a; }

// Merge of sorted runs: every lane of a group of W lanes holds R keys that
// are already ascending (one sorted run per lane, positions q = l * R + e as
// above).  The levels of the bitonic network below size 2R are skipped; each
// remaining level starts with a "flip" stage that compares position i of a
// block with its mirror (block end - 1 - i), which turns two ascending halves
// into two halves whose every key of the lower is <= every key of the upper,
// then half-cleaners at distances size/4 .. 1 sort each half.  All stages
// keep the smaller key at the lower position, so no stage needs a direction.
template <int R, int W, typename K>
__device__ __forceinline__ void group_merge_runs(K (&k)[R]) {
  const int l = lane_id() & (W - 1);
  constexpr int N = W * R;
#pragma unroll
  for (int size = 2 * R; size <= N; size <<= 1) {
    {
      const int pm = size / R - 1;                 // mirror lane within the block
      const bool lower = (l & (size / R / 2)) == 0;
      K o[R];
#pragma unroll
      for (int e = 0; e < R; ++e) o[e] = __shfl_xor_sync(FULL, k[R - 1 - e], pm);
#pragma unroll
      for (int e = 0; e < R; ++e) k[e] = lower ? kmin(k[e], o[e]) : kmax(k[e], o[e]);
    }
#pragma unroll
    for (int j = size >> 2; j > 0; j >>= 1) {
      if (j >= R) {
        const int pl = j / R;
        const bool lower = (l & pl) == 0;
#pragma unroll
        for (int e = 0; e < R; ++e) {
          const K other = __shfl_xor_sync(FULL, k[e], pl);
          k[e] = lower ? kmin(k[e], other) : kmax(k[e], other);
        }
      } else {
#pragma unroll
        for (int e = 0; e < R; ++e) {
          if ((e & j) == 0) {
            const K lo = kmin(k[e], k[e + j]);
            const K hi = kmax(k[e], k[e + j]);
            k[e] = lo;
            k[e + j] = hi;
          }
        }
      }
    }
  }
}

// Bitonic sort over aligned groups of W lanes holding R keys each (W * R
// keys per group, W a power of two <= 32).  Logical position of (lane l in
// its group, e) is q = l * R + e.  Every level starts with a flip stage and
// continues with ascending half-cleaners (as in group_merge_runs), so no
// compare-exchange needs a direction: the levels below 2R run inside a
// lane's registers and leave each lane with one ascending run, the levels
// above merge the runs.
template <int R, int W, typename K>
__device__ __forceinline__ void group_bitonic_sort(K (&k)[R]) {
#pragma unroll
  for (int size = 2; size <= R; size <<= 1) {
#pragma unroll
    for (int e = 0; e < R; ++e) {
      const int b = e & ~(size - 1);
      const int m = b + size - 1 - (e - b);  // mirror of e in its block
      if (e < m) {
        const K lo = kmin(k[e], k[m]);
        const K hi = kmax(k[e], k[m]);
        k[e] = lo;
        k[m] = hi;
      }
    }
#pragma unroll
    for (int j = size >> 2; j > 0; j >>= 1) {
#pragma unroll
      for (int e = 0; e < R; ++e) {
        if ((e & j) == 0) {
          const K lo = kmin(k[e], k[e + j]);
          const K hi = kmax(k[e], k[e + j]);
          k[e] = lo;
          k[e + j] = hi;
        }
      }
    }
  }
  if (W > 1) group_merge_runs<R, W>(k);
}

// Batcher's odd-even merge sort (Batcher 1968) of N keys in one thread's
// registers, ascending; N a power of two.  For N = 32 it takes 191
// compare-exchanges where a bitonic network takes 240.  Stage p merges
// sorted runs of length p; within it, comparators at distance q join keys
// whose indices fall in the same block of 2p.  The comparator list is built
// at compile time, so the unrolled loop indexes registers only.
template <int N>
struct OddEvenNet {
  static constexpr int count() {
    int c = 0;
    for (int p = 1; p < N; p <<= 1)
      for (int q = p; q >= 1; q >>= 1)
        for (int j = q % p; j + q < N; j += 2 * q)
          for (int i = 0; i < q && i + j + q < N; ++i)
            if ((i + j) / (2 * p) == (i + j + q) / (2 * p)) ++c;
    return c;
  }
  static constexpr int NC = count();
  struct Table {
    unsigned char lo[NC > 0 ? NC : 1], hi[NC > 0 ? NC : 1];
  };
  static constexpr Table table() {
    Table t{};
    int c = 0;
    for (int p = 1; p < N; p <<= 1)
      for (int q = p; q >= 1; q >>= 1)
        for (int j = q % p; j + q < N; j += 2 * q)
          for (int i = 0; i < q && i + j + q < N; ++i)
            if ((i + j) / (2 * p) == (i + j + q) / (2 * p)) {
              t.lo[c] = (unsigned char)(i + j);
              t.hi[c] = (unsigned char)(i + j + q);
              ++c;
            }
    return t;
  }
};

template <int N, typename K>
__device__ __forceinline__ void lane_oddeven_sort(K (&k)[N]) {
  constexpr auto T = OddEvenNet<N>::table();
#pragma unroll
  for (int c = 0; c < OddEvenNet<N>::NC; ++c) {
    const K x = k[T.lo[c]], y = k[T.hi[c]];
    k[T.lo[c]] = kmin(x, y);
    k[T.hi[c]] = kmax(x, y);
  }
}

template <int E, typename K>
__device__ __forceinline__ void warp_bitonic_sort(K (&k)[E]) {
  group_bitonic_sort<E, 32, K>(k);
}

// Scans and sums inside aligned groups of W lanes (all 32 lanes must call).
template <int W, typename T>
__device__ __forceinline__ T group_inclusive_scan(T x) {
  const int l = lane_id() & (W - 1);
#pragma unroll
  for (int d = 1; d < W; d <<= 1) {
    T y = __shfl_up_sync(FULL, x, d, W);
    if (l >= d) x += y;
  }
  return x;
}

template <int W, typename T>
__device__ __forceinline__ T group_sum(T x) {
#pragma unroll
  for (int d = W / 2; d > 0; d >>= 1) x += __shfl_xor_sync(FULL, x, d, W);
  return x;
}

__device__ __forceinline__ int upper_bound_i64(const int64_t* a, int n, int64_t x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int upper_bound_i32(const int32_t* a, int n, int32_t x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Streaming (evict-first) stores for the reorder targets: the staged
// intermediate product is written once and read once, so it should not
// displace the B rows and accumulator lines held in L2 (the GPU counterpart
// of the non-temporal stores of Sections 3.2-3.3).
__device__ __forceinline__ void st_stream(int32_t* p, int32_t v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(double* p, double v) { __stcs(p, v); }

}  // namespace magnus
