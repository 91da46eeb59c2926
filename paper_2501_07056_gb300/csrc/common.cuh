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
template <int E, typename K>
__device__ __forceinline__ void warp_bitonic_sort(K (&k)[E]) {
  const int lane = lane_id();
  constexpr int N = 32 * E;
#pragma unroll
  for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
    for (int j = size >> 1; j > 0; j >>= 1) {
      if (j >= E) {
        const int pl = j / E;
        const bool upper = (lane & pl) != 0;  // this lane holds the higher index
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int q = lane * E + e;
          const bool asc = (q & size) == 0;
          K other = __shfl_xor_sync(FULL, k[e], pl);
          // ascending block: lower index keeps min; descending: lower keeps max
          const bool keep_min = (asc != upper);
          K mn = other < k[e] ? other : k[e];
          K mx = other < k[e] ? k[e] : other;
          k[e] = keep_min ? mn : mx;
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if ((e & j) == 0) {
            const int q = lane * E + e;
            const bool asc = (q & size) == 0;
            K a = k[e], b = k[e + j];
            const bool sw = asc ? (b < a) : (a < b);
            k[e] = sw ? b : a;
            k[e + j] = sw ? a : b;
          }
        }
      }
    }
  }
}

// Block bitonic sort of n_pow2 keys in shared memory (n_pow2 a power of two,
// NT threads).  Ascending.  Contains __syncthreads.
template <int NT, typename K>
__device__ __forceinline__ void block_bitonic_sort(K* s, int n_pow2) {
  for (int size = 2; size <= n_pow2; size <<= 1) {
    for (int j = size >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < (n_pow2 >> 1); t += NT) {
        const int lo = ((t & ~(j - 1)) << 1) | (t & (j - 1));
        const int hi = lo + j;
        const bool asc = (lo & size) == 0;
        K a = s[lo], b = s[hi];
        if (asc ? (b < a) : (a < b)) {
          s[lo] = b;
          s[hi] = a;
        }
      }
      __syncthreads();
    }
  }
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
