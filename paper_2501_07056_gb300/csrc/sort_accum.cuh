// Warp-level sort accumulator (Section 3.4; expand-sort-compress of
// Algorithm 2): up to 32*E products of one row (or one chunk) are held E per
// lane, sorted with a register bitonic network on packed (column, slot) keys,
// and equal columns are merged in slot order.  Used for sort rows and for
// small coarse-level chunks.
#pragma once

#include "common.cuh"

namespace magnus {

// Key packing: (col << SB) | slot in 32 bits when the column range allows it,
// else (col << 32) | slot in 64 bits.  The slot makes every key distinct and
// orders equal columns by traversal position, so duplicates are summed in
// the order Algorithm 1 visits them.
template <typename K> struct KeyTraits;
template <> struct KeyTraits<uint32_t> {
  template <int SB> __device__ static __forceinline__ uint32_t make(int32_t col, int slot) {
    return ((uint32_t)col << SB) | (uint32_t)slot;
  }
  template <int SB> __device__ static __forceinline__ int32_t col(uint32_t k) { return (int32_t)(k >> SB); }
  template <int SB> __device__ static __forceinline__ int slot(uint32_t k) { return (int)(k & ((1u << SB) - 1)); }
};
template <> struct KeyTraits<uint64_t> {
  template <int SB> __device__ static __forceinline__ uint64_t make(int32_t col, int slot) {
    return ((uint64_t)(uint32_t)col << 32) | (uint32_t)slot;
  }
  template <int SB> __device__ static __forceinline__ int32_t col(uint64_t k) { return (int32_t)(k >> 32); }
  template <int SB> __device__ static __forceinline__ int slot(uint64_t k) { return (int)(uint32_t)k; }
};

template <int E> struct Log2Cap;
template <> struct Log2Cap<1> { static constexpr int v = 5; };
template <> struct Log2Cap<2> { static constexpr int v = 6; };
template <> struct Log2Cap<4> { static constexpr int v = 7; };
template <> struct Log2Cap<8> { static constexpr int v = 8; };

// After warp_bitonic_sort: count (and in the numeric phase, merge and write)
// the distinct columns among the first n sorted keys.
//   vals:   per-warp shared array of product values indexed by slot (numeric)
//   skeys:  per-warp shared scratch of 32*E keys (numeric)
//   col_add: added to every emitted column (chunk base)
// Returns the number of distinct columns (same value in every lane).
template <int E, typename K, bool NUMERIC>
__device__ __forceinline__ int warp_merge_emit(const K (&k)[E], int n, const double* vals, K* skeys,
                                               int32_t col_add, int32_t* __restrict__ out_col,
                                               double* __restrict__ out_val) {
  using KT = KeyTraits<K>;
  constexpr int SB = Log2Cap<E>::v;
  const int lane = lane_id();
  const K prev_last = __shfl_up_sync(FULL, k[E - 1], 1);
  bool head[E];
  int h = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int q = lane * E + e;
    const int32_t c = KT::template col<SB>(k[e]);
    int32_t pc;
    if (e == 0) pc = (lane == 0) ? -1 : KT::template col<SB>(prev_last);
    else pc = KT::template col<SB>(k[e - 1]);
    head[e] = (q < n) && (q == 0 || c != pc);
    h += head[e] ? 1 : 0;
  }
  const int inc = warp_inclusive_scan(h);
  const int total = __shfl_sync(FULL, inc, 31);
  if (NUMERIC) {
#pragma unroll
    for (int e = 0; e < E; ++e) skeys[lane * E + e] = k[e];
    __syncwarp();
    int pos = inc - h;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if (head[e]) {
        const int q = lane * E + e;
        const int32_t c = KT::template col<SB>(k[e]);
        double acc = vals[KT::template slot<SB>(k[e])];
        for (int q2 = q + 1; q2 < n; ++q2) {
          const K k2 = skeys[q2];
          if (KT::template col<SB>(k2) != c) break;
          acc += vals[KT::template slot<SB>(k2)];
        }
        out_col[pos] = c + col_add;
        out_val[pos] = acc;
        ++pos;
      }
    }
    __syncwarp();
  }
  return total;
}

// Block sort of the coarse buckets of 257..2048 products whose column
// sub-ranges overflow (the fallback of bucket_sort_keys in kernels_coarse.cu).
constexpr int BR = 8;  // keys per thread

// Bitonic sort of NT * BR keys; thread t holds positions t * BR + e.  As in
// group_bitonic_sort, every level starts with a flip stage (position q
// against the mirror position of its block) and continues with ascending
// half-cleaners, so no compare-exchange needs a direction.  Partners in the
// same thread are swapped in registers, partners in the same warp exchanged
// by shuffles, partners in other warps through s_key (NT * BR keys).
template <int NT, typename K>
__device__ __forceinline__ void block_sort_keys(K (&key)[BR], K* s_key) {
  constexpr int CAP = NT * BR;
  const int t = threadIdx.x;
  const int tb = t * BR;
  // levels inside a thread: each thread's BR keys become one ascending run
#pragma unroll
  for (int size = 2; size <= BR; size <<= 1) {
#pragma unroll
    for (int e = 0; e < BR; ++e) {
      const int b = e & ~(size - 1);
      const int m = b + size - 1 - (e - b);
      if (e < m) {
        const K lo = key[e] < key[m] ? key[e] : key[m];
        const K hi = key[e] < key[m] ? key[m] : key[e];
        key[e] = lo;
        key[m] = hi;
      }
    }
#pragma unroll
    for (int j = size >> 2; j > 0; j >>= 1) {
#pragma unroll
      for (int e = 0; e < BR; ++e) {
        if ((e & j) == 0) {
          const K lo = key[e] < key[e + j] ? key[e] : key[e + j];
          const K hi = key[e] < key[e + j] ? key[e + j] : key[e];
          key[e] = lo;
          key[e + j] = hi;
        }
      }
    }
  }
  // levels across threads: merge the runs
#pragma unroll
  for (int size = 2 * BR; size <= CAP; size <<= 1) {
    {
      const int pm = size / BR - 1;  // mirror thread within the block of `size`
      const bool lower = (t & (size / BR / 2)) == 0;
      K o[BR];
      if (pm < 32) {
#pragma unroll
        for (int e = 0; e < BR; ++e) o[e] = __shfl_xor_sync(FULL, key[BR - 1 - e], pm);
      } else {
#pragma unroll
        for (int e = 0; e < BR; ++e) s_key[tb + e] = key[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < BR; ++e) o[e] = s_key[(t ^ pm) * BR + (BR - 1 - e)];
        __syncthreads();
      }
#pragma unroll
      for (int e = 0; e < BR; ++e)
        key[e] = lower ? (o[e] < key[e] ? o[e] : key[e]) : (o[e] > key[e] ? o[e] : key[e]);
    }
#pragma unroll
    for (int j = size >> 2; j > 0; j >>= 1) {
      if (j >= BR) {
        const int pl = j / BR;  // partner thread distance
        const bool lower = (t & pl) == 0;
        if (pl < 32) {
#pragma unroll
          for (int e = 0; e < BR; ++e) {
            const K o = __shfl_xor_sync(FULL, key[e], pl);
            key[e] = lower ? (o < key[e] ? o : key[e]) : (o > key[e] ? o : key[e]);
          }
        } else {
#pragma unroll
          for (int e = 0; e < BR; ++e) s_key[tb + e] = key[e];
          __syncthreads();
#pragma unroll
          for (int e = 0; e < BR; ++e) {
            const K o = s_key[(tb + e) ^ j];
            key[e] = lower ? (o < key[e] ? o : key[e]) : (o > key[e] ? o : key[e]);
          }
          __syncthreads();
        }
      } else {
#pragma unroll
        for (int e = 0; e < BR; ++e) {
          if ((e & j) == 0) {
            const K lo = key[e] < key[e + j] ? key[e] : key[e + j];
            const K hi = key[e] < key[e + j] ? key[e + j] : key[e];
            key[e] = lo;
            key[e + j] = hi;
          }
        }
      }
    }
  }
}

}  // namespace magnus
