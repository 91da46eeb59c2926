// Block-level pieces of the dense and fine-level paths: enumeration of a
// row's intermediate product straight from A and B (Gustavson traversal,
// Eq. 1), the shared-memory dense accumulator of Algorithm 1 with ordered
// emission, and the block sort accumulator used for merged small chunks.
#pragma once

#include "common.cuh"

namespace magnus {

template <int NT>
struct TileSmem {
  int64_t off[NT + 1];   // first product of each A entry of the tile
  int64_t bs[NT];        // B.rowPtr of its B row
  double av[NT];         // its A value
  int64_t ws[NT / 32 + 1];
};

// Calls f(col, value, product_index) for every product of the A entries
// [as, ae), in tiles of NT entries.  Consecutive threads take consecutive
// products, so each B row is read with coalesced loads.  `value` is
// A.val * B.val when NUMERIC, else 0.  All threads of the block must call.
template <int NT, bool NUMERIC, class F>
__device__ __forceinline__ void block_for_each_product(const Csr& A, const Csr& B, int64_t as,
                                                       int64_t ae, TileSmem<NT>& ts, F&& f) {
  int64_t pbase = 0;
  for (int64_t j0 = as; j0 < ae; j0 += NT) {
    const int64_t j = j0 + threadIdx.x;
    int64_t bs = 0, L = 0;
    double av = 0.0;
    if (j < ae) {
      const int32_t c = A.col[j];
      bs = B.rp[c];
      L = B.rp[c + 1] - bs;
      if (NUMERIC) av = A.val[j];
    }
    int64_t tot;
    const int64_t off = block_exclusive_scan<NT>(L, ts.ws, &tot);
    ts.off[threadIdx.x] = off;
    ts.bs[threadIdx.x] = bs;
    if (NUMERIC) ts.av[threadIdx.x] = av;
    const int n_a = (int)((ae - j0) < NT ? (ae - j0) : NT);
    __syncthreads();
    for (int64_t p = threadIdx.x; p < tot; p += NT) {
      const int g = upper_bound_i64(ts.off, n_a, p) - 1;
      const int64_t k = ts.bs[g] + (p - ts.off[g]);
      const int32_t col = B.col[k];
      const double v = NUMERIC ? ts.av[g] * B.val[k] : 0.0;
      f(col, v, pbase + p);
    }
    pbase += tot;
    __syncthreads();
  }
}

// Emits the set bits of bits[0..nwords) in ascending order: column
// col_base + bit index, value acc[bit index] (when NUMERIC), written at
// out_col/out_val[outp + rank].  Returns the number of set bits.
// All threads must call; contains __syncthreads.
template <int NT, bool NUMERIC>
__device__ __forceinline__ int64_t block_emit_bitmap(const uint32_t* bits, int nwords,
                                                     const double* acc, int64_t col_base,
                                                     int32_t* __restrict__ out_col,
                                                     double* __restrict__ out_val, int64_t outp,
                                                     int64_t* ws) {
  int64_t total = 0;
  for (int w0 = 0; w0 < nwords; w0 += NT) {
    const int w = w0 + threadIdx.x;
    uint32_t m = (w < nwords) ? bits[w] : 0u;
    int64_t tot;
    int64_t pos = block_exclusive_scan<NT>((int64_t)__popc(m), ws, &tot);
    if (NUMERIC) {
      int64_t o = outp + total + pos;
      while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        const int idx = w * 32 + b;
        out_col[o] = (int32_t)(col_base + idx);
        out_val[o] = acc[idx];
        ++o;
      }
    }
    total += tot;
  }
  return total;
}

}  // namespace magnus
