// Sort-category rows (Section 3.1, category 1; Algorithm 2): one warp per
// row.  The row's intermediate product (at most 32*E products) is generated
// straight from A and B into registers, sorted by a register bitonic network
// on packed (column, slot) keys and compressed.  The symbolic pass counts
// distinct columns (precise prediction); the numeric pass multiplies, merges
// duplicates in traversal order and writes the row of C.
#include "sort_accum.cuh"

namespace magnus {

template <int E, typename K, bool NUMERIC, int NW>
__global__ void __launch_bounds__(NW * 32) k_sort_rows(SortArgs a) {
  constexpr int CAP = 32 * E;
  constexpr int SB = Log2Cap<E>::v;
  using KT = KeyTraits<K>;
  __shared__ int32_t s_off[NW][CAP];                 // first slot of each non-empty segment
  __shared__ int64_t s_bs[NW][CAP];                  // B.rowPtr of the segment's B row
  __shared__ double s_av[NW][NUMERIC ? CAP : 1];     // A value of the segment
  __shared__ uint32_t s_head[NW][E];                 // bit s: a segment (other than 0) starts at slot s
  __shared__ double s_vals[NW][NUMERIC ? CAP : 1];   // product value by slot
  __shared__ K s_keys[NW][NUMERIC ? CAP : 1];        // sorted keys (run walking)
  const int lane = lane_id(), w = warp_id();
  const int64_t stride = (int64_t)gridDim.x * NW;
  for (int64_t t = (int64_t)blockIdx.x * NW + w; t < a.n_rows; t += stride) {
    const int32_t row = a.rows[t];
    const int64_t as = a.A.rp[row], ae = a.A.rp[row + 1];
    if (lane < E) s_head[w][lane] = 0;
    // 1. Segments: the non-empty B rows referenced by row `row` of A, in
    //    stored order, with the first slot of each in the row's product list.
    int nseg = 0, P = 0;
    for (int64_t j0 = as; j0 < ae; j0 += 32) {
      const int64_t j = j0 + lane;
      int64_t bs = 0;
      int L = 0;
      double av = 0.0;
      if (j < ae) {
        const int32_t c = a.A.col[j];
        bs = a.B.rp[c];
        L = (int)(a.B.rp[c + 1] - bs);
        if (NUMERIC) av = a.A.val[j];
      }
      const unsigned nz = __ballot_sync(FULL, L > 0);
      const int inc = warp_inclusive_scan(L);
      if (L > 0) {
        const int g = nseg + __popc(nz & ((1u << lane) - 1));
        s_off[w][g] = P + inc - L;
        s_bs[w][g] = bs;
        if (NUMERIC) s_av[w][g] = av;
      }
      nseg += __popc(nz);
      P += __shfl_sync(FULL, inc, 31);
    }
    __syncwarp();
    for (int g = 1 + lane; g < nseg; g += 32) {
      const int off = s_off[w][g];
      atomicOr(&s_head[w][off >> 5], 1u << (off & 31));
    }
    __syncwarp();
    // 2. Expand: lane handles slots e*32 + lane (coalesced B reads); the
    //    segment of a slot is the number of segment starts at or before it.
    K key[E];
    int segcum = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int s = e * 32 + lane;
      const uint32_t hb = s_head[w][e];
      const int g = segcum + __popc(hb & ((2u << lane) - 1u));
      segcum += __popc(hb);
      if (s < P) {
        const int64_t k = s_bs[w][g] + (s - s_off[w][g]);
        const int32_t c = a.B.col[k];
        key[e] = KT::template make<SB>(c, s);
        if (NUMERIC) s_vals[w][s] = s_av[w][g] * a.B.val[k];
      } else {
        key[e] = ~K(0);
      }
    }
    // 3. Sort (keys are distinct; padding sorts last).
    warp_bitonic_sort<E>(key);
    // 4. Compress.
    if (NUMERIC) {
      __syncwarp();
      const int64_t ob = a.c_rp[row];
      warp_merge_emit<E, K, true>(key, P, s_vals[w], s_keys[w], 0, a.c_col + ob, a.c_val + ob);
    } else {
      const int cnt = warp_merge_emit<E, K, false>(key, P, nullptr, nullptr, 0, nullptr, nullptr);
      if (lane == 0) a.out_cnt[row] = cnt;
    }
    __syncwarp();
  }
}

template <int E, typename K, bool NUMERIC>
static cudaError_t launch_one(const SortArgs& a, int num_sms, cudaStream_t s) {
  constexpr int NW = (E >= 8) ? 4 : 8;
  int64_t blocks = (a.n_rows + NW - 1) / NW;
  const int64_t cap = (int64_t)num_sms * 32;
  if (blocks > cap) blocks = cap;
  k_sort_rows<E, K, NUMERIC, NW><<<(unsigned)blocks, NW * 32, 0, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <typename K, bool NUMERIC>
static cudaError_t launch_bin(int bin, const SortArgs& a, int num_sms, cudaStream_t s) {
  switch (bin) {
    case BIN_SORT32: return launch_one<1, K, NUMERIC>(a, num_sms, s);
    case BIN_SORT64: return launch_one<2, K, NUMERIC>(a, num_sms, s);
    case BIN_SORT128: return launch_one<4, K, NUMERIC>(a, num_sms, s);
    case BIN_SORT256: return launch_one<8, K, NUMERIC>(a, num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_sort_rows(int bin, bool numeric, const SortArgs& a, int num_sms,
                             cudaStream_t s) {
  if (a.n_rows == 0) return cudaSuccess;
  if (a.key32) {
    return numeric ? launch_bin<uint32_t, true>(bin, a, num_sms, s)
                   : launch_bin<uint32_t, false>(bin, a, num_sms, s);
  }
  return numeric ? launch_bin<uint64_t, true>(bin, a, num_sms, s)
                 : launch_bin<uint64_t, false>(bin, a, num_sms, s);
}

}  // namespace magnus
