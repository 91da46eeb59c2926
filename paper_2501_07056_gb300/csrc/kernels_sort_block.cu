// Sort-category rows of 257..1024 products (Section 3.1, category 1, with the
// sort accumulator of Algorithm 2 widened to a thread block).
//
// A row of bin SORT512 / SORT1024 is handled by one block of CAP/8 threads
// (64 or 128), eight products per thread.
//
// Symbolic: the products' (column, slot) keys are generated from A and B and
// sorted by a bitonic network (partners within a thread are swapped in
// registers, partners within a warp exchanged by shuffles, partners in other
// warps through shared memory); the runs of equal columns are counted
// (precise prediction, Section 2.1) and the sorted slot order is stored, two
// bytes per product.
//
// Numeric: the products are generated again with their values, parked in
// shared memory by slot, and visited in the recorded order: equal columns
// are adjacent with their slots ascending, so a run is summed in the
// traversal order of Algorithm 1.  Consecutive threads take consecutive
// sorted positions and write consecutive entries of the row of C.
//
// Blocks are persistent: each takes rows idx = blockIdx.x, + gridDim.x, ...
#include "sort_accum.cuh"

namespace magnus {

namespace {

template <int CAPLOG, typename K, bool NUMERIC>
__global__ void __launch_bounds__((1 << CAPLOG) / BR) k_sort_rows_block(SortArgs a) {
  constexpr int CAP = 1 << CAPLOG;
  constexpr int NT = CAP / BR;
  constexpr int NWB = NT / 32;
  constexpr int SB = CAPLOG;  // slot bits of a key
  constexpr int HW = CAP / 32;
  using KT = KeyTraits<K>;
  __shared__ K s_key[NUMERIC ? 1 : CAP];
  __shared__ int32_t s_start[CAP + 1];  // first slot of each non-empty segment
  __shared__ int64_t s_bs[CAP];         // B.rowPtr of the segment's B row
  __shared__ double s_av[NUMERIC ? CAP : 1];
  __shared__ double s_val[NUMERIC ? CAP : 1];    // product value by slot
  __shared__ int32_t s_col[NUMERIC ? CAP : 1];   // product column by slot
  __shared__ uint16_t s_perm[NUMERIC ? CAP : 1]; // slot at each sorted position
  __shared__ uint32_t s_head[HW];
  __shared__ int32_t s_pw[HW];
  __shared__ int32_t s_ws[NWB + 1];
  __shared__ int32_t s_ws2[NWB + 1];
  const int t = threadIdx.x, lane = lane_id(), w = warp_id();
  // rows [first, n) of the bin's list: all of them, or a row range's
  const int64_t first = (NUMERIC && a.range) ? a.range[0] : 0;
  const int64_t n = (NUMERIC && a.range) ? a.range[1] : a.n_rows;
  const int64_t cbase = (NUMERIC && a.c_base) ? *a.c_base : 0;

  for (int64_t idx = first + blockIdx.x; idx < n; idx += gridDim.x) {
    const RowDesc d = a.desc[idx];
    const int64_t poff = a.perm2_off[idx];
    // 1. segments: the non-empty B rows referenced by the row, in stored
    //    order, with their first slots (block scan of the lengths)
    int nseg = 0, P = 0;
    for (int j0 = 0; j0 < d.na; j0 += NT) {
      const int j = j0 + t;
      int L = 0;
      int64_t bs = 0;
      double av = 0.0;
      if (j < d.na) {
        const uint64_t sg = a.seg[d.as + j];
        L = seg_length(sg);
        bs = seg_start(sg);
        if (NUMERIC) av = a.A.val[d.as + j];
      }
      const int nz = L > 0 ? 1 : 0;
      const int incL = warp_inclusive_scan(L);
      const int incZ = warp_inclusive_scan(nz);
      if (lane == 31) {
        s_ws[w] = incL;
        s_ws2[w] = incZ;
      }
      __syncthreads();
      int offL = 0, offZ = 0, totL = 0, totZ = 0;
#pragma unroll
      for (int i = 0; i < NWB; ++i) {
        offL += (i < w) ? s_ws[i] : 0;
        offZ += (i < w) ? s_ws2[i] : 0;
        totL += s_ws[i];
        totZ += s_ws2[i];
      }
      if (L > 0) {
        const int g = nseg + offZ + incZ - 1;
        s_start[g] = P + offL + incL - L;
        s_bs[g] = bs;
        if (NUMERIC) s_av[g] = av;
      }
      nseg += totZ;
      P += totL;
      __syncthreads();
    }
    // 2. expand: slot s = e * NT + t (consecutive threads read consecutive
    //    entries of a B row); all gathers are issued before any is used
    int64_t kk[BR];
    int gg[BR];
#pragma unroll
    for (int e = 0; e < BR; ++e) {
      const int s = e * NT + t;
      kk[e] = -1;
      gg[e] = 0;
      if (s < P) {
        const int g = upper_bound_i32(s_start, nseg, s) - 1;
        gg[e] = g;
        kk[e] = s_bs[g] + (s - s_start[g]);
      }
    }
    int32_t cg[BR];
    double vg[BR];
    uint16_t pg[BR];
#pragma unroll
    for (int e = 0; e < BR; ++e) {
      cg[e] = kk[e] >= 0 ? __ldg(a.B.col + kk[e]) : 0;
      if (NUMERIC) {
        vg[e] = kk[e] >= 0 ? __ldg(a.B.val + kk[e]) : 0.0;
        const int q = e * NT + t;
        pg[e] = q < P ? a.perm2[poff + q] : (uint16_t)0;
      }
    }
    if (!NUMERIC) {
      K key[BR];
#pragma unroll
      for (int e = 0; e < BR; ++e) {
        const int s = e * NT + t;
        key[e] = (s < P) ? KT::template make<SB>(cg[e], s) : ~K(0);
      }
      // 3s. sort, store the order, count the runs of equal columns
      block_sort_keys<NT>(key, s_key);
#pragma unroll
      for (int e = 0; e < BR; ++e) {
        const int q = t * BR + e;
        s_key[q] = key[e];
        if (q < P) a.perm2[poff + q] = (uint16_t)KT::template slot<SB>(key[e]);
      }
      __syncthreads();
      uint32_t hb = 0;
#pragma unroll
      for (int e = 0; e < BR; ++e) {
        const int q = t * BR + e;
        const int32_t c = KT::template col<SB>(key[e]);
        const int32_t pc = q == 0 ? -1 : KT::template col<SB>(s_key[q - 1]);
        if (q < P && (q == 0 || c != pc)) hb |= 1u << e;
      }
      int c = __popc(hb);
      c = warp_sum(c);
      if (lane == 0) s_ws[w] = c;
      __syncthreads();
      if (t == 0) {
        int tot = 0;
        for (int i = 0; i < NWB; ++i) tot += s_ws[i];
        a.out_cnt[d.row] = tot;
      }
    } else {
      // 3n. replay the recorded order
#pragma unroll
      for (int e = 0; e < BR; ++e) {
        const int s = e * NT + t;
        if (s < P) {
          s_col[s] = cg[e];
          s_val[s] = s_av[gg[e]] * vg[e];
          s_perm[s] = pg[e];  // position s of the sorted order holds slot pg[e]
        }
      }
      __syncthreads();
      // run heads in position-major order: word m of the head bitmap covers
      // positions 32m..32m+31, one warp's lanes for one e
      int32_t cq[BR];
#pragma unroll
      for (int e = 0; e < BR; ++e) {
        const int q = e * NT + t;
        cq[e] = q < P ? s_col[pg[e]] : 0;
        const int32_t pc = (q == 0 || q >= P) ? -1 : s_col[s_perm[q - 1]];
        const unsigned hb = __ballot_sync(FULL, q < P && cq[e] != pc);
        if (lane == 0) s_head[(e * NT + w * 32) >> 5] = hb;
      }
      __syncthreads();
      if (w == 0) {
        const int c = lane < HW ? __popc(s_head[lane]) : 0;
        const int inc = warp_inclusive_scan(c);
        if (lane < HW) s_pw[lane] = inc - c;
      }
      __syncthreads();
      const int64_t crp = a.c_rp[d.row] - cbase;
#pragma unroll
      for (int e = 0; e < BR; ++e) {
        const int q = e * NT + t;
        const uint32_t hw = q < P ? s_head[q >> 5] : 0u;
        if ((hw >> (q & 31)) & 1u) {
          const int o = s_pw[q >> 5] + __popc(hw & ((1u << (q & 31)) - 1u));
          const int32_t c = cq[e];
          double acc = s_val[pg[e]];
          for (int q2 = q + 1; q2 < P; ++q2) {
            const int s2 = s_perm[q2];
            if (s_col[s2] != c) break;
            acc += s_val[s2];
          }
          a.c_col[crp + o] = c;
          a.c_val[crp + o] = acc;
        }
      }
    }
    __syncthreads();
  }
}

// Symbolic pass of the SORT512 bin with one warp per row: sixteen keys per
// lane, sorted by the warp's register network (group_bitonic_sort over 32
// lanes: swaps in registers below distance 16, shuffles above), so neither
// shared-memory exchanges nor block barriers are needed.  Segments are found
// as in the lane-group kernel (head bits at segment starts, prefix popcounts);
// the distinct columns are counted and the sorted slot order is stored, two
// bytes per product, for the block numeric replay.
constexpr int S5_NW = 4;

template <typename K>
__global__ void __launch_bounds__(S5_NW * 32) k_sort512_symbolic(SortArgs a) {
  constexpr int CAP = 512, R = 16, SB = 9, HW = CAP / 32;
  using KT = KeyTraits<K>;
  __shared__ uint16_t s_off[S5_NW][CAP];  // first slot of each non-empty segment
  __shared__ int64_t s_bs[S5_NW][CAP];    // B.rowPtr of the segment's B row
  __shared__ uint32_t s_head[S5_NW][HW];  // bit s: a segment other than the first starts at s
  const int lane = lane_id(), w = warp_id();
  const int64_t nwarps = (int64_t)gridDim.x * S5_NW;
  for (int64_t idx = (int64_t)blockIdx.x * S5_NW + w; idx < a.n_rows; idx += nwarps) {
    const RowDesc d = a.desc[idx];
    const int64_t poff = a.perm2_off[idx];
    if (lane < HW) s_head[w][lane] = 0u;
    int nseg = 0, P = 0;
    for (int j0 = 0; j0 < d.na; j0 += 32) {
      const int j = j0 + lane;
      int L = 0;
      int64_t bs = 0;
      if (j < d.na) {
        const uint64_t sg = a.seg[d.as + j];
        L = seg_length(sg);
        bs = seg_start(sg);
      }
      const unsigned nz = __ballot_sync(FULL, L > 0);
      const int inc = warp_inclusive_scan(L);
      if (L > 0) {
        const int g = nseg + __popc(nz & ((1u << lane) - 1u));
        s_off[w][g] = (uint16_t)(P + inc - L);
        s_bs[w][g] = bs;
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
    uint32_t hw[HW];
    int pw[HW];
    {
      int cum = 0;
#pragma unroll
      for (int i = 0; i < HW; ++i) {
        hw[i] = s_head[w][i];
        pw[i] = cum;
        cum += __popc(hw[i]);
      }
    }
    // slot s = e*32 + lane; all gathers issued before any is used
    int32_t cg[R];
#pragma unroll
    for (int e = 0; e < R; ++e) {
      const int s = e * 32 + lane;
      const int g = pw[e] + __popc(hw[e] & ((2u << lane) - 1u));
      cg[e] = s < P ? __ldg(a.B.col + s_bs[w][g] + (s - s_off[w][g])) : 0;
    }
    K key[R];
#pragma unroll
    for (int e = 0; e < R; ++e) {
      const int s = e * 32 + lane;
      key[e] = s < P ? KT::template make<SB>(cg[e], s) : ~K(0);
    }
    group_bitonic_sort<R, 32>(key);
    // sorted position q = lane*R + e
    const K prev_last = __shfl_up_sync(FULL, key[R - 1], 1);
    int h = 0;
#pragma unroll
    for (int e = 0; e < R; ++e) {
      const int q = lane * R + e;
      const int32_t c = KT::template col<SB>(key[e]);
      const int32_t pc = (e == 0) ? ((lane == 0) ? -1 : KT::template col<SB>(prev_last))
                                  : KT::template col<SB>(key[e - 1]);
      h += ((q < P) && (q == 0 || c != pc)) ? 1 : 0;
      if (q < P) a.perm2[poff + q] = (uint16_t)KT::template slot<SB>(key[e]);
    }
    const int cnt = warp_sum(h);
    if (lane == 0) a.out_cnt[d.row] = cnt;
    __syncwarp();
  }
}

template <typename K>
cudaError_t launch_sort512_symbolic(const SortArgs& a, int num_sms, cudaStream_t s) {
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sort512_symbolic<K>,
                                                                  S5_NW * 32, 0);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (a.n_rows + S5_NW - 1) / S5_NW;
  const int64_t cap = (int64_t)num_sms * per_sm;
  if (blocks > cap) blocks = cap;
  k_sort512_symbolic<K><<<(unsigned)blocks, S5_NW * 32, 0, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <int CAPLOG, typename K, bool NUMERIC>
cudaError_t launch_block(const SortArgs& a, int num_sms, cudaStream_t s) {
  constexpr int NT = (1 << CAPLOG) / BR;
  auto kern = k_sort_rows_block<CAPLOG, K, NUMERIC>;
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, 0);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = a.n_rows;
  const int64_t cap = (int64_t)num_sms * per_sm;
  if (blocks > cap) blocks = cap;
  kern<<<(unsigned)blocks, NT, 0, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sort_rows_block(int bin, bool numeric, const SortArgs& a, int num_sms,
                                   cudaStream_t s) {
  if (a.n_rows == 0) return cudaSuccess;
  const bool big = bin == BIN_SORT1024;
  if (numeric)  // the replay holds no keys
    return big ? launch_block<10, uint32_t, true>(a, num_sms, s)
               : launch_block<9, uint32_t, true>(a, num_sms, s);
  if (!big)  // rows of at most 512 products: one warp per row
    return a.key32 ? launch_sort512_symbolic<uint32_t>(a, num_sms, s)
                   : launch_sort512_symbolic<uint64_t>(a, num_sms, s);
  if (a.key32) {
    return big ? launch_block<10, uint32_t, false>(a, num_sms, s)
               : launch_block<9, uint32_t, false>(a, num_sms, s);
  }
  return big ? launch_block<10, uint64_t, false>(a, num_sms, s)
             : launch_block<9, uint64_t, false>(a, num_sms, s);
}

}  // namespace magnus
