// Sort-category rows of 257..1024 products (Section 3.1, category 1, with the
// sort accumulator of Algorithm 2 widened past one lane group).
//
// Symbolic (bins SORT512 and SORT1024): one warp per row.  The products'
// (column, slot) keys are generated from A and B, CAP/32 per lane, and
// sorted by the warp's register network; the runs of equal columns are
// counted (precise prediction, Section 2.1) and the sorted slot order is
// stored, two bytes per product.
//
// Numeric: the products are generated again with their values, parked in
// shared memory by slot, and visited in the recorded order: equal columns
// are adjacent with their slots ascending, so a run is summed in the
// traversal order of Algorithm 1.  Rows of at most 512 products take one
// warp each; rows of 513..1024 one block of 128 threads (eight slots per
// thread), which keeps the row's values in shared memory instead of
// registers.  Consecutive threads take consecutive sorted positions and
// write consecutive entries of the row of C.
//
// Warps and blocks are persistent: each takes rows idx, idx + its stride, ...
#include <type_traits>

#include "sort_accum.cuh"

namespace magnus {

namespace {

// Numeric pass of the SORT1024 bin: one block of CAP/8 threads per row,
// eight slots per thread (slot s = e*NT + t).  The steps of the warp kernel
// below, with the segment table, the slots and the bitmaps shared by the
// block's warps: segments by a block scan, the segment of a slot by the
// bitmap's prefix popcount, the slots parked over the segment table once
// every gather has returned, run heads by comparing each position's column
// with the previous position's (a shuffle, or shared memory across warps).
template <int CAPLOG>
__global__ void __launch_bounds__((1 << CAPLOG) / BR) k_sort_block_numeric(SortArgs a) {
  constexpr int CAP = 1 << CAPLOG;
  constexpr int NT = CAP / BR;
  constexpr int NWB = NT / 32;
  constexpr int HW = CAP / 32;
  struct SegT {
    int64_t base[CAP];  // B.rowPtr of the segment's B row minus its first slot
    double av[CAP];     // the A value that scales the segment
  };
  struct SlotT {
    double val[CAP];    // product value by slot
    int32_t col[CAP];   // product column by slot
  };
  union Area {
    SegT seg;
    SlotT slot;
  };
  __shared__ Area ar;
  __shared__ uint16_t s_perm[CAP];  // slot at each sorted position
  __shared__ uint32_t s_head[HW];   // bit s: a segment other than the first starts at s
  __shared__ int32_t s_pw[HW];      // segments starting in earlier words
  __shared__ uint32_t s_qh[HW];     // bit q: a run of equal columns starts at q
  __shared__ int32_t s_qw[HW];      // runs starting in earlier words
  __shared__ int32_t s_ws[NWB + 1];
  __shared__ int32_t s_ws2[NWB + 1];
  const int t = threadIdx.x, lane = lane_id(), w = warp_id();
  // rows [first, n) of the bin's list: all of them, or a row range's
  const int64_t first = a.range ? a.range[0] : 0;
  const int64_t n = a.range ? a.range[1] : a.n_rows;
  const int64_t cbase = a.c_base ? *a.c_base : 0;

  for (int64_t idx = first + blockIdx.x; idx < n; idx += gridDim.x) {
    const RowDesc d = a.desc[idx];
    const int64_t poff = a.perm2_off[idx];
    if (t < HW) s_head[t] = 0u;
    __syncthreads();
    // 1. segments: the non-empty B rows in stored order, their first slots
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
        av = a.A.val[d.as + j];
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
        const int off = P + offL + incL - L;
        ar.seg.base[g] = bs - off;
        ar.seg.av[g] = av;
        if (g > 0) atomicOr(&s_head[off >> 5], 1u << (off & 31));
      }
      nseg += totZ;
      P += totL;
      __syncthreads();
    }
    if (w == 0) {
      const uint32_t hw = lane < HW ? s_head[lane] : 0u;
      const int c = __popc(hw);
      const int inc = warp_inclusive_scan(c);
      if (lane < HW) s_pw[lane] = inc - c;
    }
    __syncthreads();
    // 2. gather slot s = e*NT + t (consecutive threads read consecutive
    //    entries of a B row); all loads issued before any is used
    int32_t cg[BR];
    double vg[BR];
    uint32_t pg[BR];
#pragma unroll
    for (int e = 0; e < BR; ++e) {
      const int s = e * NT + t;
      cg[e] = 0;
      vg[e] = 0.0;
      pg[e] = 0u;
      if (s < P) {
        const int g = s_pw[s >> 5] + __popc(s_head[s >> 5] & ((2u << lane) - 1u));
        const int64_t kk = ar.seg.base[g] + s;
        cg[e] = __ldg(a.B.col + kk);
        vg[e] = ar.seg.av[g] * __ldg(a.B.val + kk);
        pg[e] = a.perm2[poff + s];
      }
    }
    __syncthreads();  // the segment table is consumed; its space takes the slots
#pragma unroll
    for (int e = 0; e < BR; ++e) {
      const int s = e * NT + t;
      if (s < P) {
        ar.slot.col[s] = cg[e];
        ar.slot.val[s] = vg[e];
        s_perm[s] = (uint16_t)pg[e];
      }
    }
    __syncthreads();
    // 3. run heads in position order (position q = e*NT + t holds slot pg[e])
    int32_t cq[BR];
    uint32_t qh[BR];
#pragma unroll
    for (int e = 0; e < BR; ++e) {
      const int q = e * NT + t;
      const bool in = q < P;
      cq[e] = in ? ar.slot.col[pg[e]] : 0;
      int32_t up = __shfl_up_sync(FULL, cq[e], 1);
      if (lane == 0) up = (in && q > 0) ? ar.slot.col[s_perm[q - 1]] : -1;
      qh[e] = __ballot_sync(FULL, in && cq[e] != up);
      if (lane == 0) s_qh[q >> 5] = qh[e];
    }
    __syncthreads();
    if (w == 0) {
      const uint32_t hw = lane < HW ? s_qh[lane] : 0u;
      const int c = __popc(hw);
      const int inc = warp_inclusive_scan(c);
      if (lane < HW) s_qw[lane] = inc - c;
    }
    __syncthreads();
    // 4. one output per run, written at C.rowPtr + the run's rank
    const int64_t crp = a.c_rp[d.row] - cbase;
#pragma unroll
    for (int e = 0; e < BR; ++e) {
      const int q = e * NT + t;
      const uint32_t h = qh[e];
      if ((h >> lane) & 1u) {
        const int o = s_qw[q >> 5] + __popc(h & ((1u << lane) - 1u));
        double acc = ar.slot.val[pg[e]];
        const uint32_t next_head =
            lane < 31 ? (h >> (lane + 1)) & 1u : (q + 1 < P ? s_qh[(q + 1) >> 5] & 1u : 1u);
        if (!next_head) {
          for (int q2 = q + 1; q2 < P && !((s_qh[q2 >> 5] >> (q2 & 31)) & 1u); ++q2)
            acc += ar.slot.val[s_perm[q2]];
        }
        a.c_col[crp + o] = cq[e];
        a.c_val[crp + o] = acc;
      }
    }
    __syncthreads();
  }
}

// Symbolic pass of the SORT512 and SORT1024 bins with one warp per row.
// The row's (column, slot) keys are split by column into NB = CAP/8
// buckets of consecutive column ranges (a multiply-high of the column's
// offset from the row's smallest column; counts by shared-memory atomics,
// bucket starts by a warp scan), and every lane sorts its buckets in
// registers (odd-even merge sort: each bucket alone when all hold at most 16
// keys, else adjacent pairs of at most 32 keys): well under half the
// compare-exchanges of one warp-wide network over all CAP keys and none of
// its shuffles, which matters because the network keeps the integer pipe
// busy.  Buckets follow column order, so their concatenation is the sorted
// order.  A row with a pair of more than 32 keys (a narrow or skewed column
// range) takes the warp-wide bitonic network instead (group_bitonic_sort over 32 lanes: swaps
// in registers below distance CAP/32, shuffles above).  The distinct columns
// are counted (precise prediction, Section 2.1) and the sorted slot order
// is stored, two bytes per product, for the numeric replay.
constexpr int SW_NW = 4;

template <int CAPLOG, typename K>
__global__ void __launch_bounds__(SW_NW * 32, CAPLOG == 9 ? (sizeof(K) == 4 ? 6 : 4) : (sizeof(K) == 4 ? 4 : 3))
    k_sortw_symbolic(SortArgs a) {
  constexpr int CAP = 1 << CAPLOG, R = CAP / 32, SB = CAPLOG, HW = CAP / 32;
  constexpr int NBL = R / 8;    // buckets per lane
  constexpr int NB = 32 * NBL;  // buckets per row: at most 8 keys each on average
  using KT = KeyTraits<K>;
  union Area {
    int64_t bs[CAP];  // B.rowPtr of each segment's B row
    K key[CAP];       // then the keys, bucket by bucket
  };
  __shared__ Area s_area[SW_NW];
  __shared__ uint16_t s_off[SW_NW][CAP];  // first slot of each segment; then the sorted slots
  __shared__ uint32_t s_head[SW_NW][HW];  // bit s: a segment other than the first starts at s
  __shared__ int32_t s_pw[SW_NW][HW];     // segments starting in earlier words
  __shared__ int32_t s_cnt[SW_NW][NB];    // keys per bucket
  __shared__ int32_t s_bst[SW_NW][NB];    // first sorted position of each bucket
  const int lane = lane_id(), w = warp_id();
  const int64_t nwarps = (int64_t)gridDim.x * SW_NW;
  Area& ar = s_area[w];
  // the next row's descriptor and first 32 segment entries are loaded while
  // the current row's gathers are in flight
  int64_t idx = (int64_t)blockIdx.x * SW_NW + w;
  RowDesc d{0, 0, 0};
  int64_t poff = 0;
  uint64_t sg_pf = 0;
  if (idx < a.n_rows) {
    d = a.desc[idx];
    poff = a.perm2_off[idx];
    if (lane < d.na) sg_pf = a.seg[d.as + lane];
  }
  for (; idx < a.n_rows; idx += nwarps) {
    if (lane < HW) s_head[w][lane] = 0u;
    for (int i = lane; i < NB; i += 32) s_cnt[w][i] = 0;
    __syncwarp();
    int nseg = 0, P = 0;
    for (int j0 = 0; j0 < d.na; j0 += 32) {
      const int j = j0 + lane;
      int L = 0;
      int64_t bs = 0;
      if (j < d.na) {
        const uint64_t sg = j0 == 0 ? sg_pf : a.seg[d.as + j];
        L = seg_length(sg);
        bs = seg_start(sg);
      }
      const unsigned nz = __ballot_sync(FULL, L > 0);
      const int inc = warp_inclusive_scan(L);
      if (L > 0) {
        const int g = nseg + __popc(nz & ((1u << lane) - 1u));
        const int off = P + inc - L;
        s_off[w][g] = (uint16_t)off;
        ar.bs[g] = bs;
        if (g > 0) atomicOr(&s_head[w][off >> 5], 1u << (off & 31));
      }
      nseg += __popc(nz);
      P += __shfl_sync(FULL, inc, 31);
    }
    __syncwarp();
    {
      const uint32_t hw = lane < HW ? s_head[w][lane] : 0u;
      const int c = __popc(hw);
      const int inc = warp_inclusive_scan(c);
      if (lane < HW) s_pw[w][lane] = inc - c;
    }
    __syncwarp();
    // slot s = e*32 + lane; all gathers issued before any is used
    int32_t cg[R];
#pragma unroll
    for (int e = 0; e < R; ++e) {
      const int s = e * 32 + lane;
      cg[e] = 0;
      if (s < P) {
        const int g = s_pw[w][e] + __popc(s_head[w][e] & ((2u << lane) - 1u));
        cg[e] = __ldg(a.B.col + ar.bs[g] + (s - s_off[w][g]));
      }
    }
    RowDesc nd{0, 0, 0};
    int64_t npoff = 0;
    if (idx + nwarps < a.n_rows) {
      nd = a.desc[idx + nwarps];
      npoff = a.perm2_off[idx + nwarps];
      if (lane < nd.na) sg_pf = a.seg[nd.as + lane];
    }
    // buckets: column c goes to floor((c - mn) * NB / range), computed as a
    // multiply-high (monotone in c, clamped to the last bucket)
    int32_t mn = 0x7fffffff, mx = -1;
#pragma unroll
    for (int e = 0; e < R; ++e) {
      if (e * 32 + lane < P) {
        mn = min(mn, cg[e]);
        mx = max(mx, cg[e]);
      }
    }
    mn = warp_min(mn);
    mx = warp_max(mx);
    const uint32_t range = (uint32_t)(mx - mn) + 1u;
    const uint32_t mul =
        range <= (uint32_t)NB
            ? 0u
            : (uint32_t)fminf((float)NB * 4294967296.0f / (float)range, 4294967040.0f);
    uint32_t br[R];  // bucket << 16 | rank in the bucket
#pragma unroll
    for (int e = 0; e < R; ++e) {
      br[e] = 0u;
      if (e * 32 + lane < P) {
        const uint32_t o = (uint32_t)(cg[e] - mn);
        const uint32_t b = range <= (uint32_t)NB ? o : min(__umulhi(o, mul), (uint32_t)NB - 1u);
        br[e] = (b << 16) | (uint32_t)atomicAdd(&s_cnt[w][b], 1);
      }
    }
    __syncwarp();
    // lane l owns buckets l*NBL .. l*NBL + NBL - 1 (adjacent column ranges):
    // each sorted alone when every bucket holds at most 16 keys, else each
    // pair together when every pair holds at most 32, else the warp network
    int cb[NBL];
    int tot = 0;
    bool over16 = false, over32 = false;
#pragma unroll
    for (int j = 0; j < NBL; ++j) {
      cb[j] = s_cnt[w][lane * NBL + j];
      tot += cb[j];
      over16 = over16 || cb[j] > 16;
      if (j & 1) over32 = over32 || cb[j - 1] + cb[j] > 32;
    }
    const int start = warp_inclusive_scan(tot) - tot;
    {
      int st = start;
#pragma unroll
      for (int j = 0; j < NBL; ++j) {
        s_bst[w][lane * NBL + j] = st;
        st += cb[j];
      }
    }
    const bool fallback = __any_sync(FULL, over32);
    const bool pairs = __any_sync(FULL, over16);
    __syncwarp();  // the segment starts are consumed; their space takes the keys
#pragma unroll
    for (int e = 0; e < R; ++e) {
      const int s = e * 32 + lane;
      if (s < P) ar.key[s_bst[w][br[e] >> 16] + (br[e] & 0xffffu)] = KT::template make<SB>(cg[e], s);
    }
    __syncwarp();
    int h = 0;
    // sorts keys [st, st + c) of the lane in registers, stages their slots,
    // counts the first key of every column
    auto sort_run = [&](auto nk, int st, int c) {
      constexpr int N = decltype(nk)::value;
      K kk[N];
#pragma unroll
      for (int i = 0; i < N; ++i) kk[i] = i < c ? ar.key[st + i] : ~K(0);
      lane_oddeven_sort<N>(kk);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        if (i < c) {
          s_off[w][st + i] = (uint16_t)KT::template slot<SB>(kk[i]);
          h += (i == 0 || KT::template col<SB>(kk[i]) != KT::template col<SB>(kk[i > 0 ? i - 1 : 0]))
                   ? 1 : 0;
        }
      }
    };
    if (!fallback) {
      int st = start;
      if (!pairs) {
#pragma unroll
        for (int j = 0; j < NBL; ++j) {
          sort_run(std::integral_constant<int, 16>{}, st, cb[j]);
          st += cb[j];
        }
      } else {
#pragma unroll
        for (int j = 0; j < NBL; j += 2) {
          sort_run(std::integral_constant<int, 32>{}, st, cb[j] + cb[j + 1]);
          st += cb[j] + cb[j + 1];
        }
      }
      __syncwarp();
      // the sorted slots, written coalesced
      for (int q = lane; q < P; q += 32) a.perm2[poff + q] = s_off[w][q];
    } else {
      K key[R];
#pragma unroll
      for (int e = 0; e < R; ++e) {
        const int s = e * 32 + lane;
        key[e] = s < P ? ar.key[s] : ~K(0);
      }
      group_bitonic_sort<R, 32>(key);
      // sorted position q = lane*R + e
      const K prev_last = __shfl_up_sync(FULL, key[R - 1], 1);
#pragma unroll
      for (int e = 0; e < R; ++e) {
        const int q = lane * R + e;
        const int32_t c = KT::template col<SB>(key[e]);
        const int32_t pc = (e == 0) ? ((lane == 0) ? -1 : KT::template col<SB>(prev_last))
                                    : KT::template col<SB>(key[e > 0 ? e - 1 : 0]);
        h += ((q < P) && (q == 0 || c != pc)) ? 1 : 0;
        if (q < P) a.perm2[poff + q] = (uint16_t)KT::template slot<SB>(key[e]);
      }
    }
    const int cnt = warp_sum(h);
    if (lane == 0) a.out_cnt[d.row] = cnt;
    d = nd;
    poff = npoff;
    __syncwarp();
  }
}

// Numeric pass of the SORT512 bin with one warp per row.  The segment of
// slot s = e*32 + lane is found from the segment-start bitmap (a population
// count, no search); its B entry is gathered, scaled by the row's A value
// and parked in shared memory by slot, over the segment table, which is no
// longer needed once every gather has returned.  Position q = e*32 + lane of
// the recorded order then reads slot perm2[q]; a position starts a run of
// equal columns when its column differs from the previous position's (one
// shuffle).  A run head whose next position is also a head (the common
// case) writes its product at once; a longer run is summed in position
// order, which is slot order within the run (Algorithm 1's traversal order).
// No block barriers: the warps of a block are independent.
constexpr int S5N_NW = 4;

__global__ void __launch_bounds__(S5N_NW * 32, 4) k_sort512_numeric(SortArgs a) {
  constexpr int CAP = 512, R = CAP / 32, HW = CAP / 32;
  struct SegT {
    int64_t base[CAP];  // B.rowPtr of the segment's B row minus its first slot
    double av[CAP];     // the A value that scales the segment
  };
  struct SlotT {
    double val[CAP];    // product value by slot
    int32_t col[CAP];   // product column by slot
  };
  union Area {
    SegT seg;
    SlotT slot;
  };
  __shared__ Area s_area[S5N_NW];
  __shared__ uint16_t s_perm[S5N_NW][CAP];  // slot at each sorted position
  __shared__ uint32_t s_head[S5N_NW][HW];   // bit s: a segment other than the first starts at s
  __shared__ int32_t s_pw[S5N_NW][HW];      // segments starting in earlier words
  __shared__ uint32_t s_qh[S5N_NW][HW];     // bit q: a run of equal columns starts at q
  const int lane = lane_id(), w = warp_id();
  const int64_t first = a.range ? a.range[0] : 0;
  const int64_t n = a.range ? a.range[1] : a.n_rows;
  const int64_t cbase = a.c_base ? *a.c_base : 0;
  const int64_t nwarps = (int64_t)gridDim.x * S5N_NW;
  Area& ar = s_area[w];
  // the next row's descriptor and first 32 segment entries are loaded while
  // the current row's gathers are in flight
  int64_t idx = first + (int64_t)blockIdx.x * S5N_NW + w;
  RowDesc d{0, 0, 0};
  int64_t poff = 0;
  uint64_t sg_pf = 0;
  double av_pf = 0.0;
  if (idx < n) {
    d = a.desc[idx];
    poff = a.perm2_off[idx];
    if (lane < d.na) {
      sg_pf = a.seg[d.as + lane];
      av_pf = a.A.val[d.as + lane];
    }
  }
  for (; idx < n; idx += nwarps) {
    if (lane < HW) s_head[w][lane] = 0u;
    __syncwarp();
    // 1. segments: the non-empty B rows in stored order, their first slots
    int nseg = 0, P = 0;
    for (int j0 = 0; j0 < d.na; j0 += 32) {
      const int j = j0 + lane;
      int L = 0;
      int64_t bs = 0;
      double av = 0.0;
      if (j < d.na) {
        const uint64_t sg = j0 == 0 ? sg_pf : a.seg[d.as + j];
        L = seg_length(sg);
        bs = seg_start(sg);
        av = j0 == 0 ? av_pf : a.A.val[d.as + j];
      }
      const unsigned nz = __ballot_sync(FULL, L > 0);
      const int inc = warp_inclusive_scan(L);
      if (L > 0) {
        const int g = nseg + __popc(nz & ((1u << lane) - 1u));
        const int off = P + inc - L;
        ar.seg.base[g] = bs - off;
        ar.seg.av[g] = av;
        if (g > 0) atomicOr(&s_head[w][off >> 5], 1u << (off & 31));
      }
      nseg += __popc(nz);
      P += __shfl_sync(FULL, inc, 31);
    }
    __syncwarp();
    {
      const uint32_t hw = lane < HW ? s_head[w][lane] : 0u;
      const int c = __popc(hw);
      const int inc = warp_inclusive_scan(c);
      if (lane < HW) s_pw[w][lane] = inc - c;
    }
    __syncwarp();
    // 2. gather slot s = e*32 + lane; all loads issued before any is used
    int32_t cg[R];
    double vg[R];
    uint32_t pg[R];
#pragma unroll
    for (int e = 0; e < R; ++e) {
      const int s = e * 32 + lane;
      cg[e] = 0;
      vg[e] = 0.0;
      pg[e] = 0u;
      if (s < P) {
        const int g = s_pw[w][e] + __popc(s_head[w][e] & ((2u << lane) - 1u));
        const int64_t kk = ar.seg.base[g] + s;
        cg[e] = __ldg(a.B.col + kk);
        vg[e] = ar.seg.av[g] * __ldg(a.B.val + kk);
        pg[e] = a.perm2[poff + s];
      }
    }
    const int64_t crp = a.c_rp[d.row] - cbase;
    RowDesc nd{0, 0, 0};
    int64_t npoff = 0;
    if (idx + nwarps < n) {
      nd = a.desc[idx + nwarps];
      npoff = a.perm2_off[idx + nwarps];
      if (lane < nd.na) {
        sg_pf = a.seg[nd.as + lane];
        av_pf = a.A.val[nd.as + lane];
      }
    }
    __syncwarp();  // the segment table is consumed; its space takes the slots
#pragma unroll
    for (int e = 0; e < R; ++e) {
      const int s = e * 32 + lane;
      if (s < P) {
        ar.slot.col[s] = cg[e];
        ar.slot.val[s] = vg[e];
        s_perm[w][s] = (uint16_t)pg[e];
      }
    }
    __syncwarp();
    // 3. run heads in position order
    int32_t cq[R];
    uint32_t qh[R];
    int32_t tail = -1;  // column at the position before e*32
#pragma unroll
    for (int e = 0; e < R; ++e) {
      const int q = e * 32 + lane;
      const bool in = q < P;
      cq[e] = in ? ar.slot.col[pg[e]] : 0;
      int32_t up = __shfl_up_sync(FULL, cq[e], 1);
      if (lane == 0) up = tail;
      qh[e] = __ballot_sync(FULL, in && cq[e] != up);
      tail = __shfl_sync(FULL, cq[e], 31);
    }
    if (lane < HW) {
      uint32_t h = 0u;
#pragma unroll
      for (int e = 0; e < R; ++e) h = lane == e ? qh[e] : h;
      s_qh[w][lane] = h;
    }
    __syncwarp();
    // 4. one output per run, written at C.rowPtr + the run's rank
    int base_o = 0;
#pragma unroll
    for (int e = 0; e < R; ++e) {
      const int q = e * 32 + lane;
      const uint32_t h = qh[e];
      if ((h >> lane) & 1u) {
        const int o = base_o + __popc(h & ((1u << lane) - 1u));
        double acc = ar.slot.val[pg[e]];
        const uint32_t next_head =
            lane < 31 ? (h >> (lane + 1)) & 1u : (e + 1 < R ? qh[e + 1 < R ? e + 1 : e] & 1u : 1u);
        if (!next_head) {
          for (int q2 = q + 1; q2 < P && !((s_qh[w][q2 >> 5] >> (q2 & 31)) & 1u); ++q2)
            acc += ar.slot.val[s_perm[w][q2]];
        }
        a.c_col[crp + o] = cq[e];
        a.c_val[crp + o] = acc;
      }
      base_o += __popc(h);
    }
    d = nd;
    poff = npoff;
    __syncwarp();
  }
}

cudaError_t launch_sort512_numeric(const SortArgs& a, int num_sms, cudaStream_t s) {
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sort512_numeric,
                                                                  S5N_NW * 32, 0);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (a.n_rows + S5N_NW - 1) / S5N_NW;
  const int64_t cap = (int64_t)num_sms * per_sm;
  if (blocks > cap) blocks = cap;
  k_sort512_numeric<<<(unsigned)blocks, S5N_NW * 32, 0, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <int CAPLOG, typename K>
cudaError_t launch_sortw_symbolic(const SortArgs& a, int num_sms, cudaStream_t s) {
  auto kern = k_sortw_symbolic<CAPLOG, K>;
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SW_NW * 32, 0);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (a.n_rows + SW_NW - 1) / SW_NW;
  const int64_t cap = (int64_t)num_sms * per_sm;
  if (blocks > cap) blocks = cap;
  kern<<<(unsigned)blocks, SW_NW * 32, 0, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <int CAPLOG>
cudaError_t launch_block_numeric(const SortArgs& a, int num_sms, cudaStream_t s) {
  constexpr int NT = (1 << CAPLOG) / BR;
  auto kern = k_sort_block_numeric<CAPLOG>;
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
    return big ? launch_block_numeric<10>(a, num_sms, s) : launch_sort512_numeric(a, num_sms, s);
  if (a.key32)  // symbolic: one warp per row
    return big ? launch_sortw_symbolic<10, uint32_t>(a, num_sms, s)
               : launch_sortw_symbolic<9, uint32_t>(a, num_sms, s);
  return big ? launch_sortw_symbolic<10, uint64_t>(a, num_sms, s)
             : launch_sortw_symbolic<9, uint64_t>(a, num_sms, s);
}

}  // namespace magnus
