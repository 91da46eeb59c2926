// Sort-category rows (Section 3.1, category 1; Algorithm 2).
//
// A row of bin E holds at most 32*E products.  It is handled by a group of
// W = 4*E lanes with R = 8 products per lane, so a warp works on G = 8/E rows
// at once: every level of the load chain (row id, A.rowPtr, A.col/A.val,
// B.rowPtr, B.col/B.val) is issued for G rows together, and the sorting
// network runs mostly inside registers (three of its stage distances stay in
// a lane).
//
// Symbolic: the row's products are generated from A and B into registers,
// sorted by a bitonic network on packed (column, slot) keys and their
// distinct columns counted (precise prediction, Section 2.1).  The sorted
// order of the slots is kept, one byte per product, for the numeric pass.
//
// Numeric: the products are generated again with their values
// A.val * B.val; they are visited in the recorded sorted order, equal
// columns are summed in slot order (the traversal order of Algorithm 1), and
// the row of C is written.
//
// Rows whose nonzeros number at most W and each select a B row of 1..R
// entries ("run rows": every uniform row) number their products run-major,
// slot = j * R + x for the x-th entry of the B row of the row's j-th nonzero.
// This keeps traversal order and lets the symbolic pass skip most of the
// network: the B rows are stored sorted (an ABI requirement), so after a
// transpose through shared memory each lane holds one sorted run of R keys,
// and only the merge levels of the bitonic network remain
// (group_merge_runs).  A warp whose rows are all run rows takes that path;
// otherwise it runs the general expansion and the full network, numbering the
// products of any run rows among them the same way, so the recorded order
// means the same in both passes whichever path either took.
#include "sort_accum.cuh"

namespace magnus {

// Shared layout of one group's keys for the run transpose: run r, entry x at
// r * R + 4 * ((x >> 2) ^ ((r >> 2) & 1)) + (x & 3), groups KSTRIDE keys
// apart.  The 4-key swizzle and the group pad keep both the writes (a run
// per W/R lanes) and the 16-byte reads of whole runs free of bank conflicts.
template <int W> struct RunLayout {
  static constexpr int R = 8;
  static constexpr int CAP = W * R;
  static constexpr int KSTRIDE = CAP + (W < 32 ? W : 0);
  __device__ static __forceinline__ int at(int r, int x) {
    return r * R + 4 * ((x >> 2) ^ ((r >> 2) & 1)) + (x & 3);
  }
};

template <int E, typename K, bool NUMERIC, int NW>
__global__ void __launch_bounds__(NW * 32, (NUMERIC ? 20 : 32) / NW) k_sort_rows(SortArgs a) {
  constexpr int W = 4 * E;    // lanes per row
  constexpr int G = 32 / W;   // rows per warp
  constexpr int R = 8;        // products per lane
  constexpr int CAP = W * R;  // = 32 * E
  constexpr int SB = Log2Cap<E>::v;
  constexpr int HW = CAP / 32;  // head-bit words per row
  using KT = KeyTraits<K>;
  using RL = RunLayout<W>;
  // Per-warp shared arrays, indexed [position][group] so that the lanes of
  // the G groups interleave and a warp-wide access touches distinct banks.
  __shared__ uint8_t s_off[NW][CAP][G];    // first slot of each non-empty segment
  __shared__ int64_t s_bs[NW][CAP][G];     // B.rowPtr of the segment's B row
  __shared__ double s_av[NW][NUMERIC ? CAP : 1][G];
  __shared__ uint32_t s_head[NW][HW][G];   // bit s: a segment other than the first starts at slot s
  __shared__ int32_t s_col[NW][NUMERIC ? CAP : 1][G];
  __shared__ double s_val[NW][NUMERIC ? CAP : 1][G];
  __shared__ uint8_t s_perm[NW][NUMERIC ? CAP : 1][G];
  __shared__ uint8_t s_len[NW][W][G];      // run rows: entries of the j-th nonzero's B row
  __shared__ __align__(16) K s_key[NW][NUMERIC ? 1 : G * RL::KSTRIDE];
  const int lane = lane_id(), w = warp_id();
  const int grp = lane / W, l = lane & (W - 1);
  const int gshift = grp * W;
  const unsigned gbits = (W == 32) ? FULL : ((1u << W) - 1u);
  const int64_t stride = (int64_t)gridDim.x * NW * G;
  // rows [first, n) of the bin's list: all of them, or a row range's
  const int64_t first = (NUMERIC && a.range) ? a.range[0] : 0;
  const int64_t n = (NUMERIC && a.range) ? a.range[1] : a.n_rows;
  const int64_t cbase = (NUMERIC && a.c_base) ? *a.c_base : 0;

  // Level 1 of the load chain: the row descriptor (and the recorded order).
  struct Pre1 { RowDesc d; uint64_t perm; };
  // Level 2: output offset and the first W segment-table entries of the row.
  struct Pre2 { int64_t crp; int64_t bs; int32_t L; double av; };
  auto load1 = [&](int64_t base) -> Pre1 {
    Pre1 p{{0, 0, 0}, 0};
    const int64_t idx = base + grp;
    if (idx < n) {
      p.d = a.desc[idx];
      if (NUMERIC) p.perm = *reinterpret_cast<const uint64_t*>(a.perm + idx * CAP + l * R);
    }
    return p;
  };
  auto load2 = [&](int64_t base, const Pre1& p1) -> Pre2 {
    Pre2 q{0, 0, 0, 0.0};
    if (base + grp < n) {
      if (NUMERIC) q.crp = a.c_rp[p1.d.row] - cbase;
      if (l < p1.d.na) {
        const uint64_t sg = a.seg[p1.d.as + l];
        q.bs = seg_start(sg);
        q.L = seg_length(sg);
        if (NUMERIC) q.av = a.A.val[p1.d.as + l];
      }
    }
    return q;
  };

  auto process = [&](int64_t base, const Pre1& p1, const Pre2& p2) {
    const int64_t idx = base + grp;
    const bool valid = idx < n;
    const RowDesc d = p1.d;
    const uint64_t perm = p1.perm;
    const int64_t crp = p2.crp;
    // Run row: at most W nonzeros, each selecting a B row of 1..R entries
    // (empty groups past the end count as run rows).
    const bool mine_ok = (l >= d.na) || (p2.L >= 1 && p2.L <= R);
    const unsigned okb = (__ballot_sync(FULL, mine_ok) >> gshift) & gbits;
    const bool run_row = d.na <= W && okb == gbits;
    const bool fast = __all_sync(FULL, run_row);
    int P = 0;
    K key[R];
    if (fast) {
      // Run path.  Lane l of the group publishes its nonzero's B row; the
      // B rows are then read whole by consecutive lanes (W / R runs per
      // load instruction, or half a run when W = 4).
      const int L = (l < d.na) ? p2.L : 0;
      if (l < d.na) {
        s_bs[w][l][grp] = p2.bs;
        s_len[w][l][grp] = (uint8_t)L;
        if (NUMERIC) s_av[w][l][grp] = p2.av;
      }
      P = group_sum<W>(L);
      __syncwarp();
      constexpr int RPI = W >= R ? W / R : 1;  // runs per load instruction
      int32_t cg[R];
      double vg[R];
      bool on[R];
#pragma unroll
      for (int it = 0; it < R; ++it) {
        const int r = (W >= R) ? it * RPI + (l >> 3) : (it >> 1);
        const int x = (W >= R) ? (l & 7) : (l + 4 * (it & 1));
        on[it] = r < d.na && x < (int)s_len[w][r < W ? r : 0][grp];
        cg[it] = 0;
        vg[it] = 0.0;
        if (on[it]) {
          const int64_t k = s_bs[w][r][grp] + x;
          cg[it] = __ldg(a.B.col + k);
          if (NUMERIC) vg[it] = __ldg(a.B.val + k);
        }
      }
#pragma unroll
      for (int it = 0; it < R; ++it) {
        const int r = (W >= R) ? it * RPI + (l >> 3) : (it >> 1);
        const int x = (W >= R) ? (l & 7) : (l + 4 * (it & 1));
        const int slot = r * R + x;
        if (NUMERIC) {
          if (on[it]) {
            s_col[w][slot][grp] = cg[it];
            s_val[w][slot][grp] = s_av[w][r][grp] * vg[it];
          }
        } else {
          s_key[w][grp * RL::KSTRIDE + RL::at(r, x)] =
              on[it] ? KT::template make<SB>(cg[it], slot) : ~K(0);
        }
      }
      __syncwarp();
      if (!NUMERIC) {
        // lane l takes run l: ascending (B rows are sorted, slots increase)
        const K* src = &s_key[w][grp * RL::KSTRIDE + l * R];
        const int sw = (l >> 2) & 1;
        if (sizeof(K) == 4) {
          const uint4 q0 = *reinterpret_cast<const uint4*>(src + 4 * sw);
          const uint4 q1 = *reinterpret_cast<const uint4*>(src + 4 * (sw ^ 1));
          const uint32_t t[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
          for (int e = 0; e < R; ++e) key[e] = (K)t[e];
        } else {
#pragma unroll
          for (int e = 0; e < R; ++e) key[e] = src[4 * ((e >> 2) ^ sw) + (e & 3)];
        }
        group_merge_runs<R, W>(key);
      }
    } else {
      if (l < HW) s_head[w][l][grp] = 0;
      // 1. Segments: the non-empty B rows referenced by the row, in stored
      //    order, each with its first slot in the row's product list.
      int nseg = 0;
      for (int j0 = 0; __any_sync(FULL, j0 < d.na); j0 += W) {
        const int j = j0 + l;
        int64_t bs = 0;
        int L = 0;
        double av = 0.0;
        if (j0 == 0) {
          bs = p2.bs;  // prefetched one iteration ahead
          L = p2.L;
          av = p2.av;
        } else if (j < d.na) {
          const uint64_t sg = a.seg[d.as + j];
          bs = seg_start(sg);
          L = seg_length(sg);
          if (NUMERIC) av = a.A.val[d.as + j];
        }
        const unsigned nz = (__ballot_sync(FULL, L > 0) >> gshift) & gbits;
        const int inc = group_inclusive_scan<W>(L);
        if (L > 0) {
          const int g = nseg + __popc(nz & ((1u << l) - 1u));
          s_off[w][g][grp] = (uint8_t)(P + inc - L);
          s_bs[w][g][grp] = bs;
          if (NUMERIC) s_av[w][g][grp] = av;
        }
        nseg += __popc(nz);
        P += __shfl_sync(FULL, inc, gshift + W - 1);
      }
      __syncwarp();
      for (int g = 1 + l; g < nseg; g += W) {
        const int off = s_off[w][g][grp];
        atomicOr(&s_head[w][off >> 5][grp], 1u << (off & 31));
      }
      __syncwarp();
      uint32_t hw[HW];
      int pw[HW];
      {
        int cum = 0;
#pragma unroll
        for (int i = 0; i < HW; ++i) {
          hw[i] = s_head[w][i][grp];
          pw[i] = cum;
          cum += __popc(hw[i]);
        }
      }
      // 2. Expand: slot s = e*W + l (consecutive lanes read consecutive
      //    entries of a B row).  The segment of s is the number of segment
      //    starts at or before s.  A run row numbers its products run-major
      //    (its segments are its nonzeros: no B row is empty).
      // All gathers of the row are issued before any of them is used, so
      // the R loads of a lane (2R in the numeric pass) are in flight together.
      int32_t cg[R];
      double vg[R];
      double ag[R];
      int sl[R];
#pragma unroll
      for (int e = 0; e < R; ++e) {
        const int s = e * W + l;
        const int wi = (e * W) >> 5;
        const int g = pw[wi] + __popc(hw[wi] & ((2u << (s & 31)) - 1u));
        cg[e] = 0;
        vg[e] = 0.0;
        ag[e] = 0.0;
        sl[e] = s;
        if (s < P) {
          const int x = s - s_off[w][g][grp];
          const int64_t k = s_bs[w][g][grp] + x;
          if (run_row) sl[e] = g * R + x;
          cg[e] = __ldg(a.B.col + k);
          if (NUMERIC) {
            vg[e] = __ldg(a.B.val + k);
            ag[e] = s_av[w][g][grp];
          }
        }
      }
#pragma unroll
      for (int e = 0; e < R; ++e) {
        const int s = e * W + l;
        if (NUMERIC) {
          if (s < P) {
            s_col[w][sl[e]][grp] = cg[e];
            s_val[w][sl[e]][grp] = ag[e] * vg[e];
          }
        } else {
          key[e] = (s < P) ? KT::template make<SB>(cg[e], sl[e]) : ~K(0);
        }
      }
      if (!NUMERIC) group_bitonic_sort<R, W>(key);
    }
    if (!NUMERIC) {
      // 3s. Count distinct columns, record the sorted slot order.
      const K prev_last = __shfl_up_sync(FULL, key[R - 1], 1, W);
      int h = 0;
      uint64_t pb = 0;
#pragma unroll
      for (int e = 0; e < R; ++e) {
        const int q = l * R + e;
        const int32_t c = KT::template col<SB>(key[e]);
        const int32_t pc = (e == 0) ? ((l == 0) ? -1 : KT::template col<SB>(prev_last))
                                    : KT::template col<SB>(key[e - 1]);
        h += ((q < P) && (q == 0 || c != pc)) ? 1 : 0;
        pb |= (uint64_t)(KT::template slot<SB>(key[e]) & 0xff) << (8 * e);
      }
      const int cnt = group_sum<W>(h);
      if (valid) {
        if (l == 0) a.out_cnt[d.row] = cnt;
        // Store the order so that the numeric pass, whose lane l visits
        // sorted positions e*W + l, reads its 8 slots as one 8-byte word:
        // position q goes to byte (q % W) * 8 + q / W.
        uint8_t* dst = a.perm + idx * CAP;
#pragma unroll
        for (int e = 0; e < R; ++e) {
          const int q = l * R + e;
          dst[(q % W) * R + q / W] = (uint8_t)(pb >> (8 * e));
        }
      }
    } else {
      // 3n. Replay the recorded order: lane l visits sorted positions
      //     q = e*W + l, so consecutive lanes write consecutive entries of C.
      int sl[R];
#pragma unroll
      for (int e = 0; e < R; ++e) {
        sl[e] = (int)((perm >> (8 * e)) & 0xff);
        s_perm[w][e * W + l][grp] = (uint8_t)sl[e];
      }
      __syncwarp();
      int run = 0;                 // distinct columns before this e-row
      int32_t last_col = -1;       // column of the position before this e-row
#pragma unroll
      for (int e = 0; e < R; ++e) {
        const int q = e * W + l;
        const bool in = q < P;
        const int32_t c = in ? s_col[w][sl[e]][grp] : 0x7fffffff;
        const int32_t up = __shfl_up_sync(FULL, c, 1, W);
        const int32_t prev = (l == 0) ? last_col : up;
        const bool head = in && (q == 0 || c != prev);
        const unsigned hb = (__ballot_sync(FULL, head) >> gshift) & gbits;
        const int32_t dn = __shfl_down_sync(FULL, c, 1, W);
        if (head) {
          const int o = run + __popc(hb & ((1u << l) - 1u));
          double acc = s_val[w][sl[e]][grp];
          // the next sorted position holds the same column: sum the run in
          // slot order (the recorded order keeps equal columns slot-sorted)
          const bool more = (l < W - 1) ? (dn == c) : (q + 1 < P);
          if (more) {
            for (int q2 = q + 1; q2 < P; ++q2) {
              const int s2 = s_perm[w][q2][grp];
              if (s_col[w][s2][grp] != c) break;
              acc += s_val[w][s2][grp];
            }
          }
          a.c_col[crp + o] = c;
          a.c_val[crp + o] = acc;
        }
        run += __popc(hb);
        last_col = __shfl_sync(FULL, c, gshift + W - 1);
      }
    }
    __syncwarp();
  };

  // Two-stage software pipeline over this warp's groups of rows: while a
  // group is finished, level 2 of the next group and level 1 of the one
  // after it are in flight.  The loop is written as two halves so that each
  // stage keeps its own registers (no copies of values still being loaded).
  int64_t b = first + ((int64_t)blockIdx.x * NW + w) * G;
  Pre1 p1a = load1(b), p1b = load1(b + stride);
  Pre2 p2a = load2(b, p1a), p2b;
  while (b < n) {
    p2b = load2(b + stride, p1b);
    {
      const Pre1 cur = p1a;
      p1a = load1(b + 2 * stride);
      process(b, cur, p2a);
    }
    b += stride;
    if (b >= n) break;
    p2a = load2(b + stride, p1a);
    {
      const Pre1 cur = p1b;
      p1b = load1(b + 2 * stride);
      process(b, cur, p2b);
    }
    b += stride;
  }
}

template <int E, typename K, bool NUMERIC, int NW>
static cudaError_t launch_nw(const SortArgs& a, int num_sms, cudaStream_t s) {
  constexpr int G = 8 / E;
  auto kern = k_sort_rows<E, K, NUMERIC, NW>;
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NW * 32, 0);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (a.n_rows + NW * G - 1) / (NW * G);
  const int64_t cap = (int64_t)num_sms * per_sm;  // one resident wave
  if (blocks > cap) blocks = cap;
  kern<<<(unsigned)blocks, NW * 32, 0, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

// Warps per block: the requested shape, else 4 (numeric) / 8 (symbolic).
template <int E, typename K, bool NUMERIC>
static cudaError_t launch_one(const SortArgs& a, int num_sms, cudaStream_t s) {
  switch (a.block_warps) {
    case 2: return launch_nw<E, K, NUMERIC, 2>(a, num_sms, s);
    case 4: return launch_nw<E, K, NUMERIC, 4>(a, num_sms, s);
    case 8: return launch_nw<E, K, NUMERIC, 8>(a, num_sms, s);
    default: return launch_nw<E, K, NUMERIC, NUMERIC ? 4 : 8>(a, num_sms, s);
  }
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
  if (numeric) return launch_bin<uint32_t, true>(bin, a, num_sms, s);  // no keys in the replay
  if (a.key32) return launch_bin<uint32_t, false>(bin, a, num_sms, s);
  return launch_bin<uint64_t, false>(bin, a, num_sms, s);
}

}  // namespace magnus
