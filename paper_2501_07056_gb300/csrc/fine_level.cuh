// Fine-level chunk accumulation shared by fine rows and large coarse chunks
// (Algorithm 3 accumulation step with the hybrid accumulator of Section 3.4).
//
// The staged products of a row (or coarse chunk) are grouped by fine chunk.
// Each chunk is accumulated by one warp, chosen chunk by chunk:
//   * fewer than `dthr` products (at most 256): sort accumulator - the
//     chunk's (column, position) keys are sorted by the warp's bitonic
//     network and runs of equal columns are merged (Algorithm 2); runs of
//     consecutive small chunks are first merged into groups of up to 32
//     products, one warp sort each;
//   * otherwise: dense accumulator - each warp owns a private accumulator of
//     one chunk's columns in shared memory (FP64 values and a bitmap in the
//     numeric phase, the bitmap alone in the symbolic phase).
// Warps take consecutive chunks, a round of FNW chunks at a time, so a round
// needs two block barriers for the prefix of its chunk counts instead of
// barriers per chunk.  Dense emission walks the bitmap in column order and
// resets exactly the entries it touched, as Algorithm 1's output loop resets
// its bitmap, so the accumulators are clean for the next chunk without
// clearing the whole array.
#pragma once

#include "block_accum.cuh"
#include "sort_accum.cuh"

namespace magnus {

constexpr int FNT = DENSE_NT;      // threads per block
constexpr int FNW = FNT / 32;      // warps per block
constexpr int WARP_ACC_LOG2 = 10;  // numeric: 1024 FP64 columns per warp accumulator
constexpr int WARP_BITS_LOG2 = 13; // symbolic: 8192 columns per warp bitmap
constexpr int DIRECT_BITS_LOG2 = 19;  // symbolic: block bitmap for a whole row's range
constexpr int FINE_SORT_MAX = 256;    // largest chunk the warp sort accumulator takes
constexpr int FINE_HASH_LOG2 = 8;     // slots of a warp's hash table (in the sort staging)
constexpr int FINE_HASH_MAX = 128;    // largest chunk the hash accumulator takes (load <= 1/2)

struct FineSmem {
  int32_t* cnt;     // [FINE_MAX_CHUNKS]     chunk histogram, then reorder cursor, then
                    //                       first chunk of each merged group
  int32_t* off;     // [FINE_MAX_CHUNKS + 1] chunk offsets in staging
  double* acc;      // [FNW << shift]        warp accumulators (numeric)
  uint32_t* bits;   // [FNW][words]          warp bitmaps
  int words;        // bitmap words per warp
  uint32_t* direct; // symbolic: block bitmap of a whole row (aliases the above)
  int64_t* wcnt;    // [FNW + 1]             chunk counts of the current round; [FNW]:
                    //                       number of merged chunk groups
  double* svals;    // [FNW][FINE_SORT_MAX]  sort accumulator: values by position (numeric)
  uint32_t* skeys;  // [FNW][FINE_SORT_MAX]  sort accumulator: sorted keys (numeric)
};

__host__ __device__ inline int fine_words(int shift) { return shift >= 5 ? (1 << (shift - 5)) : 1; }

// Shared memory of the fine kernels for a chunk shift (numeric: shift <=
// WARP_ACC_LOG2; symbolic: shift <= WARP_BITS_LOG2).  `hybrid`: a hybrid
// threshold above 1 is in use, so the numeric sort accumulator's per-warp
// staging is reserved as well (dense-only launches do without it).
__host__ __device__ inline size_t fine_smem_bytes(bool numeric, int shift, bool hybrid) {
  size_t b = (size_t)FINE_MAX_CHUNKS * 4 + (size_t)(FINE_MAX_CHUNKS + 1) * 4;
  b = (b + 15) & ~(size_t)15;
  if (numeric) b += (size_t)FNW * ((size_t)1 << shift) * 8;
  b += (size_t)FNW * fine_words(shift) * 4;
  b = (b + 15) & ~(size_t)15;
  if (!numeric) {
    const size_t direct = ((size_t)1 << DIRECT_BITS_LOG2) / 8;
    if (direct > b) b = direct;
  }
  b = (b + 15) & ~(size_t)15;
  b += (FNW + 1) * 8;
  if (numeric && hybrid) b += (size_t)FNW * FINE_SORT_MAX * (8 + 4);
  return b;
}

__device__ inline FineSmem fine_carve(unsigned char* base, bool numeric, int shift, bool hybrid) {
  FineSmem f;
  size_t o = 0;
  f.cnt = reinterpret_cast<int32_t*>(base + o);
  o += (size_t)FINE_MAX_CHUNKS * 4;
  f.off = reinterpret_cast<int32_t*>(base + o);
  o += (size_t)(FINE_MAX_CHUNKS + 1) * 4;
  o = (o + 15) & ~(size_t)15;
  f.acc = reinterpret_cast<double*>(base + o);
  if (numeric) o += (size_t)FNW * ((size_t)1 << shift) * 8;
  f.words = fine_words(shift);
  f.bits = reinterpret_cast<uint32_t*>(base + o);
  o += (size_t)FNW * f.words * 4;
  o = (o + 15) & ~(size_t)15;
  f.direct = reinterpret_cast<uint32_t*>(base);
  if (!numeric) {
    const size_t direct = ((size_t)1 << DIRECT_BITS_LOG2) / 8;
    if (direct > o) o = direct;
  }
  o = (o + 15) & ~(size_t)15;
  f.wcnt = reinterpret_cast<int64_t*>(base + o);
  o += (FNW + 1) * 8;
  f.svals = (numeric && hybrid) ? reinterpret_cast<double*>(base + o) : nullptr;
  if (numeric && hybrid) o += (size_t)FNW * FINE_SORT_MAX * 8;
  f.skeys = (numeric && hybrid) ? reinterpret_cast<uint32_t*>(base + o) : nullptr;
  return f;
}

// Zeroes every warp accumulator and bitmap (once per block; emission keeps
// them clean afterwards).  All threads must call; ends with a barrier.
template <bool NUMERIC>
__device__ inline void fine_clear(const FineSmem& f, int shift) {
  const int cl = 1 << shift;
  if (NUMERIC)
    for (int i = threadIdx.x; i < FNW * cl; i += FNT) f.acc[i] = 0.0;
  for (int i = threadIdx.x; i < FNW * f.words; i += FNT) f.bits[i] = 0u;
  __syncthreads();
}

// Sort accumulator of one group of n <= 32*E products: keys (column from the
// group's first chunk on, position in the staging) sorted by the warp;
// returns the distinct count and leaves the sorted keys in k[0..E).
template <int E>
__device__ __forceinline__ int fine_sort_count(uint32_t (&k)[8], const int32_t* __restrict__ cols,
                                               int n, int32_t sub) {
  constexpr int SB = Log2Cap<E>::v;
  uint32_t kk[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int s = e * 32 + lane_id();
    kk[e] = s < n ? KeyTraits<uint32_t>::template make<SB>(cols[s] - sub, s) : ~0u;
  }
  warp_bitonic_sort<E>(kk);
#pragma unroll
  for (int e = 0; e < E; ++e) k[e] = kk[e];
  return warp_merge_emit<E, uint32_t, false>(kk, n, nullptr, nullptr, 0, nullptr, nullptr);
}

// Hash-map accumulator of one chunk of n <= FINE_HASH_MAX products
// (Section 2.1's extension of Algorithm 1: the dense array and bitmap become
// a hash map).  The warp's table has 2^FINE_HASH_LOG2 slots: keys (column in
// the chunk, EMPTY when free) in hk, FP64 sums in hv; a product claims its
// column's slot by compare-and-swap (multiplicative hash, linear probing)
// and adds its value there.  The occupied slots are then compacted to the
// front of the table (hk[0..d) columns, hv[0..d) sums), so the caller sorts
// the d distinct columns with the sort accumulator's warp network and emits
// them with the sums read by position.  The table is cleared on entry; at
// most half of it fills, so every probe sequence ends within the table.
// Returns d.
constexpr uint32_t HASH_EMPTY = 0xffffffffu;

__device__ __forceinline__ int fine_hash_compact(const int32_t* __restrict__ cols,
                                                 const double* __restrict__ vals, int n,
                                                 int cmask, uint32_t* hk, double* hv) {
  constexpr int HT = 1 << FINE_HASH_LOG2;
  constexpr int PER = HT / 32;  // slots per lane
  static_assert(HT <= FINE_SORT_MAX && HT % 32 == 0, "the table lives in the sort staging");
  const int lane = lane_id();
  for (int i = lane; i < HT; i += 32) {
    hk[i] = HASH_EMPTY;
    hv[i] = 0.0;
  }
  __syncwarp();
  for (int s = lane; s < n; s += 32) {
    const uint32_t c = (uint32_t)(cols[s] & cmask);
    const double v = vals[s];
    uint32_t h = (c * 0x9E3779B1u) >> (32 - FINE_HASH_LOG2);
    for (int probe = 0; probe < HT; ++probe) {
      const uint32_t prev = atomicCAS(&hk[h], HASH_EMPTY, c);
      if (prev == HASH_EMPTY || prev == c) {
        atomicAdd(&hv[h], v);
        break;
      }
      h = (h + 1) & (HT - 1);
    }
  }
  __syncwarp();
  uint32_t kc[PER];
  double vc[PER];
  int occ = 0;
#pragma unroll
  for (int e = 0; e < PER; ++e) {
    kc[e] = hk[lane * PER + e];
    vc[e] = hv[lane * PER + e];
    occ += kc[e] != HASH_EMPTY ? 1 : 0;
  }
  const int inc = warp_inclusive_scan(occ);
  const int d = __shfl_sync(FULL, inc, 31);
  __syncwarp();
  int idx = inc - occ;
#pragma unroll
  for (int e = 0; e < PER; ++e) {
    if (kc[e] != HASH_EMPTY) {
      hk[idx] = kc[e];
      hv[idx] = vc[e];
      ++idx;
    }
  }
  __syncwarp();
  return d;
}

template <int E>
__device__ __forceinline__ void fine_sort_emit(const uint32_t (&k)[8], int n, const double* vals,
                                               uint32_t* skeys, int32_t col_add,
                                               int32_t* __restrict__ out_col,
                                               double* __restrict__ out_val) {
  uint32_t kk[E];
#pragma unroll
  for (int e = 0; e < E; ++e) kk[e] = k[e];
  warp_merge_emit<E, uint32_t, true>(kk, n, vals, skeys, col_add, out_col, out_val);
}

// Chunk merging (Section 4.1.1: sort sizes near 32 are the sort
// accumulator's best): with the hybrid on, consecutive chunks of at most 32
// products (and below dthr) are combined greedily in column order into
// groups of at most 32 products, one key per lane of a warp sort.  Empty
// chunks join the open group.  Writes the first chunk of group g to f.cnt[g]
// (the reorder cursors are dead once the leading barrier has passed) and
// returns the number of groups.  Warp 0 walks the chunks 32 at a time with
// the group state kept identical in all its lanes.  All threads must call.
__device__ inline int fine_merge_groups(const FineSmem& f, int nch, int dthr) {
  __syncthreads();
  if (warp_id() == 0) {
    const int lane = lane_id();
    int ng = 0, cur = 0;
    bool open = false;  // the last group takes more small chunks
    for (int c0 = 0; c0 < nch; c0 += 32) {
      const int ch = c0 + lane;
      const int n = ch < nch ? f.off[ch + 1] - f.off[ch] : 0;
      const unsigned small = __ballot_sync(FULL, ch < nch && n <= 32 && n < dthr);
      const unsigned valid = (nch - c0 >= 32) ? FULL : ((1u << (nch - c0)) - 1u);
      unsigned starts = 0;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int nj = __shfl_sync(FULL, n, j);
        if ((small >> j) & 1u) {
          if (open && cur + nj <= 32) {
            cur += nj;
          } else {
            starts |= 1u << j;
            cur = nj;
            open = true;
          }
        } else {
          starts |= 1u << j;
          open = false;
        }
      }
      starts &= valid;
      if ((starts >> lane) & 1u) f.cnt[ng + __popc(starts & ((1u << lane) - 1u))] = ch;
      ng += __popc(starts);
    }
    if (lane == 0) f.wcnt[FNW] = ng;
  }
  __syncthreads();
  return (int)f.wcnt[FNW];
}

// Accumulates the staged chunks [0, nch): chunk ch holds
// stage_col/stage_val[off[ch] .. off[ch + 1]), columns relative to col_base
// (chunk index << shift | column inside the chunk).  Writes the sorted unique
// entries to out_col/out_val[0..) (numeric) and returns their number.  A
// chunk with fewer than dthr products (dthr <= FINE_SORT_MAX + 1) takes the
// sort accumulator, the others the dense one; with dthr > 1 the small chunks
// are first merged into groups (fine_merge_groups) and each warp takes a
// group.  With `hash` (numeric), the other chunks of at most FINE_HASH_MAX
// products take the hash-map accumulator (fine_hash_compact) and larger
// ones the dense one.  HYBRID = false compiles the dense accumulator alone
// (dthr <= 1, no hash), which keeps the sort and hash paths' registers out
// of the dense-only kernels.  All threads must call; the warp accumulators
// must be clean on entry and are clean on exit.
template <bool NUMERIC, bool HYBRID>
__device__ int64_t warp_chunks_accumulate(const FineSmem& f, int nch, int shift,
                                          const int32_t* __restrict__ stage_col,
                                          const double* __restrict__ stage_val,
                                          int64_t col_base, int32_t* __restrict__ out_col,
                                          double* __restrict__ out_val, int dthr, int hash) {
  const int lane = lane_id(), w = warp_id();
  const int cl = 1 << shift;
  const int words = f.words;
  double* acc = f.acc + (size_t)w * cl;
  uint32_t* bits = f.bits + (size_t)w * words;
  double* svals = NUMERIC ? f.svals + (size_t)w * FINE_SORT_MAX : nullptr;
  uint32_t* skeys = NUMERIC ? f.skeys + (size_t)w * FINE_SORT_MAX : nullptr;
  const int wpl = (words + 31) / 32;  // bitmap words per lane, in column order
  const bool sorting = HYBRID && dthr > 1 && (!NUMERIC || f.svals != nullptr);
  const bool hashing = HYBRID && NUMERIC && hash && f.svals != nullptr;
  const int ngr = sorting ? fine_merge_groups(f, nch, dthr) : nch;
  int64_t outp = 0;
  for (int r0 = 0; r0 < ngr; r0 += FNW) {
    const int g = r0 + w;
    int g0 = g, g1 = g + 1;
    if (sorting && g < ngr) {
      g0 = f.cnt[g];
      g1 = g + 1 < ngr ? f.cnt[g + 1] : nch;
    }
    int cnt = 0, lane_cnt = 0, n = 0, sort_e = 0;
    uint32_t key[8];
    if (g < ngr) {
      const int p0 = f.off[g0], p1 = f.off[g1];
      n = p1 - p0;
      if (n > 0 && sorting && (g1 - g0 > 1 || (n < dthr && n <= FINE_SORT_MAX))) {
        // sort accumulator (warp-uniform branch: n is the same in all lanes);
        // a merged group holds at most 32 products
        if (NUMERIC)
          for (int s = lane; s < n; s += 32) svals[s] = stage_val[p0 + s];
        sort_e = n <= 32 ? 1 : n <= 64 ? 2 : n <= 128 ? 4 : 8;
        const int32_t* cc = stage_col + p0;
        const int32_t sub = g0 << shift;
        if (sort_e == 1) cnt = fine_sort_count<1>(key, cc, n, sub);
        else if (sort_e == 2) cnt = fine_sort_count<2>(key, cc, n, sub);
        else if (sort_e == 4) cnt = fine_sort_count<4>(key, cc, n, sub);
        else cnt = fine_sort_count<8>(key, cc, n, sub);
      } else if (NUMERIC && hashing && n > 0 && n <= FINE_HASH_MAX) {
        // hash-map accumulator, then the d distinct columns (compacted at
        // the front of the table) are sorted and emitted like a sort chunk
        // of d products
        n = fine_hash_compact(stage_col + p0, stage_val + p0, n, cl - 1, skeys, svals);
        sort_e = n <= 32 ? 1 : n <= 64 ? 2 : 4;
        const int32_t* hc = reinterpret_cast<const int32_t*>(skeys);
        if (sort_e == 1) cnt = fine_sort_count<1>(key, hc, n, 0);
        else if (sort_e == 2) cnt = fine_sort_count<2>(key, hc, n, 0);
        else cnt = fine_sort_count<4>(key, hc, n, 0);
      } else if (n > 0) {
        for (int p = p0 + lane; p < p1; p += 32) {
          const int idx = stage_col[p] & (cl - 1);
          atomicOr(&bits[idx >> 5], 1u << (idx & 31));
          if (NUMERIC) atomicAdd(&acc[idx], stage_val[p]);
        }
        __syncwarp();
        for (int k = 0; k < wpl; ++k) {
          const int wd = lane * wpl + k;
          if (wd < words) lane_cnt += __popc(bits[wd]);
        }
        cnt = warp_sum(lane_cnt);
      }
    }
    if (lane == 0) f.wcnt[w] = cnt;
    __syncthreads();
    int64_t before = 0, total = 0;
#pragma unroll
    for (int i = 0; i < FNW; ++i) {
      const int64_t c = f.wcnt[i];
      before += (i < w) ? c : 0;
      total += c;
    }
    if (g < ngr && cnt > 0) {
      const int64_t cb = col_base + ((int64_t)g0 << shift);
      if (sort_e > 0) {
        if (NUMERIC) {
          int32_t* oc = out_col + outp + before;
          double* ov = out_val + outp + before;
          const int32_t add = (int32_t)cb;
          if (sort_e == 1) fine_sort_emit<1>(key, n, svals, skeys, add, oc, ov);
          else if (sort_e == 2) fine_sort_emit<2>(key, n, svals, skeys, add, oc, ov);
          else if (sort_e == 4) fine_sort_emit<4>(key, n, svals, skeys, add, oc, ov);
          else fine_sort_emit<8>(key, n, svals, skeys, add, oc, ov);
        }
      } else if (NUMERIC) {
        const int inc = warp_inclusive_scan(lane_cnt);
        int64_t o = outp + before + inc - lane_cnt;
        for (int k = 0; k < wpl; ++k) {
          const int wd = lane * wpl + k;
          if (wd >= words) break;
          uint32_t m = bits[wd];
          bits[wd] = 0u;
          while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            const int idx = wd * 32 + b;
            out_col[o] = (int32_t)(cb + idx);
            out_val[o] = acc[idx];
            acc[idx] = 0.0;
            ++o;
          }
        }
      } else {
        for (int k = 0; k < wpl; ++k) {
          const int wd = lane * wpl + k;
          if (wd < words) bits[wd] = 0u;
        }
      }
    }
    outp += total;
    __syncthreads();
  }
  return outp;
}

}  // namespace magnus
