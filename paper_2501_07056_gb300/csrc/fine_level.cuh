// Fine-level chunk accumulation shared by fine rows and large coarse chunks
// (Algorithm 3 accumulation step with the Section 3.4 dense accumulator).
//
// The staged products of a row (or coarse chunk) are grouped by fine chunk;
// each warp of the block owns a private dense accumulator of one chunk's
// columns in shared memory (FP64 values and a bitmap in the numeric phase,
// the bitmap alone in the symbolic phase).  Warps take consecutive chunks, a
// round of FNW chunks at a time, so a round needs two block barriers for the
// prefix of its chunk counts instead of barriers per chunk.  Emission walks
// the bitmap in column order and resets exactly the entries it touched, as
// Algorithm 1's output loop resets its bitmap, so the accumulators are clean
// for the next chunk without clearing the whole array.
#pragma once

#include "block_accum.cuh"

namespace magnus {

constexpr int FNT = DENSE_NT;      // threads per block
constexpr int FNW = FNT / 32;      // warps per block
constexpr int WARP_ACC_LOG2 = 10;  // numeric: 1024 FP64 columns per warp accumulator
constexpr int WARP_BITS_LOG2 = 13; // symbolic: 8192 columns per warp bitmap
constexpr int DIRECT_BITS_LOG2 = 19;  // symbolic: block bitmap for a whole row's range

struct FineSmem {
  int32_t* cnt;     // [FINE_MAX_CHUNKS]     chunk histogram, then reorder cursor
  int32_t* off;     // [FINE_MAX_CHUNKS + 1] chunk offsets in staging
  double* acc;      // [FNW << shift]        warp accumulators (numeric)
  uint32_t* bits;   // [FNW][words]          warp bitmaps
  int words;        // bitmap words per warp
  uint32_t* direct; // symbolic: block bitmap of a whole row (aliases the above)
  int64_t* wcnt;    // [FNW + 1]             chunk counts of the current round
};

__host__ __device__ inline int fine_words(int shift) { return shift >= 5 ? (1 << (shift - 5)) : 1; }

// Shared memory of the fine kernels for a chunk shift (numeric: shift <=
// WARP_ACC_LOG2; symbolic: shift <= WARP_BITS_LOG2).
__host__ __device__ inline size_t fine_smem_bytes(bool numeric, int shift) {
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
  return b;
}

__device__ inline FineSmem fine_carve(unsigned char* base, bool numeric, int shift) {
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

// Accumulates the staged chunks [0, nch): chunk ch holds
// stage_col/stage_val[off[ch] .. off[ch + 1]), columns relative to col_base
// (chunk index << shift | column inside the chunk).  Writes the sorted unique
// entries to out_col/out_val[0..) (numeric) and returns their number.  All
// threads must call; the warp accumulators must be clean on entry and are
// clean on exit.
template <bool NUMERIC>
__device__ int64_t warp_chunks_accumulate(const FineSmem& f, int nch, int shift,
                                          const int32_t* __restrict__ stage_col,
                                          const double* __restrict__ stage_val,
                                          int64_t col_base, int32_t* __restrict__ out_col,
                                          double* __restrict__ out_val) {
  const int lane = lane_id(), w = warp_id();
  const int cl = 1 << shift;
  const int words = f.words;
  double* acc = f.acc + (size_t)w * cl;
  uint32_t* bits = f.bits + (size_t)w * words;
  const int wpl = (words + 31) / 32;  // bitmap words per lane, in column order
  int64_t outp = 0;
  for (int r0 = 0; r0 < nch; r0 += FNW) {
    const int ch = r0 + w;
    int cnt = 0;
    if (ch < nch) {
      const int p0 = f.off[ch], p1 = f.off[ch + 1];
      for (int p = p0 + lane; p < p1; p += 32) {
        const int idx = stage_col[p] & (cl - 1);
        atomicOr(&bits[idx >> 5], 1u << (idx & 31));
        if (NUMERIC) atomicAdd(&acc[idx], stage_val[p]);
      }
      __syncwarp();
      for (int k = 0; k < wpl; ++k) {
        const int wd = lane * wpl + k;
        if (wd < words) cnt += __popc(bits[wd]);
      }
    }
    const int lane_cnt = cnt;
    cnt = warp_sum(cnt);
    if (lane == 0) f.wcnt[w] = cnt;
    __syncthreads();
    int64_t before = 0, total = 0;
#pragma unroll
    for (int i = 0; i < FNW; ++i) {
      const int64_t c = f.wcnt[i];
      before += (i < w) ? c : 0;
      total += c;
    }
    if (ch < nch && cnt > 0) {
      if (NUMERIC) {
        const int inc = warp_inclusive_scan(lane_cnt);
        int64_t o = outp + before + inc - lane_cnt;
        const int64_t cb = col_base + ((int64_t)ch << shift);
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
