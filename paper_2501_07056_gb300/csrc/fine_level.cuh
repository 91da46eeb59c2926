// Fine-level chunk accumulation shared by fine rows and coarse chunks
// (Algorithm 3 accumulation step with the Section 3.4 hybrid).
#pragma once

#include "block_accum.cuh"

namespace magnus {

constexpr int FNT = DENSE_NT;

struct FineSmem {
  int32_t* cnt;
  int32_t* off;
  double* acc;
  uint32_t* bits;
  uint64_t* keys;
  double* vals;
};

__host__ __device__ inline size_t fine_smem_bytes(bool numeric, int shift, int max_chunks) {
  const size_t cl = (size_t)1 << shift;
  size_t b = (size_t)max_chunks * 4 + (size_t)(max_chunks + 1) * 4;
  b = (b + 15) & ~(size_t)15;
  if (numeric) b += cl * 8;
  b += ((cl + 31) / 32) * 4;
  b = (b + 15) & ~(size_t)15;
  b += (size_t)GROUP_SORT_CAP * 8;
  if (numeric) b += (size_t)GROUP_SORT_CAP * 8;
  return b;
}

__device__ inline FineSmem fine_carve(unsigned char* base, bool numeric, int shift, int max_chunks) {
  FineSmem f;
  const size_t cl = (size_t)1 << shift;
  size_t o = 0;
  f.cnt = reinterpret_cast<int32_t*>(base + o);
  o += (size_t)max_chunks * 4;
  f.off = reinterpret_cast<int32_t*>(base + o);
  o += (size_t)(max_chunks + 1) * 4;
  o = (o + 15) & ~(size_t)15;
  f.acc = reinterpret_cast<double*>(base + o);
  if (numeric) o += cl * 8;
  f.bits = reinterpret_cast<uint32_t*>(base + o);
  o += ((cl + 31) / 32) * 4;
  o = (o + 15) & ~(size_t)15;
  f.keys = reinterpret_cast<uint64_t*>(base + o);
  o += (size_t)GROUP_SORT_CAP * 8;
  f.vals = reinterpret_cast<double*>(base + o);
  return f;
}

// Accumulates the staged chunks [0, nch) of one row (or one coarse chunk).
// stage_col/stage_val point at the row's staging region; off[] are the chunk
// offsets inside it.  Columns in staging are relative to col_base.  Writes
// sorted unique entries at out_col/out_val[0..) (numeric) and returns the
// number of distinct columns.  All threads must call.
template <bool NUMERIC>
__device__ int64_t fine_accumulate_chunks(const FineSmem& f, int nch, int shift, int dthr,
                                          const int32_t* __restrict__ stage_col,
                                          const double* __restrict__ stage_val, int64_t col_base,
                                          int32_t* __restrict__ out_col,
                                          double* __restrict__ out_val, int64_t* ws) {
  const int cl = 1 << shift;
  const int cl_words = (cl + 31) >> 5;
  // a chunk below the threshold must fit one sort group
  if (dthr > GROUP_SORT_CAP) dthr = GROUP_SORT_CAP;
  if (dthr < 1) dthr = 1;
  int64_t outp = 0;
  int ch = 0;
  while (ch < nch) {
    const int n = f.off[ch + 1] - f.off[ch];
    if (n == 0) {
      ++ch;
      continue;
    }
    if (n >= dthr) {
      // dense accumulator over the chunk's 2^shift columns (Algorithm 1)
      for (int i = threadIdx.x; i < cl_words; i += FNT) f.bits[i] = 0u;
      if (NUMERIC)
        for (int i = threadIdx.x; i < cl; i += FNT) f.acc[i] = 0.0;
      __syncthreads();
      const int p0 = f.off[ch], p1 = f.off[ch + 1];
      for (int p = p0 + threadIdx.x; p < p1; p += FNT) {
        const int idx = stage_col[p] & (cl - 1);
        atomicOr(&f.bits[idx >> 5], 1u << (idx & 31));
        if (NUMERIC) atomicAdd(&f.acc[idx], stage_val[p]);
      }
      __syncthreads();
      const int64_t cb = col_base + ((int64_t)ch << shift);
      outp += block_emit_bitmap<FNT, NUMERIC>(f.bits, cl_words, f.acc, cb,
                                             out_col, out_val, outp, ws);
      __syncthreads();  // emission reads acc/bits before the next chunk clears them
      ++ch;
    } else {
      // merge consecutive small chunks and sort them together (Algorithm 2)
      int g = ch;
      int tot = 0;
      while (g < nch) {
        const int m = f.off[g + 1] - f.off[g];
        if (m >= dthr || tot + m > GROUP_SORT_CAP) break;
        tot += m;
        ++g;
      }
      int np2 = 1;
      while (np2 < tot) np2 <<= 1;
      const int p0 = f.off[ch];
      const int32_t rel0 = ch << shift;
      for (int i = threadIdx.x; i < np2; i += FNT) {
        if (i < tot) {
          const int32_t rel = stage_col[p0 + i] - rel0;
          f.keys[i] = ((uint64_t)(uint32_t)rel << 32) | (uint32_t)i;
          if (NUMERIC) f.vals[i] = stage_val[p0 + i];
        } else {
          f.keys[i] = ~0ull;
        }
      }
      __syncthreads();
      block_bitonic_sort<FNT>(f.keys, np2);
      // compress: each thread takes IPT consecutive sorted keys
      constexpr int IPT = GROUP_SORT_CAP / FNT;
      int h = 0;
      bool head[IPT];
#pragma unroll
      for (int r = 0; r < IPT; ++r) {
        const int i = threadIdx.x * IPT + r;
        head[r] = (i < tot) && (i == 0 || (f.keys[i] >> 32) != (f.keys[i - 1] >> 32));
        h += head[r] ? 1 : 0;
      }
      int64_t gtot;
      int64_t pos = block_exclusive_scan<FNT>((int64_t)h, ws, &gtot);
      if (NUMERIC) {
        const int64_t cb = col_base + rel0;
#pragma unroll
        for (int r = 0; r < IPT; ++r) {
          if (!head[r]) continue;
          const int i = threadIdx.x * IPT + r;
          const uint32_t c = (uint32_t)(f.keys[i] >> 32);
          double acc = f.vals[(uint32_t)f.keys[i]];
          for (int i2 = i + 1; i2 < tot && (uint32_t)(f.keys[i2] >> 32) == c; ++i2)
            acc += f.vals[(uint32_t)f.keys[i2]];
          out_col[outp + pos] = (int32_t)(cb + c);
          out_val[outp + pos] = acc;
          ++pos;
        }
      }
      outp += gtot;
      __syncthreads();
      ch = g;
    }
  }
  return outp;
}

}  // namespace magnus
