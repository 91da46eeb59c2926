// On-device generators of the synthetic benchmark inputs (ragged, stratified
// and stencil matrices, uniform index streams).  Input generation only: no SpGEMM
// arithmetic here, and nothing here is shared with the SpGEMM library.  The
// definitions are stated in magnus_inputs.h; inputs.py holds the host twin.
#include <cuda_runtime.h>
#include <stdint.h>

#include "magnus_inputs.h"

namespace {

constexpr int KMAX = 64;
constexpr int DRAWS = 1024;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t ctr(uint64_t key, uint64_t i) {
  return mix64(key + (i + 1) * 0x9E3779B97F4A7C15ull);
}

uint64_t gen_key(uint64_t seed, uint64_t id, uint64_t t) {
  return mix64(mix64(seed * 0x9E3779B97F4A7C15ull + 0xD1B54A32D192ED03ull) ^
               (id * 0xA24BAED4963EE407ull + t));
}

__device__ __forceinline__ int64_t scale32(uint64_t x, int64_t m) {
  return (int64_t)(((x >> 32) * (uint64_t)m) >> 32);
}

__global__ void k_ragged_len(int64_t n, int64_t n_cols, int kmin, int span, uint64_t kl,
                             int64_t* __restrict__ len) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    int64_t L = kmin + scale32(ctr(kl, (uint64_t)r), span);
    len[r + 1] = L < n_cols ? L : n_cols;
  }
}

__global__ void k_ragged_fill(int64_t n, int64_t n_cols, uint64_t kc, uint64_t kv, double lo,
                              double hi, const int64_t* __restrict__ rp, int32_t* __restrict__ col,
                              double* __restrict__ val) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = rp[r];
    const int L = (int)(rp[r + 1] - s);
    int32_t c[KMAX];
    int got = 0;
    for (int j = 0; j < DRAWS && got < L; ++j) {
      const int32_t cand = (int32_t)scale32(ctr(kc, (uint64_t)r * DRAWS + j), n_cols);
      bool dup = false;
      for (int q = 0; q < got; ++q) dup |= c[q] == cand;
      if (!dup) c[got++] = cand;
    }
    for (int32_t v = 0; got < L; ++v) {  // smallest unused columns
      bool dup = false;
      for (int q = 0; q < got; ++q) dup |= c[q] == v;
      if (!dup) c[got++] = v;
    }
    for (int i = 1; i < L; ++i) {  // insertion sort
      const int32_t x = c[i];
      int q = i - 1;
      while (q >= 0 && c[q] > x) {
        c[q + 1] = c[q];
        --q;
      }
      c[q + 1] = x;
    }
    const double w = hi - lo;
    for (int k = 0; k < L; ++k) {
      col[s + k] = c[k];
      const double u = (double)(ctr(kv, (uint64_t)r * 64 + k) >> 11) * 0x1.0p-53;
      val[s + k] = __dadd_rn(lo, __dmul_rn(w, u));
    }
  }
}

__global__ void k_stratified(int64_t n, int64_t n_cols, int k, uint64_t kc, uint64_t kv,
                             double lo, double hi, int64_t* __restrict__ rp,
                             int32_t* __restrict__ col, double* __restrict__ val) {
  const int64_t total = n * k;
  const double w = hi - lo;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / k, j = e - r * k;
    const int64_t s0 = j * n_cols / k, s1 = (j + 1) * n_cols / k;
    col[e] = (int32_t)(s0 + scale32(ctr(kc, (uint64_t)e), s1 - s0));
    const double u = (double)(ctr(kv, (uint64_t)e) >> 11) * 0x1.0p-53;
    val[e] = __dadd_rn(lo, __dmul_rn(w, u));
    if (j == 0) rp[r] = e;
    if (e == total - 1) rp[n] = total;
  }
}

__global__ void k_uniform_stream(int64_t n, int64_t m, uint64_t kc, uint64_t kv, double lo,
                                 double hi, int32_t* __restrict__ col, double* __restrict__ val) {
  const double w = hi - lo;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    col[i] = (int32_t)scale32(ctr(kc, (uint64_t)i), m);
    const double u = (double)(ctr(kv, (uint64_t)i) >> 11) * 0x1.0p-53;
    val[i] = __dadd_rn(lo, __dmul_rn(w, u));
  }
}

__global__ void k_stencil_len(int k, int64_t* __restrict__ len) {
  const int64_t n = (int64_t)k * k * k;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t z = r / ((int64_t)k * k), y = (r / k) % k, x = r % k;
    auto d = [k](int64_t v) { return (int64_t)1 + (v > 0) + (v < k - 1); };
    len[r + 1] = d(z) * d(y) * d(x);
  }
}

__global__ void k_stencil_fill(int k, const int64_t* __restrict__ rp, int32_t* __restrict__ col,
                               double* __restrict__ val) {
  const int64_t n = (int64_t)k * k * k;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t z = r / ((int64_t)k * k), y = (r / k) % k, x = r % k;
    int64_t o = rp[r];
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int64_t zz = z + dz, yy = y + dy, xx = x + dx;
          if (zz < 0 || zz >= k || yy < 0 || yy >= k || xx < 0 || xx >= k) continue;
          const int64_t c = (zz * k + yy) * k + xx;
          col[o] = (int32_t)c;
          val[o] = c == r ? 26.0 : -1.0;
          ++o;
        }
  }
}

// In-place inclusive scan of a[1..n] (a[0] is set to 0): per-block sums,
// a sequential pass over the block sums, then the block offsets are added.
constexpr int SCAN_NT = 1024;

__global__ void k_scan_block(int64_t* __restrict__ a, int64_t n, int64_t* __restrict__ sums) {
  __shared__ int64_t sh[SCAN_NT];
  const int64_t i = (int64_t)blockIdx.x * SCAN_NT + threadIdx.x + 1;
  int64_t v = i <= n ? a[i] : 0;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < SCAN_NT; off <<= 1) {
    const int64_t t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  if (i <= n) a[i] = sh[threadIdx.x];
  if (threadIdx.x == SCAN_NT - 1) sums[blockIdx.x] = sh[SCAN_NT - 1];
  if (blockIdx.x == 0 && threadIdx.x == 0) a[0] = 0;
}

__global__ void k_scan_sums(int64_t* __restrict__ sums, int64_t nb) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int64_t run = 0;
    for (int64_t b = 0; b < nb; ++b) {
      const int64_t v = sums[b];
      sums[b] = run;
      run += v;
    }
  }
}

__global__ void k_scan_add(int64_t* __restrict__ a, int64_t n, const int64_t* __restrict__ sums) {
  const int64_t i = (int64_t)blockIdx.x * SCAN_NT + threadIdx.x + 1;
  if (i <= n) a[i] += sums[blockIdx.x];
}

int scan_lengths(int64_t* a, int64_t n, cudaStream_t s) {
  const int64_t nb = (n + SCAN_NT - 1) / SCAN_NT;
  if (nb == 0) return cudaMemsetAsync(a, 0, sizeof(int64_t), s) == cudaSuccess ? 0 : 5;
  int64_t* sums = nullptr;
  if (cudaMallocAsync(&sums, (size_t)nb * sizeof(int64_t), s) != cudaSuccess) return 5;
  k_scan_block<<<(unsigned)nb, SCAN_NT, 0, s>>>(a, n, sums);
  k_scan_sums<<<1, 32, 0, s>>>(sums, nb);
  k_scan_add<<<(unsigned)nb, SCAN_NT, 0, s>>>(a, n, sums);
  cudaFreeAsync(sums, s);
  return cudaGetLastError() == cudaSuccess ? 0 : 5;
}

unsigned grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 65535) b = 65535;
  return (unsigned)b;
}

}  // namespace

extern "C" {

int magnus_gen_ragged_rowptr(int64_t n_rows, int64_t n_cols, int32_t kmin, int32_t kmax,
                             uint64_t seed, uint64_t matrix_id, int64_t* row_ptr,
                             int64_t* nnz_out, void* stream) {
  if (n_rows < 0 || n_cols < 1 || n_cols >= ((int64_t)1 << 31) || !row_ptr || kmin < 1 ||
      kmax < kmin || kmax > KMAX)
    return 1;
  cudaStream_t s = (cudaStream_t)stream;
  if (n_rows > 0)
    k_ragged_len<<<grid_for(n_rows), 256, 0, s>>>(n_rows, n_cols, kmin, kmax - kmin + 1,
                                                  gen_key(seed, matrix_id, 1), row_ptr);
  if (cudaGetLastError() != cudaSuccess) return 5;
  int st = scan_lengths(row_ptr, n_rows, s);
  if (st != 0) return st;
  if (nnz_out) {
    if (cudaMemcpyAsync(nnz_out, row_ptr + n_rows, sizeof(int64_t), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return 5;
  }
  return 0;
}

int magnus_gen_ragged_fill(int64_t n_rows, int64_t n_cols, int32_t kmin, int32_t kmax,
                           uint64_t seed, uint64_t matrix_id, double lo, double hi,
                           const int64_t* row_ptr, int32_t* col, double* val, void* stream) {
  if (n_rows < 0 || n_cols < 1 || n_cols >= ((int64_t)1 << 31) || !row_ptr || kmin < 1 ||
      kmax < kmin || kmax > KMAX)
    return 1;
  if (n_rows == 0) return 0;
  if (!col || !val) return 1;
  cudaStream_t s = (cudaStream_t)stream;
  k_ragged_fill<<<grid_for(n_rows), 256, 0, s>>>(n_rows, n_cols, gen_key(seed, matrix_id, 2),
                                                 gen_key(seed, matrix_id, 3), lo, hi, row_ptr,
                                                 col, val);
  return cudaGetLastError() == cudaSuccess ? 0 : 5;
}

int magnus_gen_stratified(int64_t n_rows, int64_t n_cols, int32_t k, uint64_t seed,
                          uint64_t matrix_id, double lo, double hi, int64_t* row_ptr,
                          int32_t* col, double* val, void* stream) {
  if (n_rows < 0 || n_cols < 1 || n_cols >= ((int64_t)1 << 31) || k < 1 || k > n_cols ||
      !row_ptr || (n_rows > 0 && (!col || !val)))
    return 1;
  cudaStream_t s = (cudaStream_t)stream;
  if (n_rows == 0) return cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), s) == cudaSuccess ? 0 : 5;
  int64_t blocks = (n_rows * k + 255) / 256;
  if (blocks > 65535 * 8) blocks = 65535 * 8;
  k_stratified<<<(unsigned)blocks, 256, 0, s>>>(n_rows, n_cols, k, gen_key(seed, matrix_id, 4),
                                               gen_key(seed, matrix_id, 5), lo, hi, row_ptr, col,
                                               val);
  return cudaGetLastError() == cudaSuccess ? 0 : 5;
}

int magnus_gen_uniform_stream(int64_t n, int64_t m, uint64_t seed, uint64_t stream_id, double lo,
                              double hi, int32_t* col, double* val, void* stream) {
  if (n < 0 || m < 1 || m > ((int64_t)1 << 31) || (n > 0 && (!col || !val))) return 1;
  if (n == 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 65535 * 8) blocks = 65535 * 8;
  k_uniform_stream<<<(unsigned)blocks, 256, 0, s>>>(n, m, gen_key(seed, stream_id, 6),
                                                   gen_key(seed, stream_id, 7), lo, hi, col, val);
  return cudaGetLastError() == cudaSuccess ? 0 : 5;
}

int magnus_gen_stencil27(int32_t k, int64_t* row_ptr, int32_t* col, double* val, void* stream) {
  if (k < 1 || k > 1290 || !row_ptr || !col || !val) return 1;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = (int64_t)k * k * k;
  k_stencil_len<<<grid_for(n), 256, 0, s>>>(k, row_ptr);
  if (cudaGetLastError() != cudaSuccess) return 5;
  int st = scan_lengths(row_ptr, n, s);
  if (st != 0) return st;
  k_stencil_fill<<<grid_for(n), 256, 0, s>>>(k, row_ptr, col, val);
  return cudaGetLastError() == cudaSuccess ? 0 : 5;
}

}  // extern "C"
