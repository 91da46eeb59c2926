/*
 * magnus_inputs.h - on-device generators of the synthetic benchmark inputs.
 *
 * These functions only draw sparse matrices; they contain none of the
 * SpGEMM arithmetic and live in their own library (libmagnus_inputs.so).
 * Every matrix is a pure function of (seed, matrix_id) through a
 * counter-based generator, so a host implementation of the same definition
 * (paper_2501_07056_gb300/inputs.py: ragged_ctr, stencil27) reproduces it bit
 * for bit and the CPU oracle can check any product built from it.
 *
 * Counter-based generator (SplitMix64 output function, Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014):
 *   mix64(z)       = z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
 *                    z ^= z >> 27; z *= 0x94D049BB133111EB; z ^ (z >> 31)
 *   ctr(key, i)    = mix64(key + (i + 1) * 0x9E3779B97F4A7C15)
 *   key(s, id, t)  = mix64(mix64(s * 0x9E3779B97F4A7C15 + 0xD1B54A32D192ED03)
 *                          ^ (id * 0xA24BAED4963EE407 + t))
 * (all arithmetic modulo 2^64).
 *
 * Ragged matrix (the batched and served workloads' random operands): row r
 * has L_r = kmin + floor(hi32(ctr(key(s,id,1), r)) * (kmax-kmin+1) / 2^32)
 * distinct columns (at most n_cols).  Candidates are drawn in order
 * j = 0, 1, ... < 1024 as floor(hi32(ctr(key(s,id,2), r*1024 + j)) * n_cols
 * / 2^32); a candidate already taken is skipped.  Should 1024 draws not fill
 * the row, the smallest unused columns complete it.  The row is sorted
 * ascending; its k-th entry gets the value
 * lo + (hi - lo) * (ctr(key(s,id,3), r*64 + k) >> 11) * 2^-53,
 * rounded as one product and one sum (no fused multiply-add).
 * Requires 1 <= kmin <= kmax <= 64.
 *
 * Stratified matrix (the massive nonsquare uniform workload, rows of hundreds
 * or thousands of entries): every row has exactly k entries; entry j lies in
 * the stratum [floor(j*n_cols/k), floor((j+1)*n_cols/k)) at offset
 * floor(hi32(ctr(key(s,id,4), r*k + j)) * width / 2^32), so the columns are
 * distinct, ascending and spread uniformly; its value is
 * lo + (hi - lo) * (ctr(key(s,id,5), r*k + j) >> 11) * 2^-53 (one product,
 * one sum).  Requires 1 <= k <= n_cols.
 *
 * Uniform stream (the building-block microbenchmark): element i has index
 * floor(hi32(ctr(key(s,id,6), i)) * m / 2^32) and value
 * lo + (hi - lo) * (ctr(key(s,id,7), i) >> 11) * 2^-53.
 *
 * 27-point stencil on a k x k x k grid, lexicographic numbering, truncated at
 * the boundary: 26 on the diagonal and -1 at every in-range neighbour;
 * nnz = (3k - 2)^3.
 *
 * Status codes are those of magnus.h (0 = OK, 1 = invalid argument,
 * 5 = CUDA error).  All pointers are device pointers owned by the caller;
 * every call is stream-ordered on `stream` and does not synchronise unless
 * stated.
 */
#ifndef MAGNUS_INPUTS_H
#define MAGNUS_INPUTS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Row pointers of the ragged matrix: row_ptr[0..n_rows] (device, n_rows+1
 * int64).  If nnz_out is non-NULL the call synchronises `stream` and stores
 * row_ptr[n_rows] there. */
int magnus_gen_ragged_rowptr(int64_t n_rows, int64_t n_cols, int32_t kmin, int32_t kmax,
                             uint64_t seed, uint64_t matrix_id, int64_t* row_ptr,
                             int64_t* nnz_out, void* stream);

/* Columns and values of the ragged matrix into col/val (device, nnz
 * entries), given the row pointers from magnus_gen_ragged_rowptr. */
int magnus_gen_ragged_fill(int64_t n_rows, int64_t n_cols, int32_t kmin, int32_t kmax,
                           uint64_t seed, uint64_t matrix_id, double lo, double hi,
                           const int64_t* row_ptr, int32_t* col, double* val, void* stream);

/* The stratified matrix: row_ptr (n_rows + 1, = r * k), col and val
 * (n_rows * k entries each). */
int magnus_gen_stratified(int64_t n_rows, int64_t n_cols, int32_t k, uint64_t seed,
                          uint64_t matrix_id, double lo, double hi, int64_t* row_ptr,
                          int32_t* col, double* val, void* stream);

/* The uniform stream: col and val (n entries each), 1 <= m <= 2^31. */
int magnus_gen_uniform_stream(int64_t n, int64_t m, uint64_t seed, uint64_t stream_id, double lo,
                              double hi, int32_t* col, double* val, void* stream);

/* The 27-point stencil on a k^3 grid: row_ptr (k^3 + 1), col and val
 * ((3k-2)^3 each).  1 <= k <= 1290. */
int magnus_gen_stencil27(int32_t k, int64_t* row_ptr, int32_t* col, double* val, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MAGNUS_INPUTS_H */
