/*
 * CPU oracle for C = A * B in CSR (FP64 values, int32 columns, int64 row
 * pointers).  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * benchmark's CPU-baseline leg call it; the library never does.  It shares no
 * code, header or constant with the CUDA path.
 *
 * Everything here is the plain definition, written for obviousness rather
 * than speed:
 *
 *   - Row product count (Section 5, definition of n_interProd):
 *       P_i = sum over j in S(A_i) of nnz(B_j).
 *   - Numeric result (Eq. 1, Gustavson's row formulation, with the
 *     accumulation semantics of Algorithm 1): for every row i, visit the
 *     nonzeros of A_i in stored order and, for each, the nonzeros of row
 *     B_{A.col[j]} in stored order; the product A.val[j] * B.val[k] is added
 *     into an accumulator for column B.col[k] that starts at 0.0.  Each
 *     structurally touched column is an entry of C even if its sum is zero
 *     (precise prediction counts structure, Section 2.1).  Entries are
 *     emitted in ascending column order.
 *   - Symbolic result (Section 2.1, precise prediction): the number of
 *     distinct columns touched in each row.
 *   - Chunk histogram (Algorithm 3 / Algorithm 4 histogram step): the number
 *     of products of row i whose column falls in chunk (col >> shift).
 *   - The symbolic and numeric results once more with Algorithm 1's dense
 *     accumulator (oracle_*_dense, at the end of this file): the same sums in
 *     the same order, bit-identical to the sort formulation, but linear in
 *     the products, for the full-size checks of power-law matrices.
 *
 * The products of one row are materialised as (col, slot, value) triples and
 * sorted by (col, slot): this is the expand-sort-compress formulation of
 * Algorithm 2, and because the slot is the traversal position, the sum over a
 * column runs in exactly the traversal order that Algorithm 1 uses.
 * Compile with -ffp-contract=off so a product and its sum are rounded
 * separately (no fused multiply-add).
 *
 * Besides the value, the numeric routine returns for every entry the sum of
 * |A.val[j] * B.val[k]| over its terms, which bounds the rounding error of
 * any summation order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t col;
  int64_t slot;
  double prod;
} oracle_term;

static int cmp_term(const void* x, const void* y) {
  const oracle_term* a = (const oracle_term*)x;
  const oracle_term* b = (const oracle_term*)y;
  if (a->col != b->col) return a->col < b->col ? -1 : 1;
  if (a->slot != b->slot) return a->slot < b->slot ? -1 : 1;
  return 0;
}

static int cmp_i32(const void* x, const void* y) {
  int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
  return (a > b) - (a < b);
}

/* P_i for each listed row (Section 5: n_interProd summed per row). */
void oracle_row_products(const int64_t* a_rp, const int32_t* a_col, const int64_t* b_rp,
                         const int64_t* rows, int64_t n_list, int64_t* out) {
  for (int64_t t = 0; t < n_list; ++t) {
    int64_t i = rows[t], p = 0;
    for (int64_t j = a_rp[i]; j < a_rp[i + 1]; ++j) p += b_rp[a_col[j] + 1] - b_rp[a_col[j]];
    out[t] = p;
  }
}

/* Exact nnz of each listed row of C (precise prediction, Section 2.1):
 * the number of distinct B.col values reached from the row.
 * Returns 0, or -1 if memory could not be allocated. */
int oracle_symbolic(const int64_t* a_rp, const int32_t* a_col, const int64_t* b_rp,
                    const int32_t* b_col, const int64_t* rows, int64_t n_list, int64_t* cnt) {
  int32_t* buf = NULL;
  int64_t cap = 0;
  for (int64_t t = 0; t < n_list; ++t) {
    int64_t i = rows[t], n = 0;
    for (int64_t j = a_rp[i]; j < a_rp[i + 1]; ++j) n += b_rp[a_col[j] + 1] - b_rp[a_col[j]];
    if (n > cap) {
      free(buf);
      cap = n;
      buf = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
      if (!buf) return -1;
    }
    int64_t m = 0;
    for (int64_t j = a_rp[i]; j < a_rp[i + 1]; ++j)
      for (int64_t k = b_rp[a_col[j]]; k < b_rp[a_col[j] + 1]; ++k) buf[m++] = b_col[k];
    qsort(buf, (size_t)m, sizeof(int32_t), cmp_i32);
    int64_t u = 0;
    for (int64_t q = 0; q < m; ++q)
      if (q == 0 || buf[q] != buf[q - 1]) ++u;
    cnt[t] = u;
  }
  free(buf);
  return 0;
}

/* Numeric rows.  Row rows[t] is written at c_col/c_val/c_abs + off[t]; the
 * caller sizes the output with oracle_symbolic.  c_abs may be NULL.
 * Returns 0, or -1 if memory could not be allocated. */
int oracle_numeric(const int64_t* a_rp, const int32_t* a_col, const double* a_val,
                   const int64_t* b_rp, const int32_t* b_col, const double* b_val,
                   const int64_t* rows, int64_t n_list, const int64_t* off,
                   int32_t* c_col, double* c_val, double* c_abs) {
  oracle_term* buf = NULL;
  int64_t cap = 0;
  for (int64_t t = 0; t < n_list; ++t) {
    int64_t i = rows[t], n = 0;
    for (int64_t j = a_rp[i]; j < a_rp[i + 1]; ++j) n += b_rp[a_col[j] + 1] - b_rp[a_col[j]];
    if (n > cap) {
      free(buf);
      cap = n;
      buf = (oracle_term*)malloc((size_t)cap * sizeof(oracle_term));
      if (!buf) return -1;
    }
    int64_t m = 0;
    for (int64_t j = a_rp[i]; j < a_rp[i + 1]; ++j) {
      int32_t r = a_col[j];
      for (int64_t k = b_rp[r]; k < b_rp[r + 1]; ++k) {
        buf[m].col = b_col[k];
        buf[m].slot = m;
        buf[m].prod = a_val[j] * b_val[k];
        ++m;
      }
    }
    qsort(buf, (size_t)m, sizeof(oracle_term), cmp_term);
    int64_t w = off[t];
    int64_t q = 0;
    while (q < m) {
      int32_t c = buf[q].col;
      double acc = 0.0, s = 0.0;
      while (q < m && buf[q].col == c) {
        acc += buf[q].prod;
        s += fabs(buf[q].prod);
        ++q;
      }
      c_col[w] = c;
      c_val[w] = acc;
      if (c_abs) c_abs[w] = s;
      ++w;
    }
  }
  free(buf);
  return 0;
}

/* Chunk histogram of each listed row's intermediate product:
 * counts[t * n_chunks + h] = number of products of row rows[t] whose column
 * satisfies (col >> shift) == h.  Columns with (col >> shift) >= n_chunks are
 * an error (returns -1). */
int oracle_chunk_histogram(const int64_t* a_rp, const int32_t* a_col, const int64_t* b_rp,
                           const int32_t* b_col, const int64_t* rows, int64_t n_list,
                           int shift, int64_t n_chunks, int64_t* counts) {
  memset(counts, 0, (size_t)(n_list * n_chunks) * sizeof(int64_t));
  for (int64_t t = 0; t < n_list; ++t) {
    int64_t i = rows[t];
    for (int64_t j = a_rp[i]; j < a_rp[i + 1]; ++j)
      for (int64_t k = b_rp[a_col[j]]; k < b_rp[a_col[j] + 1]; ++k) {
        int64_t h = (int64_t)((uint32_t)b_col[k] >> shift);
        if (h >= n_chunks) return -1;
        counts[t * n_chunks + h] += 1;
      }
  }
  return 0;
}

/* The symbolic and numeric results again, by Algorithm 1 itself: one dense
 * accumulator over all n_cols columns of C (value, sum of |terms|, touched
 * flag).  Terms are added in traversal order (nonzeros of A_i in stored
 * order, then the stored order of each B row), so every entry is the same
 * sequence of additions into 0.0 as in the sort formulation above and the
 * results are bit-identical to it; a row costs O(P_i + nnz_i log nnz_i)
 * instead of O(P_i log P_i), which is what the heavy rows of a power-law
 * matrix need.  The touched columns are listed as they are first reached and
 * sorted before emission; the accumulator is cleared entry by entry after
 * each row.  Returns 0, or -1 if memory could not be allocated. */
int oracle_symbolic_dense(const int64_t* a_rp, const int32_t* a_col, const int64_t* b_rp,
                          const int32_t* b_col, int64_t n_cols, const int64_t* rows,
                          int64_t n_list, int64_t* cnt) {
  unsigned char* seen = (unsigned char*)calloc((size_t)(n_cols > 0 ? n_cols : 1), 1);
  int32_t* touched = (int32_t*)malloc((size_t)(n_cols > 0 ? n_cols : 1) * sizeof(int32_t));
  if (!seen || !touched) {
    free(seen);
    free(touched);
    return -1;
  }
  for (int64_t t = 0; t < n_list; ++t) {
    int64_t i = rows[t], u = 0;
    for (int64_t j = a_rp[i]; j < a_rp[i + 1]; ++j)
      for (int64_t k = b_rp[a_col[j]]; k < b_rp[a_col[j] + 1]; ++k)
        if (!seen[b_col[k]]) {
          seen[b_col[k]] = 1;
          touched[u++] = b_col[k];
        }
    for (int64_t q = 0; q < u; ++q) seen[touched[q]] = 0;
    cnt[t] = u;
  }
  free(seen);
  free(touched);
  return 0;
}

int oracle_numeric_dense(const int64_t* a_rp, const int32_t* a_col, const double* a_val,
                         const int64_t* b_rp, const int32_t* b_col, const double* b_val,
                         int64_t n_cols, const int64_t* rows, int64_t n_list, const int64_t* off,
                         int32_t* c_col, double* c_val, double* c_abs) {
  const size_t nc = (size_t)(n_cols > 0 ? n_cols : 1);
  double* acc = (double*)calloc(nc, sizeof(double));
  double* sabs = (double*)calloc(nc, sizeof(double));
  unsigned char* seen = (unsigned char*)calloc(nc, 1);
  int32_t* touched = (int32_t*)malloc(nc * sizeof(int32_t));
  if (!acc || !sabs || !seen || !touched) {
    free(acc);
    free(sabs);
    free(seen);
    free(touched);
    return -1;
  }
  for (int64_t t = 0; t < n_list; ++t) {
    int64_t i = rows[t], u = 0;
    for (int64_t j = a_rp[i]; j < a_rp[i + 1]; ++j) {
      int32_t r = a_col[j];
      for (int64_t k = b_rp[r]; k < b_rp[r + 1]; ++k) {
        int32_t c = b_col[k];
        double prod = a_val[j] * b_val[k];
        if (!seen[c]) {
          seen[c] = 1;
          touched[u++] = c;
        }
        acc[c] += prod;
        sabs[c] += fabs(prod);
      }
    }
    qsort(touched, (size_t)u, sizeof(int32_t), cmp_i32);
    int64_t w = off[t];
    for (int64_t q = 0; q < u; ++q) {
      int32_t c = touched[q];
      c_col[w] = c;
      c_val[w] = acc[c];
      if (c_abs) c_abs[w] = sabs[c];
      ++w;
      acc[c] = 0.0;
      sabs[c] = 0.0;
      seen[c] = 0;
    }
  }
  free(acc);
  free(sabs);
  free(seen);
  free(touched);
  return 0;
}
