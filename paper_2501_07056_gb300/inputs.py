"""Seeded synthetic workload generators (CSR, FP64 values, int32 columns).

This module only draws random sparse matrices; it contains none of the
SpGEMM arithmetic.  Both the CUDA path and the CPU oracle consume what it
produces, so the two sides always see identical inputs.

Every generator is deterministic given ``(seed, matrix_id)``: it builds a
numpy ``Generator(PCG64(SeedSequence([seed, matrix_id, ...])))``, whose
output is platform independent.

Workloads (the shapes of the paper's test sets, Section 4.2-4.3):
  * ``uniform``   - Erdos-Renyi-like rows: exactly ``k`` distinct columns per
                    row drawn uniformly, values U(lo, hi).
  * ``rmat``      - Graph500 R-MAT power-law matrix (Table 3 generator shape:
                    a=.57, b=c=.19, d=.05, edge factor 16), duplicates merged,
                    values U(0, 1).
  * ``ragged``    - rows with a uniformly drawn number of distinct columns
                    (batched products).
  * ``stencil27`` - 27-point stencil on a k^3 grid, truncated at the boundary
                    (served requests).
  * ``ragged_ctr`` - ragged rows from a counter-based generator (SplitMix64
                    output function); the on-device generator in
                    libmagnus_inputs.so implements the same definition, so
                    matrices drawn on the GPU are reproduced here bit for bit.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "CSR", "rng_for", "uniform", "ragged", "rmat", "stencil27", "identity",
    "permutation", "from_dense", "batched_sizes", "batched_problems", "served_stream",
    "workload", "ctr_key", "ctr_u64", "ragged_ctr", "ragged_ctr_nnz", "stratified",
    "uniform_stream",
]


@dataclasses.dataclass
class CSR:
    """Host CSR matrix: int64 row pointers, int32 columns, float64 values."""
    n_rows: int
    n_cols: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def validate(self) -> None:
        """Raise ValueError unless this is a well-formed CSR with rows that
        hold strictly ascending, in-range column indices."""
        rp, c = self.row_ptr, self.col
        if rp.dtype != np.int64 or c.dtype != np.int32 or self.val.dtype != np.float64:
            raise ValueError("dtypes must be int64/int32/float64")
        if rp.shape != (self.n_rows + 1,) or rp[0] != 0:
            raise ValueError("bad row_ptr shape or start")
        if np.any(np.diff(rp) < 0):
            raise ValueError("row_ptr not nondecreasing")
        if c.shape != (self.nnz,) or self.val.shape != (self.nnz,):
            raise ValueError("col/val length != nnz")
        if self.nnz:
            if c.min() < 0 or c.max() >= self.n_cols:
                raise ValueError("column out of range")
            d = np.diff(c.astype(np.int64))
            starts = np.zeros(self.nnz, dtype=bool)
            starts[rp[:-1][np.diff(rp) > 0]] = True
            if np.any(d[~starts[1:]] <= 0):
                raise ValueError("columns not strictly ascending within a row")

    def to_dense(self) -> np.ndarray:
        out = np.zeros((self.n_rows, self.n_cols), dtype=np.float64)
        rows = np.repeat(np.arange(self.n_rows), np.diff(self.row_ptr))
        out[rows, self.col] = self.val
        return out

    def row(self, i: int):
        s, e = int(self.row_ptr[i]), int(self.row_ptr[i + 1])
        return self.col[s:e], self.val[s:e]


def rng_for(seed: int, matrix_id: int, stream: int = 0) -> np.random.Generator:
    """Deterministic generator keyed by (seed, matrix id, sub-stream)."""
    return np.random.Generator(np.random.PCG64(
        np.random.SeedSequence([int(seed), int(matrix_id), int(stream)])))


def _distinct_sorted_rows(rng, lengths: np.ndarray, n_cols: int) -> np.ndarray:
    """Columns for rows of the given lengths: distinct within each row, drawn
    uniformly from [0, n_cols), ascending within each row.  Collisions are
    redrawn until none remain (rejection sampling keeps the draw uniform over
    distinct sets)."""
    lengths = lengths.astype(np.int64)
    if np.any(lengths > n_cols):
        raise ValueError("row longer than the number of columns")
    n = lengths.shape[0]
    total = int(lengths.sum())
    row_of = np.repeat(np.arange(n, dtype=np.int64), lengths)
    cols = rng.integers(0, n_cols, size=total, dtype=np.int64)
    dense_rows = lengths * 2 > n_cols
    if np.any(dense_rows):
        # Rows that take more than half the columns: draw without replacement.
        starts = np.concatenate(([0], np.cumsum(lengths)))
        for i in np.nonzero(dense_rows)[0]:
            cols[starts[i]:starts[i + 1]] = rng.choice(n_cols, size=lengths[i], replace=False)
    while True:
        key = row_of * n_cols + cols
        order = np.argsort(key, kind="stable")
        key = key[order]
        cols = cols[order]
        dup = np.zeros(total, dtype=bool)
        if total > 1:
            dup[1:] = key[1:] == key[:-1]
        nd = int(dup.sum())
        if nd == 0:
            return cols.astype(np.int32)
        cols[dup] = rng.integers(0, n_cols, size=nd, dtype=np.int64)


def _csr_from_lengths(n_rows, n_cols, lengths, cols, vals) -> CSR:
    rp = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(lengths, out=rp[1:])
    return CSR(n_rows, n_cols, rp, np.ascontiguousarray(cols, dtype=np.int32),
               np.ascontiguousarray(vals, dtype=np.float64))


def uniform(n_rows: int, n_cols: int, k: int, seed: int = 0, matrix_id: int = 0,
            lo: float = -1.0, hi: float = 1.0) -> CSR:
    """Exactly ``k`` distinct uniform-random columns per row, values U(lo, hi)."""
    rng = rng_for(seed, matrix_id)
    lengths = np.full(n_rows, k, dtype=np.int64)
    if k == 0 or n_rows == 0:
        return _csr_from_lengths(n_rows, n_cols, lengths, np.zeros(0, np.int32), np.zeros(0))
    if n_cols >= 64 * k:
        # Fast path: sort a (n_rows, k) block, redraw only rows with a repeat.
        cols = rng.integers(0, n_cols, size=(n_rows, k), dtype=np.int32)
        cols.sort(axis=1)
        while True:
            bad = np.nonzero(np.any(cols[:, 1:] == cols[:, :-1], axis=1))[0]
            if bad.size == 0:
                break
            redraw = rng.integers(0, n_cols, size=(bad.size, k), dtype=np.int32)
            redraw.sort(axis=1)
            cols[bad] = redraw
        cols = cols.reshape(-1)
    else:
        cols = _distinct_sorted_rows(rng, lengths, n_cols)
    vals = rng.uniform(lo, hi, size=n_rows * k)
    return _csr_from_lengths(n_rows, n_cols, lengths, cols, vals)


def ragged(n_rows: int, n_cols: int, kmin: int, kmax: int, seed: int = 0,
           matrix_id: int = 0, lo: float = -1.0, hi: float = 1.0) -> CSR:
    """Rows with a number of distinct columns drawn uniformly from
    {kmin..kmax}; columns uniform, values U(lo, hi)."""
    rng = rng_for(seed, matrix_id)
    lengths = rng.integers(kmin, kmax + 1, size=n_rows, dtype=np.int64)
    lengths = np.minimum(lengths, n_cols)
    cols = _distinct_sorted_rows(rng, lengths, n_cols)
    vals = rng.uniform(lo, hi, size=int(lengths.sum()))
    return _csr_from_lengths(n_rows, n_cols, lengths, cols, vals)


# ---------------------------------------------------------------------------
# counter-based generator (definition in include/magnus_inputs.h)

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z ^ (z >> np.uint64(30))
        z = z * np.uint64(0xBF58476D1CE4E5B9)
        z = z ^ (z >> np.uint64(27))
        z = z * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def ctr_u64(key, i):
    """ctr(key, i) = mix64(key + (i + 1) * golden), arithmetic mod 2^64."""
    i = np.asarray(i, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(np.uint64(key) + (i + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15))


def ctr_key(seed: int, matrix_id: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        a = _mix64(np.uint64(seed) * np.uint64(0x9E3779B97F4A7C15)
                   + np.uint64(0xD1B54A32D192ED03))
        b = np.uint64(matrix_id) * np.uint64(0xA24BAED4963EE407) + np.uint64(stream)
        return np.uint64(_mix64(a ^ b))


def _scale32(x, m: int):
    return ((x >> np.uint64(32)) * np.uint64(m)) >> np.uint64(32)


def _ragged_ctr_lengths(n_rows, n_cols, kmin, kmax, seed, matrix_id):
    kl = ctr_key(seed, matrix_id, 1)
    L = kmin + _scale32(ctr_u64(kl, np.arange(n_rows, dtype=np.uint64)), kmax - kmin + 1)
    return np.minimum(L.astype(np.int64), n_cols)


def ragged_ctr_nnz(n_rows: int, n_cols: int, kmin: int, kmax: int, seed: int = 0,
                   matrix_id: int = 0) -> int:
    return int(_ragged_ctr_lengths(n_rows, n_cols, kmin, kmax, seed, matrix_id).sum())


def ragged_ctr(n_rows: int, n_cols: int, kmin: int, kmax: int, seed: int = 0,
               matrix_id: int = 0, lo: float = -1.0, hi: float = 1.0) -> CSR:
    """Ragged matrix from the counter-based generator: the host twin of
    magnus_gen_ragged_rowptr/_fill (definition in include/magnus_inputs.h)."""
    if not (1 <= kmin <= kmax <= 64) or n_cols < 1:
        raise ValueError("need 1 <= kmin <= kmax <= 64 and n_cols >= 1")
    L = _ragged_ctr_lengths(n_rows, n_cols, kmin, kmax, seed, matrix_id)
    kc = ctr_key(seed, matrix_id, 2)
    kv = ctr_key(seed, matrix_id, 3)
    acc = np.full((n_rows, kmax), -1, dtype=np.int64)
    cnt = np.zeros(n_rows, dtype=np.int64)
    rows_all = np.arange(n_rows, dtype=np.int64)
    for j in range(1024):
        act = rows_all[cnt < L]
        if act.size == 0:
            break
        x = ctr_u64(kc, act.astype(np.uint64) * np.uint64(1024) + np.uint64(j))
        cand = _scale32(x, n_cols).astype(np.int64)
        present = (acc[act] == cand[:, None]).any(axis=1)
        take = act[~present]
        acc[take, cnt[take]] = cand[~present]
        cnt[take] += 1
    for r in rows_all[cnt < L]:  # smallest unused columns complete the row
        v = 0
        while cnt[r] < L[r]:
            if not (acc[r, :cnt[r]] == v).any():
                acc[r, cnt[r]] = v
                cnt[r] += 1
            v += 1
    big = np.int64(1) << np.int64(40)
    acc[np.arange(kmax)[None, :] >= L[:, None]] = big
    acc.sort(axis=1)
    mask = np.arange(kmax)[None, :] < L[:, None]
    cols = acc[mask].astype(np.int32)
    k = np.nonzero(mask)[1].astype(np.uint64)
    r = np.nonzero(mask)[0].astype(np.uint64)
    u = (ctr_u64(kv, r * np.uint64(64) + k) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    vals = lo + (hi - lo) * u
    return _csr_from_lengths(n_rows, n_cols, L, cols, vals)


def stratified(n_rows: int, n_cols: int, k: int, seed: int = 0, matrix_id: int = 0,
               lo: float = -1.0, hi: float = 1.0, rows=None) -> CSR:
    """Exactly k distinct ascending columns per row, one uniform draw in each
    of k equal strata of [0, n_cols): the host twin of magnus_gen_stratified
    (definition in include/magnus_inputs.h).  ``rows`` (optional) lists the
    rows to fill; the others are left empty (for the oracle, which needs only
    the rows of B that sampled rows of A reference)."""
    if not (1 <= k <= n_cols):
        raise ValueError("need 1 <= k <= n_cols")
    rows = np.arange(n_rows, dtype=np.int64) if rows is None else np.unique(np.asarray(rows, np.int64))
    lengths = np.zeros(n_rows, dtype=np.int64)
    lengths[rows] = k
    j = np.arange(k, dtype=np.int64)
    e = (rows[:, None] * k + j[None, :]).astype(np.uint64).reshape(-1)
    s0 = (j * n_cols) // k
    width = ((j + 1) * n_cols) // k - s0
    kc = ctr_key(seed, matrix_id, 4)
    kv = ctr_key(seed, matrix_id, 5)
    x = ctr_u64(kc, e).reshape(len(rows), k) >> np.uint64(32)
    off = (x * width.astype(np.uint64)[None, :]) >> np.uint64(32)
    cols = (s0[None, :] + off.astype(np.int64)).reshape(-1).astype(np.int32)
    u = (ctr_u64(kv, e) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    vals = lo + (hi - lo) * u
    return _csr_from_lengths(n_rows, n_cols, lengths, cols, vals)


def uniform_stream(n: int, m: int, seed: int = 0, stream_id: int = 0, lo: float = -1.0,
                   hi: float = 1.0):
    """(col, val) of a stream of n uniform indices in [0, m): the host twin
    of magnus_gen_uniform_stream (building-block microbenchmark)."""
    i = np.arange(n, dtype=np.uint64)
    col = _scale32(ctr_u64(ctr_key(seed, stream_id, 6), i), m).astype(np.int32)
    u = (ctr_u64(ctr_key(seed, stream_id, 7), i) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return col, lo + (hi - lo) * u


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 0, matrix_id: int = 0) -> CSR:
    """Square R-MAT matrix with 2^scale rows and edge_factor * 2^scale drawn
    edges.  Each edge picks one quadrant per level with probabilities
    (a, b, c, 1-a-b-c); no noise and no vertex permutation, so nonzeros
    cluster at the top left.  Repeated (row, col) pairs are merged, then one
    U(0, 1) value is drawn per distinct entry."""
    rng = rng_for(seed, matrix_id)
    n = 1 << scale
    m = edge_factor * n
    row = np.zeros(m, dtype=np.int64)
    col = np.zeros(m, dtype=np.int64)
    t_ab = a + b
    t_abc = a + b + c
    for level in range(scale):
        u = rng.random(m)
        bit = np.int64(1) << np.int64(scale - 1 - level)
        # quadrant 0: (0,0)  1: (0,1)  2: (1,0)  3: (1,1)
        row_bit = u >= t_ab
        col_bit = ((u >= a) & (u < t_ab)) | (u >= t_abc)
        row += row_bit.astype(np.int64) * bit
        col += col_bit.astype(np.int64) * bit
    key = np.unique(row * n + col)
    rows = key // n
    cols = (key % n).astype(np.int32)
    lengths = np.bincount(rows, minlength=n).astype(np.int64)
    vals = rng.uniform(0.0, 1.0, size=key.shape[0])
    return _csr_from_lengths(n, n, lengths, cols, vals)


def stencil27(k: int) -> CSR:
    """27-point stencil on a k x k x k grid (lexicographic numbering),
    truncated at the boundary: 26 on the diagonal, -1 off it."""
    n = k ** 3
    idx = np.arange(n, dtype=np.int64)
    z, y, x = idx // (k * k), (idx // k) % k, idx % k
    cols_l, rows_l = [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                zz, yy, xx = z + dz, y + dy, x + dx
                ok = (zz >= 0) & (zz < k) & (yy >= 0) & (yy < k) & (xx >= 0) & (xx < k)
                rows_l.append(idx[ok])
                cols_l.append((zz * k * k + yy * k + xx)[ok])
    rows = np.concatenate(rows_l)
    cols = np.concatenate(cols_l)
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    vals = np.where(rows == cols, 26.0, -1.0)
    lengths = np.bincount(rows, minlength=n).astype(np.int64)
    return _csr_from_lengths(n, n, lengths, cols.astype(np.int32), vals)


def identity(n: int) -> CSR:
    return _csr_from_lengths(n, n, np.ones(n, np.int64), np.arange(n, dtype=np.int32),
                             np.ones(n))


def permutation(perm: np.ndarray) -> CSR:
    """Permutation matrix P with P[i, perm[i]] = 1."""
    n = perm.shape[0]
    return _csr_from_lengths(n, n, np.ones(n, np.int64), perm.astype(np.int32), np.ones(n))


def from_dense(d: np.ndarray, pattern: np.ndarray | None = None) -> CSR:
    """CSR holding the entries of ``d`` where ``pattern`` is true (default:
    where d != 0).  Explicit zeros in the pattern are kept."""
    if pattern is None:
        pattern = d != 0
    rows, cols = np.nonzero(pattern)
    lengths = np.bincount(rows, minlength=d.shape[0]).astype(np.int64)
    return _csr_from_lengths(d.shape[0], d.shape[1], lengths, cols.astype(np.int32),
                             d[rows, cols].astype(np.float64))


def batched_sizes(count: int, seed: int = 0, n_lo: int = 256, n_hi: int = 65536) -> np.ndarray:
    """n_i = round(exp(U(ln n_lo, ln n_hi))) for the batched workload."""
    rng = rng_for(seed, 1_000_000)
    return np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count))).astype(np.int64)


def batched_problems(count: int, seed: int = 0, n_lo: int = 256, n_hi: int = 65536,
                     kmin: int = 2, kmax: int = 32):
    """Independent products C_i = A_i B_i: n_i = round(exp(U(ln n_lo, ln n_hi))),
    A_i and B_i square n_i x n_i with per-row nnz uniform in {kmin..kmax},
    values U(-1, 1)."""
    ns = batched_sizes(count, seed, n_lo, n_hi)
    out = []
    for i, n in enumerate(ns):
        A = ragged(int(n), int(n), kmin, kmax, seed, 2 * i + 1)
        B = ragged(int(n), int(n), kmin, kmax, seed, 2 * i + 2)
        out.append((A, B))
    return out


def served_stream(count: int, seed: int = 0, k_lo: int = 16, k_hi: int = 96,
                  b_kmin: int = 4, b_kmax: int = 16):
    """Request descriptors for the served workload: grid size k (uniform in
    {k_lo..k_hi}) and the matrix id of B, plus unit-rate exponential
    inter-arrival gaps (scale them by 1/lambda).  Matrices are built on demand
    with ``stencil27(k)`` and ``ragged(k^3, k^3, b_kmin, b_kmax, seed, id)``."""
    rng = rng_for(seed, 2_000_000)
    ks = rng.integers(k_lo, k_hi + 1, size=count)
    gaps = rng.exponential(1.0, size=count)
    return [dict(req=i, k=int(ks[i]), b_id=3_000_000 + i, gap=float(gaps[i]))
            for i in range(count)]


def workload(name: str, seed: int = 0):
    """(A, B) for a named single-product workload.  B is A for the A^2 cases."""
    if name == "uniform4096":
        A = uniform(4096, 4096, 8, seed, 0)
        return A, A
    if name == "uniform2^22":
        A = uniform(1 << 22, 1 << 22, 8, seed, 0)
        return A, A
    if name == "uniform2^24":
        A = uniform(1 << 24, 1 << 24, 8, seed, 0)
        return A, A
    if name.startswith("rmat"):
        A = rmat(int(name[4:]), 16, seed=seed, matrix_id=0)
        return A, A
    raise KeyError(name)
