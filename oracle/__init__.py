"""CPU oracle for MAGNUS SpGEMM (C = A * B, CSR, FP64).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs import this package.  The
library (``paper_2501_07056_gb300``) never imports it, and it imports
nothing from the library: the only shared module is the seeded input
generator, which holds no SpGEMM arithmetic.

``magnus_oracle.c`` holds the plain definitions (Eq. 1 with Algorithm 1's
accumulation order, precise prediction of Section 2.1, and the chunk
histogram of Algorithms 3/4; ``spgemm_dense`` computes the same C with
Algorithm 1's dense accumulator, bit-identical and linear in the products);
``params.py`` holds the paper's chunk-count model (Eq. 2-7).  ``build()`` compiles the C file with gcc and
``-ffp-contract=off``.
"""
from __future__ import annotations

import concurrent.futures as _fut
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "magnus_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (plain gcc, -O2, no FMA
    contraction, no -march flags so the result is identical on x86 and Arm)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        p = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.oracle_row_products.argtypes = [p, p, p, p, i64, p]
        lib.oracle_row_products.restype = None
        lib.oracle_symbolic.argtypes = [p, p, p, p, p, i64, p]
        lib.oracle_symbolic.restype = ctypes.c_int
        lib.oracle_numeric.argtypes = [p, p, p, p, p, p, p, i64, p, p, p, p]
        lib.oracle_numeric.restype = ctypes.c_int
        lib.oracle_symbolic_dense.argtypes = [p, p, p, p, i64, p, i64, p]
        lib.oracle_symbolic_dense.restype = ctypes.c_int
        lib.oracle_numeric_dense.argtypes = [p, p, p, p, p, p, i64, p, i64, p, p, p, p]
        lib.oracle_numeric_dense.restype = ctypes.c_int
        lib.oracle_chunk_histogram.argtypes = [p, p, p, p, p, i64, ctypes.c_int, i64, p]
        lib.oracle_chunk_histogram.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class Result:
    """Rows of C computed by the oracle: ``row_ptr`` (relative to the listed
    rows), ``col``, ``val`` and ``abs`` (sum of |terms| per entry)."""

    def __init__(self, rows, row_ptr, col, val, abs_):
        self.rows, self.row_ptr, self.col, self.val, self.abs = rows, row_ptr, col, val, abs_

    def row(self, t):
        s, e = int(self.row_ptr[t]), int(self.row_ptr[t + 1])
        return self.col[s:e], self.val[s:e], self.abs[s:e]


def _split(rows, threads):
    if threads <= 1 or rows.shape[0] < 2 * threads:
        return [rows]
    return np.array_split(rows, threads)


def row_products(A, B, rows=None) -> np.ndarray:
    lib = _load()
    rows = _c(np.arange(A.n_rows) if rows is None else rows, np.int64)
    out = np.zeros(rows.shape[0], np.int64)
    lib.oracle_row_products(_ptr(A.row_ptr), _ptr(A.col), _ptr(B.row_ptr), _ptr(rows),
                            rows.shape[0], _ptr(out))
    return out


def symbolic(A, B, rows=None, threads: int = 1) -> np.ndarray:
    """Exact nnz of each listed row of A*B."""
    lib = _load()
    rows = _c(np.arange(A.n_rows) if rows is None else rows, np.int64)
    out = np.zeros(rows.shape[0], np.int64)
    parts = _split(rows, threads)
    outs = np.split(out, np.cumsum([p.shape[0] for p in parts])[:-1])

    def run(k):
        rc = lib.oracle_symbolic(_ptr(A.row_ptr), _ptr(A.col), _ptr(B.row_ptr), _ptr(B.col),
                                 _ptr(parts[k]), parts[k].shape[0], _ptr(outs[k]))
        if rc != 0:
            raise MemoryError("oracle_symbolic")

    _run_all(run, len(parts))
    return out


def _run_all(fn, n):
    if n == 1:
        fn(0)
        return
    with _fut.ThreadPoolExecutor(n) as ex:
        list(ex.map(fn, range(n)))


def spgemm(A, B, rows=None, threads: int = 1) -> Result:
    """Rows of C = A*B (all rows by default) with per-entry |term| sums."""
    lib = _load()
    rows = _c(np.arange(A.n_rows) if rows is None else rows, np.int64)
    cnt = symbolic(A, B, rows, threads)
    rp = np.zeros(rows.shape[0] + 1, np.int64)
    np.cumsum(cnt, out=rp[1:])
    nnz = int(rp[-1])
    col = np.zeros(nnz, np.int32)
    val = np.zeros(nnz, np.float64)
    ab = np.zeros(nnz, np.float64)
    parts = _split(rows, threads)
    starts = np.concatenate(([0], np.cumsum([p.shape[0] for p in parts])))

    def run(k):
        off = _c(rp[starts[k]:starts[k + 1]], np.int64)
        rc = lib.oracle_numeric(_ptr(A.row_ptr), _ptr(A.col), _ptr(A.val), _ptr(B.row_ptr),
                                _ptr(B.col), _ptr(B.val), _ptr(parts[k]), parts[k].shape[0],
                                _ptr(off), _ptr(col), _ptr(val), _ptr(ab))
        if rc != 0:
            raise MemoryError("oracle_numeric")

    _run_all(run, len(parts))
    return Result(rows, rp, col, val, ab)


def _split_by_products(A, B, rows, parts):
    """Contiguous pieces of ``rows`` holding about equal products."""
    if parts <= 1 or rows.shape[0] < 2:
        return [rows]
    P = row_products(A, B, rows)
    cs = np.cumsum(P)
    cuts = np.searchsorted(cs, np.linspace(0, cs[-1], parts + 1)[1:-1], side="right")
    return [r for r in np.split(rows, np.unique(cuts)) if r.shape[0] > 0]


def spgemm_dense(A, B, rows=None, threads: int = 1) -> Result:
    """The same result as ``spgemm`` (bit for bit), computed with Algorithm 1's
    dense accumulator: linear in the products, for the full-size checks of
    power-law matrices whose heavy rows hold millions of products.  Work is
    split into pieces of about equal products."""
    lib = _load()
    rows = _c(np.arange(A.n_rows) if rows is None else rows, np.int64)
    parts = _split_by_products(A, B, rows, 4 * threads)
    cnts = [np.zeros(p.shape[0], np.int64) for p in parts]

    def sym(k):
        rc = lib.oracle_symbolic_dense(_ptr(A.row_ptr), _ptr(A.col), _ptr(B.row_ptr),
                                       _ptr(B.col), B.n_cols, _ptr(parts[k]), parts[k].shape[0],
                                       _ptr(cnts[k]))
        if rc != 0:
            raise MemoryError("oracle_symbolic_dense")

    _run_pool(sym, len(parts), threads)
    cnt = np.concatenate(cnts) if cnts else np.zeros(0, np.int64)
    rp = np.zeros(rows.shape[0] + 1, np.int64)
    np.cumsum(cnt, out=rp[1:])
    nnz = int(rp[-1])
    col = np.zeros(nnz, np.int32)
    val = np.zeros(nnz, np.float64)
    ab = np.zeros(nnz, np.float64)
    starts = np.concatenate(([0], np.cumsum([p.shape[0] for p in parts])))

    def num(k):
        off = _c(rp[starts[k]:starts[k + 1]], np.int64)
        rc = lib.oracle_numeric_dense(_ptr(A.row_ptr), _ptr(A.col), _ptr(A.val), _ptr(B.row_ptr),
                                      _ptr(B.col), _ptr(B.val), B.n_cols, _ptr(parts[k]),
                                      parts[k].shape[0], _ptr(off), _ptr(col), _ptr(val),
                                      _ptr(ab))
        if rc != 0:
            raise MemoryError("oracle_numeric_dense")

    _run_pool(num, len(parts), threads)
    return Result(rows, rp, col, val, ab)


def _run_pool(fn, n, threads):
    if n == 1 or threads <= 1:
        for k in range(n):
            fn(k)
        return
    with _fut.ThreadPoolExecutor(min(threads, n)) as ex:
        list(ex.map(fn, range(n)))


def numeric_into(A, B, rows, off, col, val, ab=None) -> None:
    """Low-level numeric call into caller buffers (used for timing)."""
    lib = _load()
    rc = lib.oracle_numeric(_ptr(A.row_ptr), _ptr(A.col), _ptr(A.val), _ptr(B.row_ptr),
                            _ptr(B.col), _ptr(B.val), _ptr(rows), rows.shape[0], _ptr(off),
                            _ptr(col), _ptr(val), _ptr(ab) if ab is not None else None)
    if rc != 0:
        raise MemoryError("oracle_numeric")


def chunk_histogram(A, B, rows, shift: int, n_chunks: int) -> np.ndarray:
    """counts[t, h] = products of row rows[t] with (col >> shift) == h."""
    lib = _load()
    rows = _c(rows, np.int64)
    out = np.zeros((rows.shape[0], n_chunks), np.int64)
    rc = lib.oracle_chunk_histogram(_ptr(A.row_ptr), _ptr(A.col), _ptr(B.row_ptr), _ptr(B.col),
                                    _ptr(rows), rows.shape[0], int(shift), int(n_chunks),
                                    _ptr(out))
    if rc != 0:
        raise ValueError("column beyond the last chunk")
    return out
