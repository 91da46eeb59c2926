"""The oracle pins must catch plausible mistakes.  Each case plants one bug in
a copy of the oracle source (built on the CPU into a temporary directory) and
checks that the dense-product / identity / order pins reject it."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_2501_07056_gb300 import inputs
from tests._util import random_pattern_csr

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "magnus_oracle.c")

MUTANTS = {
    # wrong B row: the position inside row i of A instead of its column index
    "wrong_b_row": ("int32_t r = a_col[j];", "int32_t r = (int32_t)(j - a_rp[i]);"),
    "dropped_term": ("for (int64_t k = b_rp[r]; k < b_rp[r + 1]; ++k) {",
                     "for (int64_t k = b_rp[r]; k + 1 < b_rp[r + 1]; ++k) {"),
    "wrong_sign": ("acc += buf[q].prod;", "acc -= buf[q].prod;"),
    "reverse_order": ("if (a->slot != b->slot) return a->slot < b->slot ? -1 : 1;",
                      "if (a->slot != b->slot) return a->slot > b->slot ? -1 : 1;"),
    "wrong_value_index": ("buf[m].prod = a_val[j] * b_val[k];",
                          "buf[m].prod = a_val[j] * b_val[b_rp[r]];"),
}


# the same kinds of mistake in the dense-accumulator form (Algorithm 1)
DENSE_MUTANTS = {
    "dense_wrong_b_row": ("      int32_t r = a_col[j];\n      for (int64_t k = b_rp[r]; k < b_rp[r + 1]; ++k) {\n        int32_t c = b_col[k];",
                          "      int32_t r = (int32_t)(j - a_rp[i]);\n      for (int64_t k = b_rp[r]; k < b_rp[r + 1]; ++k) {\n        int32_t c = b_col[k];"),
    "dense_dropped_term": ("        acc[c] += prod;", "        if (k + 1 < b_rp[r + 1]) acc[c] += prod;"),
    "dense_wrong_sign": ("        acc[c] += prod;", "        acc[c] -= prod;"),
    "dense_reverse_order": ("    for (int64_t j = a_rp[i]; j < a_rp[i + 1]; ++j) {\n      int32_t r = a_col[j];\n      for (int64_t k = b_rp[r]; k < b_rp[r + 1]; ++k) {\n        int32_t c = b_col[k];",
                            "    for (int64_t j = a_rp[i + 1] - 1; j >= a_rp[i]; --j) {\n      int32_t r = a_col[j];\n      for (int64_t k = b_rp[r]; k < b_rp[r + 1]; ++k) {\n        int32_t c = b_col[k];"),
    "dense_wrong_value_index": ("        double prod = a_val[j] * b_val[k];",
                                "        double prod = a_val[j] * b_val[b_rp[r]];"),
    "dense_stale_accumulator": ("      acc[c] = 0.0;\n      sabs[c] = 0.0;", "      sabs[c] = 0.0;"),
}


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert old in src, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new, 1))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                           str(path), "-lm"])
    lib = ctypes.CDLL(str(so))
    p, i64 = ctypes.c_void_p, ctypes.c_int64
    lib.oracle_symbolic.argtypes = [p, p, p, p, p, i64, p]
    lib.oracle_numeric.argtypes = [p, p, p, p, p, p, p, i64, p, p, p, p]
    lib.oracle_symbolic_dense.argtypes = [p, p, p, p, i64, p, i64, p]
    lib.oracle_numeric_dense.argtypes = [p, p, p, p, p, p, i64, p, i64, p, p, p, p]
    return lib


def _run(lib, A, B, dense=False):
    P = lambda a: ctypes.c_void_p(a.ctypes.data)
    rows = np.arange(A.n_rows, dtype=np.int64)
    cnt = np.zeros(A.n_rows, np.int64)
    if dense:
        lib.oracle_symbolic_dense(P(A.row_ptr), P(A.col), P(B.row_ptr), P(B.col), B.n_cols,
                                  P(rows), A.n_rows, P(cnt))
    else:
        lib.oracle_symbolic(P(A.row_ptr), P(A.col), P(B.row_ptr), P(B.col), P(rows), A.n_rows,
                            P(cnt))
    rp = np.concatenate(([0], np.cumsum(cnt))).astype(np.int64)
    col = np.zeros(max(1, rp[-1]), np.int32)
    val = np.zeros(max(1, rp[-1]))
    ab = np.zeros(max(1, rp[-1]))
    if dense:
        lib.oracle_numeric_dense(P(A.row_ptr), P(A.col), P(A.val), P(B.row_ptr), P(B.col),
                                 P(B.val), B.n_cols, P(rows), A.n_rows, P(rp[:-1].copy()),
                                 P(col), P(val), P(ab))
    else:
        lib.oracle_numeric(P(A.row_ptr), P(A.col), P(A.val), P(B.row_ptr), P(B.col), P(B.val),
                           P(rows), A.n_rows, P(rp[:-1].copy()), P(col), P(val), P(ab))
    out = np.zeros((A.n_rows, B.n_cols))
    for i in range(A.n_rows):
        out[i, col[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]]
    return out


def _pins_pass(lib, dense=False):
    rng = np.random.default_rng(0)
    for _ in range(6):
        n, k, m = rng.integers(2, 12, size=3)
        A = random_pattern_csr(rng, n, k, 0.5)
        B = random_pattern_csr(rng, k, m, 0.5)
        d = A.to_dense() @ B.to_dense()
        if not np.allclose(_run(lib, A, B, dense), d, rtol=1e-12, atol=1e-15):
            return False
    A = inputs.CSR(1, 3, np.array([0, 3]), np.array([0, 1, 2], np.int32),
                   np.array([1.0, 1e16, -1e16]))
    B = inputs.CSR(3, 1, np.array([0, 1, 2, 3]), np.array([0, 0, 0], np.int32), np.ones(3))
    return _run(lib, A, B, dense)[0, 0] == 0.0


def test_unmutated_copy_passes(tmp_path):
    assert _pins_pass(_build(tmp_path, "same", "acc += buf[q].prod;", "acc += buf[q].prod;"))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    assert not _pins_pass(_build(tmp_path, name, old, new))


def test_unmutated_dense_form_passes(tmp_path):
    assert _pins_pass(_build(tmp_path, "same_dense", "acc[c] += prod;", "acc[c] += prod;"),
                      dense=True)


@pytest.mark.parametrize("name", sorted(DENSE_MUTANTS))
def test_dense_mutant_is_caught(tmp_path, name):
    old, new = DENSE_MUTANTS[name]
    assert not _pins_pass(_build(tmp_path, name, old, new), dense=True)
