"""Pins for the CPU oracle against facts fixed by mathematics, not by the
oracle itself: dense matrix products, identities, permutations, the transpose
rule, brute-force column unions, row-sum invariants and the summation order
of Algorithm 1."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2501_07056_gb300 import inputs
from tests._util import random_pattern_csr, transpose, values_close

pytestmark = pytest.mark.filterwarnings("ignore")


def _dense_of(res, n_cols):
    out = np.zeros((res.rows.shape[0], n_cols))
    pat = np.zeros((res.rows.shape[0], n_cols), dtype=bool)
    for t in range(res.rows.shape[0]):
        c, v, _ = res.row(t)
        out[t, c] = v
        pat[t, c] = True
    return out, pat


def _check_against_dense(A, B):
    res = oracle.spgemm(A, B)
    dense = A.to_dense() @ B.to_dense()
    # Structural product: entry (i, c) exists iff some j has A_ij and B_jc
    # stored (integer matmul of the 0/1 patterns).
    pa = np.zeros((A.n_rows, A.n_cols), np.int64)
    pa[np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr)), A.col] = 1
    pb = np.zeros((B.n_rows, B.n_cols), np.int64)
    pb[np.repeat(np.arange(B.n_rows), np.diff(B.row_ptr)), B.col] = 1
    struct = (pa @ pb) > 0
    got, pat = _dense_of(res, B.n_cols)
    assert np.array_equal(pat, struct)
    abs_dense = np.abs(A.to_dense()) @ np.abs(B.to_dense())
    assert np.all(values_close(got, dense, abs_dense, rtol=1e-13))
    # The returned |term| sums are the absolute product.
    absg = np.zeros_like(got)
    for t in range(A.n_rows):
        c, _, s = res.row(t)
        absg[t, c] = s
    assert np.allclose(absg, abs_dense, rtol=1e-14, atol=0)
    for t in range(A.n_rows):
        c, _, _ = res.row(t)
        assert np.all(np.diff(c) > 0)


@pytest.mark.parametrize("seed", range(12))
def test_dense_matmul_small(seed):
    rng = np.random.default_rng(seed)
    n, k, m = rng.integers(1, 17, size=3)
    A = random_pattern_csr(rng, n, k, rng.uniform(0.05, 0.9))
    B = random_pattern_csr(rng, k, m, rng.uniform(0.05, 0.9))
    _check_against_dense(A, B)


def test_all_patterns_2x2():
    rng = np.random.default_rng(7)
    pats = [np.array(p, dtype=bool).reshape(2, 2) for p in itertools.product([0, 1], repeat=4)]
    for pa, pb in itertools.product(pats, pats):
        A = inputs.from_dense(np.where(pa, rng.uniform(-1, 1, (2, 2)), 0.0), pa)
        B = inputs.from_dense(np.where(pb, rng.uniform(-1, 1, (2, 2)), 0.0), pb)
        _check_against_dense(A, B)


def test_random_patterns_3x3():
    rng = np.random.default_rng(11)
    for _ in range(300):
        pa = rng.random((3, 3)) < 0.5
        pb = rng.random((3, 3)) < 0.5
        A = inputs.from_dense(np.where(pa, rng.uniform(-1, 1, (3, 3)), 0.0), pa)
        B = inputs.from_dense(np.where(pb, rng.uniform(-1, 1, (3, 3)), 0.0), pb)
        _check_against_dense(A, B)


def _assert_same_csr(res, M):
    assert np.array_equal(res.row_ptr, M.row_ptr)
    assert np.array_equal(res.col, M.col)
    assert np.array_equal(res.val.view(np.int64), M.val.view(np.int64))


def test_identity_products_bit_exact():
    A = inputs.uniform(300, 300, 9, seed=3, matrix_id=5)
    I = inputs.identity(300)
    _assert_same_csr(oracle.spgemm(A, I), A)
    _assert_same_csr(oracle.spgemm(I, A), A)


def test_permutation_products_bit_exact():
    rng = np.random.default_rng(5)
    A = inputs.ragged(257, 257, 0, 20, seed=1, matrix_id=2)
    perm = rng.permutation(257)
    P = inputs.permutation(perm)
    # (P A)_i = A_{perm[i]}
    res = oracle.spgemm(P, A)
    for i in range(257):
        c, v, _ = res.row(i)
        c0, v0 = A.row(perm[i])
        assert np.array_equal(c, c0) and np.array_equal(v.view(np.int64), v0.view(np.int64))
    # (A P)_{i, perm[j]} = A_{i, j}  (P^T maps column j to perm[j])
    PT = transpose(P)
    res = oracle.spgemm(A, P)
    for i in range(257):
        c, v, _ = res.row(i)
        c0, v0 = A.row(i)
        order = np.argsort(perm[c0])
        assert np.array_equal(c, perm[c0][order])
        assert np.array_equal(v.view(np.int64), v0[order].view(np.int64))
    assert PT.nnz == 257


def test_transpose_rule():
    A = inputs.ragged(120, 90, 0, 12, seed=4, matrix_id=1)
    B = inputs.ragged(90, 150, 0, 12, seed=4, matrix_id=2)
    AB = oracle.spgemm(A, B)
    BtAt = oracle.spgemm(transpose(B), transpose(A))
    ABc = inputs.CSR(120, 150, AB.row_ptr, AB.col, AB.val)
    T = transpose(ABc)
    assert np.array_equal(T.row_ptr, BtAt.row_ptr)
    assert np.array_equal(T.col, BtAt.col)
    # values: same terms, maybe a different order
    abs_t = transpose(inputs.CSR(120, 150, AB.row_ptr, AB.col, AB.abs)).val
    assert np.all(values_close(BtAt.val, T.val, abs_t))


def test_symbolic_equals_column_union():
    A = inputs.ragged(200, 500, 0, 15, seed=9, matrix_id=1)
    B = inputs.ragged(500, 400, 0, 15, seed=9, matrix_id=2)
    cnt = oracle.symbolic(A, B)
    for i in range(A.n_rows):
        ca, _ = A.row(i)
        u = set()
        for j in ca:
            u.update(B.row(j)[0].tolist())
        assert cnt[i] == len(u)


def test_row_sums_invariant():
    A = inputs.uniform(2000, 2000, 8, seed=0, matrix_id=0)
    res = oracle.spgemm(A, A)
    ones = np.ones(2000)
    b1 = np.add.reduceat(A.val, A.row_ptr[:-1]) * (np.diff(A.row_ptr) > 0)
    rows = np.repeat(np.arange(2000), np.diff(A.row_ptr))
    a_b1 = np.zeros(2000)
    np.add.at(a_b1, rows, A.val * b1[A.col])
    abs_b1 = np.zeros(2000)
    absb = np.add.reduceat(np.abs(A.val), A.row_ptr[:-1])
    np.add.at(abs_b1, rows, np.abs(A.val) * absb[A.col])
    c1 = np.add.reduceat(res.val, res.row_ptr[:-1]) * (np.diff(res.row_ptr) > 0)
    assert np.all(np.abs(c1 - a_b1) <= 1e-12 * abs_b1)
    assert ones.shape == (2000,)


def test_row_products_two_ways():
    A = inputs.ragged(1000, 800, 0, 30, seed=2, matrix_id=3)
    B = inputs.ragged(800, 700, 0, 30, seed=2, matrix_id=4)
    p = oracle.row_products(A, B)
    lens = np.diff(B.row_ptr)
    assert int(p.sum()) == int(lens[A.col].sum())
    assert p[17] == sum(int(lens[j]) for j in A.row(17)[0])


def test_chunk_histogram_matches_expansion():
    A = inputs.ragged(50, 1 << 12, 0, 20, seed=6, matrix_id=1)
    B = inputs.ragged(1 << 12, 1 << 12, 0, 20, seed=6, matrix_id=2)
    rows = np.arange(50)
    h = oracle.chunk_histogram(A, B, rows, 8, 16)
    p = oracle.row_products(A, B, rows)
    assert np.array_equal(h.sum(axis=1), p)
    for i in (0, 13, 49):
        cols = np.concatenate([B.row(j)[0] for j in A.row(i)[0]] + [np.zeros(0, np.int32)])
        assert np.array_equal(h[i], np.bincount(cols >> 8, minlength=16))


def test_accumulation_order_is_traversal_order():
    # Row 0 of A has three entries whose B rows all hit column 0 with
    # products 1, 1e16, -1e16 in traversal order.  In that order the sum is
    # (1 + 1e16) - 1e16 = 0 in binary64 (1e16 + 1 rounds to 1e16); the
    # reverse order gives (-1e16 + 1e16) + 1 = 1.
    A = inputs.CSR(1, 3, np.array([0, 3]), np.array([0, 1, 2], np.int32),
                   np.array([1.0, 1e16, -1e16]))
    B = inputs.CSR(3, 1, np.array([0, 1, 2, 3]), np.array([0, 0, 0], np.int32),
                   np.array([1.0, 1.0, 1.0]))
    res = oracle.spgemm(A, B)
    assert res.col.tolist() == [0] and res.val[0] == 0.0
    assert res.abs[0] == 2e16 + 1.0 or res.abs[0] == 2e16


def test_structural_zero_kept():
    A = inputs.CSR(1, 2, np.array([0, 2]), np.array([0, 1], np.int32), np.array([1.0, -1.0]))
    B = inputs.CSR(2, 3, np.array([0, 1, 2]), np.array([2, 2], np.int32), np.array([1.0, 1.0]))
    res = oracle.spgemm(A, B)
    assert res.col.tolist() == [2] and res.val.tolist() == [0.0]
    assert oracle.symbolic(A, B).tolist() == [1]


def test_empty_cases():
    E = inputs.CSR(0, 5, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    B = inputs.uniform(5, 7, 2, seed=1)
    res = oracle.spgemm(E, B)
    assert res.row_ptr.tolist() == [0] and res.col.size == 0
    Z = inputs.CSR(4, 5, np.zeros(5, np.int64), np.zeros(0, np.int32), np.zeros(0))
    assert oracle.spgemm(Z, B).row_ptr.tolist() == [0] * 5
    Bz = inputs.CSR(5, 7, np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0))
    A = inputs.uniform(4, 5, 3, seed=2)
    assert oracle.symbolic(A, Bz).tolist() == [0] * 4


def test_threads_do_not_change_results():
    A = inputs.uniform(3000, 3000, 8, seed=0)
    r1 = oracle.spgemm(A, A, threads=1)
    r4 = oracle.spgemm(A, A, threads=4)
    assert np.array_equal(r1.row_ptr, r4.row_ptr)
    assert np.array_equal(r1.col, r4.col)
    assert np.array_equal(r1.val.view(np.int64), r4.val.view(np.int64))


def test_uniform4096_nnz_band():
    # Each row of A*A for 8 distinct uniform columns per row in n=4096 has 64
    # products over 4096 columns: expected distinct count 4096(1-(1-1/4096)^64).
    A, B = inputs.workload("uniform4096")
    cnt = oracle.symbolic(A, B)
    expect = 4096 * (1 - (1 - 1 / 4096) ** 64)
    assert abs(cnt.mean() - expect) < 0.05
    assert cnt.max() <= 64


# ---- the dense-accumulator form (Algorithm 1), used by the full-size checks


@pytest.mark.parametrize("seed", range(6))
def test_dense_form_against_dense_matmul(seed):
    rng = np.random.default_rng(100 + seed)
    n, k, m = rng.integers(1, 17, size=3)
    A = random_pattern_csr(rng, n, k, rng.uniform(0.05, 0.9))
    B = random_pattern_csr(rng, k, m, rng.uniform(0.05, 0.9))
    res = oracle.spgemm_dense(A, B)
    got, pat = _dense_of(res, B.n_cols)
    pa = (A.to_dense() != 0) | _pattern(A)
    pb = _pattern(B)
    assert np.array_equal(pat, (pa.astype(np.int64) @ pb.astype(np.int64)) > 0)
    abs_dense = np.abs(A.to_dense()) @ np.abs(B.to_dense())
    assert np.all(values_close(got, A.to_dense() @ B.to_dense(), abs_dense, rtol=1e-13))


def _pattern(M):
    p = np.zeros((M.n_rows, M.n_cols), dtype=bool)
    p[np.repeat(np.arange(M.n_rows), np.diff(M.row_ptr)), M.col] = True
    return p


def test_dense_form_order_and_zeros():
    A = inputs.CSR(1, 3, np.array([0, 3]), np.array([0, 1, 2], np.int32),
                   np.array([1.0, 1e16, -1e16]))
    B = inputs.CSR(3, 1, np.array([0, 1, 2, 3]), np.array([0, 0, 0], np.int32), np.ones(3))
    res = oracle.spgemm_dense(A, B)
    assert res.col.tolist() == [0] and res.val[0] == 0.0  # traversal order
    A = inputs.CSR(1, 2, np.array([0, 2]), np.array([0, 1], np.int32), np.array([1.0, -1.0]))
    B = inputs.CSR(2, 3, np.array([0, 1, 2]), np.array([2, 2], np.int32), np.array([1.0, 1.0]))
    res = oracle.spgemm_dense(A, B)
    assert res.col.tolist() == [2] and res.val.tolist() == [0.0]  # structural zero kept
    I = inputs.identity(50)
    M = inputs.ragged(50, 50, 0, 9, seed=4)
    for X, Y in ((M, I), (I, M)):
        r = oracle.spgemm_dense(X, Y)
        assert np.array_equal(r.row_ptr, M.row_ptr) and np.array_equal(r.col, M.col)
        assert np.array_equal(r.val, M.val)


@pytest.mark.parametrize("kind", ["rmat", "ragged", "uniform", "empty_rows"])
def test_dense_form_bit_identical_to_sort_form(kind):
    if kind == "rmat":
        A = inputs.rmat(11, 16, seed=3)
        B = A
    elif kind == "ragged":
        A = inputs.ragged(700, 900, 0, 30, seed=5, matrix_id=1)
        B = inputs.ragged(900, 5000, 0, 30, seed=5, matrix_id=2)
    elif kind == "uniform":
        A = inputs.uniform(2000, 2000, 8, seed=6)
        B = A
    else:
        A = inputs.ragged(300, 400, 0, 2, seed=7, matrix_id=1)
        B = inputs.ragged(400, 300, 0, 3, seed=7, matrix_id=2)
    rows = np.arange(A.n_rows, dtype=np.int64)[::3]
    for rr in (None, rows):
        r1 = oracle.spgemm(A, B, rows=rr, threads=3)
        r2 = oracle.spgemm_dense(A, B, rows=rr, threads=3)
        assert np.array_equal(r1.row_ptr, r2.row_ptr)
        assert np.array_equal(r1.col, r2.col)
        assert np.array_equal(r1.val.view(np.int64), r2.val.view(np.int64))
        assert np.array_equal(r1.abs, r2.abs)
