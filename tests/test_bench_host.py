"""Host-side logic of bench.py (no GPU): the row and product samples of the
CPU baselines, the row-product counts they rely on, the massive workload's
partial host operands, and the served workload's expected product counts."""
import numpy as np

import bench
from paper_2501_07056_gb300 import inputs, serve


def test_row_products_matches_definition():
    A = inputs.ragged(300, 500, 0, 20, seed=1, matrix_id=1)
    B = inputs.ragged(500, 800, 0, 20, seed=1, matrix_id=2)
    lens = np.diff(B.row_ptr)
    want = np.array([lens[A.col[A.row_ptr[i]:A.row_ptr[i + 1]]].sum() for i in range(A.n_rows)])
    assert np.array_equal(bench.row_products(A, B), want)
    S = inputs.ragged(400, 400, 0, 20, seed=2, matrix_id=3)
    ls = np.diff(S.row_ptr)
    assert np.array_equal(bench.row_products(S), np.array(
        [ls[S.col[S.row_ptr[i]:S.row_ptr[i + 1]]].sum() for i in range(S.n_rows)]))


def test_sample_rows_bounded_and_spread():
    A = inputs.rmat(12, 16, seed=0)
    P = bench.row_products(A)
    rows, prods = bench.sample_rows(A, 2000000)
    assert prods == int(P[rows].sum()) and prods <= 2000000
    assert rows.size > 64  # more than the one-row-per-block floor
    floor_rows, _ = bench.sample_rows(A, 10)
    assert floor_rows.size == 64
    assert np.all(np.diff(rows) > 0)
    assert rows.min() < A.n_rows // 64 and rows.max() > A.n_rows * 62 // 64  # spread over A
    all_rows, total = bench.sample_rows(A, int(P.sum()))
    assert all_rows.size == A.n_rows and total == int(P.sum())


def test_massive_host_rows_of_b():
    A, B, rows = bench.massive_host("massive20", 1 << 22)
    assert A.n_rows == bench.MASSIVE_ROWS and np.all(np.diff(A.row_ptr) == bench.MASSIVE_NNZ)
    need = np.unique(np.concatenate([A.col[A.row_ptr[r]:A.row_ptr[r + 1]] for r in rows]))
    lens = np.diff(B.row_ptr)
    assert np.all(lens[need] == bench.MASSIVE_NNZ)
    assert int(lens.sum()) == need.size * bench.MASSIVE_NNZ  # only the referenced rows
    full = inputs.stratified(bench.MASSIVE_K, 1 << 20, bench.MASSIVE_NNZ, 0, 2, rows=need[:3])
    assert np.array_equal(full.col[:bench.MASSIVE_NNZ],
                          B.col[B.row_ptr[need[0]]:B.row_ptr[need[0] + 1]])


def test_served_expected_products():
    descs = inputs.served_stream(30, seed=0, k_lo=3, k_hi=7)
    est = serve.make_requests(descs, rate=10.0, exact=False)
    ex = serve.make_requests(descs, rate=10.0, exact=True)
    assert [r.arrival for r in est] == [r.arrival for r in ex]
    # expected = 10 * nnz(stencil); exact counts scatter around it
    ratio = np.array([e.products / x.products for e, x in zip(est, ex)])
    assert np.all(ratio > 0.7) and np.all(ratio < 1.4)
    assert abs(ratio.mean() - 1.0) < 0.1
