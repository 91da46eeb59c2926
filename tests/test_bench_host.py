"""Host-side logic of bench.py (no GPU): the row and product samples of the
CPU baselines, the row-product counts they rely on, the massive workload's
partial host operands, the served workload's expected product counts, and
the byte counts behind T_ideal and the roofline (against access walks)."""
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


class _Tally:
    """Byte counter for the access walk below."""

    def __init__(self):
        self.read = 0
        self.write = 0


def _gustavson_volume(A, B, nnz_c):
    """Walks the two phases of a Gustavson SpGEMM and counts every element
    read or written once per access, with int64 row pointers, int32 columns
    and FP64 values: the accounting behind Section 4.3's ideal volumes (no
    reuse of B rows, start and end pointer of every B row read in each
    phase, values only in the numeric phase)."""
    t = _Tally()
    for phase in ("symbolic", "numeric"):
        t.read += 8 * (A.n_rows + 1)  # A.rowPtr
        for i in range(A.n_rows):
            for j in range(A.row_ptr[i], A.row_ptr[i + 1]):
                t.read += 4  # A.col[j]
                if phase == "numeric":
                    t.read += 8  # A.val[j]
                k = A.col[j]
                t.read += 8 + 8  # B.rowPtr[k], B.rowPtr[k + 1]
                for _ in range(B.row_ptr[k], B.row_ptr[k + 1]):
                    t.read += 4  # B.col
                    if phase == "numeric":
                        t.read += 8  # B.val
    t.write += 8 * (A.n_rows + 1) + 12 * nnz_c  # C.rowPtr, C.col + C.val
    return t.read + t.write


def test_ideal_bytes_is_the_gustavson_access_count():
    # bench.ideal_bytes (Eq. 8 + Eq. 9 with 8/4/8-byte types) equals a plain
    # count of the accesses, so a dropped or doubled term fails here.
    import oracle
    A = inputs.ragged(60, 90, 0, 9, seed=4, matrix_id=1)
    B = inputs.ragged(90, 120, 0, 9, seed=4, matrix_id=2)
    C = oracle.spgemm(A, B)
    nnz_c = int(C.row_ptr[-1])
    P = int(bench.row_products(A, B).sum())
    assert bench.ideal_bytes(A.n_rows, A.nnz, P, nnz_c) == _gustavson_volume(A, B, nnz_c)


def test_numeric_sort_alg_bytes_is_the_numeric_access_count():
    # The roofline's algorithmic bytes of the numeric sort-row kernel: the
    # numeric phase alone, reading C.rowPtr (computed by the symbolic phase)
    # instead of writing it.
    import oracle
    A = inputs.ragged(50, 70, 0, 8, seed=5, matrix_id=1)
    B = inputs.ragged(70, 100, 0, 8, seed=5, matrix_id=2)
    nnz_c = int(oracle.spgemm(A, B).row_ptr[-1])
    read = 8 * (A.n_rows + 1) * 2  # A.rowPtr, C.rowPtr
    for j in range(A.nnz):
        k = A.col[j]
        read += 4 + 8 + 16  # A.col, A.val, B.rowPtr[k], B.rowPtr[k + 1]
        read += 12 * int(B.row_ptr[k + 1] - B.row_ptr[k])  # B.col + B.val
    want = read + 12 * nnz_c
    P = int(bench.row_products(A, B).sum())
    assert bench.numeric_sort_alg_bytes(A.n_rows, A.nnz, P, nnz_c) == want
