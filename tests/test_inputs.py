"""The seeded generators produce valid, deterministic CSR of the stated shape."""
import numpy as np

from paper_2501_07056_gb300 import inputs


def test_uniform_shape_and_validity():
    A = inputs.uniform(4096, 4096, 8, seed=0)
    A.validate()
    assert A.nnz == 4096 * 8 and np.all(np.diff(A.row_ptr) == 8)
    assert A.val.min() >= -1 and A.val.max() < 1
    B = inputs.uniform(4096, 4096, 8, seed=0)
    assert np.array_equal(A.col, B.col) and np.array_equal(A.val, B.val)
    C = inputs.uniform(4096, 4096, 8, seed=1)
    assert not np.array_equal(A.col, C.col)


def test_uniform_small_columns_path():
    A = inputs.uniform(100, 20, 15, seed=3)
    A.validate()
    assert np.all(np.diff(A.row_ptr) == 15)


def test_ragged_lengths():
    A = inputs.ragged(5000, 1000, 2, 32, seed=0, matrix_id=4)
    A.validate()
    L = np.diff(A.row_ptr)
    assert L.min() >= 2 and L.max() <= 32 and abs(L.mean() - 17) < 0.5


def test_rmat_small():
    A = inputs.rmat(12, 16, seed=0)
    A.validate()
    assert A.n_rows == 4096
    # duplicates merged: fewer than 16n distinct entries, but most survive
    assert 0.8 * 16 * 4096 < A.nnz < 16 * 4096
    # mass concentrates at the top-left (a = .57 is the (0, 0) quadrant)
    top = A.row_ptr[2048]
    assert top > 0.7 * A.nnz
    assert A.val.min() >= 0 and A.val.max() < 1


def test_stencil27():
    for k in (1, 2, 5):
        S = inputs.stencil27(k)
        S.validate()
        assert S.nnz == (3 * k - 2) ** 3
        d = S.to_dense() if k <= 5 else None
        if d is not None:
            assert np.all(np.diag(d) == 26.0)
            assert np.allclose(d, d.T)


def test_batched_and_served_descriptors():
    probs = inputs.batched_problems(3, seed=0)
    for A, B in probs:
        A.validate(); B.validate()
        assert 256 <= A.n_rows <= 65536 and A.n_cols == B.n_rows
    reqs = inputs.served_stream(50, seed=0)
    assert all(16 <= r["k"] <= 96 for r in reqs)
    assert inputs.served_stream(50, seed=0) == reqs


def test_splitmix64_first_output():
    # SplitMix64 seeded with 0: its first output is 0xE220A8397B1DCDAF
    # (Steele, Lea and Flood 2014; the reference sequence of the generator).
    assert int(inputs.ctr_u64(np.uint64(0), 0)) == 0xE220A8397B1DCDAF


def test_ragged_ctr_properties():
    A = inputs.ragged_ctr(4000, 700, 2, 32, seed=0, matrix_id=9)
    A.validate()
    L = np.diff(A.row_ptr)
    assert L.min() >= 2 and L.max() <= 32 and abs(L.mean() - 17) < 0.6
    assert A.nnz == inputs.ragged_ctr_nnz(4000, 700, 2, 32, seed=0, matrix_id=9)
    assert A.val.min() >= -1 and A.val.max() < 1
    B = inputs.ragged_ctr(4000, 700, 2, 32, seed=0, matrix_id=9)
    assert np.array_equal(A.col, B.col) and np.array_equal(A.val, B.val)
    C = inputs.ragged_ctr(4000, 700, 2, 32, seed=0, matrix_id=10)
    assert not np.array_equal(A.row_ptr, C.row_ptr)
    # columns are spread over the whole range
    assert A.col.min() < 10 and A.col.max() > 690


def test_ragged_ctr_full_rows():
    # rows as long as the column range: every column once (the fill-in rule)
    A = inputs.ragged_ctr(50, 20, 20, 32, seed=3, matrix_id=1)
    A.validate()
    assert np.all(np.diff(A.row_ptr) == 20)
    assert np.array_equal(A.col.reshape(50, 20), np.tile(np.arange(20, dtype=np.int32), (50, 1)))


def test_stratified_rows():
    A = inputs.stratified(200, 10000, 64, seed=0, matrix_id=3)
    A.validate()
    assert np.all(np.diff(A.row_ptr) == 64)
    # one column in each of the 64 strata [floor(j n/k), floor((j+1) n/k))
    j = np.arange(64, dtype=np.int64)
    c = A.col.reshape(200, 64).astype(np.int64)
    assert np.all(c >= (j * 10000) // 64) and np.all(c < ((j + 1) * 10000) // 64)
    # partial generation fills exactly the listed rows, with the same entries
    P = inputs.stratified(200, 10000, 64, seed=0, matrix_id=3, rows=[3, 150])
    assert P.nnz == 128
    assert np.array_equal(P.col[:64], A.col[3 * 64:4 * 64])
    assert np.array_equal(P.val[64:], A.val[150 * 64:151 * 64])
