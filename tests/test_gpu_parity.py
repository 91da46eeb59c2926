"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Structure (row pointers, column indices) must match bit-exactly; values must
satisfy |c - c_ref| <= 1e-12 * max(|c_ref|, sum of |terms|).  Every
category (sort, dense, fine, coarse) is exercised both where the setup picks
it and where it is forced, on inputs spanning several tiles and ragged tails.
"""
import numpy as np
import pytest

from paper_2501_07056_gb300 import inputs
from tests._gpu import assert_parity, run_gpu
from tests._util import random_pattern_csr

pytestmark = pytest.mark.gpu

SORT, DENSE, FINE, COARSE = 0, 1, 2, 3


def P(**kw):
    from paper_2501_07056_gb300 import magnus
    return magnus.make_params(**kw)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_uniform4096_auto():
    A, B = inputs.workload("uniform4096")
    got = run_gpu(A, B, same=True)
    assert_parity(got, A, B)
    info = got["info"]
    assert info["n_interprod"] == 4096 * 64
    assert info["rows_per_category"][SORT] == 4096


@pytest.mark.parametrize("force,extra", [
    (SORT, {}), (DENSE, {}), (FINE, {}), (FINE, dict(chunk_len_fine_log2=6)),
    (COARSE, {}), (COARSE, dict(chunk_len_coarse_log2=10)),
    (COARSE, dict(chunk_len_coarse_log2=8, chunk_len_fine_log2=5)),
])
def test_uniform4096_forced(force, extra):
    A, B = inputs.workload("uniform4096")
    got = run_gpu(A, B, P(force_category=force, validate=1, **extra), same=True)
    assert_parity(got, A, B)
    cats = got["info"]["rows_per_category"]
    if force == DENSE:
        assert cats[DENSE] == 4096
    elif force != SORT:
        assert cats[force] == 4096


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("T", [0, 16, 100])
def test_ragged_mixed_categories(seed, T):
    A = inputs.ragged(3000, 20000, 0, 60, seed=seed, matrix_id=1)
    B = inputs.ragged(20000, 70000, 0, 120, seed=seed, matrix_id=2)
    got = run_gpu(A, B, P(sort_threshold=T, validate=1))
    assert_parity(got, A, B)


@pytest.mark.parametrize("force", [-1, SORT, DENSE, FINE, COARSE])
def test_sparse_a_long_b_rows(force):
    """A with at most 8 nonzeros per row on average (the row analysis runs
    one lane per row, eight entries per step) over B rows of 0..400 entries:
    rows from empty to several thousand products, so the products alone place
    some rows and the column range places the others (dense or sort), and
    every forced category reads the range of every row."""
    A = inputs.ragged(3000, 4000, 0, 12, seed=21, matrix_id=1)
    B = inputs.ragged(4000, 6000, 0, 400, seed=21, matrix_id=2)
    assert A.nnz <= 8 * A.n_rows
    got = run_gpu(A, B, P(force_category=force, validate=1))
    assert_parity(got, A, B)
    cats = got["info"]["rows_per_category"]
    if force < 0:
        assert cats[SORT] > 0 and cats[DENSE] > 0
    elif force != SORT:
        assert cats[force] > 0


@pytest.mark.parametrize("T,wide", [(512, 0), (1025, 0), (0, 0), (0, -1), (100, 300)])
def test_block_sort_bins(T, wide):
    # rows of about 200-1600 products over 200000 columns: the block sort bins
    # (257..1024 products), the wide-row rule, and coarse rows above 1024
    A = inputs.ragged(2500, 6000, 8, 40, seed=4, matrix_id=1)
    B = inputs.ragged(6000, 200000, 8, 40, seed=4, matrix_id=2)
    got = run_gpu(A, B, P(sort_threshold=T, wide_sort_max=wide, validate=1))
    assert_parity(got, A, B)
    lens = np.diff(A.row_ptr)
    Bl = np.diff(B.row_ptr)
    Prow = np.add.reduceat(Bl[A.col], A.row_ptr[:-1]) * (lens > 0)
    cats = got["info"]["rows_per_category"]
    limit = max(T - 1 if T else 255, {0: 1024, -1: 0}.get(wide, wide))
    assert cats[SORT] == int(((Prow > 0) & (Prow <= limit)).sum())


@pytest.mark.parametrize("b_cols", [700, 4000])
@pytest.mark.parametrize("wide", [0, -1])
def test_sparse_rows_sort_rule(b_cols, wide):
    # rows of about 100-1600 products whose column range fits the dense
    # accumulator: rows with at least sort_threshold products take the dense
    # accumulator only when they fill half of their range (wide_sort_max on),
    # else the sort bins; with the rule off every such row is dense
    A = inputs.ragged(2000, 3000, 8, 40, seed=9, matrix_id=1)
    B = inputs.ragged(3000, b_cols, 8, 40, seed=9, matrix_id=2)
    got = run_gpu(A, B, P(wide_sort_max=wide, validate=1))
    assert_parity(got, A, B)
    info = got["info"]
    Bl = np.diff(B.row_ptr)
    first = np.where(Bl > 0, B.col[np.minimum(B.row_ptr[:-1], B.col.size - 1)], np.iinfo(np.int32).max)
    last = np.where(Bl > 0, B.col[np.maximum(B.row_ptr[1:] - 1, 0)], -1)
    n_sort = n_dense = 0
    for i in range(A.n_rows):
        js = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        p = int(Bl[js].sum())
        if p == 0:
            continue
        rng = int(last[js].max()) - int(first[js].min()) + 1
        lim = 1024 if wide == 0 else 0
        if p < info["sort_threshold"]:
            n_sort += 1
        elif rng <= info["dense_cols"] and (p > lim or rng <= 2 * p):
            n_dense += 1
        elif p <= lim:
            n_sort += 1
    cats = info["rows_per_category"]
    assert cats[SORT] == n_sort and cats[DENSE] == n_dense
    if wide == 0:
        assert cats[SORT] > 0 and (b_cols > 1000 or cats[DENSE] > 0)


@pytest.mark.parametrize("force", [-1, SORT])
def test_block_sort_skewed_columns(force):
    # four in five B rows hold column 0: rows of A with more than 32 such B
    # rows put more than 32 keys in one column bucket and take the warp-wide
    # network, the others the per-lane bucket sorts (both block-sort bins)
    rng = np.random.default_rng(11)
    b_rows = []
    for r in range(2000):
        others = rng.choice(np.arange(1, 60000), size=int(rng.integers(7, 16)), replace=False)
        cols = np.sort(others)
        if r % 5:
            cols = np.concatenate(([0], cols))
        b_rows.append(cols.tolist())
    a_rows = [np.sort(rng.choice(2000, size=int(rng.integers(24, 61)), replace=False)).tolist()
              for _ in range(700)]
    A = _csr(700, 2000, a_rows)
    B = _csr(2000, 60000, b_rows)
    got = run_gpu(A, B, P(force_category=force, validate=1))
    assert_parity(got, A, B)
    assert got["info"]["rows_per_category"][SORT] > 0


def test_block_sort_64bit_keys():
    # 2^27 columns: column + 10 slot bits exceed 32 bits
    A = inputs.ragged(1500, 3000, 10, 40, seed=6, matrix_id=1)
    B = inputs.ragged(3000, 1 << 27, 10, 40, seed=6, matrix_id=2)
    got = run_gpu(A, B, P(sort_threshold=1025))
    assert_parity(got, A, B)
    assert got["info"]["key_bits32"] == 0


@pytest.mark.parametrize("m_log2,k", [(26, 128), (20, 200), (30, 64)])
def test_massive_nonsquare_sampled(m_log2, k):
    # the massive nonsquare uniform workload at reduced size: rows of k*k
    # products spread over 2^m_log2 columns go to the coarse level, whose
    # chunks widen with the sparsity of the rows
    import torch
    from paper_2501_07056_gb300 import gen_device, magnus
    rows_a, kdim = 64, 1 << 14
    dA = gen_device.stratified(rows_a, kdim, k, 0, 11)
    dB = gen_device.stratified(kdim, 1 << m_log2, k, 0, 12)
    plan = magnus.Plan(dA, dB)
    plan.symbolic()
    col, val = plan.numeric()
    torch.cuda.synchronize()
    info = plan.info()
    assert info["rows_per_category"][COARSE] == rows_a
    if m_log2 >= 26:
        assert info["chunk_len_coarse_log2"] > 13
    A = inputs.stratified(rows_a, kdim, k, 0, 11)
    B = inputs.stratified(kdim, 1 << m_log2, k, 0, 12, rows=np.unique(A.col))
    got = dict(row_ptr=plan.c_row_ptr.cpu().numpy(), col=col.cpu().numpy(), val=val.cpu().numpy())
    assert_parity(got, A, B)
    plan.free()


@pytest.mark.parametrize("force", [-1, SORT, DENSE, FINE, COARSE])
def test_rmat_small(force):
    A = inputs.rmat(13, 16, seed=0)
    got = run_gpu(A, A, P(force_category=force, chunk_len_coarse_log2=10 if force == COARSE else 0),
                  same=True)
    assert_parity(got, A, A)


@pytest.mark.parametrize("dthr", [1, 8, 65, 200, 1024])
@pytest.mark.parametrize("force", [FINE, COARSE])
def test_hybrid_threshold_extremes(dthr, force):
    A = inputs.rmat(12, 16, seed=1)
    got = run_gpu(A, A, P(force_category=force, dense_chunk_threshold=dthr,
                          chunk_len_fine_log2=7, chunk_len_coarse_log2=9), same=True)
    assert_parity(got, A, A)


@pytest.mark.parametrize("force", [FINE, COARSE])
def test_small_staging_budget(force):
    # An 8 MB staging budget: fine rows with more products than one block's
    # slab (about 1500 here) are split by the coarse level, and coarse rows
    # run in several batches.
    A = inputs.ragged(2000, 5000, 20, 60, seed=3, matrix_id=1)
    B = inputs.ragged(5000, 30000, 10, 50, seed=3, matrix_id=2)
    got = run_gpu(A, B, P(force_category=force, max_scratch_bytes=8 << 20,
                          chunk_len_coarse_log2=12))
    assert_parity(got, A, B)
    info = got["info"]
    if force == FINE:
        assert info["rows_per_category"][FINE] > 0 and info["rows_per_category"][COARSE] > 0
    else:
        assert info["n_batches_coarse"] > 1


def _csr(n_rows, n_cols, rows_cols, vals=None):
    lengths = np.array([len(r) for r in rows_cols], np.int64)
    rp = np.concatenate(([0], np.cumsum(lengths))).astype(np.int64)
    col = np.array([c for r in rows_cols for c in r], np.int32)
    val = np.array(vals if vals is not None else np.linspace(-1, 1, col.size) + 0.5, np.float64)
    return inputs.CSR(n_rows, n_cols, rp, col, val)


@pytest.mark.parametrize("force", [-1, SORT, DENSE, FINE, COARSE])
def test_edge_cases(force):
    p = P(force_category=force)
    # all products of a row land in one column (maximal duplication)
    A = inputs.ragged(300, 400, 1, 200, seed=5, matrix_id=1)
    B1 = _csr(400, 7, [[3]] * 400, np.random.default_rng(0).uniform(-1, 1, 400))
    assert_parity(run_gpu(A, B1, p), A, B1)
    # single column of C
    B2 = _csr(400, 1, [[0]] * 400, np.random.default_rng(1).uniform(-1, 1, 400))
    assert_parity(run_gpu(A, B2, p), A, B2)
    # empty rows in A and in B, nonsquare, ragged
    rng = np.random.default_rng(2)
    A3 = random_pattern_csr(rng, 97, 131, 0.05)
    B3 = random_pattern_csr(rng, 131, 3001, 0.02)
    assert_parity(run_gpu(A3, B3, p), A3, B3)
    # 1x1
    A4 = _csr(1, 1, [[0]], [2.5])
    assert_parity(run_gpu(A4, A4, p), A4, A4)


def test_empty_matrices():
    Z = inputs.CSR(5, 6, np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0))
    B = inputs.uniform(6, 9, 2, seed=1)
    got = run_gpu(Z, B)
    assert got["nnz"] == 0 and got["row_ptr"].tolist() == [0] * 6
    E = inputs.CSR(0, 6, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    got = run_gpu(E, B)
    assert got["nnz"] == 0 and got["row_ptr"].tolist() == [0]
    A = inputs.uniform(5, 6, 3, seed=2)
    Bz = inputs.CSR(6, 9, np.zeros(7, np.int64), np.zeros(0, np.int32), np.zeros(0))
    got = run_gpu(A, Bz)
    assert got["nnz"] == 0


@pytest.mark.parametrize("force", [-1, DENSE, FINE, COARSE])
def test_wide_columns_64bit_keys(force):
    # columns near 2^31 force 64-bit sort keys and many coarse chunks
    n_cols = (1 << 31) - 1
    rng = np.random.default_rng(4)
    A = inputs.ragged(500, 800, 1, 40, seed=4, matrix_id=1)
    rows = []
    for _ in range(800):
        k = int(rng.integers(0, 30))
        rows.append(sorted(set(rng.integers(n_cols - (1 << 20), n_cols, size=k).tolist()) |
                           set(rng.integers(0, 1 << 20, size=3).tolist())))
    B = _csr(800, n_cols, rows, rng.uniform(-1, 1, sum(len(r) for r in rows)))
    got = run_gpu(A, B, P(force_category=force))
    assert_parity(got, A, B)


def test_plan_reuse_new_values():
    import torch
    A = inputs.rmat(12, 16, seed=3)
    got = run_gpu(A, A, same=True, keep_plan=True)
    assert_parity(got, A, A)
    plan, (dA, _) = got["plan"], got["dev"]
    A2 = inputs.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val * -3.0 + 0.25)
    v2 = torch.as_tensor(A2.val).cuda()
    col, val = plan.numeric(a_val=v2, b_val=v2)
    torch.cuda.synchronize()
    got2 = dict(row_ptr=got["row_ptr"], col=col.cpu().numpy(), val=val.cpu().numpy())
    assert_parity(got2, A2, A2)
    plan.free()


def test_validate_rejects_unsorted():
    from paper_2501_07056_gb300 import magnus
    A = _csr(2, 4, [[2, 1], [0]], [1.0, 2.0, 3.0])
    B = inputs.uniform(4, 4, 2, seed=0)
    with pytest.raises(magnus.MagnusError) as ei:
        run_gpu(A, B, P(validate=1))
    assert ei.value.status == 2
    Aout = _csr(2, 4, [[0, 7], [1]], [1.0, 2.0, 3.0])
    with pytest.raises(magnus.MagnusError):
        run_gpu(Aout, B, P(validate=1))


def test_numeric_before_symbolic():
    import torch
    from paper_2501_07056_gb300 import magnus
    A = inputs.uniform(64, 64, 4, seed=0)
    dA = magnus.DeviceCSR.from_host(A)
    plan = magnus.Plan(dA, dA)
    c = torch.zeros(10, dtype=torch.int64, device="cuda")
    with pytest.raises(magnus.MagnusError) as ei:
        magnus.magnus_numeric(plan.handle, dA.val.data_ptr(), dA.val.data_ptr(), c.data_ptr(),
                              c.data_ptr(), c.data_ptr(), 0)
    assert ei.value.status == 7
    plan.free()


def test_launch_counter_advances():
    from paper_2501_07056_gb300 import magnus
    A, B = inputs.workload("uniform4096")
    n0 = magnus.magnus_launch_count()
    run_gpu(A, B, same=True)
    assert magnus.magnus_launch_count() > n0


def test_wide_coarse_chunks_use_fine_level():
    # Coarse chunks of 2^16 columns are wider than one block's dense
    # accumulator, so each large (row, chunk) runs the fine level inside it.
    A = inputs.ragged(1500, 1 << 17, 5, 40, seed=8, matrix_id=1)
    B = inputs.ragged(1 << 17, 1 << 18, 20, 200, seed=8, matrix_id=2)
    got = run_gpu(A, B, P(force_category=COARSE, chunk_len_coarse_log2=16, chunk_len_fine_log2=8))
    assert_parity(got, A, B)
    assert got["info"]["chunk_len_coarse_log2"] == 16


@pytest.mark.parametrize("zero_frac", [0.0, 0.02, 0.3, 1.0])
def test_coarse_negative_zero_products(zero_frac):
    # Products equal to -0.0 (A entries -0.0, B positive): a column reached
    # only by them is still part of C's structure, whichever accumulator the
    # coarse buckets use (warp sort, dense bitmap, fine level inside), and
    # its value is a zero.  Planted at several rates, up to every product.
    A = inputs.rmat(12, 16, seed=2)
    rng = np.random.default_rng(11)
    A.val = np.abs(A.val) + 0.25
    A.val[rng.random(A.nnz) < zero_frac] = -0.0
    B = inputs.rmat(12, 16, seed=3)
    B.val = np.abs(B.val) + 0.5
    for cl in (9, 10, 13):
        got = run_gpu(A, B, P(force_category=COARSE, chunk_len_coarse_log2=cl))
        assert_parity(got, A, B)
        if zero_frac == 1.0:
            assert np.all(got["val"] == 0.0)


@pytest.mark.parametrize("dthr", [2, 9, 33, 257])
@pytest.mark.parametrize("fine_log2", [5, 7])
@pytest.mark.parametrize("force", [FINE, COARSE])
def test_chunk_merging_sparse_chunks(dthr, fine_log2, force):
    # Sparse rows over a wide column range: most fine chunks hold 0-3
    # products, so long runs of small chunks merge into groups of up to 32
    # products (one warp sort each), cut by the chunks at or above dthr.
    # Coarse chunks of 2^15 columns hold several hundred products each and
    # run the fine level inside.
    A = inputs.ragged(600, 2000, 10, 40, seed=12, matrix_id=1)
    B = inputs.ragged(2000, 1 << 16, 5, 40, seed=12, matrix_id=2)
    got = run_gpu(A, B, P(force_category=force, dense_chunk_threshold=dthr,
                          chunk_len_fine_log2=fine_log2, chunk_len_coarse_log2=15))
    assert_parity(got, A, B)


@pytest.mark.parametrize("dthr", [1, 9])
@pytest.mark.parametrize("force", [FINE, COARSE])
@pytest.mark.parametrize("inp", ["rmat", "sparse", "dup"])
def test_hash_chunk_accumulator(inp, force, dthr):
    # chunk_accumulator = 1: fine chunks of at most 128 products accumulate
    # in the warp's open-addressing table (linear probing), the distinct
    # columns are sorted by the warp; larger chunks stay dense, chunks below
    # dthr sort (merged).  R-MAT (duplicates on hub columns), sparse rows
    # (chunks of 0-3 products), and every product of a row in a handful of
    # columns (long probe chains on one slot).
    if inp == "rmat":
        A = B = inputs.rmat(12, 16, seed=4)
        extra = dict(chunk_len_fine_log2=7, chunk_len_coarse_log2=15)
    elif inp == "sparse":
        A = inputs.ragged(600, 2000, 10, 40, seed=13, matrix_id=1)
        B = inputs.ragged(2000, 1 << 16, 5, 40, seed=13, matrix_id=2)
        extra = dict(chunk_len_fine_log2=8, chunk_len_coarse_log2=15)
    else:
        rng = np.random.default_rng(14)
        n, m = 300, 1 << 15
        rows = [sorted(rng.choice(n, size=rng.integers(1, 120), replace=False).tolist())
                for _ in range(n)]
        A = _csr(n, n, rows)
        # B rows: a few fixed columns each (every chunk sees heavy duplication)
        cols = np.sort(rng.choice(m, size=6, replace=False)).tolist()
        B = _csr(n, m, [cols[: 1 + (i % 6)] for i in range(n)],
                 np.concatenate([rng.uniform(-1, 1, 1 + (i % 6)) for i in range(n)]))
        extra = dict(chunk_len_fine_log2=5, chunk_len_coarse_log2=14)
    p = P(force_category=force, dense_chunk_threshold=dthr, chunk_accumulator=1, **extra)
    got = run_gpu(A, B, p, same=A is B)
    assert_parity(got, A, B)


@pytest.mark.parametrize("reorder,bsort", [(1, 1), (2, 1), (1, -1), (2, -1)])
@pytest.mark.parametrize("case", ["rmat", "rmat_forced_small_budget", "ragged_coarse",
                                  "wide_chunks", "hub_rows"])
def test_coarse_reorder_forms(case, reorder, bsort):
    """Both stagings of Algorithm 4's reorder (outer product over A^CSC, and
    row-wise with sub-tiles counting-sorted by chunk and written as runs)
    give the oracle's C: R-MAT with its automatic coarse rows; every row
    forced coarse under an 8 MB staging budget (several batches); ragged rows
    with 2^10-column chunks; chunks wider than the block accumulator (fine
    level inside); rows of A with more than 256 nonzeros over long B rows
    (several work items per row, B rows longer than a sub-tile).  Each with
    buckets of 257..2048 products block-sorted (bsort 1) or accumulated by
    the dense accumulator / fine level (bsort -1)."""
    if case == "rmat":
        A = B = inputs.rmat(14, 16, seed=1)
        params = P(coarse_reorder=reorder, coarse_bucket_sort=bsort)
    elif case == "rmat_forced_small_budget":
        A = B = inputs.rmat(13, 16, seed=2)
        params = P(coarse_reorder=reorder, coarse_bucket_sort=bsort, force_category=COARSE,
                   max_scratch_bytes=8 << 20)
    elif case == "ragged_coarse":
        A = inputs.ragged(2000, 5000, 0, 40, seed=3, matrix_id=1)
        B = inputs.ragged(5000, 60000, 0, 40, seed=3, matrix_id=2)
        params = P(coarse_reorder=reorder, coarse_bucket_sort=bsort, force_category=COARSE,
                   chunk_len_coarse_log2=10)
    elif case == "wide_chunks":
        A = inputs.ragged(1500, 5000, 5, 60, seed=4, matrix_id=1)
        B = inputs.ragged(5000, 1 << 20, 5, 60, seed=4, matrix_id=2)
        params = P(coarse_reorder=reorder, coarse_bucket_sort=bsort, force_category=COARSE,
                   chunk_len_coarse_log2=15)
    else:
        A = inputs.ragged(40, 3000, 300, 700, seed=5, matrix_id=1)
        B = inputs.ragged(3000, 200000, 500, 3000, seed=5, matrix_id=2)
        params = P(coarse_reorder=reorder, coarse_bucket_sort=bsort, force_category=COARSE)
    got = run_gpu(A, B, params, same=A is B)
    assert got["info"]["rows_per_category"][COARSE] > 0
    assert_parity(got, A, B)
    from paper_2501_07056_gb300 import magnus
    assert magnus.device_status() == 0  # no bounded wait of the bucket sort gave up
