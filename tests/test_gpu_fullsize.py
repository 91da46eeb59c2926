"""Parity at the full sizes of the benchmark workloads, in the launch
configuration bench.py times (automatic parameters).

  * uniform n = 2^24, 8 nnz/row, C = A*A (1.07e9 products): C.rowPtr is
    compared with the oracle's precise prediction for every row; values are
    compared on sampled rows; the row-sum invariant C*1 = A*(A*1) is checked
    for every row.
  * R-MAT scale 20, edge factor 16, C = A*A (2.09e10 products, nnz(C) about
    1e10, 120 GB of output): the heaviest rows and random rows are compared
    with the oracle; the row-sum invariant is checked for every row; nnz(C) is
    checked against the band of Table 3 (9.94e9 for scale 20; the paper's
    generator keeps duplicate edges, this one merges them).

The row-sum check: in exact arithmetic sum_c C_ic = sum_j A_ij (sum_k B_jk).
Both sides are computed in FP64 by different routes, so they may differ by
the rounding of a sum of |terms|; with P_i products in row i the bound used
is 4 * P_i * 2^-53 * sum |terms|.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2501_07056_gb300 import inputs
from tests._util import values_close

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

THREADS = os.cpu_count() or 8


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _run(A):
    import torch
    from paper_2501_07056_gb300 import magnus
    torch.cuda.empty_cache()  # earlier tests' cached blocks (C alone is 108 GB here)
    dA = magnus.DeviceCSR.from_host(A)
    plan = magnus.Plan(dA, dA)
    nnz = plan.symbolic()
    col, val = plan.numeric()
    torch.cuda.synchronize()
    info = plan.info()
    rp = plan.c_row_ptr
    plan.free()
    return dA, rp, col, val, nnz, info


def _row_sum_check(dA, rp, val):
    """C*1 versus A*(A*1) for every row, on the device (torch ops, test only)."""
    import torch
    n = dA.n_rows
    c1 = torch.zeros(n, dtype=torch.float64, device="cuda")
    rp_host = rp.cpu().numpy()
    r0 = 0
    while r0 < n:  # row blocks of at most 2^30 entries of C
        r1 = int(np.searchsorted(rp_host, rp_host[r0] + (1 << 30), side="right")) - 1
        r1 = min(max(r1, r0 + 1), n)
        s0, s1 = int(rp_host[r0]), int(rp_host[r1])
        if s1 > s0:
            idx = torch.repeat_interleave(torch.arange(r0, r1, device="cuda"),
                                          rp[r0 + 1:r1 + 1] - rp[r0:r1])
            c1.index_add_(0, idx, val[s0:s1])
            del idx
        r0 = r1
    lens = dA.row_ptr[1:] - dA.row_ptr[:-1]
    rows_a = torch.repeat_interleave(torch.arange(n, device="cuda"), lens)
    b1 = torch.zeros(n, dtype=torch.float64, device="cuda").index_add_(0, rows_a, dA.val)
    babs = torch.zeros(n, dtype=torch.float64, device="cuda").index_add_(0, rows_a, dA.val.abs())
    ab1 = torch.zeros(n, dtype=torch.float64, device="cuda").index_add_(
        0, rows_a, dA.val * b1[dA.col.long()])
    sabs = torch.zeros(n, dtype=torch.float64, device="cuda").index_add_(
        0, rows_a, dA.val.abs() * babs[dA.col.long()])
    P = torch.zeros(n, dtype=torch.float64, device="cuda").index_add_(
        0, rows_a, lens[dA.col.long()].double())
    bound = 4.0 * (P + 2.0) * 2.0 ** -53 * sabs
    bad = ((c1 - ab1).abs() > bound).sum().item()
    assert bad == 0, "%d rows break the row-sum invariant" % bad


def _sampled_rows(A, rp_host, col, val, rows):
    ref = oracle.spgemm(A, A, rows=np.asarray(rows, np.int64), threads=THREADS)
    for t, i in enumerate(rows):
        s, e = int(rp_host[i]), int(rp_host[i + 1])
        rc, rv, ra = ref.row(t)
        assert e - s == rc.size, "row %d: nnz %d vs oracle %d" % (i, e - s, rc.size)
        c = col[s:e].cpu().numpy()
        v = val[s:e].cpu().numpy()
        assert np.array_equal(c, rc), "row %d columns differ" % i
        ok = values_close(v, rv, ra)
        assert ok.all(), "row %d: %d values differ" % (i, int((~ok).sum()))


def test_uniform_2_24_full_size():
    A, _ = inputs.workload("uniform2^24")
    dA, rp, col, val, nnz, info = _run(A)
    assert info["n_interprod"] == 64 * (1 << 24)
    rp_host = rp.cpu().numpy()
    cnt = oracle.symbolic(A, A, threads=THREADS)
    assert int(cnt.sum()) == nnz
    assert np.array_equal(np.diff(rp_host), cnt)
    rng = np.random.default_rng(1)
    rows = np.concatenate(([0, 1, A.n_rows - 1], rng.choice(A.n_rows, 3000, replace=False)))
    _sampled_rows(A, rp_host, col, val, rows)
    _row_sum_check(dA, rp, val)


def test_rmat20_full_size():
    A, _ = inputs.workload("rmat20")
    dA, rp, col, val, nnz, info = _run(A)
    lens = np.diff(A.row_ptr)
    P = np.bincount(np.repeat(np.arange(A.n_rows), lens), weights=lens[A.col],
                    minlength=A.n_rows).astype(np.int64)
    assert info["n_interprod"] == int(P.sum())
    # Table 3: 9,940,402,266 nonzeros of A^2 at scale 20 (duplicates kept there)
    assert 0.5 * 9.94e9 < nnz < 1.5 * 9.94e9
    rp_host = rp.cpu().numpy()
    counts = np.diff(rp_host)
    assert np.all(counts <= np.minimum(P, A.n_cols)) and np.all((counts > 0) == (P > 0))
    heavy = np.argsort(P)[-6:]
    rng = np.random.default_rng(2)
    nonempty = np.nonzero(P)[0]
    rows = np.concatenate((heavy, rng.choice(nonempty, 400, replace=False), [0, 1, 2]))
    _sampled_rows(A, rp_host, col, val, np.unique(rows))
    _row_sum_check(dA, rp, val)
