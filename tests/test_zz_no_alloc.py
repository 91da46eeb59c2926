"""Allocation-free numeric entry point (magnus_numeric_noalloc).

Some callers may not allocate device memory once they are running (a solver
that re-multiplies a fixed structure with new values inside a framework whose
allocator owns the whole device, or a loop that must not let cudaMalloc /
cudaFree synchronise the device).  For them the library offers a numeric
phase whose fine-level staging lives in a fixed static device buffer.  These
tests call it through the C ABI and compare it with magnus_numeric on the
same plan, twice in a row (the buffer keeps the previous call's contents),
and check that a plan too large for the buffer is refused before any work.
"""
import numpy as np
import pytest

from paper_2501_07056_gb300 import inputs
from tests._util import values_close

pytestmark = pytest.mark.gpu

FINE = 2


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _fine_plan(max_scratch, n_rows=3000):
    import torch
    from paper_2501_07056_gb300 import magnus
    A = inputs.ragged(n_rows, 40000, 10, 60, seed=11, matrix_id=1)
    B = inputs.ragged(40000, 300000, 5, 40, seed=11, matrix_id=2)
    dA = magnus.DeviceCSR.from_host(A)
    dB = magnus.DeviceCSR.from_host(B)
    params = magnus.make_params(force_category=FINE, chunk_len_fine_log2=10,
                                max_scratch_bytes=max_scratch)
    plan = magnus.Plan(dA, dB, params)
    nnz = plan.symbolic()
    torch.cuda.synchronize()
    return plan, (dA, dB), nnz, (A, B)


def test_noalloc_matches_numeric_on_two_calls():
    import torch
    from paper_2501_07056_gb300 import magnus
    import oracle
    plan, (dA, dB), nnz, (A, B) = _fine_plan(16 << 20)
    ref = oracle.spgemm(A, B, threads=8)  # only for the |terms| sums of the tolerance
    info = plan.info()
    assert info["rows_per_category"][FINE] == 3000 and info["n_batches_fine"] >= 1
    col_ref, val_ref = plan.numeric()
    torch.cuda.synchronize()
    col_ref = col_ref.cpu().numpy()
    val_ref = val_ref.cpu().numpy()
    assert np.array_equal(col_ref, ref.col)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        c_col = torch.full((nnz,), -1, dtype=torch.int32, device="cuda")
        c_val = torch.full((nnz,), float("nan"), dtype=torch.float64, device="cuda")
        magnus.magnus_numeric_noalloc(plan.handle, dA.val.data_ptr(), dB.val.data_ptr(),
                                      plan.c_row_ptr.data_ptr(), c_col.data_ptr(),
                                      c_val.data_ptr(), stream)
        torch.cuda.synchronize()
        assert np.array_equal(c_col.cpu().numpy(), col_ref)
        # the two calls may sum duplicates in different orders: compare with
        # the parity rule |c - c_ref| <= 1e-12 * max(|c_ref|, sum |terms|)
        got = c_val.cpu().numpy()
        assert np.all(values_close(got, val_ref, ref.abs))
    plan.free()


def test_noalloc_refuses_plan_with_coarse_rows():
    import torch
    from paper_2501_07056_gb300 import magnus
    # coarse rows need several staging buffers the fixed array cannot hold
    A = inputs.ragged(500, 4000, 10, 40, seed=12, matrix_id=1)
    B = inputs.ragged(4000, 9000, 5, 20, seed=12, matrix_id=2)
    dA, dB = magnus.DeviceCSR.from_host(A), magnus.DeviceCSR.from_host(B)
    plan = magnus.Plan(dA, dB, magnus.make_params(force_category=3))
    nnz = plan.symbolic()
    c_col = torch.empty(nnz, dtype=torch.int32, device="cuda")
    c_val = torch.empty(nnz, dtype=torch.float64, device="cuda")
    with pytest.raises(magnus.MagnusError) as ei:
        magnus.magnus_numeric_noalloc(plan.handle, dA.val.data_ptr(), dB.val.data_ptr(),
                                      plan.c_row_ptr.data_ptr(), c_col.data_ptr(),
                                      c_val.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == 9
    plan.free()
