"""Allocation-free numeric entry point (magnus_numeric_noalloc).

Some callers may not allocate device memory once they are running (a solver
that re-multiplies a fixed structure with new values inside a framework whose
allocator owns the whole device, or a loop that must not let cudaMalloc /
cudaFree synchronise the device).  For them the library offers a numeric
phase whose fine-level staging lives in a fixed static device buffer.  These
tests call it through the C ABI twice in a row (the buffer keeps the
previous call's contents) and compare each result with the oracle's C and
with magnus_numeric on the same plan; they check that the calls leave the
device's memory untouched, that the fine rows run on the grid the plan
reports, and that a plan too large for the buffer is refused before any
work.
"""
import ctypes

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


def _memory_state():
    """(bytes in use in the default stream-ordered pool, free device bytes)
    after a synchronize: any device allocation changes one of them."""
    import torch
    torch.cuda.synchronize()
    rt = ctypes.CDLL("libcudart.so.13")  # the runtime libmagnus.so already loaded
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    used = ctypes.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, 7, ctypes.byref(used)) == 0  # UsedMemCurrent
    return used.value, torch.cuda.mem_get_info()[0]


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
    ref = oracle.spgemm(A, B, threads=8)
    info = plan.info()
    assert info["rows_per_category"][FINE] == 3000 and info["n_batches_fine"] >= 1
    # a 16 MB staging budget keeps the slabs small enough for a full wave
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert info["noalloc_fine_blocks"] >= sms
    col_ref, val_ref = plan.numeric()
    torch.cuda.synchronize()
    col_ref = col_ref.cpu().numpy()
    val_ref = val_ref.cpu().numpy()
    assert np.array_equal(col_ref, ref.col)
    stream = torch.cuda.current_stream().cuda_stream
    c_col = torch.empty((nnz,), dtype=torch.int32, device="cuda")
    c_val = torch.empty((nnz,), dtype=torch.float64, device="cuda")
    for call in range(2):
        c_col.fill_(-1)
        c_val.fill_(float("nan"))
        if call == 1:
            before = _memory_state()
        magnus.magnus_numeric_noalloc(plan.handle, dA.val.data_ptr(), dB.val.data_ptr(),
                                      plan.c_row_ptr.data_ptr(), c_col.data_ptr(),
                                      c_val.data_ptr(), stream)
        torch.cuda.synchronize()
        if call == 1:  # (the first call may load device code once)
            assert _memory_state() == before, "the allocation-free call allocated"
        got_col = c_col.cpu().numpy()
        got = c_val.cpu().numpy()
        assert np.array_equal(got_col, ref.col)
        # the oracle's values under the parity rule
        # |c - c_ref| <= 1e-12 * max(|c_ref|, sum |terms|), and the pool path's
        assert np.all(values_close(got, ref.val, ref.abs))
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
    assert plan.info()["noalloc_fine_blocks"] == -1
    c_col = torch.empty(nnz, dtype=torch.int32, device="cuda")
    c_val = torch.empty(nnz, dtype=torch.float64, device="cuda")
    with pytest.raises(magnus.MagnusError) as ei:
        magnus.magnus_numeric_noalloc(plan.handle, dA.val.data_ptr(), dB.val.data_ptr(),
                                      plan.c_row_ptr.data_ptr(), c_col.data_ptr(),
                                      c_val.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == 9
    plan.free()
