"""Row slabs of C (magnus_numeric_rows) and the caller-owned workspace
(magnus_workspace_size, magnus_symbolic_ws, magnus_numeric_ws), through the
C ABI.

The phase split of Section 2.1 makes C.rowPtr an input of the numeric
phase, so any row range of C can be computed on a plan of the whole
product; Section 3.3 bounds memory by batching rows.  Every slab is compared
with the oracle's rows (structure bit-exact, values within
1e-12 * max(|c_ref|, sum |terms|)), on inputs that reach every category:
R-MAT (sort, block-sort and coarse rows), and the forced categories with a
small staging budget so that slab boundaries cut through coarse batches.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2501_07056_gb300 import inputs
from tests._util import values_close

pytestmark = pytest.mark.gpu

SORT, DENSE, FINE, COARSE = 0, 1, 2, 3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _pool_state():
    """(bytes in use in the device's default stream-ordered pool, free device
    bytes) after a synchronize: an allocation anywhere changes one of them."""
    import torch
    torch.cuda.synchronize()
    rt = ctypes.CDLL("libcudart.so.13")  # the runtime libmagnus.so already loaded
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    used = ctypes.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, 7, ctypes.byref(used)) == 0  # UsedMemCurrent
    return used.value, torch.cuda.mem_get_info()[0]


def _operands(kind):
    if kind == "rmat":
        A = inputs.rmat(13, 16, seed=0)
        return A, A
    A = inputs.ragged(3000, 20000, 0, 60, seed=21, matrix_id=1)
    # "narrow": every row's column range fits the dense accumulator
    B = inputs.ragged(20000, 6000 if kind == "narrow" else 50000, 0, 40, seed=21, matrix_id=2)
    return A, B


def _slab_cuts(n, rng):
    inner = np.sort(rng.choice(np.arange(1, n), size=min(n - 1, 9), replace=False))
    cuts = np.concatenate(([0], inner, [n]))
    # an empty slab and a one-row slab
    return np.unique(np.concatenate((cuts, [cuts[3], cuts[3] + 1])))


def _check_slab(rp, ref, r0, r1, col, val):
    e0, e1 = int(rp[r0]), int(rp[r1])
    assert np.array_equal(col, ref.col[e0:e1]), "slab [%d, %d) columns differ" % (r0, r1)
    ok = values_close(val, ref.val[e0:e1], ref.abs[e0:e1])
    assert ok.all(), "slab [%d, %d): %d values differ" % (r0, r1, int((~ok).sum()))


@pytest.mark.parametrize("kind,force,scratch", [
    ("rmat", -1, 0), ("rmat", COARSE, 8 << 20), ("rmat", FINE, 0),
    ("ragged", SORT, 0), ("narrow", DENSE, 0), ("ragged", FINE, 4 << 20),
    ("ragged", COARSE, 4 << 20)])
def test_numeric_rows_slabs_equal_oracle(kind, force, scratch):
    import torch
    from paper_2501_07056_gb300 import magnus
    A, B = _operands(kind)
    ref = oracle.spgemm(A, B, threads=8)
    dA = magnus.DeviceCSR.from_host(A)
    dB = dA if B is A else magnus.DeviceCSR.from_host(B)
    plan = magnus.Plan(dA, dB, magnus.make_params(force_category=force,
                                                  max_scratch_bytes=scratch))
    nnz = plan.symbolic()
    rp = plan.c_row_ptr.cpu().numpy()
    assert nnz == int(ref.row_ptr[-1]) and np.array_equal(rp, ref.row_ptr)
    info = plan.info()
    if force == COARSE and scratch:
        assert info["n_batches_coarse"] > 1  # slab boundaries cut through batches
    rng = np.random.default_rng(5)
    cuts = _slab_cuts(A.n_rows, rng)
    guard = 16
    for r0, r1 in zip(cuts[:-1], cuts[1:]):
        m = int(rp[r1] - rp[r0])
        col = torch.full((m + guard,), -7, dtype=torch.int32, device="cuda")
        val = torch.full((m + guard,), 123.0, dtype=torch.float64, device="cuda")
        plan.numeric_rows(int(r0), int(r1), col, val)
        torch.cuda.synchronize()
        c, v = col.cpu().numpy(), val.cpu().numpy()
        assert np.all(c[m:] == -7) and np.all(v[m:] == 123.0), "slab wrote past its entries"
        _check_slab(rp, ref, int(r0), int(r1), c[:m], v[:m])
    # the whole-matrix call on the same plan still matches
    col, val = plan.numeric()
    torch.cuda.synchronize()
    assert np.array_equal(col.cpu().numpy(), ref.col)
    assert values_close(val.cpu().numpy(), ref.val, ref.abs).all()
    plan.free()


def test_numeric_rows_arguments():
    import torch
    from paper_2501_07056_gb300 import magnus
    A, B = _operands("ragged")
    dA, dB = magnus.DeviceCSR.from_host(A), magnus.DeviceCSR.from_host(B)
    plan = magnus.Plan(dA, dB)
    c = torch.empty(8, dtype=torch.int32, device="cuda")
    v = torch.empty(8, dtype=torch.float64, device="cuda")
    with pytest.raises(magnus.MagnusError) as ei:  # before the symbolic phase
        magnus.magnus_numeric_rows(plan.handle, 0, 1, dA.val.data_ptr(), dB.val.data_ptr(),
                                   c.data_ptr(), c.data_ptr(), v.data_ptr(), 0, 0,
                                   torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == 7
    plan.symbolic()
    for r0, r1 in ((5, 4), (-1, 3), (0, A.n_rows + 1)):
        with pytest.raises(magnus.MagnusError) as ei:
            plan.numeric_rows(r0, r1, c, v)
        assert ei.value.status == 1
    plan.numeric_rows(10, 10, c, v)  # empty range: no work, no error
    plan.free()


@pytest.mark.parametrize("kind,force", [("rmat", -1), ("ragged", FINE), ("ragged", COARSE)])
def test_workspace_variants_allocate_nothing(kind, force):
    import torch
    from paper_2501_07056_gb300 import magnus
    A, B = _operands(kind)
    ref = oracle.spgemm(A, B, threads=8)
    dA = magnus.DeviceCSR.from_host(A)
    dB = dA if B is A else magnus.DeviceCSR.from_host(B)
    plan = magnus.Plan(dA, dB, magnus.make_params(force_category=force))
    nbytes = plan.workspace_size()
    assert nbytes > 0
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    base = ws.data_ptr()
    assert base % 256 == 0
    s = torch.cuda.current_stream().cuda_stream
    rp = torch.empty(A.n_rows + 1, dtype=torch.int64, device="cuda")
    # too small and misaligned workspaces are refused before any work: the
    # symbolic phase always needs its C.rowPtr scan temporaries (more than 8
    # bytes); a numeric phase needs scratch only for fine or coarse rows
    with pytest.raises(magnus.MagnusError) as ei:
        magnus.magnus_symbolic_ws(plan.handle, rp.data_ptr(), base, 8, s)
    assert ei.value.status == 10
    with pytest.raises(magnus.MagnusError) as ei:
        magnus.magnus_symbolic_ws(plan.handle, rp.data_ptr(), base + 8, nbytes, s)
    assert ei.value.status == 1
    nnz_ref = int(ref.row_ptr[-1])
    col = torch.empty(max(nnz_ref, 1), dtype=torch.int32, device="cuda")
    val = torch.empty(max(nnz_ref, 1), dtype=torch.float64, device="cuda")

    def both():
        n = magnus.magnus_symbolic_ws(plan.handle, rp.data_ptr(), base, nbytes, s)
        magnus.magnus_numeric_ws(plan.handle, dA.val.data_ptr(), dB.val.data_ptr(),
                                 rp.data_ptr(), col.data_ptr(), val.data_ptr(), base, nbytes, s)
        return n
    # the first call also loads the kernels' code (lazy module loading takes
    # device memory once); the second must leave device memory untouched
    both()
    before = _pool_state()
    nnz = both()
    after = _pool_state()
    assert after == before, "the _ws calls allocated device memory: %s -> %s" % (before, after)
    if force in (FINE, COARSE):
        with pytest.raises(magnus.MagnusError) as ei:
            magnus.magnus_numeric_ws(plan.handle, dA.val.data_ptr(), dB.val.data_ptr(),
                                     rp.data_ptr(), col.data_ptr(), val.data_ptr(), base, 8, s)
        assert ei.value.status == 10
    assert nnz == nnz_ref
    assert np.array_equal(rp.cpu().numpy(), ref.row_ptr)
    assert np.array_equal(col[:nnz].cpu().numpy(), ref.col)
    assert values_close(val[:nnz].cpu().numpy(), ref.val, ref.abs).all()
    # a row slab through the same workspace
    plan.c_row_ptr = rp
    plan.nnz_c = nnz
    r0, r1 = A.n_rows // 3, (2 * A.n_rows) // 3
    m = int(ref.row_ptr[r1] - ref.row_ptr[r0])
    sc = torch.empty(max(m, 1), dtype=torch.int32, device="cuda")
    sv = torch.empty(max(m, 1), dtype=torch.float64, device="cuda")
    plan.numeric_rows(r0, r1, sc, sv, workspace=ws[:nbytes])
    before = _pool_state()
    plan.numeric_rows(r0, r1, sc, sv, workspace=ws[:nbytes])
    after = _pool_state()
    assert after == before
    _check_slab(ref.row_ptr, ref, r0, r1, sc[:m].cpu().numpy(), sv[:m].cpu().numpy())
    plan.free()


def test_host_buffers_round_trip():
    """magnus_host_alloc buffers are page-locked host memory: asynchronous
    copies to and from the device return the data unchanged, and the region
    is released with the last tensor using it."""
    import torch
    from paper_2501_07056_gb300 import magnus
    x = np.arange(1 << 20, dtype=np.float64) * 0.5
    h = magnus.host_copy(x)
    assert h.is_pinned() and h.dtype == torch.float64 and np.array_equal(h.numpy(), x)
    d = h.to("cuda", non_blocking=True)
    out = magnus.host_empty(x.size, torch.float64)
    assert out.is_pinned()
    out.copy_(d * 2, non_blocking=True)
    torch.cuda.synchronize()
    assert np.array_equal(out.numpy(), 2 * x)
    e = magnus.host_empty(0, torch.int32)
    assert e.numel() == 0
    del h, out, e
    with pytest.raises(magnus.MagnusError):
        magnus._HostRegion(0)
