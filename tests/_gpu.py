"""GPU-side helpers for the parity tests: run the library through the C ABI
and compare with the CPU oracle under the parity rule."""
import numpy as np

import oracle
from tests._util import values_close


def run_gpu(A, B, params=None, same=False, keep_plan=False):
    import torch
    from paper_2501_07056_gb300 import magnus
    dA = magnus.DeviceCSR.from_host(A, "cuda")
    dB = dA if same else magnus.DeviceCSR.from_host(B, "cuda")
    plan = magnus.Plan(dA, dB, params)
    nnz = plan.symbolic()
    col, val = plan.numeric()
    torch.cuda.synchronize()
    out = dict(row_ptr=plan.c_row_ptr.cpu().numpy(), col=col.cpu().numpy(),
               val=val.cpu().numpy(), nnz=nnz, info=plan.info())
    if keep_plan:
        out["plan"] = plan
        out["dev"] = (dA, dB)
    else:
        plan.free()
    return out


def assert_parity(got, A, B, rows=None, threads=8):
    """Structure bit-exact, values within 1e-12 * max(|ref|, sum|terms|)."""
    ref = oracle.spgemm(A, B, rows=rows, threads=threads)
    if rows is None:
        assert np.array_equal(got["row_ptr"], ref.row_ptr), "row_ptr differs"
        assert np.array_equal(got["col"], ref.col), "columns differ"
        ok = values_close(got["val"], ref.val, ref.abs)
        assert ok.all(), "values differ at %s" % np.nonzero(~ok)[0][:10]
        return ref
    rp = got["row_ptr"]
    for t, i in enumerate(rows):
        s, e = int(rp[i]), int(rp[i + 1])
        rc, rv, ra = ref.row(t)
        assert e - s == rc.size, "row %d nnz %d vs %d" % (i, e - s, rc.size)
        assert np.array_equal(got["col"][s:e], rc), "row %d columns differ" % i
        ok = values_close(got["val"][s:e], rv, ra)
        assert ok.all(), "row %d values differ" % i
    return ref
