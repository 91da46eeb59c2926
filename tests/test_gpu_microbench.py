"""Building-block microbenchmark: the per-chunk accumulation it times gives
each chunk's unique indices and sums of a uniform stream (checked against a
numpy grouping), and the device stream equals its host twin."""
import numpy as np
import pytest

from paper_2501_07056_gb300 import inputs
from tests._util import values_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("n,m,lg", [(200000, 1 << 16, 4), (200000, 1 << 16, 8), (50000, 5000, 3),
                                    (300000, 1 << 20, 12), (1000, 7, 0)])
def test_chunk_accumulation(n, m, lg):
    import torch
    from paper_2501_07056_gb300 import gen_device, magnus
    col, val = gen_device.uniform_stream(n, m, 0, 5)
    hc, hv = inputs.uniform_stream(n, m, 0, 5)
    assert np.array_equal(col.cpu().numpy(), hc)
    assert np.array_equal(val.cpu().numpy().view(np.uint64), hv.view(np.uint64))
    res, oc, ov, nnz = magnus.microbench_chunks(col, val, m, lg)
    torch.cuda.synchronize()
    shift = res["chunk_len_log2"]
    assert res["n_chunks"] == (m + (1 << shift) - 1) >> shift
    assert res["copy_ms"] > 0 and res["reorder_ms"] > 0 and res["global_accumulate_ms"] > 0
    if res["n_chunks"] <= 4096:
        assert res["reorder_staged_ms"] > 0
    if shift > 13:
        assert res["accumulate_ms"] < 0
        return
    oc, ov, nnz = oc.cpu().numpy(), ov.cpu().numpy(), nnz.cpu().numpy()
    chunk = hc.astype(np.int64) >> shift
    counts = np.bincount(chunk, minlength=res["n_chunks"])
    starts = np.concatenate(([0], np.cumsum(counts)))
    for c in range(res["n_chunks"]):
        sel = chunk == c
        u, inv = np.unique(hc[sel], return_inverse=True)
        sums = np.zeros(u.size)
        np.add.at(sums, inv, hv[sel])
        abss = np.zeros(u.size)
        np.add.at(abss, inv, np.abs(hv[sel]))
        assert nnz[c] == u.size
        s0 = starts[c]
        assert np.array_equal(oc[s0:s0 + u.size], u)
        assert values_close(ov[s0:s0 + u.size], sums, abss).all()


def test_device_rates_are_consistent():
    """magnus_microbench_rates: every rate is positive; byte rates grow with
    the chunk size while chunk rates do not (a random gather costs at least
    one DRAM transaction); an 8-lanes-per-address FP64 atomic is slower than
    one at distinct addresses."""
    from paper_2501_07056_gb300 import magnus
    r = magnus.microbench_rates()
    assert r["sms"] > 0
    assert all(v > 0 for k, v in r.items() if k != "sms")
    assert r["gather_256"] * 256 > r["gather_32"] * 32
    assert r["gather_256"] <= r["gather_32"] * 1.1
    assert r["smem_f64_atomic_8_per_address"] < r["smem_f64_atomic_distinct"]
