"""Bounded device waits report through magnus_device_status.

The coarse bucket sort waits on mbarriers for the bulk copies of its
buckets; every wait gives up after a bounded number of SM clocks, raises a
flag and ends its block.  magnus_wait_selftest makes one such wait run out
(an announced copy that is never issued, so no copy is ever in flight), and
the host must see MAGNUS_TIMEOUT once, then MAGNUS_OK, with the context
still usable for products checked against the oracle.
"""
import numpy as np
import pytest

from paper_2501_07056_gb300 import inputs
from tests._gpu import assert_parity, run_gpu

pytestmark = pytest.mark.gpu

MAGNUS_OK, MAGNUS_TIMEOUT = 0, 6


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_bounded_wait_reports_timeout_once():
    from paper_2501_07056_gb300 import magnus
    assert magnus.device_status() == MAGNUS_OK
    magnus.wait_selftest(1 << 20)  # about half a millisecond of SM clock
    assert magnus.device_status() == MAGNUS_TIMEOUT
    assert magnus.device_status() == MAGNUS_OK  # the flag is cleared
    # the context is still usable, including the coarse bucket sort
    A = inputs.ragged(300, 3000, 20, 60, seed=7, matrix_id=1)
    B = inputs.ragged(3000, 1 << 20, 10, 40, seed=7, matrix_id=2)
    got = run_gpu(A, B, magnus.make_params(force_category=3, coarse_bucket_sort=1,
                                           chunk_len_coarse_log2=19))
    assert_parity(got, A, B)
    assert magnus.device_status() == MAGNUS_OK


def test_symbolic_reports_a_pending_timeout():
    # a timeout raised before a symbolic call is reported by that call
    from paper_2501_07056_gb300 import magnus
    A = inputs.ragged(500, 500, 2, 10, seed=3, matrix_id=1)
    dA = magnus.DeviceCSR.from_host(A, "cuda")
    plan = magnus.Plan(dA, dA)
    try:
        magnus.wait_selftest(1 << 16)
        with pytest.raises(RuntimeError, match="timed out"):
            plan.symbolic()
        assert magnus.device_status() == MAGNUS_OK
        assert np.isfinite(plan.symbolic())
    finally:
        plan.free()
