"""Autotuner: the chosen parameters compute the oracle's C, the search never
returns something slower than its starting point, repeated calls hit the
cache, and row sampling runs on a copy of evenly spaced row blocks."""
import numpy as np
import pytest

from paper_2501_07056_gb300 import inputs
from tests._gpu import assert_parity, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_autotune_mixed_rows():
    from paper_2501_07056_gb300 import magnus
    A = inputs.rmat(12, 16, seed=2, matrix_id=1)
    dA = magnus.DeviceCSR.from_host(A)
    best, rep = magnus.autotune(dA, dA, max_trials=12)
    assert 1 < rep["trials"] <= 12 and rep["from_cache"] == 0
    assert rep["best_ms"] <= rep["base_ms"]
    got = run_gpu(A, A, best, same=True)
    assert_parity(got, A, A)
    best2, rep2 = magnus.autotune(dA, dA, max_trials=12)
    assert rep2["from_cache"] == 1 and rep2["trials"] == 0
    assert magnus.params_dict(best2) == magnus.params_dict(best)


def test_autotune_sampled_rows():
    from paper_2501_07056_gb300 import magnus
    A = inputs.ragged(20000, 20000, 2, 40, seed=3, matrix_id=1)
    B = inputs.ragged(20000, 300000, 2, 40, seed=3, matrix_id=2)
    dA, dB = magnus.DeviceCSR.from_host(A), magnus.DeviceCSR.from_host(B)
    lens = np.diff(B.row_ptr)
    full = int(lens[A.col].sum())
    best, rep = magnus.autotune(dA, dB, sample_products=full // 10, max_trials=6)
    assert rep["products_full"] == full
    assert 0 < rep["sampled_rows"] < A.n_rows
    got = run_gpu(A, B, best)
    assert_parity(got, A, B)


def test_autotune_cache_keyed_by_base_params():
    # The same operands tuned from another starting point (a forced
    # category) are a separate cache entry, and the search keeps the base's
    # fixed choices.
    from paper_2501_07056_gb300 import magnus
    A = inputs.rmat(11, 16, seed=5, matrix_id=1)
    dA = magnus.DeviceCSR.from_host(A)
    _, rep = magnus.autotune(dA, dA, max_trials=3)
    base = magnus.make_params(force_category=3)
    best, rep2 = magnus.autotune(dA, dA, base, max_trials=3)
    assert rep2["from_cache"] == 0
    assert best.force_category == 3
    got = run_gpu(A, A, best, same=True)
    assert_parity(got, A, A)
    _, rep3 = magnus.autotune(dA, dA, base, max_trials=3)
    assert rep3["from_cache"] == 1


def test_autotune_batched():
    # tuned on a batch's packed products; a batch planned with the result
    # still computes every product's oracle C
    from paper_2501_07056_gb300 import magnus
    import oracle
    from tests._util import values_close
    rng = np.random.default_rng(5)
    ns = [int(x) for x in rng.integers(200, 3000, size=12)]
    As = [inputs.ragged(n, n, 2, 32, seed=11, matrix_id=2 * i + 1) for i, n in enumerate(ns)]
    Bs = [inputs.ragged(n, n, 2, 32, seed=11, matrix_id=2 * i + 2) for i, n in enumerate(ns)]
    dAs = [magnus.DeviceCSR.from_host(a) for a in As]
    dBs = [magnus.DeviceCSR.from_host(b) for b in Bs]
    bp = magnus.BatchPlan(dAs, dBs)
    best, rep = bp.autotune(max_trials=8)
    bp.free()
    assert 1 <= rep["trials"] <= 8 and rep["best_ms"] <= rep["base_ms"]
    bp = magnus.BatchPlan(dAs, dBs, best)
    bp.symbolic()
    bp.numeric()
    for i in range(len(ns)):
        C = bp.result(i)
        ref = oracle.spgemm(As[i], Bs[i], threads=8)
        assert np.array_equal(C.row_ptr.cpu().numpy(), ref.row_ptr)
        assert np.array_equal(C.col.cpu().numpy(), ref.col)
        assert values_close(C.val.cpu().numpy(), ref.val, ref.abs).all()
    bp.free()
