"""The on-device input generators reproduce their host twins bit for bit."""
import numpy as np
import pytest

from paper_2501_07056_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _host(M):
    return (M.row_ptr.cpu().numpy(), M.col.cpu().numpy(), M.val.cpu().numpy())


@pytest.mark.parametrize("n,m,kmin,kmax,seed,mid", [
    (5000, 700, 2, 32, 0, 9),        # batched-workload row lengths
    (50, 20, 20, 32, 3, 1),          # rows filled by the smallest-unused rule
    (257, 256, 2, 32, 0, 7),         # smallest batched product size
    (70000, 70000, 4, 16, 0, 3000001),  # served-workload B
    (1, 5, 1, 1, 0, 0),
])
def test_ragged_matches_host(n, m, kmin, kmax, seed, mid):
    from paper_2501_07056_gb300 import gen_device
    D = gen_device.ragged(n, m, kmin, kmax, seed, mid)
    H = inputs.ragged_ctr(n, m, kmin, kmax, seed, mid)
    rp, c, v = _host(D)
    assert np.array_equal(rp, H.row_ptr)
    assert np.array_equal(c, H.col)
    assert np.array_equal(v.view(np.uint64), H.val.view(np.uint64))


@pytest.mark.parametrize("k", [1, 2, 3, 7, 16])
def test_stencil_matches_host(k):
    from paper_2501_07056_gb300 import gen_device
    D = gen_device.stencil27(k)
    H = inputs.stencil27(k)
    rp, c, v = _host(D)
    assert np.array_equal(rp, H.row_ptr)
    assert np.array_equal(c, H.col)
    assert np.array_equal(v, H.val)
    assert H.nnz == (3 * k - 2) ** 3


@pytest.mark.parametrize("n,m,k,mid", [(300, 1 << 20, 512, 1), (64, 1000, 1000, 2), (7, 5, 3, 3),
                                        (1000, 1 << 30, 37, 4)])
def test_stratified_matches_host(n, m, k, mid):
    from paper_2501_07056_gb300 import gen_device
    D = gen_device.stratified(n, m, k, 0, mid)
    H = inputs.stratified(n, m, k, 0, mid)
    rp, c, v = _host(D)
    assert np.array_equal(rp, H.row_ptr)
    assert np.array_equal(c, H.col)
    assert np.array_equal(v.view(np.uint64), H.val.view(np.uint64))
