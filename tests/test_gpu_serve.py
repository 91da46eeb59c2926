"""Serving loop on the GPU: every request's result, computed inside shared
batched launches while other requests are in flight, equals the oracle's and
the result of the same product computed alone (one call per product):
structure bit-exact, values within the parity rule."""
import numpy as np
import pytest

import oracle
from paper_2501_07056_gb300 import inputs
from tests._util import values_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _requests(count, rate, k_lo=3, k_hi=14):
    from paper_2501_07056_gb300 import serve
    descs = inputs.served_stream(count, seed=0, k_lo=k_lo, k_hi=k_hi)
    return serve.make_requests(descs, seed=0, rate=rate)


def _oracle(req):
    k, b_id = req.payload
    A = inputs.stencil27(k)
    B = inputs.ragged_ctr(k ** 3, k ** 3, 4, 16, 0, b_id)
    return oracle.spgemm(A, B)


def _same(C, ref):
    assert np.array_equal(C.row_ptr, ref.row_ptr)
    assert np.array_equal(C.col, ref.col)
    assert values_close(C.val, ref.val, ref.abs).all()


@pytest.mark.parametrize("mem_budget", [48 << 30, 1])
def test_results_alone_and_in_the_mix(mem_budget):
    from paper_2501_07056_gb300 import serve
    reqs = _requests(40, rate=4000.0)
    mix = serve.Server(serve.StencilTimesRandom(), mode="batched", n_streams=3,
                       max_requests=8, mem_budget=mem_budget, keep_results=True)
    mix.run(reqs)
    assert all(r.done >= r.arrival for r in reqs)
    assert mix.n_batches < len(reqs)  # requests shared launches
    alone = serve.Server(serve.StencilTimesRandom(), mode="single", keep_results=True)
    reqs2 = _requests(40, rate=4000.0)
    alone.run(reqs2)
    for r, r2 in zip(reqs, reqs2):
        ref = _oracle(r)
        _same(mix.results[r.rid], ref)
        _same(alone.results[r2.rid], ref)
        assert r.nnz == r2.nnz == ref.row_ptr[-1]


def test_config_grid_sizes_alone_and_in_the_mix():
    """Requests at the served workload's own grid sizes, k in {16..96}: the
    smallest and the largest k (884,736 rows, 2.3e8 products) share batches
    with sizes between them; every result equals the oracle's and the one
    computed alone."""
    from paper_2501_07056_gb300 import serve
    ks = [16, 96, 33, 80, 16, 57, 96, 24, 70, 45]
    rng = np.random.default_rng(3)
    descs = [dict(req=i, k=k, b_id=3_000_000 + i, gap=float(g))
             for i, (k, g) in enumerate(zip(ks, rng.exponential(1.0, len(ks))))]
    # all arrive at once: the first batches take requests in order, so k = 16
    # and k = 96 share the first two batches
    reqs = serve.make_requests(descs, seed=0, rate=1e12)
    mix = serve.Server(serve.StencilTimesRandom(), mode="batched", n_streams=3,
                       max_requests=4, keep_results=True)
    mix.run(reqs)
    assert mix.n_batches < len(reqs)
    by = {r.rid: r for r in reqs}
    assert by[0].batch == by[1].batch and by[4].batch == by[6].batch
    alone = serve.Server(serve.StencilTimesRandom(), mode="single", keep_results=True)
    reqs2 = serve.make_requests(descs, seed=0, rate=1e12)
    alone.run(reqs2)
    for r, r2 in zip(sorted(reqs, key=lambda q: q.rid), sorted(reqs2, key=lambda q: q.rid)):
        ref = _oracle(r)
        _same(mix.results[r.rid], ref)
        _same(alone.results[r2.rid], ref)


def test_waits_when_free_memory_is_short():
    """A memory figure that never admits a second batch: batches run one at
    a time (each planned only after the previous one retired), and every
    result still equals the oracle's."""
    from paper_2501_07056_gb300 import serve
    reqs = _requests(12, rate=1e12)
    srv = serve.Server(serve.StencilTimesRandom(), mode="batched", n_streams=3,
                       max_requests=3, mem_source=lambda: 0, keep_results=True)
    srv.run(reqs)
    assert srv.n_batches >= 4 and srv.plan_waits >= 1
    spans = {}
    for r in reqs:
        s0, d0 = spans.get(r.batch, (r.start, r.done))
        spans[r.batch] = (min(s0, r.start), max(d0, r.done))
    order = [spans[b] for b in sorted(spans)]
    for (s0, d0), (s1, d1) in zip(order, order[1:]):
        assert s1 >= d0  # the next batch started after the previous retired
    for r in reqs:
        _same(srv.results[r.rid], _oracle(r))


def test_free_memory_figure():
    import torch
    from paper_2501_07056_gb300 import magnus, serve
    free, idle = magnus.magnus_device_memory()
    assert 0 < free <= torch.cuda.get_device_properties(0).total_memory and idle >= 0
    srv = serve.Server(serve.StencilTimesRandom(), mem_reserve=0)
    assert srv.free_memory() >= free


def test_reclaims_pytorch_cache_when_the_library_is_short():
    """Blocks PyTorch cached on another stream count as free memory but the
    library's pool cannot take them: when the library's own figure is short,
    the server hands them back before it allocates; when it is not, it keeps
    them."""
    import torch
    from paper_2501_07056_gb300 import serve
    dev = torch.device("cuda", 0)
    side = torch.cuda.Stream(dev)
    with torch.cuda.stream(side):
        x = torch.empty(64 << 20, dtype=torch.uint8, device=dev)
    del x
    torch.cuda.synchronize()

    def cached():
        return torch.cuda.memory_reserved(dev) - torch.cuda.memory_allocated(dev)
    before = cached()
    assert before >= 64 << 20
    roomy = serve.Server(serve.StencilTimesRandom(), mem_reserve=0)
    roomy._reclaim(1 << 20)
    assert roomy.reclaims == 0 and cached() == before
    total = torch.cuda.get_device_properties(dev).total_memory
    short = serve.Server(serve.StencilTimesRandom(), mem_reserve=total)
    short._reclaim(1 << 20)
    assert short.reclaims == 1
    # the side stream's block was a segment of its own; segments that still
    # hold live blocks of earlier tests stay
    assert cached() <= before - (64 << 20)


def test_latency_accounting():
    from paper_2501_07056_gb300 import serve
    reqs = _requests(30, rate=200.0, k_lo=3, k_hi=8)
    srv = serve.Server(serve.StencilTimesRandom(), mode="batched", n_streams=2, max_requests=4)
    srv.run(reqs)
    st = serve.latency_stats(reqs)
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    # open loop: nothing starts before it arrives
    assert all(r.start >= r.arrival - 1e-9 for r in reqs)
    assert srv.makespan >= reqs[-1].arrival
