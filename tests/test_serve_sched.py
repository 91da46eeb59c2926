"""Host logic of the serving loop (no GPU): FIFO batch formation under the
product and request budgets, output-memory admission, and when the server
hands PyTorch's unused cache back before the library allocates."""
from paper_2501_07056_gb300.serve import Request, Scheduler, make_requests, stencil_products
from paper_2501_07056_gb300 import inputs


def _reqs(prods):
    return [Request(rid=i, arrival=float(i), products=p) for i, p in enumerate(prods)]


def test_fifo_batches_respect_budgets():
    s = Scheduler(max_products=100, max_requests=3, mem_budget=1000)
    s.admit(_reqs([40, 40, 40, 10, 200, 5]))
    b1 = s.next_batch()
    assert [r.rid for r in b1] == [0, 1]          # 40 + 40 + 40 > 100
    b2 = s.next_batch()
    assert [r.rid for r in b2] == [2, 3]          # 10 fits, 200 does not
    b3 = s.next_batch()
    assert [r.rid for r in b3] == [4]             # an oversized request goes alone
    b4 = s.next_batch()
    assert [r.rid for r in b4] == [5]
    assert s.next_batch() == []


def test_request_count_budget():
    s = Scheduler(max_products=10 ** 9, max_requests=2, mem_budget=1)
    s.admit(_reqs([1, 1, 1, 1, 1]))
    assert [len(s.next_batch()) for _ in range(3)] == [2, 2, 1]


def test_memory_admission():
    s = Scheduler(max_products=10, max_requests=1, mem_budget=100)
    assert s.reserve(60)
    assert not s.reserve(60)       # would exceed the budget while 60 are in flight
    assert s.reserve(40)
    s.release(60)
    s.release(40)
    assert s.reserve(500)          # alone, an oversized batch is admitted
    assert not s.reserve(1)
    s.release(500)
    assert s.mem_in_use == 0


def test_admission_by_free_memory_waits_when_short():
    free = {"bytes": 100}
    s = Scheduler(max_products=10, max_requests=1, mem_source=lambda: free["bytes"])
    assert s.fits(10 ** 12)        # nothing in flight: always admitted
    assert s.reserve(80)           # the first batch (its memory is then allocated)
    free["bytes"] = 20
    assert not s.fits(50) and not s.reserve(50)   # short of memory: waits
    assert s.reserve(20)           # fits what is left
    free["bytes"] = 0
    assert not s.reserve(1)
    s.release(80)
    free["bytes"] = 80             # the retired batch's memory is free again
    assert s.reserve(50)
    s.release(20)
    s.release(50)
    assert s.in_flight == 0 and s.fits(10 ** 12)


def test_peek_matches_next_batch():
    s = Scheduler(max_products=100, max_requests=3, mem_budget=1)
    s.admit(_reqs([40, 40, 40, 10]))
    peek = [r.rid for r in s.peek_batch()]
    assert peek == [r.rid for r in s.next_batch()] == [0, 1]
    assert [r.rid for r in s.peek_batch()] == [2, 3]


def test_stencil_products_closed_form():
    # with every B row of length L, products = L * nnz(stencil) = L (3k-2)^3
    for k in (1, 2, 5):
        p = stencil_products(k, 0, 7, b_kmin=6, b_kmax=6)
        assert p == min(6, k ** 3) * (3 * k - 2) ** 3  # rows hold at most n columns
    # and against a direct count from the generated matrices
    k, b_id = 4, 3_000_011
    A = inputs.stencil27(k)
    B = inputs.ragged_ctr(k ** 3, k ** 3, 4, 16, 0, b_id)
    lens = __import__("numpy").diff(B.row_ptr)
    assert stencil_products(k, 0, b_id) == int(lens[A.col].sum())


def test_make_requests_arrivals():
    descs = inputs.served_stream(50, seed=0, k_lo=2, k_hi=5)
    reqs = make_requests(descs, rate=100.0)
    arr = [r.arrival for r in reqs]
    assert arr == sorted(arr) and arr[0] > 0
    assert abs(arr[-1] - sum(d["gap"] for d in descs) / 100.0) < 1e-9


def test_reclaim_decision_on_the_host(monkeypatch):
    """The server hands PyTorch's unused cache back only when it holds some
    and free device memory plus the library pool's idle bytes, less the
    reserve, is short of the bytes about to be allocated (fake memory
    figures, no GPU)."""
    from paper_2501_07056_gb300 import magnus, serve

    class FakeCuda:
        def __init__(self):
            self.reserved, self.allocated, self.emptied = 0, 0, 0

        def memory_reserved(self, dev=None):
            return self.reserved

        def memory_allocated(self, dev=None):
            return self.allocated

        def empty_cache(self):
            self.emptied += 1
            self.reserved = self.allocated

    class FakeTorch:
        cuda = FakeCuda()

    mem = {"free": 0, "idle": 0}
    monkeypatch.setattr(magnus, "magnus_device_memory", lambda: (mem["free"], mem["idle"]))
    srv = object.__new__(serve.Server)
    srv.torch, srv.device, srv.mem_reserve, srv.reclaims = FakeTorch, None, 100, 0
    cuda = FakeTorch.cuda

    # nothing cached: nothing to hand back, however short the library is
    srv._reclaim(10 ** 9)
    assert srv.reclaims == 0 and cuda.emptied == 0
    # cached blocks, and free + idle - reserve covers the request: kept
    cuda.reserved, cuda.allocated = 5000, 1000
    mem["free"], mem["idle"] = 600, 500
    srv._reclaim(1000)
    assert srv.reclaims == 0 and cuda.reserved == 5000
    # one byte more than that: handed back
    srv._reclaim(1001)
    assert srv.reclaims == 1 and cuda.emptied == 1 and cuda.reserved == 1000
