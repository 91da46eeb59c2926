"""Serving loop: SpGEMM requests admitted continuously and packed into
shared batched launches.

A request asks for C = A * B.  The server keeps the operands it was given
resident until the request completes, and runs a loop that

  * admits the requests that have arrived into a FIFO queue,
  * whenever one of its CUDA streams is idle, takes the oldest pending
    requests (up to a product and request budget) and plans them as one
    batch (``BatchPlan``: every launch serves the rows of all of them),
  * plans a batch only if an estimate of its plan and operands fits the
    device memory still free, then runs the symbolic phase, which gives the
    exact size of every C, and allocates the outputs and the numeric
    scratch only if they fit the free device memory (otherwise the batch
    waits, planned, until earlier batches retire and free theirs),
  * enqueues the numeric phase and goes on with the next batch on another
    stream, so batches overlap on the device, and
  * retires a batch when its completion event fires: each request's latency
    is completion time minus arrival time.

The free-memory figure counts the blocks PyTorch's caching allocator holds
unused, which the library's own stream-ordered pool cannot take: before the
library allocates, the server hands that cache back to the device when free
memory and the pool's idle bytes alone fall short.

The one-call-per-product server (``mode="single"``) runs the same loop with
one request at a time through the single-product API, on one stream.

Scheduling decisions live in ``Scheduler`` (host logic only, testable without
a GPU); ``Server`` drives the GPU.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float            # seconds after the start of the run
    products: int             # intermediate products (for budgets and rates)
    payload: object = None    # whatever the executor needs to build the operands
    start: float = -1.0       # when its batch was planned
    done: float = -1.0        # completion time
    nnz: int = -1
    batch: int = -1


class Scheduler:
    """FIFO admission and batch formation (no GPU).

    ``max_products`` / ``max_requests`` bound one batch.  Memory admission:
    with ``mem_source`` (a callable returning the device bytes new work may
    still use, read at every decision) a batch is admitted when what it
    still has to allocate fits that figure; otherwise ``mem_budget`` bounds
    the bytes of all batches in flight.  A batch is always admitted when
    nothing is in flight (it may then fail with an out-of-memory error
    instead of waiting forever)."""

    def __init__(self, max_products: int, max_requests: int, mem_budget: int | None = None,
                 mem_source=None):
        if mem_budget is None and mem_source is None:
            raise ValueError("need a memory budget or a source of free memory")
        self.max_products = max_products
        self.max_requests = max_requests
        self.mem_budget = mem_budget
        self.mem_source = mem_source
        self.pending: collections.deque = collections.deque()
        self.mem_in_use = 0
        self.in_flight = 0

    def admit(self, reqs):
        for r in reqs:
            self.pending.append(r)

    def peek_batch(self):
        """The requests next_batch would take, left pending."""
        out, prods = [], 0
        for r in self.pending:
            if len(out) >= self.max_requests or (out and prods + r.products > self.max_products):
                break
            out.append(r)
            prods += r.products
        return out

    def next_batch(self):
        """The oldest pending requests that fit one batch (at least one)."""
        out = self.peek_batch()
        for _ in out:
            self.pending.popleft()
        return out

    def fits(self, nbytes: int) -> bool:
        """Whether work that still has to allocate ``nbytes`` may start now."""
        if self.in_flight == 0:
            return True
        if self.mem_source is not None:
            return nbytes <= self.mem_source()
        return self.mem_in_use + nbytes <= self.mem_budget

    def reserve(self, nbytes: int) -> bool:
        """Admit a batch whose allocations still to come are ``nbytes`` if
        they fit (a batch is admitted when nothing else is in flight)."""
        if not self.fits(nbytes):
            return False
        self.mem_in_use += nbytes
        self.in_flight += 1
        return True

    def release(self, nbytes: int):
        self.mem_in_use -= nbytes
        self.in_flight -= 1


class _Flight:
    __slots__ = ("reqs", "plan", "event", "outputs", "operands", "nbytes", "stream", "batch",
                 "single")


class Server:
    """Drives the GPU.  ``executor`` builds a request's operands on the device:
    ``executor.operands(req, stream) -> (A: DeviceCSR, B: DeviceCSR)``."""

    def __init__(self, executor, params=None, mode="batched", n_streams=2,
                 max_products=1 << 31, max_requests=64, mem_budget=None,
                 mem_reserve=2 << 30, mem_source=None, keep_results=False, device="cuda"):
        """Admission is by free device memory (``free_memory()``, less
        ``mem_reserve`` bytes kept back), unless ``mem_source`` replaces that
        figure or a fixed ``mem_budget`` of bytes in flight is given."""
        import torch
        self.torch = torch
        self.executor = executor
        self.params = params
        self.mode = mode
        self.device = torch.device(device)
        self.mem_reserve = mem_reserve
        n = 1 if mode == "single" else max(1, n_streams)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(n)]
        if mem_budget is None and mem_source is None:
            mem_source = self.free_memory
        self.sched = Scheduler(max_products, 1 if mode == "single" else max_requests,
                               mem_budget=mem_budget, mem_source=mem_source)
        self.keep_results = keep_results
        self.results = {}
        self.executed_products = 0
        self.plan_waits = 0       # batches whose planning waited for memory
        self.launch_waits = 0     # planned batches whose launch waited for memory
        self.reclaims = 0         # times PyTorch's unused cache was handed back

    def free_memory(self) -> int:
        """Device bytes new work may use: free device memory, plus what the
        library's stream-ordered pool and PyTorch's caching allocator hold
        unused (each reuses its own first), less the reserve."""
        from . import magnus
        torch = self.torch
        free, pool_idle = magnus.magnus_device_memory()
        cached = torch.cuda.memory_reserved(self.device) - torch.cuda.memory_allocated(self.device)
        return free + pool_idle + cached - self.mem_reserve

    def _reclaim(self, nbytes: int):
        """PyTorch's cached blocks count in ``free_memory()``, but the
        library's stream-ordered pool cannot take them (nor can PyTorch reuse
        blocks cached on another server's streams).  When free device memory
        plus the pool's idle bytes, less the reserve, falls short of the
        ``nbytes`` that the next step allocates, PyTorch's unused cache goes
        back to the device first."""
        from . import magnus
        torch = self.torch
        cached = torch.cuda.memory_reserved(self.device) - torch.cuda.memory_allocated(self.device)
        if cached <= 0:
            return
        free, pool_idle = magnus.magnus_device_memory()
        if free + pool_idle - self.mem_reserve < nbytes:
            torch.cuda.empty_cache()
            self.reclaims += 1

    def _estimate(self, reqs) -> int:
        est = getattr(self.executor, "estimate_bytes", None)
        return sum(est(r) for r in reqs) if est is not None else 0

    # -- one batch -----------------------------------------------------------
    def _plan(self, reqs, stream, batch_id):
        from . import magnus
        torch = self.torch
        self._reclaim(self._estimate(reqs))
        f = _Flight()
        f.reqs, f.stream, f.batch = reqs, stream, batch_id
        with torch.cuda.stream(stream):
            ops = [self.executor.operands(r, stream) for r in reqs]
            f.operands = ops
            # a batch of one request takes the single-product path (packing
            # its operands would only add work)
            f.single = self.mode == "single" or len(reqs) == 1
            if f.single:
                A, B = ops[0]
                plan = magnus.Plan(A, B, self.params, stream)
                nnz = plan.symbolic()
                offs = [0, nnz]
            else:
                plan = magnus.BatchPlan([a for a, _ in ops], [b for _, b in ops], self.params, stream)
                offs = plan.symbolic()
        f.plan = plan
        info = plan.info()
        self.executed_products += info["n_interprod"]
        # still to allocate: C (row pointers, columns, values) and the
        # numeric phase's scratch
        f.nbytes = (12 * offs[-1] + 8 * (sum(a.n_rows for a, _ in ops) + 1)
                    + info["workspace_bytes"])
        for i, r in enumerate(reqs):
            r.nnz = offs[i + 1] - offs[i]
        return f

    def _launch(self, f):
        torch = self.torch
        self._reclaim(f.nbytes)
        with torch.cuda.stream(f.stream):
            f.outputs = f.plan.numeric()
            f.event = torch.cuda.Event()
            f.event.record(f.stream)

    def _retire(self, f, now):
        for r in f.reqs:
            r.done = now
        if self.keep_results:
            for i, r in enumerate(f.reqs):
                if f.single:
                    self.results[r.rid] = _host_csr(f.plan.A.n_rows, f.plan.B.n_cols,
                                                    f.plan.c_row_ptr, f.outputs[0], f.outputs[1])
                else:
                    C = f.plan.result(i)
                    self.results[r.rid] = _host_csr(C.n_rows, C.n_cols, C.row_ptr, C.col, C.val)
        f.plan.free()
        f.plan = f.outputs = f.operands = None
        self.sched.release(f.nbytes)

    # -- the loop --------------------------------------------------------------
    def run(self, requests, time_scale=1.0):
        """Open-loop run: request r arrives at r.arrival * time_scale seconds
        after the start.  Returns the requests with start/done filled."""
        torch = self.torch
        order = sorted(requests, key=lambda r: r.arrival)
        nxt = 0
        idle = list(self.streams)
        flights = []
        waiting = None           # a planned batch whose outputs do not fit yet
        batch_id = 0
        plan_blocked = False
        t0 = time.perf_counter()
        while nxt < len(order) or flights or waiting is not None or self.sched.pending:
            now = time.perf_counter() - t0
            arrived = []
            while nxt < len(order) and order[nxt].arrival * time_scale <= now:
                arrived.append(order[nxt])
                nxt += 1
            self.sched.admit(arrived)
            # retire finished batches
            still = []
            for f in flights:
                if f.event.query():
                    self._retire(f, time.perf_counter() - t0)
                    idle.append(f.stream)
                else:
                    still.append(f)
            flights = still
            progressed = False
            if waiting is not None and self.sched.reserve(waiting.nbytes):
                self._launch(waiting)
                flights.append(waiting)
                waiting = None
                progressed = True
            if (waiting is None and idle and self.sched.pending
                    and not self.sched.fits(self._estimate(self.sched.peek_batch()))):
                # planning the next batch waits for memory
                if not plan_blocked:
                    self.plan_waits += 1
                plan_blocked = True
            elif waiting is None and idle and self.sched.pending:
                plan_blocked = False
                reqs = self.sched.next_batch()
                stream = idle.pop()
                t = time.perf_counter() - t0
                for r in reqs:
                    r.start, r.batch = t, batch_id
                f = self._plan(reqs, stream, batch_id)
                batch_id += 1
                if self.sched.reserve(f.nbytes):
                    self._launch(f)
                    flights.append(f)
                else:
                    waiting = f
                    self.launch_waits += 1
                progressed = True
            if not progressed:
                if flights:
                    time.sleep(5e-5)
                elif nxt < len(order):
                    wait = order[nxt].arrival * time_scale - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 1e-3))
        torch.cuda.synchronize(self.device)
        self.makespan = time.perf_counter() - t0
        self.n_batches = batch_id
        return order


def _host_csr(n_rows, n_cols, rp, col, val):
    from .inputs import CSR
    return CSR(int(n_rows), int(n_cols), rp.cpu().numpy().astype(np.int64),
               col.cpu().numpy().astype(np.int32), val.cpu().numpy().astype(np.float64))


class StencilTimesRandom:
    """Operands of the served workload: A is the 27-point stencil on a k^3
    grid (kept resident per k), B is an n x n ragged matrix with b_kmin..b_kmax
    nonzeros per row drawn on the device from (seed, request's matrix id)."""

    def __init__(self, device="cuda", seed=0, b_kmin=4, b_kmax=16):
        self.device = device
        self.seed = seed
        self.b_kmin, self.b_kmax = b_kmin, b_kmax
        self.stencils = {}

    def estimate_bytes(self, req) -> int:
        """Device bytes planning a request takes before its C is sized: B
        (about (b_kmin + b_kmax) / 2 entries per row, 12 B each, plus row
        pointers), the plan's per-row arrays (about 48 B per row), its
        segment table (8 B per nonzero of the stencil) and the sort order of
        its products (at most 2 B per product)."""
        k = req.payload[0]
        n = k ** 3
        nnz_b = n * (self.b_kmin + self.b_kmax) // 2
        return 8 * (n + 1) + 12 * nnz_b + 48 * n + 8 * (3 * k - 2) ** 3 + 2 * req.products

    def operands(self, req, stream):
        from . import gen_device
        k, b_id = req.payload
        if k not in self.stencils:
            self.stencils[k] = gen_device.stencil27(k, self.device, stream)
        A = self.stencils[k]
        n = k ** 3
        B = gen_device.ragged(n, n, self.b_kmin, self.b_kmax, self.seed, b_id,
                              device=self.device, stream=stream)
        return A, B


def stencil_products(k: int, seed: int, b_id: int, b_kmin=4, b_kmax=16) -> int:
    """Exact intermediate products of stencil27(k) * ragged B (host, from the
    counter-based generator's row lengths): sum_j nnz(B_j) * (A's column j
    count), and the stencil is symmetric in structure."""
    from .inputs import _ragged_ctr_lengths
    n = k ** 3
    L = _ragged_ctr_lengths(n, n, b_kmin, b_kmax, seed, b_id)
    idx = np.arange(n, dtype=np.int64)
    z, y, x = idx // (k * k), (idx // k) % k, idx % k

    def cnt(v):
        return 1 + (v > 0).astype(np.int64) + (v < k - 1).astype(np.int64)
    deg = cnt(z) * cnt(y) * cnt(x)
    return int((L * deg).sum())


def make_requests(descs, seed=0, rate=1.0, exact=True, b_kmin=4, b_kmax=16):
    """Requests of the served workload from ``inputs.served_stream`` entries;
    arrival gaps are the unit-rate gaps divided by ``rate`` (requests/s).
    ``exact=False`` budgets each request by its expected product count,
    (b_kmin + b_kmax) / 2 * nnz(stencil), instead of counting it on the host;
    the executed product counts are then taken from the plans."""
    out, t = [], 0.0
    for d in descs:
        t += d["gap"] / rate
        k = d["k"]
        if exact:
            p = stencil_products(k, seed, d["b_id"], b_kmin, b_kmax)
        else:
            p = int(round((b_kmin + b_kmax) / 2 * (3 * k - 2) ** 3))
        out.append(Request(rid=d["req"], arrival=t, products=p, payload=(k, d["b_id"])))
    return out


def latency_stats(reqs):
    lat = np.array([r.done - r.arrival for r in reqs])
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3)}
