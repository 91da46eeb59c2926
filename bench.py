#!/usr/bin/env python
"""Benchmark of the MAGNUS SpGEMM hot path on GB300.

Workload (one step = the whole hot path on one product): C = A*A with A a
uniform random square matrix, n = 2^24, exactly 8 distinct uniform columns per
row, FP64 values U(-1, 1), seed 0 (1.07e9 intermediate products).  A step is
plan (setup, Section 3.1) + symbolic (Section 2.1) + allocation of C +
numeric (Algorithms 1-4) + freeing the plan, timed with CUDA events on the
calling stream.  The
inputs (1.6 GB) are larger than the 126 MB L2, so no flush is needed between
steps.

Output: one JSON line (rank 0).  ``value`` is whole-job GFLOP/s
(2 x intermediate products / s, Section 5 definition of n_interProd), ``e2e``
the same metric through the public API with host buffers (H2D of A and D2H of
C inside the timed region; C is computed in row slabs by magnus_numeric_rows
and each slab is copied back while the next computes, magnus.spgemm_host),
``roofline`` the dominant kernel's algorithmic bytes per launch over its
measured duration against the measured HBM copy bandwidth, ``cpu_baseline``
the CPU oracle on a bounded row sample.

Other workloads (``--workload``): uniform4096 and uniform2^22 (smaller
uniform), rmat20 / rmat18 / rmat16 (R-MAT, edge factor 16), massive20..30
(the nonsquare uniform workload of Section 4.3), batched4096 (many
independent products, batched plans against one call per product), served
(open-loop request stream, continuous batching against one call per
product, p50/p99 latency) and ablation (the building-block microbenchmark).

``--impl reference`` times the CPU oracle instead (the reference arm): each
step is the oracle on a bounded sample of the same workload on all host cores.

Multi-GPU: rows of C are independent, but every product here fits one GPU,
so N GPUs run N replicas of the workload (weak scaling); ranks synchronise
with a barrier and the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "uniform2^24": "C=A*A, A uniform random square n=2^24, 8 distinct uniform cols/row, "
                   "FP64 U(-1,1), int32 cols, seed 0",
    "uniform2^22": "C=A*A, A uniform random square n=2^22, 8 distinct uniform cols/row, "
                   "FP64 U(-1,1), int32 cols, seed 0",
    "uniform4096": "C=A*A, A uniform random square n=4096, 8 distinct uniform cols/row, "
                   "FP64 U(-1,1), int32 cols, seed 0",
    "rmat20": "C=A*A, A R-MAT scale 20, edge factor 16, (a,b,c)=(.57,.19,.19), "
              "duplicates merged, FP64 U(0,1), seed 0",
    "rmat18": "C=A*A, A R-MAT scale 18, edge factor 16, (a,b,c)=(.57,.19,.19), "
              "duplicates merged, FP64 U(0,1), seed 0",
    "rmat16": "C=A*A, A R-MAT scale 16, edge factor 16, (a,b,c)=(.57,.19,.19), "
              "duplicates merged, FP64 U(0,1), seed 0 (profiling size)",
    "served": "open-loop stream of SpGEMM requests, Poisson arrivals, each C=A*B with A the "
              "27-point stencil on a k^3 grid (k uniform in {16..96}) and B n x n (n=k^3) with "
              "nnz/row uniform in {4..16} (counter-based generator, drawn on the device), FP64, "
              "seed 0",
    "massive20": "C=A*B, A 4096 x 2^21 and B 2^21 x 2^20, 512 stratified-uniform cols/row in "
                 "both (counter-based generator, drawn on the device), FP64 U(-1,1), seed 0",
    "massive24": "C=A*B, A 4096 x 2^21 and B 2^21 x 2^24, 512 stratified-uniform cols/row in "
                 "both (counter-based generator, drawn on the device), FP64 U(-1,1), seed 0",
    "massive28": "C=A*B, A 4096 x 2^21 and B 2^21 x 2^28, 512 stratified-uniform cols/row in "
                 "both (counter-based generator, drawn on the device), FP64 U(-1,1), seed 0",
    "massive30": "C=A*B, A 4096 x 2^21 and B 2^21 x 2^30, 512 stratified-uniform cols/row in "
                 "both (counter-based generator, drawn on the device), FP64 U(-1,1), seed 0",
    "ablation": "building blocks of one reorder level (histogram, scan, reorder, per-chunk "
                "dense accumulation) on a uniform stream of 2^28 (int32 index, FP64 value) "
                "pairs with indices in [0, 2^16), [0, 2^20) and [0, 2^24), against a stream "
                "copy and a global dense accumulator; chunk count swept 2^0..2^14",
    "rates": "device rates that bound the kernels: random gathers of 16-256 byte chunks and "
             "of 8-entry CSR B rows from 2 GB arrays, shared-memory FP64 and u32 accumulation "
             "(distinct, random and 8-lanes-per-address atomics, plain adds)",
    "batched4096": "4096 independent products C_i=A_i*B_i, n_i log-uniform in [256, 65536], "
                   "A_i and B_i n_i x n_i with nnz/row uniform in {2..32} (counter-based "
                   "generator, drawn on the device), FP64 U(-1,1), seed 0",
}
CPU_SAMPLE_PRODUCTS = 1 << 29   # cpu_baseline: about 2-15 s of oracle time
E2E_BLOCKS = 8                  # e2e: row slabs of C copied back while the next computes
REF_STEP_PRODUCTS = 1 << 27     # reference arm: one step
PROFILE_DIR = os.path.join(ROOT, "profiles")


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="uniform2^24", choices=sorted(WORKLOADS))
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--e2e-blocks", type=int, default=E2E_BLOCKS,
                   help="e2e: row slabs of C whose entries are copied back while the next "
                        "compute")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-configs", action="store_true",
                   help="default workload only: skip the R-MAT 20, batched and served lines "
                        "appended under detail.configs")
    p.add_argument("--force-category", type=int, default=-1)
    p.add_argument("--sort-threshold", type=int, default=0)
    p.add_argument("--chunk-coarse", type=int, default=0,
                   help="log2 of the coarse chunk length (0 = planner's choice)")
    p.add_argument("--chunk-fine", type=int, default=0,
                   help="log2 of the fine chunk length (0 = planner's choice)")
    p.add_argument("--dthr", type=int, default=0,
                   help="fine-level hybrid threshold (0 = planner's choice; 1 = dense only)")
    p.add_argument("--chunk-accumulator", type=int, default=0, choices=[0, 1],
                   help="fine-level chunk accumulator: 0 dense array, 1 hash map")
    p.add_argument("--coarse-reorder", type=int, default=0, choices=[0, 1, 2],
                   help="coarse staging: 0 automatic, 1 outer product, 2 row-wise runs")
    p.add_argument("--coarse-bucket-sort", type=int, default=0, choices=[-1, 0, 1],
                   help="coarse buckets of 257..2048 products: block sort 1, off -1, "
                        "0 automatic")
    p.add_argument("--batch-count", type=int, default=4096,
                   help="batched workload: number of products")
    p.add_argument("--batch-waves", type=int, default=4,
                   help="batched workload: products are planned in this many waves")
    p.add_argument("--requests", type=int, default=2000,
                   help="served workload: number of requests")
    p.add_argument("--rho", type=float, default=0.8,
                   help="served workload: offered load as a fraction of the one-call capacity")
    p.add_argument("--rho-high", type=float, default=1.1,
                   help="served workload: a second, overloading offered load (0 = skip)")
    p.add_argument("--autotune", type=int, default=0,
                   help="1 = run magnus_autotune (row sample of about 2^27 products, at most "
                        "16 runs; batched workload: magnus_autotune_batched on the first "
                        "wave, 2^28 products) before the warm-up and time its choice")
    p.add_argument("--numeric-graph", type=int, default=0,
                   help="1 = capture the numeric phase in a CUDA graph")
    p.add_argument("--l2-fetch", type=int, default=0,
                   help="L2 fetch granularity hint in bytes (0 = leave the setting alone)")
    return p.parse_args(argv)


# ---------------------------------------------------------------------------
# multi-rank plumbing (torchrun: one process per GPU)

class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local_rank)
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg is not None:
            self.pg.barrier()

    def max(self, x: float) -> float:
        return self._reduce(x, "max")

    def sum(self, x: float) -> float:
        return self._reduce(x, "sum")

    def _reduce(self, x, op):
        if self.pg is None:
            return float(x)
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX if op == "max" else self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg is not None:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("index,timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append(dict(sm=float(parts[2]), smax=float(parts[3]),
                                 power=float(parts[4]) if parts[4] not in ("[N/A]", "N/A") else None,
                                 hw=parts[6], hwt=parts[7], swt=parts[8], swp=parts[9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        pw = [r["power"] for r in rows if r["power"] is not None]
        return {"sm_mhz": statistics.median(r["sm"] for r in rows),
                "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(pw) if pw else None}


# ---------------------------------------------------------------------------
# roofline bookkeeping

def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


SORT_KERNEL_SOURCES = ("kernels_sort.cu", "sort_accum.cuh", "common.cuh", "internal.h")
COARSE_KERNEL_SOURCES = ("kernels_coarse.cu", "fine_level.cuh", "block_accum.cuh",
                         "sort_accum.cuh", "common.cuh", "internal.h")


def csrc_hash(files=SORT_KERNEL_SOURCES) -> str:
    """Hash of the sources that define the profiled kernel (not of the host
    orchestration), so a stored ncu figure is used only for that code."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2501_07056_gb300", "csrc")
    for fn in files:
        with open(os.path.join(d, fn), "rb") as f:
            h.update(fn.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_tag: str, workload: str, sources=SORT_KERNEL_SOURCES):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    path = os.path.join(PROFILE_DIR, "%s_%s.md" % (kernel_tag, workload.replace("^", "")))
    try:
        text = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("csrc_sha256") != csrc_hash(sources):
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def numeric_sort_alg_bytes(n_rows, nnz_a, n_inter, nnz_c):
    """Algorithmic bytes of the numeric sort-row kernel (Eq. 8-9 split by
    phase): A.rowPtr and C.rowPtr (8 B per row each), A.col + A.val (12 B)
    and the begin/end B.rowPtr of its B row (16 B) per nonzero of A, B.col +
    B.val per intermediate product (12 B), C.col + C.val per nonzero of C
    (12 B)."""
    return 16 * (n_rows + 1) + 28 * nnz_a + 12 * n_inter + 12 * nnz_c


def coarse_big_alg_bytes(products, nnz, buckets):
    """Algorithmic bytes of the large-bucket accumulator of the coarse level:
    every staged product of those buckets is read once (4 B chunk-local
    column + 8 B value), every entry of C they produce is written once
    (12 B), and each bucket reads its staging offsets, output offset and row
    pointer (24 B)."""
    return 12 * products + 12 * nnz + 24 * buckets


def ideal_bytes(n_rows, nnz_a, n_inter, nnz_c):
    """Eq. 8 + Eq. 9 with s_rowPtr = 8, s_colIdx = 4, s_val = 8."""
    read = 2 * (n_rows + 1) * 8 + nnz_a * (4 * 8 + 2 * 4 + 8) + n_inter * (2 * 4 + 8)
    write = (n_rows + 1) * 8 + nnz_c * (4 + 8)
    return read + write


def workload_config(args, n_rows, nnz_a, n_inter, dist):
    return {"workload": WORKLOADS[args.workload], "n": n_rows, "nnz_a": nnz_a,
            "n_interprod": int(n_inter),
            "parallelism": "replicas" if dist.world > 1 else "single",
            "l2": "inputs larger than L2 (A and B exceed the 126 MB L2), no flush",
            "step": "plan+symbolic+alloc C+numeric+free plan"}


# The paper's massive nonsquare uniform workload (Section 4.3): C has 4096
# rows and m_C columns; A is 4096 x K, B is K x m_C, 512 nonzeros per row in
# both (the paper uses 2048 with float values; 512 with FP64 keeps B and C
# within one GPU).
MASSIVE_ROWS, MASSIVE_K, MASSIVE_NNZ = 4096, 1 << 21, 512


def massive_operands(name, dev):
    from paper_2501_07056_gb300 import gen_device
    m_c = 1 << int(name[len("massive"):])
    dA = gen_device.stratified(MASSIVE_ROWS, MASSIVE_K, MASSIVE_NNZ, 0, 1, device=dev)
    dB = gen_device.stratified(MASSIVE_K, m_c, MASSIVE_NNZ, 0, 2, device=dev)
    return dA, dB


def massive_host(name, max_products):
    """Host A and the rows of B referenced by a sample of A's rows."""
    from paper_2501_07056_gb300 import inputs
    m_c = 1 << int(name[len("massive"):])
    A = inputs.stratified(MASSIVE_ROWS, MASSIVE_K, MASSIVE_NNZ, 0, 1)
    n = max(1, min(MASSIVE_ROWS, max_products // (MASSIVE_NNZ * MASSIVE_NNZ)))
    rows = (np.arange(n, dtype=np.int64) * (MASSIVE_ROWS // n)).astype(np.int64)
    need = np.unique(np.concatenate([A.col[A.row_ptr[r]:A.row_ptr[r + 1]] for r in rows]))
    B = inputs.stratified(MASSIVE_K, m_c, MASSIVE_NNZ, 0, 2, rows=need)
    return A, B, rows


# ---------------------------------------------------------------------------

def row_products(A, B=None):
    B = A if B is None else B
    lens = np.diff(B.row_ptr)
    per_nz = lens[A.col].astype(np.int64)
    cs = np.concatenate(([0], np.cumsum(per_nz)))
    return cs[A.row_ptr[1:]] - cs[A.row_ptr[:-1]]


def sample_rows(A, max_products, n_blocks=64):
    """Rows of n_blocks evenly spaced equal row blocks holding at most
    max_products intermediate products (all rows if they fit; one row per
    block if even that exceeds the budget)."""
    P = row_products(A)
    if P.sum() <= max_products:
        return np.arange(A.n_rows, dtype=np.int64), int(P.sum())
    cs = np.concatenate(([0], np.cumsum(P)))
    starts = (np.arange(n_blocks) * (A.n_rows // n_blocks)).astype(np.int64)
    lo, hi = 1, max(1, A.n_rows // n_blocks)
    while lo < hi:  # largest block length within the budget
        mid = (lo + hi + 1) // 2
        if int((cs[starts + mid] - cs[starts]).sum()) <= max_products:
            lo = mid
        else:
            hi = mid - 1
    rows = (starts[:, None] + np.arange(lo)[None, :]).reshape(-1)
    return rows, int(P[rows].sum())


def cpu_oracle_rate(A, rows, threads, B=None):
    import oracle
    B = A if B is None else B
    prods = int(row_products(A, B)[rows].sum())
    t0 = time.perf_counter()
    oracle.spgemm(A, B, rows=rows, threads=threads)
    dt = time.perf_counter() - t0
    return 2.0 * prods / dt / 1e9, prods, dt


def run_reference_products(args, dist):
    """Reference arm of the batched and served workloads: the CPU oracle on
    all host cores over a bounded sample of products (regenerated on the host
    from the counter-based generator), one product after another, in the
    metric of our arm (GFLOP/s for batched, products/s for served)."""
    import oracle
    from paper_2501_07056_gb300 import inputs, serve
    threads = os.cpu_count() or 1
    if args.workload == "batched4096":
        ns = inputs.batched_sizes(args.batch_count, seed=0)
        probs = [(int(n), 2 * i + 1, 2 * i + 2) for i, n in enumerate(ns)][:16]

        def make(p):
            n, ia, ib = p
            return (inputs.ragged_ctr(n, n, 2, 32, 0, ia), inputs.ragged_ctr(n, n, 2, 32, 0, ib))
        metric, unit = "SpGEMM GFLOP/s", "GFLOP/s"
    else:
        descs = inputs.served_stream(args.requests, seed=0)[:4]
        probs = [(d["k"], d["b_id"]) for d in descs]

        def make(p):
            k, b_id = p
            return inputs.stencil27(k), inputs.ragged_ctr(k ** 3, k ** 3, 4, 16, 0, b_id)
        metric, unit = "served products/s", "products/s"
    mats = [make(p) for p in probs]
    flops = sum(2 * int(row_products(A, B).sum()) for A, B in mats)
    total_t = 0.0
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for A, B in mats:
            oracle.spgemm(A, B, threads=threads)
        if step >= args.warmup:
            total_t += time.perf_counter() - t0
    per_step = total_t / args.steps
    value = (flops / per_step / 1e9) if unit == "GFLOP/s" else len(mats) / per_step
    sample = "the first %d products of the workload, one after another" % len(mats)
    return {
        "impl": "reference", "metric": metric, "value": value, "unit": unit,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "products": len(mats)},
        "cpu_baseline": {"value": value, "unit": unit, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_reference(args, dist):
    """Reference arm: the CPU oracle as it stands on all host cores, each step
    a bounded row sample of the workload."""
    from paper_2501_07056_gb300 import inputs
    if dist.rank != 0:
        return None
    if args.workload in ("batched4096", "served"):
        return run_reference_products(args, dist)
    if args.workload == "ablation":
        return {"impl": "reference",
                "unavailable": "the building-block microbenchmark has no CPU program to compare"}
    threads = os.cpu_count() or 1
    if args.workload.startswith("massive"):
        A, B, rows = massive_host(args.workload, REF_STEP_PRODUCTS)
    else:
        A, B = inputs.workload(args.workload)
        rows, _ = sample_rows(A, REF_STEP_PRODUCTS)
    for _ in range(args.warmup):
        cpu_oracle_rate(A, rows, threads, B)
    rates, total_prods, total_t = [], 0, 0.0
    for _ in range(args.steps):
        r, prods, dt = cpu_oracle_rate(A, rows, threads, B)
        rates.append(r)
        total_prods += prods
        total_t += dt
    value = 2.0 * total_prods / total_t / 1e9
    sample = ("%d rows of the workload in 64 evenly spaced row blocks (%d products per step), "
              "C rows via Eq. 1" % (rows.size, total_prods // args.steps))
    return {
        "impl": "reference", "metric": "SpGEMM GFLOP/s", "value": value, "unit": "GFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, A.n_rows, A.nnz, int(row_products(A, B).sum())
                                  if not args.workload.startswith("massive") else -1, dist),
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def run_ours(args, dist):
    import torch

    from paper_2501_07056_gb300 import inputs, magnus

    dev = torch.device("cuda", dist.local_rank if dist.world > 1 else 0)
    torch.cuda.set_device(dev)
    magnus._lib()  # fail loudly if the library is missing
    massive = args.workload.startswith("massive")
    if massive:
        A = None
        dA, dB = massive_operands(args.workload, dev)
    else:
        A, _ = inputs.workload(args.workload)
        dA = magnus.DeviceCSR.from_host(A, dev)
        dB = dA
    torch.cuda.synchronize()
    params = magnus.make_params(force_category=args.force_category,
                                sort_threshold=args.sort_threshold,
                                chunk_len_coarse_log2=args.chunk_coarse,
                                chunk_len_fine_log2=args.chunk_fine,
                                dense_chunk_threshold=args.dthr,
                                chunk_accumulator=args.chunk_accumulator,
                                coarse_reorder=args.coarse_reorder,
                                coarse_bucket_sort=args.coarse_bucket_sort,
                                l2_fetch_bytes=args.l2_fetch)
    stream = torch.cuda.current_stream()
    tuned = None
    if args.autotune:
        t0 = time.perf_counter()
        params, rep = magnus.autotune(dA, dB, params, sample_products=1 << 27, max_trials=16,
                                      stream=stream)
        tuned = {"report": rep, "seconds": time.perf_counter() - t0,
                 "params": magnus.params_dict(params)}
        torch.cuda.empty_cache()

    # The end-to-end leg runs first, in the process as it starts: device
    # memory released and mapped again (the device loop's plans and outputs)
    # slows the copy engines for a while afterwards, which would charge the
    # host-link copies with the device loop's bookkeeping.
    e2e = None
    if not args.no_e2e and not massive:
        sizing = magnus.Plan(dA, dB, params, stream)
        nnz_e2e = sizing.symbolic()
        n_inter_e2e = sizing.info()["n_interprod"]
        sizing.free()
        torch.cuda.synchronize()
        e2e = run_e2e(args, dist, A, dev, params, n_inter_e2e, nnz_e2e)

    stage = {k: [] for k in magnus.STAGES}

    def retire(keep, record):
        # The previous step's plan: its stage times (reading them waits for
        # its numeric pass to complete), then it is freed, before the next
        # step plans, as one call per product (magnus.spgemm) does.  Keeping
        # it alive while the next plan is built cost about 0.9 ms per step.
        old = keep.pop(0)
        if record:
            for k, v in old.stage_times().items():
                stage[k].append(v)
        old.free()

    def step(keep, record):
        while keep:
            retire(keep, record)
        plan = magnus.Plan(dA, dB, params, stream)
        plan.enable_timing(True)
        plan.symbolic()
        c_col, c_val = plan.numeric()
        # C is dropped once its computation is enqueued; the caching allocator
        # reuses the memory in stream order for the next step's C
        del c_col, c_val
        keep.append(plan)
        return plan

    # warm-up (also gives the sizes)
    keep = []
    for _ in range(args.warmup):
        plan = step(keep, False)
        torch.cuda.synchronize()
    info = plan.info()
    nnz_c = info["nnz_c"]
    n_inter = info["n_interprod"]
    while keep:
        retire(keep, False)
    torch.cuda.synchronize()

    clocks = ClockSampler(dev.index).start()
    dist.barrier()
    torch.cuda.synchronize()
    n_launch0 = magnus.magnus_launch_count()
    # one event per step boundary: the total, and the mean / median / min of
    # the single steps
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record(stream)
    for i in range(args.steps):
        step(keep, True)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    n_launch = magnus.magnus_launch_count() - n_launch0
    clk = clocks.stop()
    ms_local = evs[0].elapsed_time(evs[-1])
    step_list = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    while keep:
        retire(keep, True)
    ms_max = dist.max(ms_local)
    total_units = dist.sum(2.0 * n_inter * args.steps)
    value = total_units / (ms_max * 1e-3) / 1e9
    stage_ms = {k: (sum(v) / len(v) if v else 0.0) for k, v in stage.items()}

    # roofline of the dominant kernel: the numeric sort-row kernel, or the
    # large-bucket accumulator when the coarse level carries the work
    peak, peak_kind = peak_hbm()
    if stage_ms["num_coarse"] > stage_ms["num_sort"]:
        kern_ms = stage_ms["num_coarse_big"]
        alg = coarse_big_alg_bytes(info["coarse_dense_products"], info["coarse_dense_nnz"],
                                   info["coarse_dense_buckets"])
        kernel = "k_bucket_dense numeric (coarse buckets of > 256 products)"
        traffic = profiled_traffic("bucket_dense_numeric", args.workload, COARSE_KERNEL_SOURCES)
    else:
        kern_ms = stage_ms["num_sort"]
        alg = numeric_sort_alg_bytes(dA.n_rows, dA.nnz, n_inter, nnz_c)
        kernel = "k_sort_rows numeric"
        traffic = profiled_traffic("sort_rows_numeric", args.workload)
    achieved = alg / (kern_ms * 1e-3) / 1e9 if kern_ms > 0 else 0.0
    t_ideal_ms = ideal_bytes(dA.n_rows, dA.nnz, n_inter, nnz_c) / (peak * 1e9) * 1e3

    result = {
        "metric": "SpGEMM GFLOP/s", "value": value, "unit": "GFLOP/s", "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(args, dA.n_rows, dA.nnz, n_inter, dist),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": kernel,
                     "alg_bytes_per_launch": alg, "kernel_ms": kern_ms,
                     "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind
                     if peak_kind == "measured" else "fallback 6.8 TB/s"},
        "clocks": clk,
        "gpu_launches": n_launch,
        "detail": {"nnz_c": nnz_c, "autotune": tuned,
                   "stage_ms": stage_ms,
                   "step_ms": {"mean": statistics.mean(step_list),
                               "median": statistics.median(step_list), "min": min(step_list)},
                   "t_over_t_ideal": (ms_max / args.steps) / t_ideal_ms,
                   "t_ideal_ms": t_ideal_ms, "rows_per_category": info["rows_per_category"],
                   "sort_threshold": info["sort_threshold"]},
    }
    if e2e is not None:
        result["e2e"] = e2e
    if not args.no_cpu and dist.rank == 0:
        threads = os.cpu_count() or 1
        if massive:
            A, Bh, rows = massive_host(args.workload, 1 << 26)
        else:
            Bh = A
            rows, _ = sample_rows(A, CPU_SAMPLE_PRODUCTS)
        rate, prods, dt = cpu_oracle_rate(A, rows, threads, Bh)
        result["cpu_baseline"] = {
            "value": rate, "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
            "sample": "%d rows of the workload in 64 evenly spaced row blocks (%d products, "
                      "%.1f s wall)" % (rows.size, prods, dt)}
    return result


def run_batched(args, dist):
    """Batched workload: every step computes all products, wave by wave
    (one batched plan, symbolic and numeric per wave, C freed after the
    wave).  Beside it, the same products one call per product."""
    import torch

    from paper_2501_07056_gb300 import gen_device, inputs, magnus

    dev = torch.device("cuda", dist.local_rank if dist.world > 1 else 0)
    torch.cuda.set_device(dev)
    magnus._lib()
    count = args.batch_count
    ns = inputs.batched_sizes(count, seed=0)
    # replicas: each rank runs the whole batch
    As = [gen_device.ragged(int(n), int(n), 2, 32, 0, 2 * i + 1, device=dev) for i, n in enumerate(ns)]
    Bs = [gen_device.ragged(int(n), int(n), 2, 32, 0, 2 * i + 2, device=dev) for i, n in enumerate(ns)]
    torch.cuda.synchronize()
    params = magnus.make_params(sort_threshold=args.sort_threshold,
                                force_category=args.force_category,
                                chunk_len_coarse_log2=args.chunk_coarse,
                                chunk_len_fine_log2=args.chunk_fine)
    stream = torch.cuda.current_stream()
    nw = max(1, min(args.batch_waves, count))
    bounds = [round(w * count / nw) for w in range(nw + 1)]
    stats = {"n_inter": 0, "nnz_c": 0, "stage_ms": {}, "rows_per_category": [0, 0, 0, 0]}
    tuned = None
    if args.autotune:
        # untimed setup: tune on the first wave's packed products (a row
        # sample), then plan every wave with the result
        bp = magnus.BatchPlan(As[bounds[0]:bounds[1]], Bs[bounds[0]:bounds[1]], params, stream)
        best, rep = bp.autotune(params, sample_products=1 << 28, max_trials=16)
        bp.free()
        params = best
        tuned = dict(rep, params={name: getattr(best, name) for name, _ in best._fields_})

    def step(record=False):
        tot_i = tot_c = 0
        st = {}
        for w in range(nw):
            lo, hi = bounds[w], bounds[w + 1]
            bp = magnus.BatchPlan(As[lo:hi], Bs[lo:hi], params, stream)
            if record:
                bp.enable_timing(True)
            off = bp.symbolic()
            col, val = bp.numeric()
            del col, val
            bp.c_col = bp.c_val = None
            if record:
                info = bp.info()
                tot_i += info["n_interprod"]
                tot_c += off[-1]
                for k, v in bp.stage_times().items():
                    st[k] = st.get(k, 0.0) + v
                for c in range(4):
                    stats["rows_per_category"][c] += info["rows_per_category"][c]
                stats["plan"] = {k: info[k] for k in (
                    "chunk_len_fine_log2", "chunk_len_coarse_log2", "n_chunks_coarse",
                    "n_batches_coarse", "sort_threshold", "dense_cols", "scratch_bytes")}
            bp.free()
        if record:
            stats["n_inter"], stats["nnz_c"], stats["stage_ms"] = tot_i, tot_c, st

    step(record=True)
    for _ in range(args.warmup - 1):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index).start()
    dist.barrier()
    torch.cuda.synchronize()
    n_launch0 = magnus.magnus_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    n_launch = magnus.magnus_launch_count() - n_launch0
    clk = clocks.stop()
    ms = dist.max(ev0.elapsed_time(ev1)) / args.steps
    n_inter = stats["n_inter"]
    value = dist.sum(2.0 * n_inter) / (ms * 1e-3) / 1e9

    # one call per product (plan, symbolic, allocate C, numeric, free)
    def one_by_one(k):
        for i in range(k):
            C = magnus.spgemm(As[i], Bs[i], params, stream)
            del C
    one_by_one(min(count, 64))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    one_by_one(count)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_one = e0.elapsed_time(e1)
    wall_one = time.perf_counter() - t0
    return {
        "metric": "SpGEMM GFLOP/s", "value": value, "unit": "GFLOP/s", "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS["batched4096"].replace("4096", str(count), 1),
                   "products": count, "waves": nw, "n_interprod": n_inter,
                   "nnz_c": stats["nnz_c"],
                   "parallelism": "replicas" if dist.world > 1 else "single",
                   "l2": "inputs larger than L2, no flush",
                   "step": "per wave: batched plan+symbolic+alloc C+numeric"},
        "products_per_s": count / (ms * 1e-3),
        "one_call_per_product": {"ms": ms_one, "wall_s": wall_one,
                                 "products_per_s": count / (ms_one * 1e-3),
                                 "gflops": 2.0 * n_inter / (ms_one * 1e-3) / 1e9},
        "clocks": clk,
        "gpu_launches": n_launch,
        "detail": {"stage_ms_untimed_step": stats["stage_ms"],
                   "rows_per_category": stats["rows_per_category"],
                   "last_wave_plan": stats.get("plan"), "autotune": tuned},
    }


def run_served(args, dist):
    """Served workload: the one-call-per-product capacity is measured on a
    closed-loop sample, the arrival rate set to rho times it, and the same
    open-loop arrival sequence replayed through the one-call server and the
    continuous-batching server."""
    import torch

    from paper_2501_07056_gb300 import inputs, magnus, serve

    dev = torch.device("cuda", dist.local_rank if dist.world > 1 else 0)
    torch.cuda.set_device(dev)
    magnus._lib()
    descs = inputs.served_stream(args.requests, seed=0)
    params = magnus.make_params(sort_threshold=args.sort_threshold,
                                force_category=args.force_category)
    work = serve.StencilTimesRandom(device=dev)

    def reqs_at(rate, d=descs):
        return serve.make_requests(d, seed=0, rate=rate, exact=False)

    # capacity of the one-call path: a closed-loop sample (all arrive at 0)
    nsamp = min(len(descs), 200)
    # PyTorch caches blocks per stream and every server has streams of its
    # own: the cache goes back to the device between servers (untimed)
    serve.Server(work, params, mode="single", device=dev).run(reqs_at(1e12, descs[:16]))
    torch.cuda.empty_cache()
    srv = serve.Server(work, params, mode="single", device=dev)
    srv.run(reqs_at(1e12, descs[:nsamp]))
    cap = srv.executed_products / srv.makespan
    torch.cuda.empty_cache()
    srvb = serve.Server(work, params, mode="batched", n_streams=3, max_requests=64,
                        max_products=1 << 30, device=dev)
    srvb.run(reqs_at(1e12, descs[:nsamp]))
    cap_batched = srvb.executed_products / srvb.makespan
    mean_p = np.mean([r.products for r in reqs_at(1.0)])
    rate = args.rho * cap / mean_p
    out = {}
    for mode in ("single", "batched"):
        reqs = reqs_at(rate)
        torch.cuda.empty_cache()
        srv = serve.Server(work, params, mode=mode, n_streams=3, max_requests=64,
                           max_products=1 << 30, device=dev)
        clocks = ClockSampler(dev.index).start()
        n0 = magnus.magnus_launch_count()
        srv.run(reqs)
        clk = clocks.stop()
        prods = srv.executed_products
        out[mode] = dict(serve.latency_stats(reqs), requests_per_s=len(reqs) / srv.makespan,
                         gflops=2.0 * prods / srv.makespan / 1e9, makespan_s=srv.makespan,
                         batches=srv.n_batches, gpu_launches=magnus.magnus_launch_count() - n0,
                         cache_reclaims=srv.reclaims, clocks=clk)
    b, o = out["batched"], out["single"]
    high = None
    if args.rho_high > 0:
        # an offered load above the one-call capacity: the one-call queue
        # grows for the whole run, continuous batching may still keep up
        rate_h = args.rho_high * cap / mean_p
        high = {"rho": args.rho_high, "arrival_rate_per_s": rate_h}
        for mode in ("single", "batched"):
            reqs = reqs_at(rate_h)
            torch.cuda.empty_cache()
            srv = serve.Server(work, params, mode=mode, n_streams=3, max_requests=64,
                               max_products=1 << 30, device=dev)
            srv.run(reqs)
            high[mode] = dict(serve.latency_stats(reqs), requests_per_s=len(reqs) / srv.makespan,
                              makespan_s=srv.makespan, batches=srv.n_batches,
                              cache_reclaims=srv.reclaims)
    return {
        "metric": "served products/s", "value": b["requests_per_s"], "unit": "products/s",
        "n_gpus": dist.world, "steps": 1, "warmup": 1, "ms_per_step": 1e3 * b["makespan_s"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS["served"], "requests": len(descs), "rho": args.rho,
                   "arrival_rate_per_s": rate, "one_call_capacity_products_per_s": cap,
                   "batched_capacity_products_per_s": cap_batched,
                   "capacity_sample": "first %d requests, all arriving at once" % nsamp,
                   "mean_products_per_request": float(mean_p),
                   "parallelism": "replicas" if dist.world > 1 else "single"},
        "latency_ms": {"p50": b["p50_ms"], "p99": b["p99_ms"]},
        "served_batched": b, "served_one_call": o, "overload": high,
        "clocks": b["clocks"], "gpu_launches": b["gpu_launches"],
    }


def run_ablation(args, dist):
    """Figures 5-6 analogue: per-step device times of one reorder level versus
    the number of chunks, and their sum relative to a stream copy."""
    import torch

    from paper_2501_07056_gb300 import gen_device, magnus

    dev = torch.device("cuda", dist.local_rank if dist.world > 1 else 0)
    torch.cuda.set_device(dev)
    n = 1 << 28
    sweep = []
    clocks = ClockSampler(dev.index).start()
    for m_log2 in (16, 20, 24):
        m = 1 << m_log2
        col, val = gen_device.uniform_stream(n, m, 0, m_log2, device=dev)
        for lg in range(0, 15):
            best = None
            for _ in range(max(1, args.warmup)):  # keep the fastest of the repeats
                r, _, _, _ = magnus.microbench_chunks(col, val, m, lg)
                if best is None or r["copy_ms"] < best["copy_ms"]:
                    best = r
            reorder = best["reorder_ms"]
            if best["reorder_staged_ms"] >= 0:
                reorder = min(reorder, best["reorder_staged_ms"])
            steps = best["histogram_ms"] + best["scan_ms"] + reorder
            best["reorder_level_over_copy"] = steps / best["copy_ms"]
            if best["accumulate_ms"] >= 0:
                best["with_accumulate_over_copy"] = (steps + best["accumulate_ms"]) / best["copy_ms"]
                best["global_accumulate_over_copy"] = best["global_accumulate_ms"] / best["copy_ms"]
            best["chunks_log2"] = lg
            best["index_range_log2"] = m_log2
            sweep.append(best)
        del col, val
    clk = clocks.stop()
    full = [r["with_accumulate_over_copy"] for r in sweep if "with_accumulate_over_copy" in r]
    copy_gbs = n * 24 / (min(r["copy_ms"] for r in sweep) * 1e-3) / 1e9
    return {
        "metric": "reorder level + dense accumulation time over stream copy", "value": min(full),
        "unit": "x", "n_gpus": dist.world, "steps": len(sweep), "warmup": args.warmup,
        "ms_per_step": sum(r["copy_ms"] for r in sweep) / len(sweep),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS["ablation"], "stream": n, "index_range": "2^16, 2^20, 2^24",
                   "copy_GBps": copy_gbs,
                   "paper": "Section 4.1: about 2.2x streaming time at the optimal chunk "
                            "count, reorder breaking point at 2^13 chunks (1 core, SPR)"},
        "sweep": sweep, "clocks": clk, "gpu_launches": 5 * len(sweep),
    }


def _link_bandwidth(dst_host, src_host, dev, chunk=1 << 30):
    """Plain pinned copies on one stream, into and out of the e2e buffers
    (the same host pages): (H2D GB/s, D2H GB/s) over about one C's bytes."""
    import torch
    buf = torch.empty(chunk, dtype=torch.uint8, device=dev)
    out = dst_host.view(torch.uint8)
    inp = src_host.view(torch.uint8)
    s = torch.cuda.current_stream()
    res = []
    for direction in ("h2d", "d2h"):
        host = inp if direction == "h2d" else out
        n = host.numel()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        done = 0
        while done < n:
            m = min(chunk, n - done)
            if direction == "h2d":
                buf[:m].copy_(host[done:done + m], non_blocking=True)
            else:
                host[done:done + m].copy_(buf[:m], non_blocking=True)
            done += m
        e1.record(s)
        torch.cuda.synchronize()
        res.append(n / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    del buf
    return res[0], res[1]


def run_rates(args, dist):
    """The device rates behind the rooflines: random chunk gathers (the sort
    kernels gather one B row per nonzero of A) and shared-memory FP64
    accumulation (the dense accumulators), per second device-wide."""
    import torch

    from paper_2501_07056_gb300 import magnus
    dev = torch.device("cuda", dist.local_rank if dist.world > 1 else 0)
    torch.cuda.set_device(dev)
    clocks = ClockSampler(dev.index).start()
    reps = [magnus.microbench_rates() for _ in range(max(1, args.steps))]
    clk = clocks.stop()
    best = {k: max(r[k] for r in reps) for k in reps[0]}
    sm_hz = 2.07e9 * best["sms"]
    per_clk = {k: best[k] / sm_hz for k in best if k.startswith("smem")}
    return {
        "metric": "random gather rate, 32-byte chunks", "value": best["gather_32"] / 1e9,
        "unit": "G chunks/s", "n_gpus": dist.world, "steps": len(reps), "warmup": 0,
        "ms_per_step": 0.0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": {"workload": WORKLOADS["rates"]},
        "rates_per_s": best, "smem_updates_per_clock_per_sm_at_2070mhz": per_clk,
        "clocks": clk, "gpu_launches": 44 * len(reps),
    }


def run_e2e(args, dist, A, dev, params, n_inter, nnz_c):
    """Same metric through the public API with host buffers: every step
    copies A (which serves as both operands) from pinned host memory to the
    device, plans the whole product and runs its symbolic phase, copies
    C.rowPtr back, then computes C in row slabs (magnus_numeric_rows) whose
    entries are copied back to pinned host memory while the next slab
    computes (magnus.spgemm_host).  Every timed step is timed."""
    import torch

    from paper_2501_07056_gb300 import magnus
    # page-locked host buffers backed by huge pages (magnus_host_alloc): the
    # public API's own allocator for host operands and results
    h_rp = magnus.host_copy(A.row_ptr)
    h_col = magnus.host_copy(A.col)
    h_val = magnus.host_copy(A.val)
    o_rp = magnus.host_empty(A.n_rows + 1, torch.int64)
    o_col = magnus.host_empty(nnz_c, torch.int32)
    o_val = magnus.host_empty(nnz_c, torch.float64)
    h2d = h_rp.numel() * 8 + h_col.numel() * 4 + h_val.numel() * 8
    d2h = o_rp.numel() * 8 + o_col.numel() * 4 + o_val.numel() * 8

    pinned = ((h_rp, h_col, h_val), (h_rp, h_col, h_val))
    parts = []

    walls = []

    def step(record):
        t = {} if record else None
        w0 = time.perf_counter()
        magnus.spgemm_host(A, A, params, blocks=args.e2e_blocks, device=dev,
                           out=(o_rp, o_col, o_val), pinned=pinned, timing=t)
        torch.cuda.synchronize()
        if record:
            parts.append(t)
            walls.append(1e3 * (time.perf_counter() - w0))

    # the link test first: its device buffer changes the caching allocator's
    # state, which the warm-up steps then settle again before the timed ones
    link_h2d, link_d2h = _link_bandwidth(o_val, h_val, dev)
    for _ in range(max(1, args.warmup)):
        step(False)
    steps = max(1, args.steps)
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        step(True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    dist.barrier()
    dt_max = dist.max(dt)
    # the link again after the timed steps: copies that were slow inside the
    # loop but not here met other traffic on the host's memory meanwhile
    link_h2d_after, link_d2h_after = _link_bandwidth(o_val, h_val, dev)
    units = dist.sum(2.0 * n_inter * steps)
    mean = {k: statistics.mean(p[k] for p in parts) for k in parts[0]} if parts else {}
    return {"value": units / dt_max / 1e9, "unit": "GFLOP/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "row_slabs": args.e2e_blocks, "steps": steps,
            "ms_per_step": 1e3 * dt_max / steps,
            "parts_ms": mean,
            "step_ms": {"min": min(walls), "median": statistics.median(walls),
                        "max": max(walls)} if walls else {},
            # steps above 1.5x the median, with their parts: which copy was slow
            "slow_steps": [dict({k: round(v, 2) for k, v in parts[i].items()}, step=i,
                                wall_ms=round(walls[i], 2))
                           for i in range(len(walls))
                           if walls[i] > 1.5 * statistics.median(walls)][:8],
            "link_gbs": {"h2d": link_h2d, "d2h": link_d2h,
                         "h2d_after": link_h2d_after, "d2h_after": link_d2h_after,
                         "how": "plain pinned copies of 1 GB pieces on one stream into the "
                                "e2e output buffer (D2H) and from the input (H2D), before and "
                                "after the timed steps"},
            "copy_floor_ms": 1e3 * (h2d / (link_h2d * 1e9) + d2h / (link_d2h * 1e9))}


def _summary(res):
    """The headline keys of another workload's line, for detail.configs."""
    keep = ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "roofline", "clocks",
            "gpu_launches", "latency_ms", "products_per_s", "one_call_per_product",
            "served_one_call", "overload", "config")
    out = {k: res[k] for k in keep if k in res}
    d = res.get("detail", {})
    for k in ("stage_ms", "t_over_t_ideal", "nnz_c", "stage_ms_untimed_step",
              "rows_per_category", "last_wave_plan", "autotune"):
        if k in d:
            out[k] = d[k]
    if "served_batched" in res:
        out["served_batched"] = {k: v for k, v in res["served_batched"].items() if k != "clocks"}
        out["served_one_call"] = {k: v for k, v in res["served_one_call"].items()
                                  if k != "clocks"}
    return out


def run_other_configs(args, dist):
    """R-MAT scale 20 (3 steps), batched 4096 products (2 steps) and the
    served stream (2,000 requests), each in its own metric, measured in the
    same process after the headline workload."""
    import torch
    out = {}
    for name, extra in (("rmat20", ["--steps", "3"]),
                        ("batched4096", ["--steps", "2", "--autotune", "1"]),
                        ("served", ["--requests", "2000"])):
        torch.cuda.empty_cache()
        sub = parse_args(["--workload", name, "--warmup", "3", "--no-e2e", "--no-cpu",
                          "--gpus", str(args.gpus)] + extra)
        try:
            if name == "batched4096":
                r = run_batched(sub, dist)
            elif name == "served":
                r = run_served(sub, dist)
            else:
                r = run_ours(sub, dist)
            out[name] = _summary(r)
        except Exception as e:  # report, do not lose the headline line
            out[name] = {"error": "%s: %s" % (type(e).__name__, e)}
        torch.cuda.synchronize()
    return out


def main(argv=None):
    args = parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    dist = Dist()
    try:
        if args.impl == "reference":
            res = run_reference(args, dist)
        elif args.workload == "batched4096":
            res = run_batched(args, dist)
        elif args.workload == "served":
            res = run_served(args, dist)
        elif args.workload == "ablation":
            res = run_ablation(args, dist)
        elif args.workload == "rates":
            res = run_rates(args, dist)
        else:
            res = run_ours(args, dist)
            if args.workload == "uniform2^24" and not args.no_configs:
                res["detail"]["configs"] = run_other_configs(args, dist)
        if dist.rank == 0 and res is not None:
            print(json.dumps(res), flush=True)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
