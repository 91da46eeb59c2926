"""Thin ctypes binding of libmagnus.so (C ABI in include/magnus.h).

Only argument marshalling lives here; every step of the SpGEMM runs in the
library's CUDA kernels.  Device memory and streams come from PyTorch.  The
library is loaded on first use; if it is missing the call raises (there is no
CPU fallback).

Functions with the C names (``magnus_plan``, ``magnus_symbolic``,
``magnus_numeric``, ``magnus_free`` ...) mirror the ABI one to one.
``spgemm`` is the convenience call a user makes: it plans, runs the symbolic
phase, allocates C with PyTorch and runs the numeric phase.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmagnus.so")

c_i32, c_i64, c_p, c_u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_uint64

CAT_AUTO, CAT_SORT, CAT_DENSE, CAT_FINE, CAT_COARSE = -1, 0, 1, 2, 3
STAGES = ["sym_sort", "sym_dense", "sym_fine", "sym_coarse", "sym_scan",
          "num_sort", "num_dense", "num_fine", "num_coarse",
          "sym_coarse_big", "num_coarse_big"]


class CsrDesc(ctypes.Structure):
    _fields_ = [("n_rows", c_i64), ("n_cols", c_i64), ("nnz", c_i64),
                ("row_ptr", c_p), ("col", c_p), ("val", c_p)]


class Params(ctypes.Structure):
    _fields_ = [("sort_threshold", c_i32), ("force_category", c_i32),
                ("chunk_len_fine_log2", c_i32), ("chunk_len_coarse_log2", c_i32),
                ("dense_chunk_threshold", c_i32), ("validate", c_i32),
                ("max_scratch_bytes", c_i64), ("l2_fetch_bytes", c_i32), ("numeric_graph", c_i32), ("wide_sort_max", c_i32),
                ("chunk_accumulator", c_i32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_rows", c_i64), ("n_cols", c_i64), ("n_interprod", c_i64),
                ("max_row_products", c_i64), ("nnz_c", c_i64), ("rows_empty", c_i64),
                ("rows_per_category", c_i64 * 4), ("products_per_category", c_i64 * 4),
                ("staged_products_numeric", c_i64), ("scratch_bytes", c_i64),
                ("sort_threshold", c_i32), ("chunk_len_fine_log2", c_i32),
                ("chunk_len_fine_sym_log2", c_i32), ("chunk_len_coarse_log2", c_i32),
                ("n_chunks_coarse", c_i32), ("dense_cols", c_i32),
                ("dense_chunk_threshold", c_i32), ("key_bits32", c_i32),
                ("n_batches_fine", c_i32), ("n_batches_coarse", c_i32),
                ("coarse_dense_products", c_i64), ("coarse_dense_nnz", c_i64),
                ("coarse_dense_buckets", c_i64)]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else v
        return d


class TuneReport(ctypes.Structure):
    _fields_ = [("trials", c_i32), ("from_cache", c_i32), ("sampled_rows", c_i64),
                ("products_full", c_i64), ("base_ms", ctypes.c_float), ("best_ms", ctypes.c_float)]


class MicrobenchResult(ctypes.Structure):
    _fields_ = [("copy_ms", ctypes.c_float), ("histogram_ms", ctypes.c_float),
                ("scan_ms", ctypes.c_float), ("reorder_ms", ctypes.c_float),
                ("accumulate_ms", ctypes.c_float), ("global_accumulate_ms", ctypes.c_float),
                ("n_chunks", c_i32), ("chunk_len_log2", c_i32),
                ("reorder_staged_ms", ctypes.c_float), ("reserved", c_i32)]


class ChunkModel(ctypes.Structure):
    _fields_ = [("m_c_log2", c_i32), ("chunk_len_fine_log2", c_i32),
                ("chunk_len_fine_sym_log2", c_i32), ("n_chunks_fine_max_log2", c_i32),
                ("m_c_max_log2", c_i32), ("n_chunks_coarse", c_i32),
                ("fine_smem_bytes", c_i64)]


class MagnusError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        msg = "%s: %s" % (where, _lib().magnus_strerror(status).decode())
        if status == 5:
            msg += " (%s)" % _lib().magnus_last_cuda_error().decode()
        super().__init__(msg)


_LIB = None

# Exported symbols and their signatures (restype, argtypes).
SIGNATURES = {
    "magnus_params_default": (c_i32, [ctypes.POINTER(Params)]),
    "magnus_plan": (c_i32, [ctypes.POINTER(c_p), ctypes.POINTER(CsrDesc), ctypes.POINTER(CsrDesc),
                            ctypes.POINTER(Params), c_p]),
    "magnus_symbolic": (c_i32, [c_p, c_p, ctypes.POINTER(c_i64), c_p]),
    "magnus_numeric": (c_i32, [c_p, c_p, c_p, c_p, c_p, c_p, c_p]),
    "magnus_numeric_noalloc": (c_i32, [c_p, c_p, c_p, c_p, c_p, c_p, c_p]),
    "magnus_free": (None, [c_p]),
    "magnus_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "magnus_last_cuda_error": (ctypes.c_char_p, []),
    "magnus_plan_info": (c_i32, [c_p, ctypes.POINTER(PlanInfo)]),
    "magnus_enable_timing": (c_i32, [c_p, ctypes.c_int]),
    "magnus_stage_times": (c_i32, [c_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    "magnus_launch_count": (c_u64, []),
    "magnus_plan_batched": (c_i32, [ctypes.POINTER(c_p), c_i32, ctypes.POINTER(CsrDesc),
                                    ctypes.POINTER(CsrDesc), ctypes.POINTER(Params), c_p]),
    "magnus_batch_layout": (c_i32, [c_p, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64)]),
    "magnus_symbolic_batched": (c_i32, [c_p, c_p, ctypes.POINTER(c_i64), c_p]),
    "magnus_numeric_batched": (c_i32, [c_p, c_p, c_p, c_p, c_p]),
    "magnus_batch_info": (c_i32, [c_p, ctypes.POINTER(PlanInfo)]),
    "magnus_free_batched": (None, [c_p]),
    "magnus_batch_inner_plan": (c_p, [c_p]),
    "magnus_microbench_chunks": (c_i32, [c_p, c_p, c_i64, c_i64, c_i32, c_p, c_p, c_p,
                                         ctypes.POINTER(MicrobenchResult), c_p]),
    "magnus_autotune": (c_i32, [ctypes.POINTER(CsrDesc), ctypes.POINTER(CsrDesc),
                                ctypes.POINTER(Params), c_i64, c_i32, ctypes.POINTER(Params),
                                ctypes.POINTER(TuneReport), c_p]),
    "magnus_chunk_model": (c_i32, [c_i64, c_i64, c_i64, c_i32, ctypes.POINTER(ChunkModel)]),
}


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmagnus.so is not built (run __graft_entry__.build()); "
                               "there is no CPU fallback")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _LIB = lib
    return _LIB


def _check(st, where):
    if st != 0:
        raise MagnusError(st, where)


# ---------------------------------------------------------------------------
# One-to-one wrappers of the C entry points.

def magnus_params_default() -> Params:
    p = Params()
    _check(_lib().magnus_params_default(ctypes.byref(p)), "magnus_params_default")
    return p


def magnus_plan(A: CsrDesc, B: CsrDesc, params: Params | None, stream: int) -> int:
    h = c_p()
    _check(_lib().magnus_plan(ctypes.byref(h), ctypes.byref(A), ctypes.byref(B),
                              ctypes.byref(params) if params is not None else None,
                              c_p(stream)), "magnus_plan")
    return h.value


def magnus_symbolic(plan: int, c_row_ptr: int, stream: int) -> int:
    nnz = c_i64()
    _check(_lib().magnus_symbolic(c_p(plan), c_p(c_row_ptr), ctypes.byref(nnz), c_p(stream)),
           "magnus_symbolic")
    return nnz.value


def magnus_numeric(plan: int, a_val: int, b_val: int, c_row_ptr: int, c_col: int, c_val: int,
                   stream: int) -> None:
    _check(_lib().magnus_numeric(c_p(plan), c_p(a_val), c_p(b_val), c_p(c_row_ptr), c_p(c_col),
                                 c_p(c_val), c_p(stream)), "magnus_numeric")


def magnus_numeric_noalloc(plan: int, a_val: int, b_val: int, c_row_ptr: int, c_col: int,
                           c_val: int, stream: int) -> None:
    """Numeric phase that allocates no device memory (staging in the
    library's fixed static buffer); for callers that may not allocate once
    running.  Same arguments and results as magnus_numeric."""
    _check(_lib().magnus_numeric_noalloc(c_p(plan), c_p(a_val), c_p(b_val), c_p(c_row_ptr),
                                         c_p(c_col), c_p(c_val), c_p(stream)),
           "magnus_numeric_noalloc")


def magnus_free(plan: int) -> None:
    if plan:
        _lib().magnus_free(c_p(plan))


def magnus_plan_info(plan: int) -> dict:
    info = PlanInfo()
    _check(_lib().magnus_plan_info(c_p(plan), ctypes.byref(info)), "magnus_plan_info")
    return info.as_dict()


def magnus_enable_timing(plan: int, enable: bool = True) -> None:
    _check(_lib().magnus_enable_timing(c_p(plan), int(enable)), "magnus_enable_timing")


def magnus_stage_times(plan: int) -> dict:
    arr = (ctypes.c_double * len(STAGES))()
    _check(_lib().magnus_stage_times(c_p(plan), arr, len(STAGES)), "magnus_stage_times")
    return dict(zip(STAGES, list(arr)))


def magnus_launch_count() -> int:
    return int(_lib().magnus_launch_count())


def magnus_chunk_model(m_c: int, smem_bytes: int, l2_bytes: int, resident_blocks: int) -> dict:
    out = ChunkModel()
    _check(_lib().magnus_chunk_model(m_c, smem_bytes, l2_bytes, resident_blocks,
                                     ctypes.byref(out)), "magnus_chunk_model")
    return {name: getattr(out, name) for name, _ in out._fields_}


# ---------------------------------------------------------------------------
# PyTorch-facing convenience layer.

@dataclasses.dataclass
class DeviceCSR:
    """CSR on the GPU: int64 row_ptr, int32 col, float64 val (torch tensors)."""
    n_rows: int
    n_cols: int
    row_ptr: "torch.Tensor"
    col: "torch.Tensor"
    val: "torch.Tensor"

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    def desc(self, with_val: bool = True) -> CsrDesc:
        return CsrDesc(self.n_rows, self.n_cols, self.nnz, self.row_ptr.data_ptr(),
                       self.col.data_ptr() if self.nnz else 0,
                       self.val.data_ptr() if (with_val and self.nnz) else 0)

    @staticmethod
    def from_host(M, device="cuda", non_blocking=False) -> "DeviceCSR":
        import torch
        return DeviceCSR(M.n_rows, M.n_cols,
                         torch.as_tensor(M.row_ptr).to(device, non_blocking=non_blocking),
                         torch.as_tensor(M.col).to(device, non_blocking=non_blocking),
                         torch.as_tensor(M.val).to(device, non_blocking=non_blocking))


def make_params(sort_threshold=0, force_category=CAT_AUTO, chunk_len_fine_log2=0,
                chunk_len_coarse_log2=0, dense_chunk_threshold=0, validate=0,
                max_scratch_bytes=0, l2_fetch_bytes=0, numeric_graph=0,
                wide_sort_max=0, chunk_accumulator=0) -> Params:
    p = magnus_params_default()
    p.sort_threshold = sort_threshold
    p.force_category = force_category
    p.chunk_len_fine_log2 = chunk_len_fine_log2
    p.chunk_len_coarse_log2 = chunk_len_coarse_log2
    p.dense_chunk_threshold = dense_chunk_threshold
    p.validate = validate
    p.max_scratch_bytes = max_scratch_bytes
    p.l2_fetch_bytes = l2_fetch_bytes
    p.numeric_graph = numeric_graph
    p.wide_sort_max = wide_sort_max
    p.chunk_accumulator = chunk_accumulator
    return p


class Plan:
    """Owns a magnus plan for fixed A and B structures (values may change)."""

    def __init__(self, A: DeviceCSR, B: DeviceCSR, params: Params | None = None, stream=None):
        import torch
        self.A, self.B = A, B
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = magnus_plan(A.desc(False), B.desc(False), params, self.stream.cuda_stream)
        self.c_row_ptr = None
        self.nnz_c = None

    def symbolic(self, c_row_ptr=None) -> int:
        import torch
        if c_row_ptr is None:
            c_row_ptr = torch.empty(self.A.n_rows + 1, dtype=torch.int64, device=self.A.row_ptr.device)
        self.c_row_ptr = c_row_ptr
        self.nnz_c = magnus_symbolic(self.handle, c_row_ptr.data_ptr(), self.stream.cuda_stream)
        return self.nnz_c

    def numeric(self, c_col=None, c_val=None, a_val=None, b_val=None):
        import torch
        dev = self.A.row_ptr.device
        if c_col is None:
            c_col = torch.empty(max(self.nnz_c, 1), dtype=torch.int32, device=dev)
        if c_val is None:
            c_val = torch.empty(max(self.nnz_c, 1), dtype=torch.float64, device=dev)
        av = self.A.val if a_val is None else a_val
        bv = self.B.val if b_val is None else b_val
        magnus_numeric(self.handle, av.data_ptr() if av.numel() else 0,
                       bv.data_ptr() if bv.numel() else 0, self.c_row_ptr.data_ptr(),
                       c_col.data_ptr(), c_val.data_ptr(), self.stream.cuda_stream)
        return c_col[:self.nnz_c], c_val[:self.nnz_c]

    def info(self) -> dict:
        return magnus_plan_info(self.handle)

    def enable_timing(self, on=True):
        magnus_enable_timing(self.handle, on)

    def stage_times(self) -> dict:
        return magnus_stage_times(self.handle)

    def free(self):
        if self.handle:
            magnus_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def autotune(A: "DeviceCSR", B: "DeviceCSR", base: Params | None = None, sample_products=0,
             max_trials=16, stream=None):
    """magnus_autotune: returns (best Params, report dict)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    best = Params()
    rep = TuneReport()
    da, db = A.desc(True), B.desc(True)
    _check(_lib().magnus_autotune(ctypes.byref(da), ctypes.byref(db),
                                  ctypes.byref(base) if base is not None else None,
                                  sample_products, max_trials, ctypes.byref(best),
                                  ctypes.byref(rep), c_p(s.cuda_stream)), "magnus_autotune")
    return best, {name: getattr(rep, name) for name, _ in rep._fields_}


def microbench_chunks(col, val, m: int, n_chunks_log2: int, stream=None):
    """magnus_microbench_chunks on device tensors; returns (result dict,
    out_col, out_val, chunk_nnz)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    n = col.numel()
    out_col = torch.empty(n, dtype=torch.int32, device=col.device)
    out_val = torch.empty(n, dtype=torch.float64, device=col.device)
    nch = 1 << n_chunks_log2
    chunk_nnz = torch.zeros(nch + 1, dtype=torch.int64, device=col.device)
    res = MicrobenchResult()
    _check(_lib().magnus_microbench_chunks(c_p(col.data_ptr()), c_p(val.data_ptr()), n, m,
                                           n_chunks_log2, c_p(out_col.data_ptr()),
                                           c_p(out_val.data_ptr()), c_p(chunk_nnz.data_ptr()),
                                           ctypes.byref(res), c_p(s.cuda_stream)),
           "magnus_microbench_chunks")
    return ({name: getattr(res, name) for name, _ in res._fields_}, out_col, out_val, chunk_nnz)


def params_dict(p: Params) -> dict:
    return {name: getattr(p, name) for name, _ in p._fields_}


class BatchPlan:
    """Owns a batched plan for products C_i = A_i * B_i (one packed C)."""

    def __init__(self, As, Bs, params: Params | None = None, stream=None):
        import torch
        if len(As) != len(Bs) or not As:
            raise ValueError("need equally many A and B operands (at least one)")
        self.As, self.Bs = list(As), list(Bs)
        self.count = len(As)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        da = (CsrDesc * self.count)(*[a.desc(True) for a in self.As])
        db = (CsrDesc * self.count)(*[b.desc(True) for b in self.Bs])
        h = c_p()
        _check(_lib().magnus_plan_batched(ctypes.byref(h), self.count, da, db,
                                          ctypes.byref(params) if params is not None else None,
                                          c_p(self.stream.cuda_stream)), "magnus_plan_batched")
        self.handle = h.value
        ro = (c_i64 * (self.count + 1))()
        tot = c_i64()
        _check(_lib().magnus_batch_layout(c_p(self.handle), ro, ctypes.byref(tot)),
               "magnus_batch_layout")
        self.row_offsets = list(ro)
        self.total_rows = tot.value
        self.c_row_ptr = None
        self.c_offsets = None
        self.c_col = None
        self.c_val = None

    def symbolic(self) -> list:
        import torch
        dev = self.As[0].row_ptr.device
        self.c_row_ptr = torch.empty(self.total_rows + 1, dtype=torch.int64, device=dev)
        off = (c_i64 * (self.count + 1))()
        _check(_lib().magnus_symbolic_batched(c_p(self.handle), c_p(self.c_row_ptr.data_ptr()),
                                              off, c_p(self.stream.cuda_stream)),
               "magnus_symbolic_batched")
        self.c_offsets = list(off)
        return self.c_offsets

    def numeric(self, c_col=None, c_val=None):
        import torch
        dev = self.As[0].row_ptr.device
        nnz = self.c_offsets[-1]
        if c_col is None:
            c_col = self.c_col if self.c_col is not None else \
                torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
        if c_val is None:
            c_val = self.c_val if self.c_val is not None else \
                torch.empty(max(nnz, 1), dtype=torch.float64, device=dev)
        self.c_col, self.c_val = c_col, c_val
        _check(_lib().magnus_numeric_batched(c_p(self.handle), c_p(self.c_row_ptr.data_ptr()),
                                             c_p(c_col.data_ptr()), c_p(c_val.data_ptr()),
                                             c_p(self.stream.cuda_stream)),
               "magnus_numeric_batched")
        return c_col[:nnz], c_val[:nnz]

    def result(self, i: int) -> DeviceCSR:
        """C_i as a DeviceCSR (views into the packed C; row pointers copied)."""
        r0, r1 = self.row_offsets[i], self.row_offsets[i + 1]
        e0, e1 = self.c_offsets[i], self.c_offsets[i + 1]
        rp = self.c_row_ptr[r0:r1 + 1] - e0
        return DeviceCSR(r1 - r0, self.Bs[i].n_cols, rp, self.c_col[e0:e1], self.c_val[e0:e1])

    def info(self) -> dict:
        info = PlanInfo()
        _check(_lib().magnus_batch_info(c_p(self.handle), ctypes.byref(info)), "magnus_batch_info")
        return info.as_dict()

    def enable_timing(self, on=True):
        magnus_enable_timing(_lib().magnus_batch_inner_plan(c_p(self.handle)), on)

    def stage_times(self) -> dict:
        return magnus_stage_times(_lib().magnus_batch_inner_plan(c_p(self.handle)))

    def free(self):
        if self.handle:
            _lib().magnus_free_batched(c_p(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


_BLOCK_STREAMS: dict = {}


def _block_streams(dev, n: int):
    """The row-block streams of spgemm_host, created once per device and
    reused by later calls: the caching allocator keeps freed blocks per
    stream, so new streams on every call could not reuse the previous call's
    memory for C and would allocate (and release) it again."""
    import torch
    key = (dev.type, dev.index if dev.index is not None else torch.cuda.current_device())
    have = _BLOCK_STREAMS.setdefault(key, [])
    while len(have) < n:
        have.append(torch.cuda.Stream(dev))
    return have[:n]


def spgemm_host(A, B, params: Params | None = None, blocks: int = 4, device="cuda",
                out=None, pinned=None):
    """C = A * B for host CSR operands with a host result, pipelined: A and B
    are copied to the device, A's rows are cut into ``blocks`` row blocks
    (balanced by nonzeros), each planned and computed on its own stream, and
    each block's rows of C are copied back while the next blocks compute.
    ``pinned``: optional (A, B) pinned host copies (torch tensors
    (row_ptr, col, val)) to copy from; ``out``: optional pinned host tensors
    (row_ptr, col, val) large enough for C (else allocated).  Returns
    (row_ptr, col, val) host tensors (views of ``out`` when given)."""
    import numpy as np
    import torch
    dev = torch.device(device)
    if pinned is None:
        pa = tuple(torch.from_numpy(x).pin_memory() for x in (A.row_ptr, A.col, A.val))
        pinned = (pa, pa if B is A else
                  tuple(torch.from_numpy(x).pin_memory() for x in (B.row_ptr, B.col, B.val)))
    main = torch.cuda.current_stream(dev)
    (arp, acol, aval), (brp, bcol, bval) = pinned
    dA = DeviceCSR(A.n_rows, A.n_cols, arp.to(dev, non_blocking=True),
                   acol.to(dev, non_blocking=True), aval.to(dev, non_blocking=True))
    if B is A:  # C = A * A: one copy serves both operands
        dB = dA
    else:
        dB = DeviceCSR(B.n_rows, B.n_cols, brp.to(dev, non_blocking=True),
                       bcol.to(dev, non_blocking=True), bval.to(dev, non_blocking=True))
    up = torch.cuda.Event()
    up.record(main)
    nb = max(1, min(blocks, A.n_rows))
    targets = np.linspace(0, A.nnz, nb + 1)
    cuts = np.unique(np.concatenate(([0], np.searchsorted(A.row_ptr, targets[1:-1]), [A.n_rows])))
    streams = _block_streams(dev, len(cuts) - 1)
    parts = []
    base = 0

    def copy_back(part, o_rp, o_col, o_val):
        r0, r1, nnz, plan, col, val, s, off = part
        with torch.cuda.stream(s):
            # the block's row pointers, shifted by the entries before it
            o_rp[r0:r1].copy_(plan.c_row_ptr[:r1 - r0] + off, non_blocking=True)
            o_col[off:off + nnz].copy_(col, non_blocking=True)
            o_val[off:off + nnz].copy_(val, non_blocking=True)

    for k, s in enumerate(streams):
        r0, r1 = int(cuts[k]), int(cuts[k + 1])
        z0, z1 = int(A.row_ptr[r0]), int(A.row_ptr[r1])
        s.wait_event(up)
        with torch.cuda.stream(s):
            Ak = DeviceCSR(r1 - r0, A.n_cols, dA.row_ptr[r0:r1 + 1] - z0, dA.col[z0:z1],
                           dA.val[z0:z1])
            plan = Plan(Ak, dB, params, s)
            nnz = plan.symbolic()
            col, val = plan.numeric()
        part = (r0, r1, nnz, plan, col, val, s, base)
        base += nnz
        parts.append(part)
        if out is not None:  # copy this block back while the next ones compute
            copy_back(part, *out)
    total = base
    if out is None:
        out = (torch.empty(A.n_rows + 1, dtype=torch.int64).pin_memory(),
               torch.empty(max(total, 1), dtype=torch.int32).pin_memory(),
               torch.empty(max(total, 1), dtype=torch.float64).pin_memory())
        for part in parts:
            copy_back(part, *out)
    o_rp, o_col, o_val = out
    for part in parts:
        part[6].synchronize()
        part[3].free()
    o_rp[A.n_rows] = total
    return o_rp, o_col[:total], o_val[:total]


def spgemm(A: DeviceCSR, B: DeviceCSR, params: Params | None = None, stream=None) -> DeviceCSR:
    """C = A * B on the GPU (plan, symbolic, allocate, numeric)."""
    plan = Plan(A, B, params, stream)
    try:
        plan.symbolic()
        col, val = plan.numeric()
        return DeviceCSR(A.n_rows, B.n_cols, plan.c_row_ptr, col, val)
    finally:
        plan.free()
