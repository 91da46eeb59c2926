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
                ("chunk_accumulator", c_i32), ("coarse_reorder", c_i32),
                ("sort_block_warps", c_i32), ("coarse_bucket_sort", c_i32)]


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
                ("coarse_dense_buckets", c_i64), ("plan_bytes", c_i64),
                ("workspace_bytes", c_i64), ("noalloc_fine_blocks", c_i32), ("reserved", c_i32)]

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


class Rates(ctypes.Structure):
    _fields_ = [("gather_16", ctypes.c_double), ("gather_32", ctypes.c_double),
                ("gather_64", ctypes.c_double), ("gather_128", ctypes.c_double),
                ("gather_256", ctypes.c_double), ("gather_csr_row8", ctypes.c_double),
                ("smem_f64_atomic_distinct", ctypes.c_double),
                ("smem_f64_atomic_random", ctypes.c_double),
                ("smem_f64_atomic_8_per_address", ctypes.c_double),
                ("smem_f64_add_plain", ctypes.c_double),
                ("smem_u32_atomic_random", ctypes.c_double), ("sms", c_i32), ("reserved", c_i32)]


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
    "magnus_workspace_size": (c_i32, [c_p, ctypes.POINTER(ctypes.c_size_t)]),
    "magnus_symbolic_ws": (c_i32, [c_p, c_p, ctypes.POINTER(c_i64), c_p, ctypes.c_size_t, c_p]),
    "magnus_numeric_ws": (c_i32, [c_p, c_p, c_p, c_p, c_p, c_p, c_p, ctypes.c_size_t, c_p]),
    "magnus_numeric_rows": (c_i32, [c_p, c_i64, c_i64, c_p, c_p, c_p, c_p, c_p, c_p,
                                    ctypes.c_size_t, c_p]),
    "magnus_free": (None, [c_p]),
    "magnus_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "magnus_last_cuda_error": (ctypes.c_char_p, []),
    "magnus_plan_info": (c_i32, [c_p, ctypes.POINTER(PlanInfo)]),
    "magnus_enable_timing": (c_i32, [c_p, ctypes.c_int]),
    "magnus_stage_times": (c_i32, [c_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    "magnus_launch_count": (c_u64, []),
    "magnus_device_status": (c_i32, [c_p]),
    "magnus_wait_selftest": (c_i32, [c_i64, c_p]),
    "magnus_device_memory": (c_i32, [ctypes.POINTER(ctypes.c_size_t),
                                     ctypes.POINTER(ctypes.c_size_t)]),
    "magnus_host_alloc": (c_i32, [ctypes.c_size_t, ctypes.POINTER(c_p)]),
    "magnus_host_free": (c_i32, [c_p, ctypes.c_size_t]),
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
    "magnus_autotune_batched": (c_i32, [c_p, ctypes.POINTER(Params), c_i64, c_i32,
                                        ctypes.POINTER(Params), ctypes.POINTER(TuneReport), c_p]),
    "magnus_chunk_model": (c_i32, [c_i64, c_i64, c_i64, c_i32, ctypes.POINTER(ChunkModel)]),
    "magnus_microbench_rates": (c_i32, [ctypes.POINTER(Rates), c_p]),
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


def magnus_workspace_size(plan: int) -> int:
    n = ctypes.c_size_t()
    _check(_lib().magnus_workspace_size(c_p(plan), ctypes.byref(n)), "magnus_workspace_size")
    return n.value


def magnus_symbolic_ws(plan: int, c_row_ptr: int, workspace: int, workspace_bytes: int,
                       stream: int) -> int:
    nnz = c_i64()
    _check(_lib().magnus_symbolic_ws(c_p(plan), c_p(c_row_ptr), ctypes.byref(nnz), c_p(workspace),
                                     workspace_bytes, c_p(stream)), "magnus_symbolic_ws")
    return nnz.value


def magnus_numeric_ws(plan: int, a_val: int, b_val: int, c_row_ptr: int, c_col: int, c_val: int,
                      workspace: int, workspace_bytes: int, stream: int) -> None:
    _check(_lib().magnus_numeric_ws(c_p(plan), c_p(a_val), c_p(b_val), c_p(c_row_ptr),
                                    c_p(c_col), c_p(c_val), c_p(workspace), workspace_bytes,
                                    c_p(stream)), "magnus_numeric_ws")


def magnus_numeric_rows(plan: int, row_begin: int, row_end: int, a_val: int, b_val: int,
                        c_row_ptr: int, c_col: int, c_val: int, workspace: int,
                        workspace_bytes: int, stream: int) -> None:
    _check(_lib().magnus_numeric_rows(c_p(plan), row_begin, row_end, c_p(a_val), c_p(b_val),
                                      c_p(c_row_ptr), c_p(c_col), c_p(c_val), c_p(workspace),
                                      workspace_bytes, c_p(stream)), "magnus_numeric_rows")


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


def device_status(stream=None) -> int:
    """magnus_device_status: synchronises the stream; MAGNUS_OK, or
    MAGNUS_TIMEOUT when a bounded device wait gave up since the last call."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(_lib().magnus_device_status(c_p(s.cuda_stream)))


def wait_selftest(limit_cycles: int, stream=None) -> None:
    """magnus_wait_selftest: a bounded device wait that runs out."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(_lib().magnus_wait_selftest(int(limit_cycles), c_p(s.cuda_stream)),
           "magnus_wait_selftest")


def magnus_device_memory() -> tuple:
    """(free device bytes, bytes the stream-ordered pool holds unused)."""
    fr, idle = ctypes.c_size_t(), ctypes.c_size_t()
    _check(_lib().magnus_device_memory(ctypes.byref(fr), ctypes.byref(idle)),
           "magnus_device_memory")
    return fr.value, idle.value


def magnus_chunk_model(m_c: int, smem_bytes: int, l2_bytes: int, resident_blocks: int) -> dict:
    out = ChunkModel()
    _check(_lib().magnus_chunk_model(m_c, smem_bytes, l2_bytes, resident_blocks,
                                     ctypes.byref(out)), "magnus_chunk_model")
    return {name: getattr(out, name) for name, _ in out._fields_}


class _HostRegion:
    """A magnus_host_alloc region exposed to numpy through the array
    interface; released when the last array (or tensor) using it is gone."""

    def __init__(self, nbytes: int):
        p = c_p()
        _check(_lib().magnus_host_alloc(nbytes, ctypes.byref(p)), "magnus_host_alloc")
        self.ptr, self.nbytes = p.value, nbytes
        self.__array_interface__ = {"shape": (nbytes,), "typestr": "|u1",
                                    "data": (self.ptr, False), "version": 3}

    def __del__(self):
        if getattr(self, "ptr", None):
            _lib().magnus_host_free(c_p(self.ptr), self.nbytes)
            self.ptr = None


def host_empty(count: int, dtype):
    """A page-locked host tensor of ``count`` elements in huge-page-backed
    memory (magnus_host_alloc): copies to and from the device run at the
    host link's rate even when host memory is fragmented."""
    import numpy as np
    import torch
    npdt = {torch.int32: np.int32, torch.int64: np.int64, torch.float64: np.float64,
            torch.uint8: np.uint8}[dtype]
    nbytes = max(int(count), 1) * np.dtype(npdt).itemsize
    raw = np.asarray(_HostRegion(nbytes))  # keeps the region alive as its base
    return torch.from_numpy(raw.view(npdt)[:max(int(count), 1)])[:int(count)]


def host_copy(x):
    """A huge-page-backed page-locked copy of the numpy array ``x``."""
    import torch
    dt = {"int32": torch.int32, "int64": torch.int64, "float64": torch.float64}[str(x.dtype)]
    t = host_empty(x.size, dt)
    t.numpy()[:] = x.reshape(-1)
    return t


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
                wide_sort_max=0, chunk_accumulator=0, coarse_reorder=0,
                sort_block_warps=0, coarse_bucket_sort=0) -> Params:
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
    p.coarse_reorder = coarse_reorder
    p.sort_block_warps = sort_block_warps
    p.coarse_bucket_sort = coarse_bucket_sort
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

    def numeric_rows(self, row_begin: int, row_end: int, c_col, c_val, a_val=None, b_val=None,
                     workspace=None):
        """magnus_numeric_rows: rows [row_begin, row_end) of C into c_col /
        c_val (device tensors holding at least that slab's entries, written
        from index 0).  ``workspace``: optional uint8 device tensor of at
        least workspace_size() bytes (else scratch comes from the pool)."""
        av = self.A.val if a_val is None else a_val
        bv = self.B.val if b_val is None else b_val
        ws = workspace.data_ptr() if workspace is not None else 0
        wsb = workspace.numel() * workspace.element_size() if workspace is not None else 0
        magnus_numeric_rows(self.handle, row_begin, row_end, av.data_ptr() if av.numel() else 0,
                            bv.data_ptr() if bv.numel() else 0, self.c_row_ptr.data_ptr(),
                            c_col.data_ptr() if c_col.numel() else 0,
                            c_val.data_ptr() if c_val.numel() else 0, ws, wsb,
                            self.stream.cuda_stream)

    def workspace_size(self) -> int:
        return magnus_workspace_size(self.handle)

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


def microbench_rates(stream=None) -> dict:
    """magnus_microbench_rates: random-gather and shared-memory accumulation
    rates of the current device (per second, device-wide)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    r = Rates()
    _check(_lib().magnus_microbench_rates(ctypes.byref(r), c_p(s.cuda_stream)),
           "magnus_microbench_rates")
    return {name: getattr(r, name) for name, _ in r._fields_ if name != "reserved"}


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

    def autotune(self, base: Params | None = None, sample_products=0, max_trials=16):
        """magnus_autotune_batched: (best Params, report dict) for batches of
        products like these."""
        best = Params()
        rep = TuneReport()
        _check(_lib().magnus_autotune_batched(c_p(self.handle),
                                              ctypes.byref(base) if base is not None else None,
                                              sample_products, max_trials, ctypes.byref(best),
                                              ctypes.byref(rep), c_p(self.stream.cuda_stream)),
               "magnus_autotune_batched")
        return best, {name: getattr(rep, name) for name, _ in rep._fields_}

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


_COPY_STREAMS: dict = {}


def _copy_stream(dev):
    """The copy-back stream of spgemm_host, created once per device and
    reused by later calls (a new stream per call would create driver streams
    without bound)."""
    import torch
    key = (dev.type, dev.index if dev.index is not None else torch.cuda.current_device())
    if key not in _COPY_STREAMS:
        _COPY_STREAMS[key] = torch.cuda.Stream(dev)
    return _COPY_STREAMS[key]


def spgemm_host(A, B, params: Params | None = None, blocks: int = 4, device="cuda",
                out=None, pinned=None, timing=None):
    """C = A * B for host CSR operands with a host result.

    A and B are copied to the device; one plan and the symbolic phase cover
    the whole product; C.rowPtr is copied back and cuts C into ``blocks``
    slabs of about equal entries.  Each slab is computed by
    magnus_numeric_rows into one of two device slab buffers and copied back
    to host memory while the next slab computes, so the device holds two
    slabs of C, not all of it.
    ``pinned``: optional (A, B) page-locked host copies (torch tensors
    (row_ptr, col, val)) to copy from, else made with ``host_copy``;
    ``out``: optional page-locked host tensors (row_ptr, col, val) large
    enough for C, else allocated with ``host_empty``.  ``timing``:
    optional dict that receives the device time of each part (ms, CUDA
    events): h2d, plan_symbolic, rowptr_d2h, numeric (sum over slabs), d2h
    (first slab copy start to last copy end), slab_setup (C.rowPtr home to
    the first slab's numeric launch: the host's cut and buffer work), total.
    Returns (row_ptr,
    col, val) host tensors (views of ``out`` when given)."""
    import numpy as np
    import torch
    dev = torch.device(device)
    if pinned is None:
        pa = tuple(host_copy(x) for x in (A.row_ptr, A.col, A.val))
        pinned = (pa, pa if B is A else tuple(host_copy(x) for x in (B.row_ptr, B.col, B.val)))
    main = torch.cuda.current_stream(dev)
    cs = _copy_stream(dev)
    ev = (lambda: torch.cuda.Event(enable_timing=True)) if timing is not None else \
        (lambda: torch.cuda.Event())
    t0 = ev()
    t0.record(main)
    (arp, acol, aval), (brp, bcol, bval) = pinned
    dA = DeviceCSR(A.n_rows, A.n_cols, arp.to(dev, non_blocking=True),
                   acol.to(dev, non_blocking=True), aval.to(dev, non_blocking=True))
    if B is A:  # C = A * A: one copy serves both operands
        dB = dA
    else:
        dB = DeviceCSR(B.n_rows, B.n_cols, brp.to(dev, non_blocking=True),
                       bcol.to(dev, non_blocking=True), bval.to(dev, non_blocking=True))
    t_h2d = ev()
    t_h2d.record(main)
    plan = Plan(dA, dB, params, main)
    try:
        nnz = plan.symbolic()
        t_sym = ev()
        t_sym.record(main)
        if out is None:
            out = (host_empty(A.n_rows + 1, torch.int64), host_empty(max(nnz, 1), torch.int32),
                   host_empty(max(nnz, 1), torch.float64))
        o_rp, o_col, o_val = out
        o_rp[:A.n_rows + 1].copy_(plan.c_row_ptr)
        t_rp = ev()
        t_rp.record(main)
        rp = o_rp.numpy()
        nb = max(1, min(blocks, A.n_rows))
        # integer targets: float ones would make numpy convert all of C.rowPtr
        targets = (np.arange(1, nb, dtype=np.int64) * nnz) // nb
        cuts = np.searchsorted(rp[:A.n_rows + 1], targets, side="left")
        cuts = np.unique(np.concatenate(([0], cuts, [A.n_rows]))).astype(np.int64)
        slabs = [(int(cuts[k]), int(cuts[k + 1])) for k in range(len(cuts) - 1)]
        most = max(int(rp[r1] - rp[r0]) for r0, r1 in slabs)
        bufs = [(torch.empty(max(most, 1), dtype=torch.int32, device=dev),
                 torch.empty(max(most, 1), dtype=torch.float64, device=dev))
                for _ in range(min(2, len(slabs)))]
        copied = [None] * len(bufs)
        marks = []
        for k, (r0, r1) in enumerate(slabs):
            col, val = bufs[k % len(bufs)]
            if copied[k % len(bufs)] is not None:  # the buffer's previous slab is home
                main.wait_event(copied[k % len(bufs)])
            c0 = ev()
            c0.record(main)
            plan.numeric_rows(r0, r1, col, val)
            c1 = ev()
            c1.record(main)
            cs.wait_event(c1)
            e0, e1 = int(rp[r0]), int(rp[r1])
            with torch.cuda.stream(cs):
                d0 = ev()
                d0.record(cs)
                o_col[e0:e1].copy_(col[:e1 - e0], non_blocking=True)
                o_val[e0:e1].copy_(val[:e1 - e0], non_blocking=True)
                d1 = ev()
                d1.record(cs)
            copied[k % len(bufs)] = d1
            marks.append((c0, c1, d0, d1))
        for col, val in bufs:  # the copy stream reads them after the loop
            col.record_stream(cs)
            val.record_stream(cs)
        cs.synchronize()
        main.synchronize()
        if timing is not None:
            timing.update(
                h2d=t0.elapsed_time(t_h2d), plan_symbolic=t_h2d.elapsed_time(t_sym),
                rowptr_d2h=t_sym.elapsed_time(t_rp),
                slab_setup=t_rp.elapsed_time(marks[0][0]) if marks else 0.0,
                numeric=sum(c0.elapsed_time(c1) for c0, c1, _, _ in marks),
                d2h=marks[0][2].elapsed_time(marks[-1][3]) if marks else 0.0,
                total=t0.elapsed_time(marks[-1][3]) if marks else t0.elapsed_time(t_rp),
                slabs=len(slabs))
    finally:
        plan.free()
    return o_rp[:A.n_rows + 1], o_col[:nnz], o_val[:nnz]


def spgemm(A: DeviceCSR, B: DeviceCSR, params: Params | None = None, stream=None) -> DeviceCSR:
    """C = A * B on the GPU (plan, symbolic, allocate, numeric)."""
    plan = Plan(A, B, params, stream)
    try:
        plan.symbolic()
        col, val = plan.numeric()
        return DeviceCSR(A.n_rows, B.n_cols, plan.c_row_ptr, col, val)
    finally:
        plan.free()
