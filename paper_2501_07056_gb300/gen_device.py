"""Binding of the on-device input generators (libmagnus_inputs.so).

Input generation only: it draws the synthetic operands of the batched and
served workloads on the GPU (far faster than numpy for billions of entries).
The definitions are in include/magnus_inputs.h; ``inputs.ragged_ctr`` and
``inputs.stencil27`` are the host twins, equal bit for bit.
"""
from __future__ import annotations

import ctypes
import os

from .magnus import DeviceCSR

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmagnus_inputs.so")

c_i32, c_i64, c_u64, c_p, c_f64 = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                   ctypes.c_void_p, ctypes.c_double)
SIGNATURES = {
    "magnus_gen_ragged_rowptr": (c_i32, [c_i64, c_i64, c_i32, c_i32, c_u64, c_u64, c_p,
                                         ctypes.POINTER(c_i64), c_p]),
    "magnus_gen_ragged_fill": (c_i32, [c_i64, c_i64, c_i32, c_i32, c_u64, c_u64, c_f64, c_f64,
                                       c_p, c_p, c_p, c_p]),
    "magnus_gen_stencil27": (c_i32, [c_i32, c_p, c_p, c_p, c_p]),
    "magnus_gen_stratified": (c_i32, [c_i64, c_i64, c_i32, c_u64, c_u64, c_f64, c_f64, c_p, c_p,
                                      c_p, c_p]),
    "magnus_gen_uniform_stream": (c_i32, [c_i64, c_i64, c_u64, c_u64, c_f64, c_f64, c_p, c_p, c_p]),
}
_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmagnus_inputs.so is not built (run __graft_entry__.build())")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _LIB = lib
    return _LIB


def _check(st, where):
    if st != 0:
        raise RuntimeError("%s failed with status %d" % (where, st))


def ragged(n_rows: int, n_cols: int, kmin: int, kmax: int, seed: int = 0, matrix_id: int = 0,
           lo: float = -1.0, hi: float = 1.0, device="cuda", stream=None) -> DeviceCSR:
    """The ragged matrix of ``inputs.ragged_ctr``, drawn on the device."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream(device)
    rp = torch.empty(n_rows + 1, dtype=torch.int64, device=device)
    nnz = c_i64()
    _check(_lib().magnus_gen_ragged_rowptr(n_rows, n_cols, kmin, kmax, seed, matrix_id,
                                           rp.data_ptr(), ctypes.byref(nnz), s.cuda_stream),
           "magnus_gen_ragged_rowptr")
    col = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=device)
    val = torch.empty(max(nnz.value, 1), dtype=torch.float64, device=device)
    _check(_lib().magnus_gen_ragged_fill(n_rows, n_cols, kmin, kmax, seed, matrix_id, lo, hi,
                                         rp.data_ptr(), col.data_ptr(), val.data_ptr(),
                                         s.cuda_stream), "magnus_gen_ragged_fill")
    return DeviceCSR(n_rows, n_cols, rp, col[:nnz.value], val[:nnz.value])


def stencil27(k: int, device="cuda", stream=None) -> DeviceCSR:
    """The 27-point stencil of ``inputs.stencil27``, built on the device."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream(device)
    n = k ** 3
    nnz = (3 * k - 2) ** 3
    rp = torch.empty(n + 1, dtype=torch.int64, device=device)
    col = torch.empty(nnz, dtype=torch.int32, device=device)
    val = torch.empty(nnz, dtype=torch.float64, device=device)
    _check(_lib().magnus_gen_stencil27(k, rp.data_ptr(), col.data_ptr(), val.data_ptr(),
                                       s.cuda_stream), "magnus_gen_stencil27")
    return DeviceCSR(n, n, rp, col, val)


def stratified(n_rows: int, n_cols: int, k: int, seed: int = 0, matrix_id: int = 0,
               lo: float = -1.0, hi: float = 1.0, device="cuda", stream=None) -> DeviceCSR:
    """The stratified matrix of ``inputs.stratified``, drawn on the device."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream(device)
    nnz = n_rows * k
    rp = torch.empty(n_rows + 1, dtype=torch.int64, device=device)
    col = torch.empty(max(nnz, 1), dtype=torch.int32, device=device)
    val = torch.empty(max(nnz, 1), dtype=torch.float64, device=device)
    _check(_lib().magnus_gen_stratified(n_rows, n_cols, k, seed, matrix_id, lo, hi, rp.data_ptr(),
                                        col.data_ptr(), val.data_ptr(), s.cuda_stream),
           "magnus_gen_stratified")
    return DeviceCSR(n_rows, n_cols, rp, col[:nnz], val[:nnz])


def uniform_stream(n: int, m: int, seed: int = 0, stream_id: int = 0, lo: float = -1.0,
                   hi: float = 1.0, device="cuda", stream=None):
    """(col, val) tensors of ``inputs.uniform_stream``, drawn on the device."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream(device)
    col = torch.empty(max(n, 1), dtype=torch.int32, device=device)
    val = torch.empty(max(n, 1), dtype=torch.float64, device=device)
    _check(_lib().magnus_gen_uniform_stream(n, m, seed, stream_id, lo, hi, col.data_ptr(),
                                            val.data_ptr(), s.cuda_stream),
           "magnus_gen_uniform_stream")
    return col[:n], val[:n]
