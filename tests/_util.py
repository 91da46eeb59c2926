"""Shared test helpers: the parity rule and small CSR utilities."""
import numpy as np

from paper_2501_07056_gb300.inputs import CSR

# Parity rule for FP64 values: |c - c_ref| <= RTOL * max(|c_ref|, S) where S is
# the sum of |terms| of the entry.  S bounds the rounding error of any
# summation order ((k-1) u S with u = 2^-53), so reordered sums pass while a
# dropped or wrong term does not.
RTOL = 1e-12


def values_close(val, ref, abs_sum, rtol=RTOL):
    bound = rtol * np.maximum(np.abs(ref), abs_sum)
    return np.abs(val - ref) <= bound


def transpose(M: CSR) -> CSR:
    rows = np.repeat(np.arange(M.n_rows, dtype=np.int64), np.diff(M.row_ptr))
    order = np.lexsort((rows, M.col))
    cols_t = rows[order].astype(np.int32)
    lengths = np.bincount(M.col, minlength=M.n_cols).astype(np.int64)
    rp = np.zeros(M.n_cols + 1, np.int64)
    np.cumsum(lengths, out=rp[1:])
    return CSR(M.n_cols, M.n_rows, rp, cols_t, M.val[order].copy())


def random_pattern_csr(rng, n_rows, n_cols, density, lo=-1.0, hi=1.0) -> CSR:
    pat = rng.random((n_rows, n_cols)) < density
    d = np.where(pat, rng.uniform(lo, hi, (n_rows, n_cols)), 0.0)
    rows, cols = np.nonzero(pat)
    lengths = np.bincount(rows, minlength=n_rows).astype(np.int64)
    rp = np.zeros(n_rows + 1, np.int64)
    np.cumsum(lengths, out=rp[1:])
    return CSR(n_rows, n_cols, rp, cols.astype(np.int32), d[rows, cols].astype(np.float64))


def golden(name: str) -> dict:
    """The key = value entries of tests/golden/<name> (numbers printed in the
    paper, each commented with its place there)."""
    import os
    out = {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        key, val = (x.strip() for x in line.split("=", 1))
        out[key] = float(val) if "." in val else int(val)
    return out
