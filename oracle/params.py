"""Oracle for the paper's chunk-count model (Section 3.5, Eq. 2-7).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark baseline leg).

Each function is the equation written out in plain Python floats.  The
library's own chunk planner is re-derived for GPU shared memory and L2 and
shares nothing with this file; the tests use this module to pin the paper's
arithmetic to the numbers the paper prints (coarse-level crossovers at
m_C = 2^30 on a 1 MB L2 and 2^32 on a 2 MB L2, Section 4.3; 2^12 optimal fine
chunks for the 2^29 microbenchmark, Section 4.1.2).

Readings taken where the text leaves room:
  * "rounded to the nearest power of two" (Eq. 3 and Eq. 6) is read as the
    power of two that minimises Eq. 2.  Eq. 2 written in t = ln(n) is
    symmetric about the optimum, so this is rounding log2(n) to the nearest
    integer.
  * m_C is first ceiled to a power of two (Section 3.5); m_CmaxL2 from Eq. 5
    is floored to a power of two.
"""
from __future__ import annotations

import math


def ceil_pow2(x: float) -> int:
    """Smallest power of two >= x (x >= 1)."""
    if x <= 1:
        return 1
    return 1 << math.ceil(math.log2(x) - 1e-12)


def floor_pow2(x: float) -> int:
    """Largest power of two <= x (x >= 1)."""
    if x < 1:
        raise ValueError("x < 1")
    p = 1 << int(math.floor(math.log2(x)))
    while p * 2 <= x:
        p *= 2
    while p > x:
        p //= 2
    return p


def s_chunk_fine(s_histo: int = 4, s_prefix: int = 4, s_cache_line: int = 64) -> float:
    """Per-chunk reorder storage: histogram entry + prefix-sum entry + two
    active cache lines (colFine and valFine), Section 3.5."""
    return s_histo + s_prefix + 2 * s_cache_line


def s_dense_accum(phase: str, s_val: int = 4) -> float:
    """Bytes per accumulator column: value + bitmap byte (numeric) or the
    bitmap byte alone (symbolic), Section 3.5."""
    if phase == "numeric":
        return s_val + 1
    if phase == "symbolic":
        return 1
    raise ValueError(phase)


def s_fine_level(m_c: float, n_chunks_fine: float, s_da: float, s_cf: float) -> float:
    """Eq. 2: storage of the cached fine-level structures."""
    return m_c * s_da / n_chunks_fine + n_chunks_fine * s_cf


def n_chunks_fine_continuous(m_c: float, s_da: float, s_cf: float) -> float:
    """Eq. 3 before rounding: the minimiser of Eq. 2."""
    return math.sqrt(m_c * s_da / s_cf)


def round_pow2_min_eq2(x: float) -> int:
    """Power of two nearest to x in log2 (= the power of two minimising
    Eq. 2 when x is its continuous minimiser)."""
    return 1 << max(0, int(math.floor(math.log2(x) + 0.5)))


def n_chunks_fine(m_c: float, s_da: float, s_cf: float) -> int:
    """Eq. 3: optimal fine chunks, fine level alone."""
    return round_pow2_min_eq2(n_chunks_fine_continuous(m_c, s_da, s_cf))


def s_fine_level_optimal(m_c: float, s_da: float, s_cf: float) -> float:
    """Eq. 4: Eq. 2 evaluated at the continuous optimum of Eq. 3."""
    return 2.0 * math.sqrt(m_c * s_da * s_cf)


def m_c_max_l2(s_l2: float, s_da: float, s_cf: float) -> int:
    """Eq. 5 floored to a power of two: the widest column range whose optimal
    fine-level structures still fit in s_l2."""
    return floor_pow2(s_l2 * s_l2 / (4.0 * s_da * s_cf))


def n_chunks_fine_two_level(s_l2: float, s_da: float, s_cf: float) -> int:
    """Eq. 6: fine chunks once the coarse level is in use."""
    return round_pow2_min_eq2(math.sqrt(m_c_max_l2(s_l2, s_da, s_cf) * s_da / s_cf))


def n_chunks_coarse(m_c: int, s_l2: float, s_da: float, s_cf: float) -> int:
    """Eq. 7: coarse chunks = m_C / m_CmaxL2 (m_C ceiled to a power of two;
    1 when the fine level alone suffices)."""
    mc = ceil_pow2(m_c)
    return max(1, mc // m_c_max_l2(s_l2, s_da, s_cf))


def plan(m_c: int, s_l2: int, s_cache_line: int = 64, s_val: int = 4, phase: str = "numeric"):
    """All chunk parameters of Section 3.5 for one phase."""
    s_da = s_dense_accum(phase, s_val)
    s_cf = s_chunk_fine(4, 4, s_cache_line)
    mc = ceil_pow2(m_c)
    mmax = m_c_max_l2(s_l2, s_da, s_cf)
    if mc <= mmax:
        nf = n_chunks_fine(mc, s_da, s_cf)
        return dict(m_c=mc, coarse=False, n_chunks_coarse=1, n_chunks_fine=nf,
                    chunk_len_fine=max(1, mc // nf), m_c_max_l2=mmax)
    nf = n_chunks_fine_two_level(s_l2, s_da, s_cf)
    return dict(m_c=mc, coarse=True, n_chunks_coarse=mc // mmax, n_chunks_fine=nf,
                chunk_len_fine=max(1, mmax // nf), m_c_max_l2=mmax)
