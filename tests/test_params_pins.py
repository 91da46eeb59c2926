"""Pins for the paper's chunk-count model (Section 3.5, Eq. 2-7) against the
numbers printed in Section 4 and against brute-force minimisation."""
import math

import pytest

from oracle import params as P
from tests._util import golden

MB = 1 << 20
S_CF = P.s_chunk_fine(4, 4, 64)   # 4 + 4 + 2*64 = 136 bytes (Section 3.5)
PRINTED = golden("paper_printed_values.txt")


def test_s_chunk_fine_value():
    assert S_CF == 136


@pytest.mark.parametrize("l2,expect", [(MB, PRINTED["coarse_crossover_m_c_l2_1mb"]),
                                        (2 * MB, PRINTED["coarse_crossover_m_c_l2_2mb"])])
def test_coarse_crossovers_section_4_3(l2, expect):
    # Section 4.3: MAGNUS switches on the coarse level at m_C = 2^30 on SKX
    # (1 MB L2) and at 2^32 on SPR/EMR (2 MB L2), Table 1.  Eq. 5 reproduces
    # both with the bitmap-only accumulator footprint (s_denseAccum = 1).
    assert P.m_c_max_l2(l2, P.s_dense_accum("symbolic"), S_CF) == expect
    assert not P.plan(expect, l2, phase="symbolic")["coarse"]
    assert P.plan(2 * expect, l2, phase="symbolic")["coarse"]


def test_crossover_ratio_is_l2_squared():
    r = P.m_c_max_l2(2 * MB, 1, S_CF) / P.m_c_max_l2(MB, 1, S_CF)
    assert r == 4


def test_numeric_footprint_crossovers():
    # With s_denseAccum = s_val + 1 = 5 (float values) Eq. 5 gives 2^30/2^28.
    assert P.m_c_max_l2(2 * MB, 5, S_CF) == 1 << 30
    assert P.m_c_max_l2(MB, 5, S_CF) == 1 << 28


def test_reorder_breaking_point_section_4_1_2():
    # Section 4.1.2: reordering slows past 2^13 chunks on SPR, where the
    # histogram, prefix-sum and active-line storage (n * s_chunkFine) exceeds
    # the 2 MB L2.
    n_break = (2 * MB) / S_CF
    assert P.floor_pow2(n_break) == PRINTED["reorder_breaking_point_chunks"]
    # and the 2^31 * 2^13 = 2^44 column statement that follows it
    assert (1 << 31) * (1 << 13) == 1 << 44


def test_eq3_microbenchmark_arithmetic():
    # Stream length 2^29, float values (s_denseAccum = 5): sqrt(2^29*5/136)
    # = 4443, nearest power of two 2^12.
    x = P.n_chunks_fine_continuous(1 << 29, 5, S_CF)
    assert abs(x - 4443.0) < 1.0
    assert P.n_chunks_fine(1 << 29, 5, S_CF) == 1 << 12


@pytest.mark.parametrize("m_c", [1 << 10, 1 << 17, 1 << 24, 1 << 29, 3 << 20])
@pytest.mark.parametrize("s_da", [1, 5, 9])
def test_eq3_minimises_eq2_over_powers_of_two(m_c, s_da):
    best = min((P.s_fine_level(m_c, 1 << e, s_da, S_CF), 1 << e) for e in range(0, 40))[1]
    assert P.n_chunks_fine(m_c, s_da, S_CF) == best


@pytest.mark.parametrize("m_c", [1 << 12, 1 << 20, 1 << 31])
def test_eq4_is_eq2_at_optimum(m_c):
    n = P.n_chunks_fine_continuous(m_c, 5, S_CF)
    assert math.isclose(P.s_fine_level(m_c, n, 5, S_CF), P.s_fine_level_optimal(m_c, 5, S_CF),
                        rel_tol=1e-12)


@pytest.mark.parametrize("l2", [MB, 2 * MB, 3 * MB])
@pytest.mark.parametrize("s_da", [1, 5])
def test_eq5_is_largest_fitting_power_of_two(l2, s_da):
    m = P.m_c_max_l2(l2, s_da, S_CF)
    assert P.s_fine_level_optimal(m, s_da, S_CF) <= l2
    assert P.s_fine_level_optimal(2 * m, s_da, S_CF) > l2


def test_eq6_eq7_two_level():
    l2 = 2 * MB
    pl = P.plan(1 << 36, l2, phase="symbolic")
    assert pl["coarse"]
    assert pl["n_chunks_coarse"] * pl["m_c_max_l2"] == 1 << 36
    assert pl["n_chunks_fine"] == P.n_chunks_fine(pl["m_c_max_l2"], 1, S_CF)
    # Fine chunks stop growing once the coarse level is in use (Section 3.5).
    assert P.plan(1 << 38, l2, phase="symbolic")["n_chunks_fine"] == pl["n_chunks_fine"]


def test_m_c_ceiled():
    assert P.plan(3 << 20, 2 * MB)["m_c"] == 1 << 22


def test_golden_table3_transcription():
    # The transcribed Table 3 columns agree with each other: nnz_A is 16 per
    # row (edge factor 16, n = 2^scale) and nnz(A^2) / n is the printed
    # average to its printed precision, so a mistyped digit fails here.
    for scale in range(18, 24):
        n = PRINTED["rmat16_scale%d_n" % scale]
        assert n == 1 << scale
        assert PRINTED["rmat16_scale%d_nnz_a" % scale] == 16 * n
        avg = PRINTED["rmat16_scale%d_nnz_a2" % scale] / n
        assert abs(avg - PRINTED["rmat16_scale%d_avg_a2" % scale]) < 0.05 + 1e-9

