"""The C-ABI library loads on a machine without a GPU and exports every
function declared in include/magnus.h; host-only entry points work."""
import ctypes
import os
import re

import pytest

from paper_2501_07056_gb300 import magnus

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(magnus_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return magnus._lib()


def test_every_header_is_checked():
    assert sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")) == \
        ["magnus.h", "magnus_inputs.h"]


def test_every_declared_symbol_is_exported(lib):
    names = _declared("magnus.h")
    assert len(names) >= 10
    raw = ctypes.CDLL(magnus.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n
        assert n in magnus.SIGNATURES, n


def test_input_generator_symbols_are_exported(lib):
    from paper_2501_07056_gb300 import gen_device
    names = _declared("magnus_inputs.h")
    assert len(names) == 5
    raw = ctypes.CDLL(gen_device.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n
        assert n in gen_device.SIGNATURES, n
    # the generator library holds no SpGEMM entry point
    assert not hasattr(raw, "magnus_plan")


def test_generator_rejects_bad_args_without_gpu(lib):
    from paper_2501_07056_gb300 import gen_device
    g = gen_device._lib()
    assert g.magnus_gen_ragged_rowptr(10, 10, 0, 5, 0, 0, None, None, None) == 1
    assert g.magnus_gen_ragged_rowptr(10, 10, 2, 65, 0, 0, 8, None, None) == 1
    assert g.magnus_gen_stencil27(0, 8, 8, 8, None) == 1


def test_strerror(lib):
    for s in range(0, 9):
        assert magnus._lib().magnus_strerror(s)
    assert magnus._lib().magnus_strerror(99) == b"unknown status"


def test_params_default(lib):
    p = magnus.magnus_params_default()
    assert p.force_category == -1 and p.sort_threshold == 0 and p.validate == 0


def test_plan_rejects_bad_args_without_gpu(lib):
    # NULL descriptors and shape mismatches are rejected before any CUDA call.
    h = ctypes.c_void_p()
    assert lib.magnus_plan(ctypes.byref(h), None, None, None, None) == 1
    A = magnus.CsrDesc(4, 5, 0, 8, 0, 0)
    B = magnus.CsrDesc(6, 5, 0, 8, 0, 0)
    assert lib.magnus_plan(ctypes.byref(h), ctypes.byref(A), ctypes.byref(B), None, None) == 1
    big = magnus.CsrDesc(4, 1 << 32, 0, 8, 0, 0)
    Bb = magnus.CsrDesc(1 << 32, 5, 0, 8, 0, 0)
    assert lib.magnus_plan(ctypes.byref(h), ctypes.byref(big), ctypes.byref(Bb), None, None) == 3
    # B row starts are kept in 40 bits of the segment table
    A40 = magnus.CsrDesc(4, 5, 0, 8, 0, 0)
    B40 = magnus.CsrDesc(5, 6, 1 << 40, 8, 8, 8)
    assert lib.magnus_plan(ctypes.byref(h), ctypes.byref(A40), ctypes.byref(B40), None, None) == 3
    assert lib.magnus_numeric(None, None, None, None, None, None, None) == 1
    assert lib.magnus_symbolic(None, None, None, None) == 1
    # the bounded-wait self-test checks its limit before any CUDA call
    lib.magnus_wait_selftest.argtypes = [ctypes.c_int64, ctypes.c_void_p]
    assert lib.magnus_wait_selftest(0, None) == 1
    assert lib.magnus_wait_selftest((1 << 31) + 1, None) == 1


L2 = 126 * (1 << 20)


@pytest.mark.parametrize("m_log2", [5, 10, 12, 14, 16, 20, 22, 24, 26, 28, 31])
@pytest.mark.parametrize("smem", [32 << 10, 64 << 10, 96 << 10])
@pytest.mark.parametrize("blocks", [152, 304])
def test_chunk_model_consistency(lib, m_log2, smem, blocks):
    m = magnus.magnus_chunk_model(1 << m_log2, smem, L2, blocks)
    assert m["m_c_log2"] == m_log2
    c, mm = m["chunk_len_fine_log2"], m["m_c_max_log2"]
    # accumulator + bookkeeping of the chosen fine level fit the budget
    assert (1 << c) * (8 + 1 / 8) + (1 << (mm - c)) * 8 <= smem
    # fine chunks per row bounded by the L2 write-combining share
    assert (mm - c) <= m["n_chunks_fine_max_log2"] <= 12
    assert blocks * (1 << m["n_chunks_fine_max_log2"]) * 256 <= L2 / 2
    # coarse chunks tile the column range
    assert m["n_chunks_coarse"] * (1 << mm) >= (1 << m_log2)
    if m["n_chunks_coarse"] > 1:
        assert mm < m_log2
    # symbolic: bitmap only, so its chunks are at least as long
    assert m["chunk_len_fine_sym_log2"] >= min(c, m_log2)


def test_chunk_model_minimises_eq2(lib):
    # With a generous budget the choice is the Eq. 2 minimiser over powers of
    # two: 2^c * (8 + 1/8) + 2^(M - c) * 8.
    M = 20
    m = magnus.magnus_chunk_model(1 << M, 1 << 30, 1 << 40, 1)
    costs = {c: (1 << c) * (8 + 1 / 8) + (1 << (M - c)) * 8 for c in range(5, M + 1)
             if M - c <= 12}
    assert m["chunk_len_fine_log2"] == min(costs, key=costs.get)
    assert m["n_chunks_coarse"] == 1


def test_chunk_model_invalid(lib):
    with pytest.raises(magnus.MagnusError):
        magnus.magnus_chunk_model(0, 1, 1, 1)


def _header_structs():
    """Field lists of the `typedef struct { ... } name;` blocks of magnus.h,
    as (name, C type, array length)."""
    text = open(os.path.join(ROOT, "include", "magnus.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct \{(.*?)\}\s*(\w+);", text, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"(const )?([\w ]+?)\s*(\*?)\s*(\w+)(\[(\d+)\])?$", decl)
            assert m, "cannot parse %r in %s" % (decl, name)
            ctype = "ptr" if m.group(3) else m.group(2).strip()
            fields.append((m.group(4), ctype, int(m.group(6)) if m.group(6) else 0))
        out[name] = fields
    return out


@pytest.mark.parametrize("cname,pyname", [
    ("magnus_csr_t", "CsrDesc"), ("magnus_params_t", "Params"),
    ("magnus_plan_info_t", "PlanInfo"), ("magnus_tune_report_t", "TuneReport"),
    ("magnus_microbench_t", "MicrobenchResult"), ("magnus_chunk_model_t", "ChunkModel"),
    ("magnus_rates_t", "Rates"),
])
def test_binding_structs_match_header(cname, pyname):
    # The ctypes mirrors of the ABI structs carry the header's fields in the
    # header's order with the same widths, so a renamed or inserted field in
    # either place fails here rather than as a shifted value at run time.
    widths = {"int32_t": ctypes.sizeof(ctypes.c_int32), "int64_t": 8, "float": 4,
              "double": 8, "ptr": ctypes.sizeof(ctypes.c_void_p)}
    hdr = _header_structs()[cname]
    py = getattr(magnus, pyname)._fields_
    assert [f[0] for f in hdr] == [f[0] for f in py]
    for (name, ctype, n), (_, pytype) in zip(hdr, py):
        size = widths[ctype] * (n if n else 1)
        assert ctypes.sizeof(pytype) == size, name
