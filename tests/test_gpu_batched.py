"""Batched products (many C_i = A_i * B_i in shared launches) against the
oracle, product by product: structure bit-exact, values within the parity
rule; plus the same products computed one call at a time, CUDA-graph replay
with new values, non-square and empty products, and the device-drawn
batched workload (sampled products checked against the oracle)."""
import math

import numpy as np
import pytest

import oracle
from paper_2501_07056_gb300 import inputs
from tests._util import random_pattern_csr, values_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _check_product(bp, i, A, B):
    C = bp.result(i)
    rp = C.row_ptr.cpu().numpy()
    col = C.col.cpu().numpy()
    val = C.val.cpu().numpy()
    ref = oracle.spgemm(A, B, threads=8)
    assert np.array_equal(rp, ref.row_ptr), "product %d row_ptr" % i
    assert np.array_equal(col, ref.col), "product %d columns" % i
    ok = values_close(val, ref.val, ref.abs)
    assert ok.all(), "product %d values" % i
    return ref


def _problems(count, seed, n_lo=16, n_hi=3000, kmin=2, kmax=32):
    rng = np.random.default_rng(seed)
    ns = np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count))).astype(int)
    return [(inputs.ragged_ctr(int(n), int(n), kmin, kmax, seed, 2 * i + 1),
             inputs.ragged_ctr(int(n), int(n), kmin, kmax, seed, 2 * i + 2))
            for i, n in enumerate(ns)]


def _run(problems, params=None):
    import torch
    from paper_2501_07056_gb300 import magnus
    dev = [(magnus.DeviceCSR.from_host(A), magnus.DeviceCSR.from_host(B)) for A, B in problems]
    bp = magnus.BatchPlan([a for a, _ in dev], [b for _, b in dev], params)
    bp.symbolic()
    bp.numeric()
    torch.cuda.synchronize()
    return bp, dev


def test_batched_matches_oracle():
    probs = _problems(60, seed=0)
    bp, _ = _run(probs)
    assert bp.c_offsets[0] == 0
    for i, (A, B) in enumerate(probs):
        _check_product(bp, i, A, B)
    bp.free()


@pytest.mark.parametrize("cat", [0, 1, 2, 3])
def test_batched_forced_categories(cat):
    from paper_2501_07056_gb300 import magnus
    probs = _problems(12, seed=1, n_hi=900, kmax=20)
    params = magnus.make_params(force_category=cat)
    bp, _ = _run(probs, params)
    for i, (A, B) in enumerate(probs):
        _check_product(bp, i, A, B)
    bp.free()


def test_batched_equals_single_calls():
    import torch
    from paper_2501_07056_gb300 import magnus
    probs = _problems(20, seed=2)
    bp, dev = _run(probs)
    for i, (dA, dB) in enumerate(dev):
        C = magnus.spgemm(dA, dB)
        torch.cuda.synchronize()
        Cb = bp.result(i)
        assert torch.equal(C.row_ptr, Cb.row_ptr)
        assert torch.equal(C.col, Cb.col)
        ref = oracle.spgemm(*probs[i])
        ok = values_close(Cb.val.cpu().numpy(), C.val.cpu().numpy(), ref.abs)
        assert ok.all()
    bp.free()


def test_batched_nonsquare_and_empty():
    rng = np.random.default_rng(5)
    probs = []
    for (m, k, n, d) in [(7, 9, 4, 0.4), (0, 3, 5, 0.5), (5, 6, 8, 0.0), (1, 1, 1, 1.0),
                         (40, 30, 300, 0.2), (3, 0, 6, 0.5), (64, 64, 64, 0.1)]:
        probs.append((random_pattern_csr(rng, m, k, d), random_pattern_csr(rng, k, n, d)))
    bp, _ = _run(probs)
    for i, (A, B) in enumerate(probs):
        _check_product(bp, i, A, B)
    bp.free()


def test_batched_graph_replay_with_new_values():
    import torch
    from paper_2501_07056_gb300 import magnus
    probs = _problems(25, seed=3)
    dev = [(magnus.DeviceCSR.from_host(A), magnus.DeviceCSR.from_host(B)) for A, B in probs]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        bp = magnus.BatchPlan([a for a, _ in dev], [b for _, b in dev],
                              magnus.make_params(numeric_graph=1), s)
        bp.symbolic()
        bp.numeric()
        s.synchronize()
        for i, (A, B) in enumerate(probs):
            _check_product(bp, i, A, B)
        # new values in place, then the replayed graph
        for r in range(2):
            for i, (A, B) in enumerate(probs):
                A.val = np.cos(A.val * (r + 2)) + 0.25
                B.val = np.sin(B.val * (r + 3))
                dev[i][0].val.copy_(torch.from_numpy(A.val))
                dev[i][1].val.copy_(torch.from_numpy(B.val))
            bp.numeric()
            s.synchronize()
            for i, (A, B) in enumerate(probs):
                _check_product(bp, i, A, B)
    bp.free()


def test_single_plan_graph_replay():
    import torch
    from paper_2501_07056_gb300 import magnus
    A = inputs.rmat(11, 16, seed=0, matrix_id=4)
    dA = magnus.DeviceCSR.from_host(A)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan = magnus.Plan(dA, dA, magnus.make_params(numeric_graph=1), s)
        plan.symbolic()
        col = torch.empty(plan.nnz_c, dtype=torch.int32, device="cuda")
        val = torch.empty(plan.nnz_c, dtype=torch.float64, device="cuda")
        n0 = magnus.magnus_launch_count()
        for r in range(3):
            A.val = np.cos(A.val * (r + 1))
            dA.val.copy_(torch.from_numpy(A.val))
            plan.numeric(col, val)
            s.synchronize()
            ref = oracle.spgemm(A, A)
            assert np.array_equal(col.cpu().numpy(), ref.col)
            assert values_close(val.cpu().numpy(), ref.val, ref.abs).all()
        assert magnus.magnus_launch_count() > n0
        plan.free()


def test_batched_device_drawn_workload_sampled():
    """The batched workload's shape (n_i log-uniform, 2-32 nnz/row) drawn on
    the device; a sample of products is checked against the oracle."""
    import torch
    from paper_2501_07056_gb300 import gen_device, magnus
    rng = np.random.default_rng(7)
    ns = np.rint(np.exp(rng.uniform(math.log(256), math.log(65536), size=96))).astype(int)
    As = [gen_device.ragged(int(n), int(n), 2, 32, 0, 2 * i + 1) for i, n in enumerate(ns)]
    Bs = [gen_device.ragged(int(n), int(n), 2, 32, 0, 2 * i + 2) for i, n in enumerate(ns)]
    bp = magnus.BatchPlan(As, Bs)
    bp.symbolic()
    bp.numeric()
    torch.cuda.synchronize()
    for i in [0, 1, int(np.argmax(ns)), int(np.argmin(ns)), 50, 95]:
        n = int(ns[i])
        A = inputs.ragged_ctr(n, n, 2, 32, 0, 2 * i + 1)
        B = inputs.ragged_ctr(n, n, 2, 32, 0, 2 * i + 2)
        _check_product(bp, i, A, B)
    bp.free()


def test_batched_config_shape_first_wave():
    """The batched workload exactly as the benchmark runs it: the first of
    its four waves (products 0..1023 of 4096, n_i log-uniform in
    [256, 65536], 2-32 nnz per row, drawn on the device from the same matrix
    ids) in one batched plan with the automatic parameters; 130 products
    (every eighth, the largest and the smallest) are checked against the
    oracle entry by entry."""
    import torch
    from paper_2501_07056_gb300 import gen_device, magnus
    ns = inputs.batched_sizes(4096, seed=0)[:1024]
    As = [gen_device.ragged(int(n), int(n), 2, 32, 0, 2 * i + 1) for i, n in enumerate(ns)]
    Bs = [gen_device.ragged(int(n), int(n), 2, 32, 0, 2 * i + 2) for i, n in enumerate(ns)]
    bp = magnus.BatchPlan(As, Bs)
    bp.symbolic()
    bp.numeric()
    torch.cuda.synchronize()
    check = sorted(set(range(0, 1024, 8)) | {int(np.argmax(ns)), int(np.argmin(ns))})
    assert len(check) >= 64
    for i in check:
        n = int(ns[i])
        A = inputs.ragged_ctr(n, n, 2, 32, 0, 2 * i + 1)
        B = inputs.ragged_ctr(n, n, 2, 32, 0, 2 * i + 2)
        _check_product(bp, i, A, B)
    bp.free()


@pytest.mark.parametrize("blocks", [1, 3, 8])
def test_spgemm_host_pipelined(blocks):
    """Host operands and host result, computed in row blocks on several
    streams with the copies back overlapping the next blocks."""
    import torch
    from paper_2501_07056_gb300 import magnus
    A = inputs.ragged(5000, 3000, 0, 30, seed=8, matrix_id=1)
    B = inputs.ragged(3000, 9000, 0, 30, seed=8, matrix_id=2)
    ref = oracle.spgemm(A, B)
    for out in (None, "pre"):
        o = None
        if out == "pre":
            n = int(ref.row_ptr[-1])
            o = (torch.empty(A.n_rows + 1, dtype=torch.int64).pin_memory(),
                 torch.empty(n + 5, dtype=torch.int32).pin_memory(),
                 torch.empty(n + 5, dtype=torch.float64).pin_memory())
        rp, col, val = magnus.spgemm_host(A, B, blocks=blocks, out=o)
        assert np.array_equal(rp.numpy(), ref.row_ptr)
        assert np.array_equal(col.numpy(), ref.col)
        assert values_close(val.numpy(), ref.val, ref.abs).all()
    # C = A * A with one copy of A
    S = inputs.uniform(4096, 4096, 8, seed=0)
    rp, col, val = magnus.spgemm_host(S, S, blocks=blocks)
    refs = oracle.spgemm(S, S)
    assert np.array_equal(rp.numpy(), refs.row_ptr) and np.array_equal(col.numpy(), refs.col)
    # a product with no entries: one empty slab, nothing copied back
    Z = inputs.ragged(64, 64, 0, 0, seed=1, matrix_id=3)
    rp, col, val = magnus.spgemm_host(Z, Z, blocks=blocks)
    assert rp.numel() == 65 and int(rp.sum()) == 0 and col.numel() == 0 and val.numel() == 0
