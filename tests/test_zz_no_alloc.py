"""The allocation-free entry point (paco_lcs_boundaries_static) against the
context entry point and the oracle, bit-exact, on calls in a row that share
its one scratch array.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2011_01441_gb300 as P
from paper_2011_01441_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _both(ctx, a_np, b_np):
    import torch
    a = torch.from_numpy(a_np).cuda()
    b = torch.from_numpy(b_np).cuda()
    L1, r1, c1 = P.paco_lcs_boundaries(ctx, a, b)
    ctx.sync()
    L2, r2, c2 = P.paco_lcs_boundaries_static(a, b, checked=True)
    torch.cuda.synchronize()
    assert int(L2.item()) == int(L1.item())
    assert torch.equal(r1, r2) and torch.equal(c1, c2)
    return int(L2.item()), r2.cpu().numpy(), c2.cpu().numpy()


def test_static_scratch_matches_context_path_twice():
    import __graft_entry__
    __graft_entry__.build()
    ctx = P.Context(0)
    try:
        a0 = W.symbols(71, 0, 7000, 20)
        a1 = W.symbols(72, 0, 2500, 4)
        cases = [(a0, W.mutate_rate(a0, 20, 0.15, 71, 1)),
                 (a1, W.symbols(72, 1, 9000, 4))]  # wider than tall: bits along b
        for a_np, b_np in cases:  # two calls in a row on the shared scratch
            L, row, col = _both(ctx, a_np, b_np)
            Lo, rowo, colo = oracle.lcs(a_np, b_np)
            assert L == Lo and np.array_equal(row, rowo) and np.array_equal(col, colo)
    finally:
        ctx.close()


def test_static_scratch_two_words_per_lane_and_empty_sides():
    # a tall, narrow table: the planner gives each lane two 31-row words and
    # the kernel computes the strip split in place (no strip table)
    plan = P.paco_plan_pair(300000, 256, 152)
    assert plan["words_per_lane"] == 2
    ctx = P.Context(0)
    try:
        a = W.symbols(73, 0, 300000, 4)
        b = W.symbols(73, 1, 256, 4)
        L, row, col = _both(ctx, a, b)
        Lo, rowo, colo = oracle.lcs(a, b)
        assert L == Lo and np.array_equal(row, rowo) and np.array_equal(col, colo)
        for n, m in ((0, 50), (50, 0), (0, 0)):
            _both(ctx, W.symbols(74, 0, n, 4), W.symbols(74, 1, m, 4))
    finally:
        ctx.close()


def test_static_scratch_just_under_its_limit():
    # 350000 x 350000: the carry rows take about 31 of the 32 MiB
    ctx = P.Context(0)
    try:
        a = W.symbols(75, 0, 350000, 20)
        b = W.mutate_rate(a, 20, 0.15, 75, 1)[:350000]
        _both(ctx, a, b)
    finally:
        ctx.close()


def test_static_scratch_rejects_tables_beyond_its_limit_and_a_missing_length():
    import torch
    big = torch.zeros(9_000_000, dtype=torch.uint8, device="cuda")
    with pytest.raises(P.PacoError) as e:
        P.paco_lcs_boundaries_static(big, big, want_rows=False, want_cols=False)
    assert e.value.status == P.PACO_EINVAL
    small = torch.zeros(100, dtype=torch.uint8, device="cuda")
    rc = P.load().paco_lcs_boundaries_static(ctypes.c_void_p(small.data_ptr()), 100,
                                             ctypes.c_void_p(small.data_ptr()), 100, None, None, None, None)
    assert rc == P.PACO_EINVAL  # no d_len: a device-side error would have nowhere to go
