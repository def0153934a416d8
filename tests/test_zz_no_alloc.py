"""The allocation-free entry point (paco_lcs_boundaries_static) against the
context entry point, bit-exact, on two calls in a row.  This file is
collected last on purpose."""
import numpy as np
import pytest

import paper_2011_01441_gb300 as P
from paper_2011_01441_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_static_scratch_matches_context_path_twice():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    ctx = P.Context(0)
    try:
        cases = [(W.symbols(71, 0, 7000, 20), None), (W.symbols(72, 0, 2500, 4), None)]
        cases[0] = (cases[0][0], W.mutate_rate(cases[0][0], 20, 0.15, 71, 1))
        cases[1] = (cases[1][0], W.symbols(72, 1, 9000, 4))  # wider than tall: bits along b
        for a_np, b_np in cases:  # two calls in a row on the shared scratch
            a = torch.from_numpy(a_np).cuda()
            b = torch.from_numpy(b_np).cuda()
            L1, r1, c1 = P.paco_lcs_boundaries(ctx, a, b)
            ctx.sync()
            L2, r2, c2 = P.paco_lcs_boundaries_static(a, b)
            torch.cuda.synchronize()
            assert int(L2.item()) == int(L1.item())
            assert torch.equal(r1, r2) and torch.equal(c1, c2)
    finally:
        ctx.close()


def test_static_scratch_rejects_tables_beyond_its_limit():
    import torch
    big = torch.zeros(9_000_000, dtype=torch.uint8, device="cuda")
    with pytest.raises(P.PacoError) as e:
        P.paco_lcs_boundaries_static(big, big, want_rows=False, want_cols=False)
    assert e.value.status == P.PACO_EINVAL
