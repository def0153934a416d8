"""GPU parity of the tile schedules (the paper's comparison: PACO partition,
PA p x p blocks, PO divide and conquer) run on the batch kernel: L, bottom
row and right column equal the oracle's bit for bit."""
import numpy as np
import pytest

import oracle
import paper_2011_01441_gb300 as P
from paper_2011_01441_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    c = P.Context(0)
    yield c
    c.close()


def run(ctx, a, b, kind, base=0):
    import torch
    ctx.set_option(P.OPT_TILES, kind)
    ctx.set_option(P.OPT_TILE_BASE, base)
    try:
        L, row, col = P.paco_lcs_boundaries(ctx, torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
        ctx.sync()
        return int(L.item()), row.cpu().numpy(), col.cpu().numpy()
    finally:
        ctx.set_option(P.OPT_TILES, 0)
        ctx.set_option(P.OPT_TILE_BASE, 0)


@pytest.mark.parametrize("kind", [P.TILES_PACO, P.TILES_PA, P.TILES_PO])
@pytest.mark.parametrize("n,m", [(1, 1000), (1000, 1), (62, 64), (4096, 4096), (5000, 3001), (3001, 5000),
                                 (20000, 19000)])
def test_tile_schedules_match_oracle(ctx, kind, n, m):
    a = W.symbols(n + m + kind, 0, n, 4)
    b = W.mutate_rate(a, 4, 0.15, kind, 1)[:m] if m <= n else W.symbols(n + m + kind, 1, m, 4)
    got = run(ctx, a, b, kind)
    want = oracle.lcs(a, b)
    assert got[0] == want[0]
    assert np.array_equal(got[1], want[1]) and np.array_equal(got[2], want[2])


@pytest.mark.parametrize("kind,base", [(P.TILES_PACO, 1), (P.TILES_PACO, 16), (P.TILES_PO, 1), (P.TILES_PO, 4)])
def test_tile_bases(ctx, kind, base):
    a = W.symbols(70 + base, 0, 9000, 20)
    b = W.symbols(70 + base, 1, 7000, 20)
    got = run(ctx, a, b, kind, base)
    want = oracle.lcs(a, b)
    assert got[0] == want[0]
    assert np.array_equal(got[1], want[1]) and np.array_equal(got[2], want[2])


def test_tile_schedules_take_zero_boundaries_only(ctx):
    import torch
    a = torch.from_numpy(W.symbols(1, 0, 100, 4)).cuda()
    b = torch.from_numpy(W.symbols(1, 1, 100, 4)).cuda()
    top = torch.zeros(101, dtype=torch.int32, device="cuda")
    ctx.set_option(P.OPT_TILES, P.TILES_PA)
    try:
        with pytest.raises(P.PacoError) as e:
            P.paco_lcs_boundaries(ctx, a, b, top)
        assert e.value.status == P.PACO_EINVAL
    finally:
        ctx.set_option(P.OPT_TILES, 0)
