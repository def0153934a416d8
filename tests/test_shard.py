"""Sharding a batch of independent pairs over ranks (include/paco_plan.h,
paco_plan_shard; paper_2011_01441_gb300/shard.py): the size-balanced greedy
split on CPU, and two gloo ranks that each run their share and gather the
lengths in the batch's order.  On CPU the per-rank computation is the oracle
(passed in by the test); on GPUs it is paco_lcs_batch."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import paper_2011_01441_gb300 as P  # noqa: E402
from paper_2011_01441_gb300 import shard  # noqa: E402
from paper_2011_01441_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("ranks", [1, 2, 3, 8])
def test_every_pair_once_and_ranks_balanced(ranks):
    bt = W.batch_pairs(npairs=600)
    owner, cells = shard.paco_plan_shard(bt.a_off, bt.b_off, ranks)
    c = np.diff(bt.a_off) * np.diff(bt.b_off)
    assert owner.shape == (600,) and owner.min() >= 0 and owner.max() < ranks
    # each pair on exactly one rank, and the per-rank totals are the pairs' sums
    for r in range(ranks):
        assert cells[r] == c[owner == r].sum()
    assert cells.sum() == c.sum()
    # greedy by decreasing size: totals differ by at most one (the largest) pair
    assert cells.max() - cells.min() <= c.max()


def test_greedy_order_on_a_small_case():
    # sizes 9, 7, 5, 3, 1 on two ranks: 9 -> r0, 7 -> r1, 5 -> r1 (7 < 9), 3 -> r0 (9 < 12), 1 -> r0 or r1
    la = np.array([1, 3, 5, 7, 9])
    off = np.concatenate([[0], np.cumsum(la)]).astype(np.int64)
    ones = np.arange(6, dtype=np.int64)  # m = 1 for every pair: cells = n
    owner, cells = shard.paco_plan_shard(off, ones, 2)
    assert list(owner[[4, 3, 2, 1]]) == [0, 1, 1, 0]
    assert sorted(cells.tolist()) == [12, 13]


def test_bad_arguments():
    with pytest.raises(P.PacoError):
        shard.paco_plan_shard(np.array([0, 5, 3]), np.array([0, 1, 2]), 2)   # decreasing offsets
    with pytest.raises(P.PacoError):
        shard.paco_plan_shard(np.array([0, 1]), np.array([0, 1]), 0)         # no ranks


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    try:
        import torch.distributed as dist
        import oracle
        from paper_2011_01441_gb300 import shard as S
        from paper_2011_01441_gb300 import workloads as Wl
        dist.init_process_group("gloo", rank=rank, world_size=ws)
        bt = Wl.batch_pairs(npairs=300, hi=2048)

        def compute(a_cat, a_off, b_cat, b_off):  # the oracle stands in for the GPU batch on CPU
            return oracle.lcs_batch(a_cat, a_off, b_cat, b_off, threads=2, boundaries=False)[0]
        lens, mine = S.run_sharded_batch(bt.a_cat, bt.a_off, bt.b_cat, bt.b_off, compute)
        dist.destroy_process_group()
        q.put((rank, lens.tolist(), mine.tolist(), None))
    except Exception as e:
        q.put((rank, None, None, repr(e)))


def test_two_gloo_ranks_gather_every_length_in_order():
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, lens, mine, err in res:
        assert err is None, err
    bt = W.batch_pairs(npairs=300, hi=2048)
    want = oracle.lcs_batch(bt.a_cat, bt.a_off, bt.b_cat, bt.b_off, boundaries=False)[0]
    assert res[0][1] == res[1][1] == want.tolist()        # every rank holds all lengths, in order
    assert sorted(res[0][2] + res[1][2]) == list(range(300))  # each pair run on exactly one rank
    assert res[0][2] and res[1][2]


@pytest.mark.gpu
def test_sharded_batch_on_the_gpu_matches_the_oracle():
    """One rank (one GPU here): the sharded path with paco_lcs_batch as the
    per-rank computation gives the oracle's lengths in the batch's order."""
    import oracle
    bt = W.batch_pairs(npairs=500, hi=4096)
    ctx = P.Context(0)
    try:
        lens, mine = shard.run_sharded_batch(bt.a_cat, bt.a_off, bt.b_cat, bt.b_off,
                                             shard.batch_on_device(ctx, alphabet=4))
    finally:
        ctx.close()
    want = oracle.lcs_batch(bt.a_cat, bt.a_off, bt.b_cat, bt.b_off, boundaries=False)[0]
    assert np.array_equal(lens, want) and mine.size == 500
