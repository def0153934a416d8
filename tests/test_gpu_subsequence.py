"""GPU recovery of one longest common subsequence (Hirschberg on the boundary
engine): the pairs must form a common subsequence (a[ai] == b[bj], both
strictly increasing) whose length is the oracle's LCS length.  Which longest
subsequence comes back is not unique, so only these properties are checked."""
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


def recover(ctx, a, b):
    import torch
    da = torch.from_numpy(np.ascontiguousarray(a)).cuda() if a.size else torch.zeros(1, dtype=torch.uint8, device="cuda")[:0]
    db = torch.from_numpy(np.ascontiguousarray(b)).cuda() if b.size else torch.zeros(1, dtype=torch.uint8, device="cuda")[:0]
    ai, bj = P.paco_lcs_subsequence(ctx, da, db)
    return ai.cpu().numpy(), bj.cpu().numpy()


def check(ctx, a, b):
    ai, bj = recover(ctx, a, b)
    L = oracle.lcs(a, b)[0] if a.size and b.size else 0
    assert ai.size == L, (ai.size, L, a.size, b.size)
    if L:
        assert np.all(np.diff(ai) > 0) and np.all(np.diff(bj) > 0)
        assert ai[0] >= 0 and ai[-1] < a.size and bj[0] >= 0 and bj[-1] < b.size
        assert np.array_equal(a[ai], b[bj])


@pytest.mark.parametrize("n,m,sigma", [(0, 5, 4), (5, 0, 4), (1, 1, 2), (1, 40, 4), (40, 1, 4), (2, 2, 2),
                                       (31, 32, 4), (100, 1000, 4), (1000, 100, 20), (2049, 1500, 4),
                                       (3001, 2999, 256), (5000, 4800, 2)])
def test_random_pairs(ctx, n, m, sigma):
    a = W.symbols(n + 7 * m + sigma, 0, n, sigma)
    b = W.symbols(n + 7 * m + sigma, 1, m, sigma)
    check(ctx, a, b)


def test_identical_disjoint_and_mutated(ctx):
    a = W.symbols(3, 0, 4000, 20)
    ai, bj = recover(ctx, a, a)
    assert np.array_equal(ai, np.arange(a.size)) and np.array_equal(bj, np.arange(a.size))
    ai, bj = recover(ctx, a % 10, (a % 10) + 10)
    assert ai.size == 0
    b = W.mutate_rate(a, 20, 0.15, 3, 1)
    check(ctx, a, b)
    check(ctx, b, a)


def test_medium_mutated_pair(ctx):
    a = W.symbols(4, 0, 20000, 4)
    b = W.mutate_rate(a, 4, 0.2, 4, 1)
    check(ctx, a, b)


@pytest.mark.slow
def test_full_size_mutated_pair(ctx):
    """The 131072-square mutated pair: length from the (parity-tested) pair
    path, validity of every index pair."""
    import torch
    p = W.single_mutated()
    da, db = torch.from_numpy(p.a).cuda(), torch.from_numpy(p.b).cuda()
    L = int(P.paco_lcs_length(ctx, da, db).item())
    ai, bj = P.paco_lcs_subsequence(ctx, da, db)
    ai, bj = ai.cpu().numpy(), bj.cpu().numpy()
    assert ai.size == L
    assert np.all(np.diff(ai) > 0) and np.all(np.diff(bj) > 0)
    assert np.array_equal(p.a[ai], p.b[bj])
