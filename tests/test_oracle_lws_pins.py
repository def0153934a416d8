"""Pins of the 1D-problem oracle (least weight subsequence, Eq. (1D) of
Sec. "PACO 1D") to facts that do not come from the oracle:

* the weight itself, written here a second time from its definition
  (MurmurHash3's fmix32 finaliser and the capped square), on random (i, j);
* D[j] as the cheapest chain 0 = i_0 < i_1 < ... < i_k = j, found by
  listing every chain (all 2^(j-1) subsets of the inner points);
* D as single-source shortest paths on the DAG i -> j (i < j) by the
  Dijkstra routine of scipy, on up to 1500 points;
* closed forms of the test weight families: (j - i)^2 -> unit steps,
  a constant -> one jump, the capped square alone -> the balanced split of
  j into parts near T;
* the returned argmin reaches D.

CPU only."""
from itertools import combinations

import numpy as np
import pytest

import oracle

T = 40


def fmix32(h):
    h &= 0xFFFFFFFF
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & 0xFFFFFFFF
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & 0xFFFFFFFF
    h ^= h >> 16
    return h


def w_def(kind, i, j, seed=0):
    if kind in (0, 3):
        d = j - i - T
        q = d * d if -4096 < d < 4096 else 1 << 24
        if kind == 0:
            q += fmix32(((i * 0x9E3779B1) & 0xFFFFFFFF) ^ j ^ seed) & 255
        return q
    if kind == 1:
        return (j - i) ** 2
    return T


def w_vec(i, j, seed):
    """The benchmark weight on numpy int64 arrays (kind 0)."""
    d = j - i - T
    q = np.where(np.abs(d) < 4096, d * d, 1 << 24)
    h = ((i * 0x9E3779B1) & 0xFFFFFFFF) ^ j ^ seed
    h = h & 0xFFFFFFFF
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & 0xFFFFFFFF
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & 0xFFFFFFFF
    h ^= h >> 16
    return q + (h & 255)


def test_fmix32_is_the_published_finaliser():
    # the finaliser is a bijection of 32-bit words that fixes 0
    assert fmix32(0) == 0
    xs = np.random.default_rng(1).integers(0, 1 << 32, 2000, dtype=np.uint64)
    assert len({fmix32(int(x)) for x in xs}) == len(set(int(x) for x in xs))


@pytest.mark.parametrize("seed", [0, 7, 0xDEADBEEF])
def test_weight_matches_its_definition(seed):
    rng = np.random.default_rng(seed & 0xFFFF)
    for _ in range(500):
        i = int(rng.integers(0, 1 << 20))
        j = i + 1 + int(rng.integers(0, 9000))
        for kind in range(4):
            assert oracle.lws_weight(kind, i, j, T, seed) == w_def(kind, i, j, seed), (kind, i, j)
    # both sides of the cap on the squared term
    for jump in (T - 4097, T - 4096, T - 4095, T + 4095, T + 4096, T + 4097, 1, T):
        if jump < 1:
            continue
        for kind in (0, 3):
            assert oracle.lws_weight(kind, 1000, 1000 + jump, T, seed) == w_def(kind, 1000, 1000 + jump, seed), jump


@pytest.mark.parametrize("kind,seed", [(0, 0), (0, 11), (3, 0), (1, 0), (2, 0)])
def test_every_chain_enumerated(kind, seed):
    n = 13
    D, arg = oracle.lws(n, 5, kind, T, seed)
    for j in range(1, n + 1):
        best = None
        for k in range(j):
            for inner in combinations(range(1, j), k):
                pts = (0,) + inner + (j,)
                cost = 5 + sum(w_def(kind, a, b, seed) for a, b in zip(pts, pts[1:]))
                best = cost if best is None else min(best, cost)
        assert D[j] == best, (kind, j)


@pytest.mark.parametrize("n,seed", [(300, 3), (1500, 1234)])
def test_dijkstra_on_the_dag(n, seed):
    """Single-source shortest paths from point 0 over the edges i -> j,
    i < j, weighted by w (explicit zero weights stay edges in a CSR matrix),
    by scipy's Dijkstra."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import dijkstra
    i, j = np.triu_indices(n + 1, k=1)
    w = w_vec(i.astype(np.int64), j.astype(np.int64), seed)
    G = csr_matrix((w.astype(np.float64), (i, j)), shape=(n + 1, n + 1))
    assert G.nnz == w.size
    dist = dijkstra(G, directed=True, indices=0)
    D, _ = oracle.lws(n, 0, 0, T, seed)
    assert np.array_equal(dist.astype(np.int64), D)


def test_closed_forms_of_test_families():
    n = 3000
    D1, _ = oracle.lws(n, 9, 1, T)
    assert np.array_equal(D1, 9 + np.arange(n + 1))          # (j - i)^2: unit steps are cheapest
    D2, _ = oracle.lws(n, 9, 2, T)
    assert D2[0] == 9 and np.all(D2[1:] == 9 + T)             # constant: one jump
    D3, _ = oracle.lws(n, 0, 3, T)
    for j in range(1, n + 1, 7):
        best = None
        for k in range(1, j + 1):
            q, r = divmod(j, k)
            cost = r * (q + 1 - T) ** 2 + (k - r) * (q - T) ** 2
            best = cost if best is None else min(best, cost)
        assert D3[j] == best, j


def test_argmin_reaches_the_minimum():
    n = 2000
    D, arg = oracle.lws(n, 0, 0, T, 99)
    for j in range(1, n + 1, 3):
        i = int(arg[j])
        assert 0 <= i < j and D[j] == D[i] + w_def(0, i, j, 99)
