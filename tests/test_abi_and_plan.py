"""CPU-only checks: the C-ABI library loads and exports every declared
symbol; the planner's partition satisfies the paper's structural claims."""
import os
import re
from collections import Counter, defaultdict

import numpy as np
import pytest

import paper_2011_01441_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(paco_[a-z0-9_]+)\s*\(", txt, re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return P.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    expected = {"paco_ctx_create", "paco_ctx_destroy", "paco_strerror", "paco_last_error",
                "paco_ctx_sync", "paco_ctx_set_option", "paco_ctx_get_option", "paco_lcs_length",
                "paco_lcs_boundaries", "paco_lcs_boundaries_host", "paco_lcs_batch",
                "paco_lcs_submit", "paco_lcs_poll", "paco_serve_get_stats",
                "paco_measure_int_peak", "paco_last_kernel_ms", "paco_plan_partition",
                "paco_plan_partition_deps", "paco_plan_pair", "paco_affine_align", "paco_affine_align_host",
                "paco_affine_batch", "paco_lws", "paco_plan_1d"}
    assert expected <= set(names), expected - set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_strerror_is_static_text(lib):
    assert P._strerror(P.PACO_ETIMEOUT) == "device wait timed out"
    assert P._strerror(P.PACO_EINVAL) == "invalid argument"


def _cover(tiles, n, m):
    grid = np.zeros((n, m), dtype=np.int32)
    for t in tiles:
        grid[t["r0"]:t["r1"], t["c0"]:t["c1"]] += 1
    return grid


@pytest.mark.parametrize("n,m,p,base", [(64, 64, 4, 2), (97, 131, 3, 2), (300, 120, 7, 3),
                                        (1000, 1000, 37, 4), (257, 257, 1, 8), (40, 40, 2, 1)])
def test_partition_exact_cover_and_topological(lib, n, m, p, base):
    tiles = P.paco_plan_partition(n, m, p, base)
    assert np.all(_cover(tiles, n, m) == 1)
    assert [t["order"] for t in tiles] == list(range(len(tiles)))
    assert all(0 <= t["owner"] < p for t in tiles)
    off, idx = P.paco_plan_partition_deps(n, m, p, base)
    for k in range(len(tiles)):
        for d in idx[off[k]:off[k + 1]]:
            assert d < k  # every dependency runs earlier on the time line
            u, t = tiles[d], tiles[k]
            touches_top = u["r1"] == t["r0"] and u["c0"] < t["c1"] and u["c1"] >= t["c0"]
            touches_left = u["c1"] == t["c0"] and u["r0"] < t["r1"] and u["r1"] >= t["r0"]
            assert touches_top or touches_left


def test_partition_dependencies_are_complete(lib):
    """Brute force: tile k must list every tile containing a cell directly
    above, directly left or diagonally above-left of one of its cells."""
    n, m, p, base = 48, 40, 3, 2
    tiles = P.paco_plan_partition(n, m, p, base)
    owner = np.full((n, m), -1)
    for k, t in enumerate(tiles):
        owner[t["r0"]:t["r1"], t["c0"]:t["c1"]] = k
    off, idx = P.paco_plan_partition_deps(n, m, p, base)
    for k, t in enumerate(tiles):
        need = set()
        for i in range(t["r0"], t["r1"]):
            for j in range(t["c0"], t["c1"]):
                for di, dj in ((-1, 0), (0, -1), (-1, -1)):
                    ii, jj = i + di, j + dj
                    if ii >= 0 and jj >= 0 and owner[ii, jj] != k:
                        need.add(int(owner[ii, jj]))
        assert need == set(int(x) for x in idx[off[k]:off[k + 1]]), k


def test_partition_p4_matches_figure(lib):
    """Fig. "PACO LCS (p=4)": the label-1 regions are the p regions of the
    middle anti-diagonal, each of side n/p; label 2 puts p regions on each of
    p-1 anti-diagonals of every corner triangle (2(p-1) per processor)."""
    n, p = 256, 4
    tiles = P.paco_plan_partition(n, n, p, 8)
    lab = defaultdict(list)
    for t in tiles:
        lab[t["label"]].append(t)
    one = lab[1]
    assert len(one) == p
    for k, t in enumerate(sorted(one, key=lambda t: t["c0"])):
        assert (t["r1"] - t["r0"], t["c1"] - t["c0"]) == (n // p, n // p)
        assert t["r0"] // (n // p) + t["c0"] // (n // p) == p - 1  # middle anti-diagonal
    two = lab[2]
    assert len(two) == 2 * p * (p - 1)
    assert all((t["r1"] - t["r0"]) == n // (2 * p) for t in two)
    assert Counter(t["owner"] for t in two) == {o: 2 * (p - 1) for o in range(p)}


@pytest.mark.parametrize("p", [2, 3, 4, 5, 7, 37])
def test_partition_label_doubling_and_balance(lib, p):
    """From label 2 on, each processor's count of label-(j+1) regions is twice
    its label-j count while regions are halved, and per-processor cell totals
    differ by no more than one base-case region per label (the "optimal
    balanced computation" criterion)."""
    n, base = 64 * p, 4
    tiles = P.paco_plan_partition(n, n, p, base)
    per_label_owner = defaultdict(Counter)
    sizes = defaultdict(set)
    for t in tiles:
        per_label_owner[t["label"]][t["owner"]] += 1
        sizes[t["label"]].add(t["r1"] - t["r0"])
    labels = sorted(per_label_owner)
    for j in labels[1:-2]:
        if j + 1 in per_label_owner and max(sizes[j + 1]) * 2 <= max(sizes[j]) + 1:
            for o in range(p):
                assert per_label_owner[j + 1][o] == 2 * per_label_owner[j][o], (j, o)
    cells = Counter()
    for t in tiles:
        cells[t["owner"]] += (t["r1"] - t["r0"]) * (t["c1"] - t["c0"])
    biggest_leaf = max((t["r1"] - t["r0"]) * (t["c1"] - t["c0"]) for t in tiles if t["label"] == labels[-1])
    assert max(cells.values()) - min(cells.values()) <= (len(labels) + 1) * max(biggest_leaf, 4 * base * base)


def test_partition_leaf_count_formula(lib):
    """Corollary on partitioning overheads: while every level is assigned in
    full groups of p, the leaves number p[1 + sum_i 2^(i-1)(p-1)]."""
    p = 4
    n = 16 * p
    tiles = P.paco_plan_partition(n, n, p, 4)
    labels = Counter(t["label"] for t in tiles)
    assert labels[1] == p
    for i in range(2, 3):
        assert labels[i] == p * (2 ** (i - 1)) * (p - 1)


@pytest.mark.parametrize("wpl", [1, 2])
@pytest.mark.parametrize("n,m,sms", [(131072, 131072, 148), (131072, 131072, 152),
                                     (1048576, 16384, 152), (16384, 1048576, 152),
                                     (4096, 4096, 152), (1000, 3, 152), (33, 1, 7)])
def test_pair_plan_balanced_strips(lib, n, m, sms, wpl):
    pl = P.paco_plan_pair(n, m, sms, words_per_lane=wpl)
    L = max(n, m)
    g = 31 * wpl  # rows of one lane: the granule of the balanced split
    assert pl["words_per_lane"] == wpl
    assert pl["L"] == L and pl["S"] == min(n, m)
    assert pl["transpose"] == (1 if m > n else 0)
    row0 = pl["row0"]
    assert row0[0] == 0 and row0[-1] == L
    h = np.diff(row0)
    assert np.all(h > 0) and np.all(row0[:-1] % g == 0)
    assert np.all(h <= pl["warps"] * 32 * g)
    if h.size > 2:
        assert h[:-1].max() - h[:-1].min() <= g  # the +-1 granule split of the p-way division
    assert pl["chunk"] in (2, 4, 8)


def test_pair_plan_default_words_per_lane(lib):
    assert P.paco_plan_pair(131072, 131072, 152)["words_per_lane"] in (1, 2)


def test_pair_plan_options(lib):
    pl = P.paco_plan_pair(5000, 7000, 152, chunk=4, warps=2, orient=1, schedule=1)
    assert pl["transpose"] == 0 and pl["chunk"] == 4 and pl["warps"] == 2
    assert list(pl["row0"]) == [0, 1984, 3968, 5000]


@pytest.mark.parametrize("kind", [1, 2, 3])
@pytest.mark.parametrize("n,m,p,base", [(131072, 131072, 152, 4), (5000, 3001, 7, 2), (62, 64, 4, 1),
                                        (100000, 1000, 152, 4)])
def test_tile_schedules_cover_and_order(lib, kind, n, m, p, base):
    """Tiles cover the table exactly, are at most 992 rows, sit on the
    31 x 64 granule grid, and every dependency precedes its tile."""
    t = P.paco_plan_tiles(n, m, p, kind, base)
    cells = 0
    for k, x in enumerate(t["tiles"]):
        assert 0 <= x["r0"] < x["r1"] <= n and 0 <= x["c0"] < x["c1"] <= m
        assert x["r1"] - x["r0"] <= 992
        assert x["r0"] % 31 == 0 and (x["r1"] % 31 == 0 or x["r1"] == n)
        assert x["c0"] % 64 == 0 and (x["c1"] % 64 == 0 or x["c1"] == m)
        cells += (x["r1"] - x["r0"]) * (x["c1"] - x["c0"])
        deps = t["dep_idx"][t["dep_off"][k]:t["dep_off"][k + 1]]
        assert np.all(deps < k)
    assert cells == n * m
    if n * m < 1e7:  # exact cover, cell by cell
        cover = np.zeros((n, m), dtype=np.int8)
        for x in t["tiles"]:
            cover[x["r0"]:x["r1"], x["c0"]:x["c1"]] += 1
        assert np.all(cover == 1)
    assert t["critical_cells"] > 0


def test_tile_schedule_critical_paths_follow_the_paper():
    """On a 131072-square table with p = 152: PA's critical path is 2 n m / p
    (its (2p - 1) blocks), PACO's is shorter, PO's fork-join path longer."""
    n = m = 131072
    p = 152
    unit = n * m / p
    pa = P.paco_plan_tiles(n, m, p, 2, 4)["critical_cells"] / unit
    paco = P.paco_plan_tiles(n, m, p, 1, 4)["critical_cells"] / unit
    po = P.paco_plan_tiles(n, m, p, 3, 16)["critical_cells"] / unit
    assert 1.95 < pa < 2.05
    assert paco < pa
    assert po > pa


# ---------------------------------------------------------------- PACO 1D

def _w1d(i, j, T=40, seed=6):
    """The benchmark weight of the 1D problem on int64 arrays (its definition)."""
    d = j - i - T
    q = np.where(np.abs(d) < 4096, d * d, 1 << 24)
    h = (((i * 0x9E3779B1) & 0xFFFFFFFF) ^ j ^ seed) & 0xFFFFFFFF
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & 0xFFFFFFFF
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & 0xFFFFFFFF
    h ^= h >> 16
    return q + (h & 255)


@pytest.mark.parametrize("n,p,base", [(100, 3, 8), (255, 4, 16), (1000, 7, 32), (513, 1, 64), (2000, 152, 64),
                                      (64, 16, 2)])
def test_plan_1d_covers_the_triangle_once(lib, n, p, base):
    r = P.paco_plan_1d(n, p, base)
    cover = np.zeros((n + 1, n + 1), dtype=np.int32)   # [i, j]
    for t in r["tasks"]:
        assert 0 <= t["proc"] < p
        if t["kind"] == 0:
            blk = cover[t["j0"]:t["j1"], t["j0"]:t["j1"]]
            blk += np.triu(np.ones_like(blk), k=1)
        else:
            assert t["i1"] <= t["j0"]                  # a square reads finished inputs only
            cover[t["i0"]:t["i1"], t["j0"]:t["j1"]] += 1
    assert np.array_equal(cover, np.triu(np.ones((n + 1, n + 1), dtype=np.int32), k=1))
    if p == 1:
        assert r["temp_words"] == 0 and all(t["merge_group"] == -1 for t in r["tasks"])


@pytest.mark.parametrize("n,p", [(4095, 4), (4095, 16), (4095, 64), (4095, 3), (4095, 152), (8191, 7)])
def test_plan_1d_square_balance_and_half_perimeters(lib, n, p):
    """Every square is split into p rectangles of area 1/p of it (up to the
    rounding of one row or column per cut), and the rectangles of the top
    square have half-perimeters O(side / sqrt(p)) (Theorem of Sec. "PACO 1D")."""
    r = P.paco_plan_1d(n, p, 64)
    by_phase = defaultdict(list)
    for t in r["tasks"]:
        if t["kind"] == 1:
            by_phase[t["phase"]].append(t)
    for ph, rects in by_phase.items():
        w = max(t["j1"] for t in rects) - min(t["j0"] for t in rects)
        h = max(t["i1"] for t in rects) - min(t["i0"] for t in rects)
        areas = Counter()
        for t in rects:
            areas[t["proc"]] += (t["j1"] - t["j0"]) * (t["i1"] - t["i0"])
        assert sum(areas.values()) == w * h
        cuts = int(np.ceil(np.log2(p))) + 1
        for a in areas.values():
            assert abs(a - w * h / p) <= cuts * (w + h), (ph, a, w * h / p)
    top = max(by_phase.values(), key=lambda rs: sum((t["j1"] - t["j0"]) * (t["i1"] - t["i0"]) for t in rs))
    side = max(t["j1"] for t in top) - min(t["j0"] for t in top)
    for t in top:
        hp = (t["j1"] - t["j0"]) + (t["i1"] - t["i0"])
        assert hp <= 4 * side / np.sqrt(p) + 2, (hp, side, p)
    if p & (p - 1) == 0:   # a power of two: alternating halvings give equal rectangles
        assert len({((t["j1"] - t["j0"]), (t["i1"] - t["i0"])) for t in top}) <= 2
    # temporary space of the input-side cuts: O(sqrt(p) n log n)
    assert r["temp_words"] <= 4 * np.sqrt(p) * (n + 1) * np.log2(n + 1)


@pytest.mark.parametrize("n,p,base", [(300, 5, 16), (777, 8, 40)])
def test_plan_1d_schedule_computes_eq_1d(lib, n, p, base):
    """Running the plan phase by phase (rectangles of a phase into the
    outputs or into their temporary buffers, merged by a min after the
    phase) gives the oracle's D: the order respects every dependency."""
    import oracle
    r = P.paco_plan_1d(n, p, base)
    D = np.full(n + 1, np.iinfo(np.int64).max // 4, dtype=np.int64)
    D[0] = 0
    by_phase = defaultdict(list)
    for t in r["tasks"]:
        by_phase[t["phase"]].append(t)
    for ph in sorted(by_phase):
        temps = {}
        for t in by_phase[ph]:
            if t["kind"] == 0:
                for j in range(max(t["j0"], 1), t["j1"]):
                    i = np.arange(t["j0"], j)
                    if i.size:
                        D[j] = min(D[j], int(np.min(D[i] + _w1d(i, j))))
            else:
                i = np.arange(t["i0"], t["i1"])[:, None]
                j = np.arange(t["j0"], t["j1"])[None, :]
                c = np.min(D[i] + _w1d(i, j), axis=0)
                if t["merge_group"] < 0:
                    D[t["j0"]:t["j1"]] = np.minimum(D[t["j0"]:t["j1"]], c)
                else:
                    temps[(t["merge_group"], t["j0"])] = (t["j0"], c)
        for j0, c in temps.values():
            D[j0:j0 + c.size] = np.minimum(D[j0:j0 + c.size], c)
    Do, _ = oracle.lws(n, 0, 0, 40, 6)
    assert np.array_equal(D, Do)
