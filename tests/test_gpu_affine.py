"""GPU parity of the affine-gap alignment kernels (include/paco_affine.h)
against the CPU oracle, bit-exact, through the C ABI: single pairs of ragged
sizes in both orientations and both band heights, degenerate pairs, batches,
the 4096-pair batch workload in full, and the 131072-square pair against the
stored oracle result and against closed forms at that size."""
import hashlib
import os

import numpy as np
import pytest

import oracle
import paper_2011_01441_gb300 as P
from paper_2011_01441_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
SCORES = (2, 3, 5, 2)
SCORE_SETS = [SCORES, (1, 0, 0, 0), (0, 1, 0, 1), (1, 1, 3, 1), (3, 1, 0, 2), (1, 5, 2, 0), (65535, 65535, 0, 1)]


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    c = P.Context(0)
    yield c
    c.close()


def _dev(x):
    import torch
    x = np.ascontiguousarray(x, dtype=np.uint8)
    return torch.from_numpy(x).cuda() if x.size else torch.zeros(0, dtype=torch.uint8, device="cuda")


def _align(ctx, a, b, scores, rows_per_lane=0):
    ctx.set_option(P.OPT_AFFINE_ROWS, rows_per_lane)
    try:
        s, row, col = P.paco_affine_align(ctx, _dev(a), _dev(b), scores, want_rows=True, want_cols=True)
        ctx.sync()
    finally:
        ctx.set_option(P.OPT_AFFINE_ROWS, 0)
    return int(s.cpu()[0]), row.cpu().numpy(), col.cpu().numpy()


def _check(ctx, a, b, scores, rows_per_lane=0):
    s, row, col = _align(ctx, a, b, scores, rows_per_lane)
    so, ro, co = oracle.affine(a, b, *scores)
    assert s == so, (a.size, b.size, scores, rows_per_lane)
    assert np.array_equal(row, ro), ("row", a.size, b.size, scores, rows_per_lane)
    assert np.array_equal(col, co), ("col", a.size, b.size, scores, rows_per_lane)


SIZES = [1, 2, 15, 16, 17, 31, 127, 128, 129, 255, 256, 257, 600, 1025]


@pytest.mark.parametrize("rows_per_lane", [2, 4, 8])
def test_ragged_sizes_both_orientations(ctx, rows_per_lane):
    rng = np.random.default_rng(100 + rows_per_lane)
    for t in range(24):
        n, m = int(rng.choice(SIZES)), int(rng.choice(SIZES))
        sigma = int(rng.choice([2, 4, 20, 256]))
        a = W.symbols(61, t, n, sigma)
        b = W.mutate_rate(a, sigma, 0.2, 62, t)[:m] if rng.random() < 0.6 else W.symbols(63, t, m, sigma)
        _check(ctx, a, b, SCORES, rows_per_lane)


@pytest.mark.parametrize("scores", SCORE_SETS)
def test_score_sets(ctx, scores):
    a = W.symbols(71, 0, 700, 4)
    b = W.mutate_rate(a, 4, 0.25, 72, 0)
    _check(ctx, a, b, scores, 4)
    _check(ctx, b[:300], a, scores, 8)


def test_many_bands_tall_and_wide(ctx):
    a = W.symbols(81, 0, 5000, 4)
    b = W.mutate_rate(a, 4, 0.15, 82, 0)
    _check(ctx, a, b, SCORES, 4)
    _check(ctx, a[:700], W.symbols(83, 0, 9000, 4), SCORES, 8)
    _check(ctx, W.symbols(84, 0, 9000, 4), a[:40], SCORES, 4)


def test_degenerate_pairs(ctx):
    e = np.zeros(0, np.uint8)
    a = W.symbols(91, 0, 37, 4)
    for x, y in [(e, e), (a, e), (e, a)]:
        _check(ctx, x, y, SCORES)


def test_rejects_bad_arguments(ctx):
    a = _dev(W.symbols(92, 0, 10, 4))
    for bad in [(-1, 1, 1, 1), (1, 1, 1, 65536)]:
        with pytest.raises(P.PacoError) as e:
            P.paco_affine_align(ctx, a, a, bad)
        assert e.value.status == P.PACO_EINVAL
    # reachable values must stay inside +-2^29
    big = _dev(np.zeros(1 << 20, np.uint8))
    with pytest.raises(P.PacoError) as e:
        P.paco_affine_align(ctx, big, big, (1000, 0, 0, 0))
    assert e.value.status == P.PACO_EINVAL


def _cat(strings):
    off = np.zeros(len(strings) + 1, dtype=np.int64)
    off[1:] = np.cumsum([s.size for s in strings])
    return (np.concatenate(strings).astype(np.uint8) if strings else np.zeros(0, np.uint8)), off


@pytest.mark.parametrize("rows_per_lane", [2, 4, 8])
def test_batch_mixed_sizes(ctx, rows_per_lane):
    rng = np.random.default_rng(200 + rows_per_lane)
    A, B = [], []
    for k in range(80):
        n, m = int(rng.choice([0] + SIZES)), int(rng.choice([0] + SIZES))
        a = W.symbols(93, k, n, 4)
        A.append(a)
        B.append(W.fit_length(W.mutate_rate(a, 4, 0.2, 94, k), m, 4, 95, k))
    a_cat, a_off = _cat(A)
    b_cat, b_off = _cat(B)
    ctx.set_option(P.OPT_AFFINE_ROWS, rows_per_lane)
    try:
        got = P.paco_affine_batch(ctx, _dev(a_cat), _dev(b_cat), a_off, b_off, SCORES)
        ctx.sync()
    finally:
        ctx.set_option(P.OPT_AFFINE_ROWS, 0)
    want = oracle.affine_batch(a_cat, a_off, b_cat, b_off, SCORES)
    assert np.array_equal(got.cpu().numpy()[:80], want)


def test_batch_plan_reuse_with_new_data(ctx):
    """Repeated calls with the same lengths reuse the uploaded plan; new
    symbols in the same layout still give the oracle's scores."""
    A = [W.symbols(96, k, 100 + 173 * k, 4) for k in range(15)]
    B = [W.mutate_rate(x, 4, 0.2, 97, k) for k, x in enumerate(A)]
    a_cat, a_off = _cat(A)
    b_cat, b_off = _cat(B)
    for it in range(3):
        x = a_cat if it % 2 == 0 else (a_cat + it) % 4
        got = P.paco_affine_batch(ctx, _dev(x), _dev(b_cat), a_off, b_off, SCORES)
        ctx.sync()
        want = oracle.affine_batch(x.astype(np.uint8), a_off, b_cat, b_off, SCORES)
        assert np.array_equal(got.cpu().numpy()[:15], want), it


def test_batch_full_workload_4096_pairs(ctx):
    """The 4096-pair workload (lengths log-uniform in [64, 8192], alphabet 4,
    15% mutation) in the configuration the benchmark times: every score
    against the oracle (spread over all host cores)."""
    bt = W.batch_pairs()
    got = P.paco_affine_batch(ctx, _dev(bt.a_cat), _dev(bt.b_cat), bt.a_off, bt.b_off, SCORES)
    ctx.sync()
    want = oracle.affine_batch(bt.a_cat, bt.a_off, bt.b_cat, bt.b_off, SCORES)
    assert np.array_equal(got.cpu().numpy(), want)


def _golden():
    rec = {}
    with open(os.path.join(HERE, "golden", "affine_pair131072.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            k, _, v = line.strip().partition(" ")
            rec[k] = v
    return rec


def test_full_pair_131072_against_stored_oracle(ctx):
    """The 131072-square mutated pair in the benchmark's launch
    configuration: score, last row and last column equal the oracle's
    (stored by tests/golden/make_affine_golden.py: hashes and samples)."""
    g = _golden()
    pair = W.single_mutated()
    assert int(g["n"]) == pair.a.size and int(g["m"]) == pair.b.size
    scores = tuple(int(v) for v in g["scores"].split())
    s, row, col = P.paco_affine_align(ctx, _dev(pair.a), _dev(pair.b), scores, want_rows=True, want_cols=True)
    ctx.sync()
    row = row.cpu().numpy()
    col = col.cpu().numpy()
    stride = int(g["stride"])
    assert int(s.cpu()[0]) == int(g["score"])
    assert list(row[::stride]) == [int(v) for v in g["bottom_row_samples"].split()]
    assert list(col[::stride]) == [int(v) for v in g["right_col_samples"].split()]
    assert hashlib.sha256(row.astype(np.int32).tobytes()).hexdigest() == g["bottom_row_sha256"]
    assert hashlib.sha256(col.astype(np.int32).tobytes()).hexdigest() == g["right_col_sha256"]


def test_full_size_closed_forms_and_symmetry(ctx):
    """At 131072 rows: a block of k symbols inserted or deleted costs one gap
    run exactly (the closed form the oracle is pinned to); the transposed
    problem has the same score."""
    M, X, O, E = SCORES
    a = W.symbols(97, 0, 131072, 20)
    block = W.symbols(98, 0, 999, 20)
    ins = np.concatenate([a[:50000], block, a[50000:]])
    dele = np.concatenate([a[:70000], a[70999:]])
    for x, y, want in [(a, ins, M * a.size - (O + E * 999)), (ins, a, M * a.size - (O + E * 999)),
                       (a, dele, M * (a.size - 999) - (O + E * 999))]:
        s, _, _ = P.paco_affine_align(ctx, _dev(x), _dev(y), SCORES)
        ctx.sync()
        assert int(s.cpu()[0]) == want
    b = W.mutate_rate(a[:20000], 20, 0.2, 99, 0)
    s1, r1, c1 = P.paco_affine_align(ctx, _dev(a[:20000]), _dev(b), SCORES, want_rows=True, want_cols=True)
    s2, r2, c2 = P.paco_affine_align(ctx, _dev(b), _dev(a[:20000]), SCORES, want_rows=True, want_cols=True)
    ctx.sync()
    assert int(s1.cpu()[0]) == int(s2.cpu()[0])
    assert np.array_equal(r1.cpu().numpy(), c2.cpu().numpy()) and np.array_equal(c1.cpu().numpy(), r2.cpu().numpy())


def test_host_buffer_entry_point(ctx):
    import ctypes
    a = W.symbols(101, 0, 3000, 4)
    b = W.mutate_rate(a, 4, 0.2, 102, 0)
    row = np.empty(b.size + 1, np.int32)
    col = np.empty(a.size + 1, np.int32)
    s = ctypes.c_int32(0)
    vp = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    P.paco_affine_align_host_ptr(ctx, vp(a), a.size, vp(b), b.size, SCORES, ctypes.byref(s), vp(row), vp(col))
    so, ro, co = oracle.affine(a, b, *SCORES)
    assert s.value == so and np.array_equal(row, ro) and np.array_equal(col, co)


def test_bounded_wait_times_out_and_recovers(ctx):
    """A band whose input never arrives (test-only switch) ends the launch
    with PACO_ETIMEOUT within the wait limit, not a hang; the context then
    aligns correctly again."""
    a = W.symbols(103, 0, 5000, 4)
    b = W.mutate_rate(a, 4, 0.2, 104, 0)
    ctx.set_option(P.OPT_WAIT_LIMIT_NS, 50_000_000)
    ctx.set_option(P.OPT_TEST_STALL, 3)
    try:
        with pytest.raises(P.PacoError) as e:
            P.paco_affine_align(ctx, _dev(a), _dev(b), SCORES)
            ctx.sync()
        assert e.value.status == P.PACO_ETIMEOUT
    finally:
        ctx.set_option(P.OPT_TEST_STALL, -1)
        ctx.set_option(P.OPT_WAIT_LIMIT_NS, 2_000_000_000)
    _check(ctx, a, b, SCORES)
