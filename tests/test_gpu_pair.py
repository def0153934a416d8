"""GPU parity of the single-pair path against the CPU oracle (bit-exact:
the work is integer).  Every call goes through the C ABI."""
import concurrent.futures as cf
import itertools

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


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run(ctx, a, b, top=None, left=None, **opts):
    for k, v in opts.items():
        ctx.set_option(getattr(P, "OPT_" + k.upper()), v)
    try:
        L, row, col = P.paco_lcs_boundaries(ctx, _dev(a), _dev(b),
                                            None if top is None else _dev(top),
                                            None if left is None else _dev(left))
        ctx.sync()
        return int(L.item()), row.cpu().numpy(), col.cpu().numpy()
    finally:
        for k in opts:
            ctx.set_option(getattr(P, "OPT_" + k.upper()), -1 if k == "test_stall" else 0)


def check(ctx, a, b, top=None, left=None, **opts):
    got = run(ctx, a, b, top, left, **opts)
    want = oracle.lcs(a, b, top, left)
    assert got[0] == want[0], (got[0], want[0], a.size, b.size, opts)
    assert np.array_equal(got[1], want[1]), ("bottom_row", a.size, b.size, opts)
    assert np.array_equal(got[2], want[2]), ("right_col", a.size, b.size, opts)


SIZES = [1, 2, 31, 32, 33, 64, 1023, 1024, 1025, 2049, 3001]


@pytest.mark.parametrize("n,m", list(itertools.product([1, 33, 1024, 1025, 3001], [1, 2, 32, 33, 1023, 2049])))
def test_shapes_sigma4(ctx, n, m):
    a = W.symbols(n * 7 + m, 0, n, 4)
    b = W.symbols(n * 7 + m, 1, m, 4)
    check(ctx, a, b)


@pytest.mark.parametrize("sigma", [1, 2, 20, 256])
def test_alphabets(ctx, sigma):
    a = W.symbols(sigma, 0, 2500, sigma)
    b = W.symbols(sigma, 1, 1900, sigma)
    check(ctx, a, b)


@pytest.mark.parametrize("chunk,warps", [(c, w) for c in (2, 4, 8) for w in (1, 3, 6)] + [(4, 2)])
def test_chunks_and_strip_heights(ctx, chunk, warps):
    # several CTA strips (inter-CTA chaining) and several warps (shared ring)
    a = W.symbols(chunk * 100 + warps, 0, 7000, 4)
    b = W.mutate_rate(a, 4, 0.15, chunk, 3)[:4567]
    check(ctx, a, b, chunk=chunk, warps=warps)


@pytest.mark.parametrize("n,m,chunk,warps", [(7000, 4567, 2, 1), (7000, 4567, 4, 2), (7000, 4567, 8, 3),
                                              (62, 33, 2, 1), (63, 1, 4, 1), (1985, 2049, 8, 1),
                                              (3001, 1023, 2, 3), (12345, 2000, 4, 1)])
def test_two_words_per_lane(ctx, n, m, chunk, warps):
    """Lanes of two 31-row words (the lower one a chunk behind the upper):
    ragged lanes, ragged chunks, several strips and warps."""
    a = W.symbols(n + 3 * m, 0, n, 4)
    b = W.mutate_rate(a, 4, 0.15, chunk, warps)[:m] if m <= n else W.symbols(n + 3 * m, 1, m, 4)
    check(ctx, a, b, chunk=chunk, warps=warps, words_per_lane=2)


def test_two_words_per_lane_boundaries_and_timeout(ctx):
    rng = np.random.default_rng(8)
    for t in range(3):
        pa = W.symbols(80 + t, 0, int(rng.integers(1, 300)), 20)
        pb = W.symbols(80 + t, 1, int(rng.integers(1, 300)), 20)
        a = W.symbols(80 + t, 2, int(rng.integers(2000, 5000)), 20)
        b = W.symbols(80 + t, 3, int(rng.integers(500, 3000)), 20)
        H = oracle.lcs_table(np.concatenate([pa, a]), np.concatenate([pb, b]))
        check(ctx, a, b, H[pa.size, pb.size:].copy(), H[pa.size:, pb.size].copy(),
              words_per_lane=2, chunk=[2, 4, 8][t])
    a = W.symbols(91, 0, 9000, 4)
    b = W.symbols(91, 1, 3000, 4)
    ctx.set_option(P.OPT_WAIT_LIMIT_NS, 50_000_000)
    try:
        with pytest.raises(P.PacoError) as e:
            run(ctx, a, b, warps=1, test_stall=2, words_per_lane=2)
        assert e.value.status == P.PACO_ETIMEOUT
    finally:
        ctx.set_option(P.OPT_WAIT_LIMIT_NS, 2_000_000_000)
    check(ctx, a, b, words_per_lane=2)


@pytest.mark.parametrize("orient", [1, 2])
def test_orientations(ctx, orient):
    a = W.symbols(31, 0, 1500, 20)
    b = W.symbols(31, 1, 5003, 20)
    check(ctx, a, b, orient=orient, warps=1)
    check(ctx, b, a, orient=orient, warps=1)


@pytest.mark.parametrize("schedule", [0, 1])
def test_schedules(ctx, schedule):
    a = W.symbols(41, 0, 9000, 4)
    b = W.symbols(41, 1, 700, 4)
    check(ctx, a, b, schedule=schedule, warps=2)


def test_input_boundaries_from_a_real_table(ctx):
    rng = np.random.default_rng(3)
    for t in range(6):
        pa = W.symbols(60 + t, 0, int(rng.integers(0, 400)), 4)
        pb = W.symbols(60 + t, 1, int(rng.integers(0, 400)), 4)
        a = W.symbols(60 + t, 2, int(rng.integers(1, 3000)), 4)
        b = W.symbols(60 + t, 3, int(rng.integers(1, 3000)), 4)
        H = oracle.lcs_table(np.concatenate([pa, a]), np.concatenate([pb, b]))
        top = H[pa.size, pb.size:].copy()
        left = H[pa.size:, pb.size].copy()
        check(ctx, a, b, top, left, warps=1 + t % 3, chunk=[2, 4, 8][t % 3])


def test_composition_chained_calls(ctx):
    """Split a into two row blocks: the first call's bottom row is the
    second call's top boundary; the result equals the unsplit table."""
    a = W.symbols(77, 0, 6000, 20)
    b = W.symbols(77, 1, 5000, 20)
    L, row, col = run(ctx, a, b)
    L1, row1, col1 = run(ctx, a[:2500], b)
    L2, row2, col2 = run(ctx, a[2500:], b, top=row1, left=np.zeros(3501, np.int32))
    assert L2 == L and np.array_equal(row2, row)
    assert np.array_equal(np.concatenate([col1, col2[1:]]), col)


def test_degenerate_tables(ctx):
    for n, m in ((0, 0), (0, 5), (7, 0)):
        a = W.symbols(5, 0, n, 4)
        b = W.symbols(5, 1, m, 4)
        check(ctx, a, b)
    top = np.arange(6, dtype=np.int32) // 2 + 3
    check(ctx, np.zeros(0, np.uint8), W.symbols(5, 1, 5, 4), top=top, left=np.array([3], np.int32))
    left = np.arange(8, dtype=np.int32) // 3 + 1
    check(ctx, W.symbols(5, 0, 7, 4), np.zeros(0, np.uint8), top=np.array([1], np.int32), left=left)


def test_invalid_boundary_reports_einval(ctx):
    a = W.symbols(9, 0, 100, 4)
    b = W.symbols(9, 1, 90, 4)
    top = np.arange(91, dtype=np.int32)
    top[50] += 5  # a step of 6: not an LCS boundary
    with pytest.raises(P.PacoError) as e:
        run(ctx, a, b, top=top)
    assert e.value.status == P.PACO_EINVAL
    check(ctx, a, b)  # the context is usable afterwards


def test_unaligned_device_inputs(ctx):
    import torch
    a = W.symbols(13, 0, 3000, 4)
    b = W.symbols(13, 1, 2500, 4)
    ta = torch.from_numpy(np.concatenate([np.zeros(3, np.uint8), a])).cuda()[3:]
    tb = torch.from_numpy(np.concatenate([np.zeros(1, np.uint8), b])).cuda()[1:]
    L, row, col = P.paco_lcs_boundaries(ctx, ta, tb)
    ctx.sync()
    want = oracle.lcs(a, b)
    assert int(L.item()) == want[0]
    assert np.array_equal(row.cpu().numpy(), want[1]) and np.array_equal(col.cpu().numpy(), want[2])


def test_length_only_and_host_entry(ctx):
    import torch
    a = W.symbols(15, 0, 5000, 20)
    b = W.symbols(15, 1, 4000, 20)
    L = P.paco_lcs_length(ctx, _dev(a), _dev(b))
    ctx.sync()
    want = oracle.lcs(a, b)
    assert int(L.item()) == want[0]
    Lh, row, col = P.paco_lcs_boundaries_host(ctx, a, b)
    assert Lh == want[0] and np.array_equal(row, want[1]) and np.array_equal(col, want[2])


def test_repeated_calls_are_identical(ctx):
    a = W.symbols(17, 0, 4000, 4)
    b = W.symbols(17, 1, 4000, 4)
    first = run(ctx, a, b, warps=1)
    for _ in range(3):
        again = run(ctx, a, b, warps=1)
        assert again[0] == first[0] and np.array_equal(again[1], first[1]) and np.array_equal(again[2], first[2])


def test_bounded_wait_times_out_and_recovers(ctx):
    """A strip whose input never arrives (test-only switch) must end the
    launch with PACO_ETIMEOUT within the wait limit, not hang."""
    a = W.symbols(19, 0, 5000, 4)
    b = W.symbols(19, 1, 3000, 4)
    ctx.set_option(P.OPT_WAIT_LIMIT_NS, 50_000_000)
    try:
        with pytest.raises(P.PacoError) as e:
            run(ctx, a, b, warps=1, test_stall=2)
        assert e.value.status == P.PACO_ETIMEOUT
    finally:
        ctx.set_option(P.OPT_WAIT_LIMIT_NS, 2_000_000_000)
    check(ctx, a, b, warps=1)


def test_config_small_4096(ctx):
    p = W.single_small()
    check(ctx, p.a, p.b)


def test_closed_form_at_full_size(ctx):
    """Independent of the oracle: b a subsequence of a (deletions only) gives
    L = |b|; a a subsequence of c (insertions only) gives L = |a|."""
    a = W.symbols(21, 0, 131072, 20)
    keep = W.unit(21, 1, a.size) > 0.05
    b = a[keep]
    L, row, col = run(ctx, a, b)
    assert L == b.size and col[-1] == b.size and row[-1] == b.size
    c = W.mutate_exact(a, 20, 0, 3000, 0, 21, 5)
    L2, _, _ = run(ctx, a, c)
    assert L2 == a.size


@pytest.mark.slow
def test_full_size_pairs_match_oracle(ctx):
    """The 131072^2 mutated pair and the 1048576 x 16384 byte pair, in the
    launch configuration the benchmark times, element by element against the
    oracle (run for both pairs at once on two host threads)."""
    p2 = W.single_mutated()
    p3 = W.single_skinny()
    with cf.ThreadPoolExecutor(2) as ex:
        f2 = ex.submit(oracle.lcs, p2.a, p2.b)
        f3 = ex.submit(oracle.lcs, p3.a, p3.b)
        g2 = run(ctx, p2.a, p2.b)
        g3 = run(ctx, p3.a, p3.b)
        for got, fut in ((g2, f2), (g3, f3)):
            want = fut.result()
            assert got[0] == want[0]
            assert np.array_equal(got[1], want[1])
            assert np.array_equal(got[2], want[2])
