"""GPU parity of the batch and serving paths against the CPU oracle
(bit-exact), through the C ABI."""
import time

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


def _cat(strings):
    off = np.zeros(len(strings) + 1, dtype=np.int64)
    off[1:] = np.cumsum([s.size for s in strings])
    cat = np.concatenate(strings).astype(np.uint8) if strings else np.zeros(0, np.uint8)
    return cat, off


def _mixed_pairs(seed, npairs, lens):
    rng = np.random.default_rng(seed)
    A, B = [], []
    for k in range(npairs):
        n = int(lens[rng.integers(0, len(lens))])
        m = int(lens[rng.integers(0, len(lens))])
        sigma = int(rng.choice([2, 4, 20, 256]))
        a = W.symbols(seed, 2 * k, n, sigma)
        b = W.mutate_rate(a, sigma, 0.2, seed, 2 * k + 1)[:m] if rng.random() < 0.5 else W.symbols(seed, 9000 + k, m, sigma)
        A.append(a)
        B.append(b)
    return A, B


def run_batch(ctx, A, B, boundaries=False, chunk=0):
    import torch
    a_cat, a_off = _cat(A)
    b_cat, b_off = _cat(B)
    npairs = len(A)
    n = np.diff(a_off)
    m = np.diff(b_off)
    row_off = np.concatenate([[0], np.cumsum(m + 1)[:-1]]).astype(np.int64)
    col_off = np.concatenate([[0], np.cumsum(n + 1)[:-1]]).astype(np.int64)
    da = torch.from_numpy(a_cat).cuda() if a_cat.size else torch.zeros(1, dtype=torch.uint8, device="cuda")
    db = torch.from_numpy(b_cat).cuda() if b_cat.size else torch.zeros(1, dtype=torch.uint8, device="cuda")
    rows = torch.full((int((m + 1).sum()),), -7, dtype=torch.int32, device="cuda") if boundaries else None
    cols = torch.full((int((n + 1).sum()),), -7, dtype=torch.int32, device="cuda") if boundaries else None
    ctx.set_option(P.OPT_CHUNK, chunk)
    try:
        L = P.paco_lcs_batch(ctx, da, db, a_off, b_off, rows_cat=rows, h_row_off=row_off if boundaries else None,
                             cols_cat=cols, h_col_off=col_off if boundaries else None)
        ctx.sync()
    finally:
        ctx.set_option(P.OPT_CHUNK, 0)
    out = [L.cpu().numpy()[:npairs]]
    if boundaries:
        out += [rows.cpu().numpy(), row_off, cols.cpu().numpy(), col_off]
    return out


def check_batch(ctx, A, B, boundaries=False, chunk=0):
    got = run_batch(ctx, A, B, boundaries, chunk)
    for k, (a, b) in enumerate(zip(A, B)):
        Lo, ro, co = oracle.lcs(a, b)
        assert got[0][k] == Lo, (k, a.size, b.size, chunk)
        if boundaries:
            rows, row_off, cols, col_off = got[1:]
            assert np.array_equal(rows[row_off[k]:row_off[k] + b.size + 1], ro), ("row", k, a.size, b.size)
            assert np.array_equal(cols[col_off[k]:col_off[k] + a.size + 1], co), ("col", k, a.size, b.size)


LENS = [0, 1, 2, 31, 32, 33, 100, 991, 992, 993, 1500, 2048, 3000]


@pytest.mark.parametrize("chunk", [0, 2, 4, 8])
def test_batch_lengths_mixed_sizes(ctx, chunk):
    A, B = _mixed_pairs(11 + chunk, 60, LENS)
    check_batch(ctx, A, B, chunk=chunk)


@pytest.mark.parametrize("chunk", [2, 8])
def test_batch_boundaries_mixed_sizes(ctx, chunk):
    A, B = _mixed_pairs(23 + chunk, 40, LENS)
    check_batch(ctx, A, B, boundaries=True, chunk=chunk)


def test_batch_size_classes_autotuned(ctx):
    """Pairs in every size class of the streamed side (< 256, < 1024, < 4096,
    >= 4096 columns) with per-class autotuned chunk widths: results match the
    oracle, and every class reports a width of 2, 4 or 8."""
    A, B = [], []
    for k, (n, m) in enumerate([(100, 90), (700, 600), (2500, 2000), (5000, 4100), (40, 3000), (4500, 300)] * 3):
        a = W.symbols(91, k, n, 4)
        A.append(a)
        B.append(W.mutate_rate(a, 4, 0.15, 92, k)[:m] if m <= n else W.fit_length(a, m, 4, 93, k))
    check_batch(ctx, A, B, boundaries=True, chunk=0)
    packed = ctx.get_option(P.OPT_BATCH_CHUNKS)
    assert all(((packed >> (4 * k)) & 15) in (2, 4, 8) for k in range(4)), hex(packed)


def test_batch_tall_pairs_chain_segments(ctx):
    # pairs taller than one warp (992 rows): segments chain through global memory
    A = [W.symbols(5, k, 5000 + 37 * k, 4) for k in range(6)]
    B = [W.mutate_rate(a, 4, 0.15, 6, k)[:700 + 100 * k] for k, a in enumerate(A)]
    check_batch(ctx, A, B, boundaries=True)
    check_batch(ctx, B, A, boundaries=True)


@pytest.mark.parametrize("chunk", [0, 2, 8])
def test_batch_tall_narrow_chains_among_square_pairs(ctx, chunk):
    """Pairs of 20000-30000 rows and 1-64 columns (chains of 21-31 segments
    with one or two words each, started early by the critical-path order and
    interleaved with other pairs' segments) mixed with square pairs, both
    orientations, with both boundaries."""
    A, B = [], []
    for k, (n, m) in enumerate([(30000, 1), (20000, 2), (25000, 31), (22000, 33), (30000, 64), (3000, 2900),
                                (1500, 1500), (993, 992), (40, 20000)]):
        a = W.symbols(97, k, n, 4)
        b = W.symbols(98, k, m, 4)
        A.append(a)
        B.append(b)
    check_batch(ctx, A, B, boundaries=True, chunk=chunk)
    check_batch(ctx, B, A, boundaries=True, chunk=chunk)


def test_batch_declared_alphabet(ctx):
    """A declared alphabet shrinks the match table; results are unchanged,
    and a symbol outside it is reported (PACO_EINVAL) without a fault."""
    A = [W.symbols(81, k, 600 + 50 * k, 4) for k in range(20)]
    B = [W.mutate_rate(a, 4, 0.2, 82, k) for k, a in enumerate(A)]
    ctx.set_option(P.OPT_ALPHABET, 4)
    try:
        check_batch(ctx, A, B, boundaries=True)
        bad = [a.copy() for a in A]
        bad[3][5] = 9
        with pytest.raises(P.PacoError) as e:
            run_batch(ctx, bad, B)
        assert e.value.status == P.PACO_EINVAL
        check_batch(ctx, A, B)
    finally:
        ctx.set_option(P.OPT_ALPHABET, 256)


def test_batch_graph_replay_and_new_data(ctx):
    A, B = _mixed_pairs(31, 30, LENS)
    first = run_batch(ctx, A, B)
    again = run_batch(ctx, A, B)
    assert np.array_equal(first[0], again[0])
    # same layout, different symbols
    A2 = [np.ascontiguousarray(a[::-1]) for a in A]
    check_batch(ctx, A2, B)


def test_batch_empty_and_all_degenerate(ctx):
    check_batch(ctx, [np.zeros(0, np.uint8)] * 3, [np.zeros(5, np.uint8), np.zeros(0, np.uint8), np.ones(2, np.uint8)],
                boundaries=True)


def test_batch_full_workload_4096_pairs(ctx):
    """The 4096-pair workload (lengths log-uniform in [64, 8192], alphabet 4,
    15% mutation) in the configuration the benchmark times (alphabet declared,
    lengths only, graph replay), then with both boundaries: every pair's
    length, last row and last column against the oracle (oracle spread over
    all host cores)."""
    import torch
    bt = W.batch_pairs()
    da = torch.from_numpy(bt.a_cat).cuda()
    db = torch.from_numpy(bt.b_cat).cuda()
    Lo, rows_o, row_off, cols_o, col_off = oracle.lcs_batch(bt.a_cat, bt.a_off, bt.b_cat, bt.b_off)
    ctx.set_option(P.OPT_ALPHABET, 4)
    try:
        L = P.paco_lcs_batch(ctx, da, db, bt.a_off, bt.b_off)
        ctx.sync()
        assert np.array_equal(L.cpu().numpy(), Lo)
        rows = torch.empty(int(row_off[-1]), dtype=torch.int32, device="cuda")
        cols = torch.empty(int(col_off[-1]), dtype=torch.int32, device="cuda")
        L2 = P.paco_lcs_batch(ctx, da, db, bt.a_off, bt.b_off, rows_cat=rows, h_row_off=row_off[:-1],
                              cols_cat=cols, h_col_off=col_off[:-1])
        ctx.sync()
    finally:
        ctx.set_option(P.OPT_ALPHABET, 256)
    assert np.array_equal(L2.cpu().numpy(), Lo)
    assert np.array_equal(rows.cpu().numpy(), rows_o)
    assert np.array_equal(cols.cpu().numpy(), cols_o)


# ---------------------------------------------------------------- serving

def _wait(ctx, tickets, sizes, want, timeout=120.0):
    res = {}
    t0 = time.time()
    while len(res) < len(tickets):
        for t, (n, m) in zip(tickets, sizes):
            if t in res:
                continue
            r = P.paco_lcs_poll(ctx, t, n, m, want)
            if r is not None:
                res[t] = r
        assert time.time() - t0 < timeout, "serving did not finish"
        time.sleep(0.0005)
    return [res[t] for t in tickets]


def test_serve_matches_oracle(ctx):
    A, B = _mixed_pairs(41, 120, LENS + [4000, 6000])
    tickets = [P.paco_lcs_submit(ctx, a, b, want_boundaries=(k % 3 == 0)) for k, (a, b) in enumerate(zip(A, B))]
    for k, (t, a, b) in enumerate(zip(tickets, A, B)):
        want = k % 3 == 0
        L, row, col = _wait(ctx, [t], [(a.size, b.size)], want)[0]
        Lo, ro, co = oracle.lcs(a, b)
        assert L == Lo
        if want:
            assert np.array_equal(row, ro) and np.array_equal(col, co)
    st = P.paco_serve_get_stats(ctx)
    assert st["completed"] >= 120 and st["batches_launched"] >= 1


def test_serve_alone_equals_in_mix(ctx):
    """Continuous batching must not change a result: the same request gives
    identical outputs (tolerance 0) alone and inside a stream of others."""
    a = W.symbols(51, 0, 3000, 20)
    b = W.mutate_rate(a, 20, 0.2, 51, 1)
    t = P.paco_lcs_submit(ctx, a, b, want_boundaries=True)
    alone = _wait(ctx, [t], [(a.size, b.size)], True)[0]
    A, B = _mixed_pairs(52, 80, LENS + [5000])
    ts = []
    for k in range(80):
        ts.append(P.paco_lcs_submit(ctx, A[k], B[k]))
        if k == 40:
            tm = P.paco_lcs_submit(ctx, a, b, want_boundaries=True)
    mixed = _wait(ctx, [tm], [(a.size, b.size)], True)[0]
    _wait(ctx, ts, [(x.size, y.size) for x, y in zip(A, B)], False)
    assert alone[0] == mixed[0]
    assert np.array_equal(alone[1], mixed[1]) and np.array_equal(alone[2], mixed[2])


def test_serve_submit_many_and_poll_many(ctx):
    """Batched submission and polling give the oracle's lengths, release
    each ticket once, and report unknown tickets."""
    A, B = _mixed_pairs(71, 90, LENS + [4000])
    a_cat, a_off = _cat(A)
    b_cat, b_off = _cat(B)
    t = P.paco_lcs_submit_many(ctx, a_cat, a_off, b_cat, b_off)
    assert t.size == 90 and np.unique(t).size == 90
    got = np.full(90, -1, dtype=np.int64)
    t0 = time.time()
    while (got < 0).any():
        idx = np.nonzero(got < 0)[0]
        st, ln = P.paco_lcs_poll_many(ctx, t[idx])
        assert np.all((st == P.PACO_OK) | (st == P.PACO_PENDING))
        fin = st == P.PACO_OK
        got[idx[fin]] = ln[fin]
        assert time.time() - t0 < 120
        time.sleep(0.0005)
    for k in range(90):
        assert got[k] == oracle.lcs(A[k], B[k])[0], k
    st, _ = P.paco_lcs_poll_many(ctx, t[:3])
    assert np.all(st == P.PACO_ENOTFOUND)


def test_serve_budget_and_tickets():
    c = P.Context(0, mem_budget_bytes=1 << 20)
    try:
        big = W.symbols(61, 0, 200000, 4)
        with pytest.raises(P.PacoError) as e:
            P.paco_lcs_submit(c, big, big)
        assert e.value.status == P.PACO_EBUSY
        # requests that fit are admitted as memory frees up
        A = [W.symbols(62, k, 20000, 4) for k in range(12)]
        ts = [P.paco_lcs_submit(c, a, a) for a in A]
        out = _wait(c, ts, [(a.size, a.size) for a in A], False)
        assert [r[0] for r in out] == [a.size for a in A]
        with pytest.raises(P.PacoError) as e:
            P.paco_lcs_poll(c, ts[0])
        assert e.value.status == P.PACO_ENOTFOUND
    finally:
        c.close()


def test_serve_arena_laps_and_full_arena(ctx):
    """Serving copies request strings into pinned FIFO arenas of 256 MiB per
    side: 150 requests with 4 MiB a-strings (600 MiB in all) lap the a-arena
    twice, a full arena answers PACO_EBUSY (the partial submit stops there),
    and space comes back as micro-batches complete.  b is one symbol, so
    L = 1 exactly when a holds it."""
    k_total = 150
    n = 4 << 20
    pending, got, k = {}, {}, 0
    t0 = time.time()
    while len(got) < k_total:
        assert time.time() - t0 < 300
        if k < k_total:
            syms = [np.uint8(3 if (j * 7) % 5 else 9) for j in range(k, min(k_total, k + 8))]
            a_list = [np.full(n, j % 3, np.uint8) for j in range(k, k + len(syms))]
            for a, j in zip(a_list, range(k, k + len(syms))):
                a[(j * 977) % n] = 9 if j % 4 == 0 else 1  # a holds 9 only when j % 4 == 0
            a_cat = np.concatenate(a_list)
            a_off = np.arange(len(syms) + 1, dtype=np.int64) * n
            b_cat = np.array(syms, np.uint8)
            b_off = np.arange(len(syms) + 1, dtype=np.int64)
            t = P.paco_lcs_submit_many(ctx, a_cat, a_off, b_cat, b_off, partial=True)
            for i, ticket in enumerate(t):
                pending[int(ticket)] = k + i
            k += len(t)
        if pending:
            tick = np.array(list(pending), np.uint64)
            st, ln = P.paco_lcs_poll_many(ctx, tick)
            for ticket, s_, l_ in zip(tick, st, ln):
                if s_ != P.PACO_PENDING:
                    assert s_ == P.PACO_OK
                    got[pending.pop(int(ticket))] = int(l_)
        time.sleep(0.001)
    # a holds the symbols j % 3 and one 9 (j % 4 == 0) or one 1; b is 3 (never
    # in a) unless j % 5 == 0, when it is 9
    for j in range(k_total):
        want = 1 if (j % 5 == 0 and j % 4 == 0) else 0
        assert got[j] == want, (j, got[j])


def test_serve_one_large_submission_in_groups(ctx):
    """One submit_many call of 600 requests with 1 MiB a-strings (600 MiB,
    more than the 256 MiB a-arena): the strings are copied by the submitting
    thread and its helpers, the call takes the requests that fit and stops
    with PACO_EBUSY partway through its first group of 512, and the rest goes
    in as arena space comes back.  b is one symbol, so L = 1 exactly when a
    holds it."""
    k_total = 600
    n = 1 << 20
    a_cat = np.empty(k_total * n, np.uint8)
    for j in range(k_total):
        a_cat[j * n:(j + 1) * n] = j % 3
        a_cat[j * n + (j * 977) % n] = 9 if j % 4 == 0 else 1  # a holds 9 only when j % 4 == 0
    a_off = np.arange(k_total + 1, dtype=np.int64) * n
    b_cat = np.array([9 if j % 5 == 0 else 3 for j in range(k_total)], np.uint8)
    b_off = np.arange(k_total + 1, dtype=np.int64)
    pending, got, k = {}, {}, 0
    first = None
    t0 = time.time()
    while len(got) < k_total:
        assert time.time() - t0 < 300
        if k < k_total:
            t = P.paco_lcs_submit_many(ctx, a_cat[a_off[k]:], a_off[k:] - a_off[k], b_cat[k:], b_off[k:] - b_off[k],
                                       partial=True)
            if first is None:
                first = t.size
            for i, ticket in enumerate(t):
                pending[int(ticket)] = k + i
            k += t.size
        if pending:
            tick = np.array(list(pending), np.uint64)
            st, ln = P.paco_lcs_poll_many(ctx, tick)
            for ticket, s_, l_ in zip(tick, st, ln):
                if s_ != P.PACO_PENDING:
                    assert s_ == P.PACO_OK
                    got[pending.pop(int(ticket))] = int(l_)
        time.sleep(0.001)
    assert 0 < first < 512  # stopped by the full arena inside the first group
    for j in range(k_total):
        want = 1 if (j % 5 == 0 and j % 4 == 0) else 0
        assert got[j] == want, (j, got[j])
