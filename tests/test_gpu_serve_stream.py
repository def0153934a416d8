"""The serving path on a seeded sample of the serving workload itself
(requests of the 100,000-request stream: side lengths log-uniform in
[32, 65536] independently, alphabet 20, b a 20%-mutated copy of a in half the
requests and independent in the rest), bit-exact against the CPU oracle.

The whole stream is about 7.4e12 cells, minutes of oracle time on all host
cores, so the test checks a 1% sample (1000 requests drawn by a seeded
generator, lengths only, through the batched submit and poll calls) plus 60
of them with both boundaries through single submit and poll, all in flight
together."""
import time

import numpy as np
import pytest

import oracle
import paper_2011_01441_gb300 as P
from paper_2011_01441_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SAMPLE_SEED = 55
NSAMPLE = 1000
NBOUND = 60


def _cat(strings):
    off = np.zeros(len(strings) + 1, dtype=np.int64)
    off[1:] = np.cumsum([s.size for s in strings])
    return np.concatenate(strings).astype(np.uint8), off


def test_serving_stream_sample_matches_oracle():
    import __graft_entry__
    __graft_entry__.build()
    ks = np.unique(W.below(SAMPLE_SEED, 0, 4 * NSAMPLE, 100000))[:NSAMPLE]
    reqs = [W.serve_request(int(k)) for k in ks]
    A = [r.a for r in reqs]
    B = [r.b for r in reqs]
    n = np.array([a.size for a in A])
    m = np.array([b.size for b in B])
    # the sample spans the stream's range of sizes and both kinds of pair
    assert n.min() < 64 and m.min() < 64 and n.max() > 32768 and m.max() > 32768
    a_cat, a_off = _cat(A)
    b_cat, b_off = _cat(B)

    ctx = P.Context(0)
    try:
        bound = list(range(0, NSAMPLE, NSAMPLE // NBOUND))[:NBOUND]
        tb = [P.paco_lcs_submit(ctx, A[k], B[k], want_boundaries=True) for k in bound]
        tickets = P.paco_lcs_submit_many(ctx, a_cat, a_off, b_cat, b_off)
        got = np.full(NSAMPLE, -1, dtype=np.int64)
        pending = np.arange(NSAMPLE)
        t0 = time.time()
        while pending.size:
            st, ln = P.paco_lcs_poll_many(ctx, tickets[pending])
            done = st == P.PACO_OK
            assert np.all((st == P.PACO_OK) | (st == P.PACO_PENDING)), st[~done]
            got[pending[done]] = ln[done]
            pending = pending[~done]
            assert time.time() - t0 < 300, "serving did not finish"
            time.sleep(0.001)
        brows = {}
        t0 = time.time()
        while len(brows) < len(tb):
            for k, t in zip(bound, tb):
                if k in brows:
                    continue
                r = P.paco_lcs_poll(ctx, t, A[k].size, B[k].size, True)
                if r is not None:
                    brows[k] = r
            assert time.time() - t0 < 300, "serving did not finish"
            time.sleep(0.001)
        assert ctx.sync() in (None, 0)
    finally:
        ctx.close()

    Lo, _, _, _, _ = oracle.lcs_batch(a_cat, a_off, b_cat, b_off, boundaries=False)
    assert np.array_equal(got, Lo.astype(np.int64)), np.flatnonzero(got != Lo)[:10]
    sa, soff = _cat([A[k] for k in bound])
    sb, sboff = _cat([B[k] for k in bound])
    Lb, rows, row_off, cols, col_off = oracle.lcs_batch(sa, soff, sb, sboff, boundaries=True)
    for i, k in enumerate(bound):
        L, row, col = brows[k]
        assert L == Lb[i]
        assert np.array_equal(row, rows[row_off[i]:row_off[i + 1]])
        assert np.array_equal(col, cols[col_off[i]:col_off[i + 1]])
