"""GPU parity of the 1D-problem kernel (include/paco_lws.h, Eq. 1D of
Sec. "PACO 1D") against the CPU oracle, bit-exact, through the C ABI:
sizes around the block and warp granules, both weight variants, several
seeds and T, D[0] values, the degenerate n = 0, argument checks, and the
n = 131072 workload against the stored oracle result and against the
closed form of the squared-term-only weight."""
import hashlib
import os

import numpy as np
import pytest

import oracle
import paper_2011_01441_gb300 as P

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    c = P.Context(0)
    yield c
    c.close()


def _gpu(ctx, n, d0=0, T=40, seed=0, noise=True):
    D = P.paco_lws(ctx, n, d0, T, seed, noise)
    ctx.sync()
    return D.cpu().numpy().astype(np.int64)


@pytest.mark.parametrize("n", [0, 1, 2, 31, 32, 33, 255, 256, 257, 511, 1000, 4095, 4097, 9000])
def test_sizes(ctx, n):
    D = _gpu(ctx, n, 3, 40, 17)
    Do, _ = oracle.lws(n, 3, 0, 40, 17)
    assert np.array_equal(D, Do), n


@pytest.mark.parametrize("T,seed,noise,d0", [(40, 0, True, 0), (1, 5, True, 100), (0, 9, True, 7),
                                             (300, 0xFFFFFFFF, True, 0), (-50, 3, True, 0), (40, 0, False, 0),
                                             (7, 0, False, 1 << 28)])
def test_weights(ctx, T, seed, noise, d0):
    n = 3000
    D = _gpu(ctx, n, d0, T, seed, noise)
    Do, _ = oracle.lws(n, d0, 0 if noise else 3, T, seed)
    assert np.array_equal(D, Do), (T, seed, noise, d0)


def test_rejects_bad_arguments(ctx):
    for kw in [dict(n=-1), dict(n=10, d0=-1), dict(n=10, d0=1 << 29), dict(n=10, T=1 << 21)]:
        args = dict(n=10, d0=0, T=40)
        args.update(kw)
        with pytest.raises(P.PacoError) as e:
            P.paco_lws(ctx, args["n"], args["d0"], args["T"])
        assert e.value.status == P.PACO_EINVAL


def test_repeated_launches_reuse_flags(ctx):
    for k in range(5):
        n = 2000 + 300 * k
        assert np.array_equal(_gpu(ctx, n, 0, 40, k), oracle.lws(n, 0, 0, 40, k)[0])


def _golden():
    rec = {}
    with open(os.path.join(HERE, "golden", "lws_n131072.txt")) as f:
        for line in f:
            if not line.startswith("#"):
                k, _, v = line.strip().partition(" ")
                rec[k] = v
    return rec


def test_full_n131072_against_stored_oracle(ctx):
    g = _golden()
    n = int(g["n"])
    D = _gpu(ctx, n, 0, int(g["T"]), int(g["seed"]))
    assert int(D[-1]) == int(g["last"])
    assert list(D[::int(g["stride"])]) == [int(v) for v in g["D_samples"].split()]
    assert hashlib.sha256(D.astype(np.int32).tobytes()).hexdigest() == g["D_sha256"]


def test_full_size_closed_form_without_noise(ctx):
    """Squared term only: D[j] is the cheapest split of j into parts, the
    balanced split into k parts for the best k (parts far from T only add
    cost); checked on sampled j of the n = 131072 run."""
    n, T = 131072, 40
    D = _gpu(ctx, n, 0, T, 0, noise=False)
    for j in list(range(1, 200)) + list(range(131000, 131073, 7)):
        k = max(1, j // T)
        best = None
        for kk in range(max(1, k - 2), k + 3):
            q, r = divmod(j, kk)
            if q == 0:
                continue
            cost = r * (q + 1 - T) ** 2 + (kk - r) * (q - T) ** 2
            best = cost if best is None else min(best, cost)
        assert D[j] == best, j


def test_bounded_wait_times_out_and_recovers(ctx):
    """A block whose inputs never arrive (test-only switch) ends the launch
    with PACO_ETIMEOUT within the wait limit, not a hang; the context then
    computes correctly again."""
    ctx.set_option(P.OPT_WAIT_LIMIT_NS, 50_000_000)
    ctx.set_option(P.OPT_TEST_STALL, 5)
    try:
        with pytest.raises(P.PacoError) as e:
            P.paco_lws(ctx, 3000, 0, 40, 1)
            ctx.sync()
        assert e.value.status == P.PACO_ETIMEOUT
    finally:
        ctx.set_option(P.OPT_TEST_STALL, -1)
        ctx.set_option(P.OPT_WAIT_LIMIT_NS, 2_000_000_000)
    assert np.array_equal(_gpu(ctx, 3000, 0, 40, 1), oracle.lws(3000, 0, 0, 40, 1)[0])
