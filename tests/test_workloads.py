"""The seeded input generators: determinism and the stated shapes."""
import numpy as np

from paper_2011_01441_gb300 import workloads as W


def test_splitmix_reference_values():
    # SplitMix64 with key = mix64(0) and counter 1.. ; recomputed here with
    # plain Python integers from the published constants.
    def mix(z):
        z &= (1 << 64) - 1
        z ^= z >> 30
        z = (z * 0xBF58476D1CE4E5B9) & ((1 << 64) - 1)
        z ^= z >> 27
        z = (z * 0x94D049BB133111EB) & ((1 << 64) - 1)
        return z ^ (z >> 31)
    key = mix((7 << 32) | 3)
    expect = [mix(key + i * 0x9E3779B97F4A7C15) for i in range(1, 6)]
    assert W.u64(7, 3, 5).tolist() == expect
    assert W.u64(7, 3, 2, offset=3).tolist() == expect[3:5]


def test_symbols_range_and_determinism():
    s = W.symbols(1, 0, 10000, 20)
    assert s.dtype == np.uint8 and s.min() >= 0 and s.max() <= 19
    assert np.array_equal(s, W.symbols(1, 0, 10000, 20))
    counts = np.bincount(s, minlength=20)
    assert counts.min() > 400  # roughly uniform


def test_single_pair_shapes():
    p1 = W.single_small()
    assert p1.a.size == 4096 and p1.b.size == 4096 and p1.a.max() <= 3
    p2 = W.single_mutated(n=20000)
    assert p2.a.size == p2.b.size == 20000
    assert p2.a.max() <= 19 and p2.b.max() <= 19
    p3 = W.single_skinny(n=4096, m=512)
    assert p3.a.size == 4096 and p3.b.size == 512


def test_mutate_exact_counts():
    a = W.symbols(9, 0, 1000, 20)
    b = W.mutate_exact(a, 20, 100, 0, 0, 9, 5)
    assert b.size == 1000 and int(np.sum(a != b)) == 100
    c = W.mutate_exact(a, 20, 0, 30, 10, 9, 6)
    assert c.size == 1020


def test_batch_lengths():
    bt = W.batch_pairs(npairs=64)
    la, lb = np.diff(bt.a_off), np.diff(bt.b_off)
    assert la.min() >= 64 and la.max() <= 8192 and lb.min() >= 64 and lb.max() <= 8192
    assert bt.a_cat.max() <= 3 and bt.b_cat.max() <= 3


def test_serve_request_deterministic():
    r1 = W.serve_request(17)
    r2 = W.serve_request(17)
    assert np.array_equal(r1.a, r2.a) and np.array_equal(r1.b, r2.b)
    assert 32 <= r1.a.size <= 65536 and 32 <= r1.b.size <= 65536
    t = W.poisson_arrivals(5, 1000, 100.0)
    assert np.all(np.diff(t) > 0) and 5.0 < t[-1] < 15.0
