"""Pins for the CPU oracle: each test ties the two-row DP of Eq. (1) to
something other than itself (brute-force enumeration of subsequences, the
indel-distance recursion, closed forms, invariants, a textbook example)."""
import itertools
import os
import random

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2011_01441_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _bin_strings(maxlen):
    for k in range(maxlen + 1):
        for t in itertools.product((0, 1), repeat=k):
            yield list(t)


def test_clrs_worked_example():
    # CLRS 3rd ed. Sec. 15.4 (the reference the paper gives for Eq. (1)):
    # X = ABCBDAB, Y = BDCABA has an LCS of length 4 (e.g. BCBA).
    L, row, col = oracle.lcs(b"ABCBDAB", b"BDCABA")
    assert L == 4
    assert row[-1] == 4 and col[-1] == 4


def test_exhaustive_binary_vs_enumeration():
    strings = list(_bin_strings(6))
    for a in strings:
        for b in strings:
            L, _, _ = oracle.lcs(np.array(a, np.uint8), np.array(b, np.uint8))
            assert L == brute.lcs_brute(a, b), (a, b)


@pytest.mark.parametrize("sigma", [2, 4, 256])
def test_random_vs_enumeration_with_boundaries_out(sigma):
    rng = random.Random(100 + sigma)
    for _ in range(60):
        a = [rng.randrange(sigma) for _ in range(rng.randint(0, 12))]
        b = [rng.randrange(sigma) for _ in range(rng.randint(0, 12))]
        L, row, col = oracle.lcs(np.array(a, np.uint8), np.array(b, np.uint8))
        assert L == brute.lcs_brute(a, b)
        # every bottom-row and right-column entry is itself an LCS of prefixes
        assert row.tolist() == brute.bottom_row_brute(a, b)
        assert col.tolist() == brute.right_col_brute(a, b)


def test_indel_distance_identity():
    rng = random.Random(7)
    for _ in range(150):
        sigma = rng.choice([2, 3, 4, 20])
        a = [rng.randrange(sigma) for _ in range(rng.randint(0, 10))]
        b = [rng.randrange(sigma) for _ in range(rng.randint(0, 10))]
        L, _, _ = oracle.lcs(np.array(a, np.uint8), np.array(b, np.uint8))
        assert len(a) + len(b) - 2 * L == brute.indel_brute(a, b), (a, b)


def test_full_table_vs_enumeration():
    rng = random.Random(11)
    for _ in range(20):
        a = [rng.randrange(3) for _ in range(rng.randint(0, 8))]
        b = [rng.randrange(3) for _ in range(rng.randint(0, 8))]
        H = oracle.lcs_table(np.array(a, np.uint8), np.array(b, np.uint8))
        for i in range(len(a) + 1):
            for j in range(len(b) + 1):
                assert H[i, j] == brute.lcs_brute(a[:i], b[:j])


def test_closed_forms():
    for k in range(0, 40, 7):
        for l in range(0, 40, 5):
            assert oracle.lcs(np.full(k, 3, np.uint8), np.full(l, 3, np.uint8))[0] == min(k, l)
    for k in range(1, 50, 6):
        a = np.array([0, 1] * k, np.uint8)
        b = np.array([1, 0] * k, np.uint8)
        assert oracle.lcs(a, b)[0] == 2 * k - 1


def test_empty_inputs():
    L, row, col = oracle.lcs(np.zeros(0, np.uint8), np.arange(5, dtype=np.uint8))
    assert L == 0 and row.tolist() == [0] * 6 and col.tolist() == [0]
    L, row, col = oracle.lcs(np.arange(5, dtype=np.uint8), np.zeros(0, np.uint8))
    assert L == 0 and row.tolist() == [0] and col.tolist() == [0] * 6


def _rand(rng, n, sigma, base=0):
    return (np.array([rng.randrange(sigma) for _ in range(n)]) + base).astype(np.uint8)


def test_invariants_medium():
    rng = random.Random(3)
    for _ in range(20):
        n, m = rng.randint(0, 300), rng.randint(0, 300)
        sigma = rng.choice([2, 4, 20, 256])
        a, b = _rand(rng, n, sigma), _rand(rng, m, sigma)
        L, row, col = oracle.lcs(a, b)
        # identity and bounds
        assert oracle.lcs(a, a)[0] == n
        assert 0 <= L <= min(n, m)
        # symmetry: the table of (b, a) is the transpose
        L2, row2, col2 = oracle.lcs(b, a)
        assert L2 == L
        assert np.array_equal(row, col2) and np.array_equal(col, row2)
        # reversal invariance of the length
        assert oracle.lcs(a[::-1].copy(), b[::-1].copy())[0] == L
        # unit steps along both outputs
        for v in (row, col):
            d = np.diff(v)
            assert np.all((d == 0) | (d == 1))
        # disjoint alphabets give 0 everywhere
        Lz, rz, cz = oracle.lcs(a % 100, (_rand(rng, m, 7, base=100)))
        assert Lz == 0 and not rz.any() and not cz.any()


def test_deletion_and_insertion_only():
    rng = np.random.default_rng(5)
    a = rng.integers(0, 20, 5000).astype(np.uint8)
    keep = rng.random(5000) > 0.2
    b = a[keep]
    assert oracle.lcs(a, b)[0] == b.size          # b is a subsequence of a
    ins = rng.integers(0, 20, 1000).astype(np.uint8)
    pos = np.sort(rng.integers(0, 5000, 1000))
    c = np.insert(a, pos, ins)
    assert oracle.lcs(a, c)[0] == a.size          # a is a subsequence of c


def test_boundaries_composition_rows_and_cols():
    """Splitting a (or b) and chaining the produced boundary through the
    first/last row (column) gives the unsplit table's boundaries."""
    rng = random.Random(9)
    for _ in range(30):
        n, m = rng.randint(2, 200), rng.randint(2, 200)
        sigma = rng.choice([2, 4, 20])
        a, b = _rand(rng, n, sigma), _rand(rng, m, sigma)
        L, row, col = oracle.lcs(a, b)
        k = rng.randint(1, n - 1)
        L1, row1, col1 = oracle.lcs(a[:k], b)
        # the lower part's first column is the table's first column: zeros
        L2, row2, col2 = oracle.lcs(a[k:], b, top=row1, left=np.zeros(n - k + 1, np.int32))
        assert L2 == L and np.array_equal(row2, row)
        assert np.array_equal(np.concatenate([col1, col2[1:]]), col)
        q = rng.randint(1, m - 1)
        La, rowa, cola = oracle.lcs(a, b[:q])
        Lb, rowb, colb = oracle.lcs(a, b[q:], top=np.zeros(m - q + 1, np.int32), left=cola)
        assert Lb == L and np.array_equal(colb, col)
        assert np.array_equal(np.concatenate([rowa, rowb[1:]]), row)


def test_boundaries_no_match_closed_form():
    """With no symbol in common, H[i][j] = max(top[j], left[i]) for valid
    (non-decreasing, unit-step) boundaries."""
    rng = random.Random(13)
    for _ in range(30):
        n, m = rng.randint(1, 60), rng.randint(1, 60)
        c0 = rng.randint(0, 50)
        top = np.concatenate([[c0], c0 + np.cumsum([rng.randint(0, 1) for _ in range(m)])]).astype(np.int32)
        left = np.concatenate([[c0], c0 + np.cumsum([rng.randint(0, 1) for _ in range(n)])]).astype(np.int32)
        a = _rand(rng, n, 4)
        b = _rand(rng, m, 4, base=10)
        H = oracle.lcs_table(a, b, top, left)
        assert np.array_equal(H, np.maximum(top[None, :], left[:, None]))


def test_golden_fixture():
    """Stored LCS values written by tests/golden/make_golden.py, which calls
    only the brute-force enumeration under oracle/."""
    path = os.path.join(GOLDEN, "lcs_bruteforce.txt")
    cases = 0
    with open(path) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            a_s, b_s, L_s = line.split()
            a = np.array([int(c) for c in a_s.strip("'")], np.uint8) if a_s != "-" else np.zeros(0, np.uint8)
            b = np.array([int(c) for c in b_s.strip("'")], np.uint8) if b_s != "-" else np.zeros(0, np.uint8)
            assert oracle.lcs(a, b)[0] == int(L_s), line
            cases += 1
    assert cases >= 50


def test_batch_matches_single():
    rng = random.Random(17)
    pairs = [(_rand(rng, rng.randint(0, 300), 4), _rand(rng, rng.randint(0, 300), 4)) for _ in range(40)]
    a_cat = np.concatenate([p[0] for p in pairs])
    b_cat = np.concatenate([p[1] for p in pairs])
    a_off = np.concatenate([[0], np.cumsum([p[0].size for p in pairs])])
    b_off = np.concatenate([[0], np.cumsum([p[1].size for p in pairs])])
    L, rows, row_off, cols, col_off = oracle.lcs_batch(a_cat, a_off, b_cat, b_off, threads=4)
    for k, (a, b) in enumerate(pairs):
        Lk, r, c = oracle.lcs(a, b)
        assert L[k] == Lk
        assert np.array_equal(rows[row_off[k]:row_off[k + 1]], r)
        assert np.array_equal(cols[col_off[k]:col_off[k + 1]], c)


def test_planted_mistakes_are_caught():
    """A plausible bug in the recurrence (dropped +1, transposed operand, or
    an off-by-one index) must disagree with enumeration somewhere; this checks
    that the pins above have the power to catch them."""
    def buggy(a, b, kind):
        n, m = len(a), len(b)
        H = [[0] * (m + 1) for _ in range(n + 1)]
        for i in range(1, n + 1):
            for j in range(1, m + 1):
                if kind == "no_plus_one":
                    H[i][j] = H[i - 1][j - 1] if a[i - 1] == b[j - 1] else max(H[i - 1][j], H[i][j - 1])
                elif kind == "diag_is_up":
                    H[i][j] = H[i - 1][j] + 1 if a[i - 1] == b[j - 1] else max(H[i - 1][j], H[i][j - 1])
                elif kind == "index_shift":
                    H[i][j] = H[i - 1][j - 1] + 1 if a[i - 1] == b[j - 2 if j > 1 else 0] else max(H[i - 1][j], H[i][j - 1])
        return H[n][m]
    rng = random.Random(21)
    for kind in ("no_plus_one", "diag_is_up", "index_shift"):
        caught = False
        for _ in range(200):
            a = [rng.randrange(3) for _ in range(rng.randint(1, 8))]
            b = [rng.randrange(3) for _ in range(rng.randint(1, 8))]
            if buggy(a, b, kind) != brute.lcs_brute(a, b):
                caught = True
                break
        assert caught, kind


# ---- the independent bit-vector routine (Allison & Dix / Hyyro) against the DP ----

def test_bitpar_against_bruteforce_exhaustive_binary():
    for n in range(0, 6):
        for m in range(0, 6):
            for x in range(1 << n):
                a = [(x >> k) & 1 for k in range(n)]
                for y in range(0, 1 << m, 3):
                    b = [(y >> k) & 1 for k in range(m)]
                    L, row, col = oracle.lcs_bitpar(np.array(a, np.uint8), np.array(b, np.uint8))
                    assert L == brute.lcs_brute(a, b)
                    assert list(row) == brute.bottom_row_brute(a, b)
                    assert list(col) == brute.right_col_brute(a, b)


@pytest.mark.parametrize("n,m,sigma", [(0, 7, 4), (7, 0, 4), (1, 1, 2), (63, 64, 4), (64, 65, 4), (65, 63, 2),
                                       (127, 128, 20), (1000, 3000, 4), (3001, 999, 256), (4096, 4096, 4)])
def test_bitpar_equals_dp(n, m, sigma):
    a = W.symbols(n + 11 * m, 0, n, sigma)
    b = W.symbols(n + 11 * m, 1, m, sigma)
    d = oracle.lcs(a, b)
    t = oracle.lcs_bitpar(a, b)
    assert d[0] == t[0]
    assert np.array_equal(d[1], t[1]) and np.array_equal(d[2], t[2])


def test_bitpar_equals_dp_mutated_20000():
    """Two independent CPU methods agree on a 20000-square mutated pair."""
    a = W.symbols(12, 0, 20000, 20)
    b = W.mutate_rate(a, 20, 0.15, 12, 1)
    d = oracle.lcs(a, b)
    t = oracle.lcs_bitpar(a, b)
    assert d[0] == t[0] and np.array_equal(d[1], t[1]) and np.array_equal(d[2], t[2])
