"""Pins of the affine-gap alignment oracle (Gotoh's recurrence, the variant
the footnote to Eq. (1) names) to facts that do not come from the oracle:

* enumeration of every alignment, scored from the definition (exhaustive on
  tiny binary inputs, random on small ones), for the score, the last row and
  the last column;
* special cases that reduce to other problems: LCS length (match 1, nothing
  else), Levenshtein distance (unit mismatch and gap extension), indel
  distance n + m - 2 LCS (mismatch 2, extension 1);
* closed forms at any size: a block of k symbols inserted into or deleted
  from a costs exactly one gap run;
* symmetries: swapping the inputs transposes the table, reversing both
  leaves the score unchanged.

CPU only."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2011_01441_gb300 import workloads as W

# (match, mismatch, gap_open, gap_extend): each term non-zero in some set,
# and sets where opening dominates, extension dominates, or mismatch is free
SCORE_SETS = [(2, 3, 5, 2), (1, 0, 0, 0), (0, 1, 0, 1), (1, 1, 3, 1), (3, 1, 0, 2), (1, 5, 2, 0), (4, 2, 7, 1)]


def _strings(alphabet, max_len):
    for n in range(max_len + 1):
        for s in itertools.product(alphabet, repeat=n):
            yield bytes(s)


@pytest.mark.parametrize("scores", SCORE_SETS)
def test_exhaustive_binary_against_enumeration(scores):
    strings = list(_strings([0, 1], 3))
    for a in strings:
        for b in strings:
            got, row, col = oracle.affine(a, b, *scores)
            assert got == brute.affine_brute(a, b, *scores), (a, b, scores)
            assert list(row) == [brute.affine_brute(a, b[:j], *scores) for j in range(len(b) + 1)]
            assert list(col) == [brute.affine_brute(a[:i], b, *scores) for i in range(len(a) + 1)]


@pytest.mark.parametrize("scores", SCORE_SETS)
def test_random_small_against_enumeration(scores):
    rng = np.random.default_rng(7 + sum(scores))
    for _ in range(12):
        n, m = int(rng.integers(0, 7)), int(rng.integers(0, 7))
        sigma = int(rng.choice([2, 3, 4]))
        a = bytes(rng.integers(0, sigma, n).tolist())
        b = bytes(rng.integers(0, sigma, m).tolist())
        got, row, col = oracle.affine(a, b, *scores)
        assert got == brute.affine_brute(a, b, *scores), (a, b, scores)
        assert row[-1] == col[-1] == got


def test_lcs_special_case():
    """match 1, no mismatch or gap cost: the score counts matched columns,
    so it is the LCS length, by the brute force and by the LCS oracle."""
    rng = np.random.default_rng(3)
    for _ in range(30):
        a = bytes(rng.integers(0, 3, int(rng.integers(0, 9))).tolist())
        b = bytes(rng.integers(0, 3, int(rng.integers(0, 9))).tolist())
        assert oracle.affine(a, b, 1, 0, 0, 0)[0] == brute.lcs_brute(a, b)
    for k in range(4):
        a = W.symbols(11, k, 300 + 17 * k, 4)
        b = W.symbols(12, k, 250 + 31 * k, 4)
        s, row, col = oracle.affine(a, b, 1, 0, 0, 0)
        L, lrow, lcol = oracle.lcs(a, b)
        assert s == L and np.array_equal(row, lrow) and np.array_equal(col, lcol)


def test_levenshtein_special_case():
    """No reward, unit mismatch, unit gap extension, no opening: minus the
    score is the edit distance with unit substitution, insertion, deletion."""
    rng = np.random.default_rng(5)
    for _ in range(40):
        a = bytes(rng.integers(0, 4, int(rng.integers(0, 10))).tolist())
        b = bytes(rng.integers(0, 4, int(rng.integers(0, 10))).tolist())
        assert -oracle.affine(a, b, 0, 1, 0, 1)[0] == brute.levenshtein_brute(a, b), (a, b)


def test_indel_special_case_at_size():
    """Mismatch 2 = one insertion plus one deletion, so substitutions never
    help: minus the score is n + m - 2 LCS (LCS oracle, pinned separately)."""
    for k in range(3):
        a = W.symbols(21, k, 1500 + 101 * k, 4)
        b = W.mutate_rate(a, 4, 0.2, 22, k)
        L = oracle.lcs(a, b)[0]
        assert -oracle.affine(a, b, 0, 2, 0, 1)[0] == a.size + b.size - 2 * L


@pytest.mark.parametrize("scores", [(2, 3, 5, 2), (1, 1, 3, 1), (3, 1, 0, 2), (1, 5, 2, 0), (0, 0, 4, 1)])
def test_gap_block_closed_forms(scores):
    """b = a with a block of k symbols inserted: at most n columns match and
    b has k more symbols, so some gap run in a covers at least k columns;
    aligning a to itself with one run reaches that bound: score =
    match*n - (open + k*extend).  The deletion case mirrors it."""
    M, X, O, E = scores
    for t, (n, k, pos) in enumerate([(1, 1, 0), (40, 3, 40), (500, 17, 123), (3000, 250, 2999), (2000, 1, 0)]):
        a = W.symbols(31, t, n, 20)
        block = W.symbols(32, t, k, 20)
        b = np.concatenate([a[:pos], block, a[pos:]])
        assert oracle.affine(a, b, *scores)[0] == M * n - (O + E * k)
        assert oracle.affine(b, a, *scores)[0] == M * n - (O + E * k)
        d = np.concatenate([a[:pos], a[pos + k:]]) if pos + k <= n else a[:n - k]
        assert oracle.affine(a, d, *scores)[0] == M * (n - k) - (O + E * k)


def test_identity_empty_and_symmetries():
    M, X, O, E = 2, 3, 5, 2
    a = W.symbols(41, 0, 777, 4)
    b = W.mutate_rate(a, 4, 0.25, 42, 0)
    assert oracle.affine(a, a, M, X, O, E)[0] == M * a.size
    e = np.zeros(0, np.uint8)
    s, row, col = oracle.affine(a, e, M, X, O, E)
    assert s == -(O + E * a.size) and list(row) == [s]
    assert list(col) == [0] + [-(O + E * i) for i in range(1, a.size + 1)]
    assert oracle.affine(e, e, M, X, O, E)[0] == 0
    s1, r1, c1 = oracle.affine(a, b, M, X, O, E)
    s2, r2, c2 = oracle.affine(b, a, M, X, O, E)
    assert s1 == s2 and np.array_equal(r1, c2) and np.array_equal(c1, r2)
    assert oracle.affine(a[::-1], b[::-1], M, X, O, E)[0] == s1


def test_batch_equals_single_pairs():
    A = [W.symbols(51, k, 50 + 40 * k, 4) for k in range(12)]
    B = [W.mutate_rate(x, 4, 0.2, 52, k) for k, x in enumerate(A)]
    a_off = np.concatenate([[0], np.cumsum([x.size for x in A])])
    b_off = np.concatenate([[0], np.cumsum([x.size for x in B])])
    got = oracle.affine_batch(np.concatenate(A), a_off, np.concatenate(B), b_off, (2, 3, 5, 2), threads=3)
    assert list(got) == [oracle.affine(x, y, 2, 3, 5, 2)[0] for x, y in zip(A, B)]
