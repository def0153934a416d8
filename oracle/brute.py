"""Brute-force LCS facts for tiny inputs (test infrastructure only).

These routines do not use the recurrence of Eq. (1) at all; they pin the
two-row oracle to definitions that are independent of it:

* `lcs_brute(a, b)` - the definition of the problem statement in Sec.
  "PACO LCS": the longest sequence that is a (not necessarily contiguous)
  subsequence of both inputs, found by enumerating every subsequence of `a`
  (all 2**|a| index subsets) and testing it against `b` greedily.
* `indel_brute(a, b)` - edit distance with insertions and deletions only
  (no substitutions), written as its own recursion.  For any two strings
  |a| + |b| - 2 LCS(a, b) equals this distance, a classical identity that
  checks the oracle through a different recurrence.

* `affine_brute(a, b, match, mismatch, gap_open, gap_extend)` - the best
  score of a global alignment with affine gap costs found by listing every
  alignment (every path of aligned columns, gaps in a and gaps in b) and
  scoring each from the definition: +match / -mismatch per aligned column,
  gap_open + k * gap_extend per maximal run of k gap columns in one
  sequence.  It never uses Gotoh's recurrence.
* `levenshtein_brute(a, b)` - edit distance with unit-cost substitution,
  insertion and deletion, as its own recursion.

Only for |a| <= 14 or so (the alignment listing only for |a|, |b| <= 7).
"""
from __future__ import annotations

import functools
from itertools import combinations


def is_subsequence(s, t) -> bool:
    """True iff `s` occurs in `t` as a subsequence (greedy left-to-right scan)."""
    it = iter(t)
    return all(any(c == d for d in it) for c in s)


def lcs_brute(a, b) -> int:
    a = list(a)
    b = list(b)
    for k in range(min(len(a), len(b)), 0, -1):
        for idx in combinations(range(len(a)), k):
            if is_subsequence([a[i] for i in idx], b):
                return k
    return 0


def indel_brute(a, b) -> int:
    a = tuple(a)
    b = tuple(b)

    @functools.lru_cache(maxsize=None)
    def d(i: int, j: int) -> int:
        if i == 0:
            return j
        if j == 0:
            return i
        best = min(d(i - 1, j) + 1, d(i, j - 1) + 1)
        if a[i - 1] == b[j - 1]:
            best = min(best, d(i - 1, j - 1))
        return best

    return d(len(a), len(b))


def bottom_row_brute(a, b):
    """H[n][j] = LCS(a, b[:j]) for j = 0..m, each by enumeration."""
    return [lcs_brute(a, b[:j]) for j in range(len(b) + 1)]


def right_col_brute(a, b):
    """H[i][m] = LCS(a[:i], b) for i = 0..n, each by enumeration."""
    return [lcs_brute(a[:i], b) for i in range(len(a) + 1)]


def alignments(n: int, m: int):
    """Every global alignment of lengths n and m as a string over 'M'
    (aligned column), 'I' (b symbol against a gap) and 'D' (a symbol against
    a gap)."""
    if n == 0 and m == 0:
        yield ""
        return
    if n > 0 and m > 0:
        for rest in alignments(n - 1, m - 1):
            yield rest + "M"
    if m > 0:
        for rest in alignments(n, m - 1):
            yield rest + "I"
    if n > 0:
        for rest in alignments(n - 1, m):
            yield rest + "D"


def alignment_score(a, b, path: str, match: int, mismatch: int, gap_open: int, gap_extend: int) -> int:
    i = j = 0
    score = 0
    prev = ""
    for op in path:
        if op == "M":
            score += match if a[i] == b[j] else -mismatch
            i += 1
            j += 1
        else:
            if op != prev:
                score -= gap_open
            score -= gap_extend
            if op == "I":
                j += 1
            else:
                i += 1
        prev = op
    return score


def affine_brute(a, b, match, mismatch, gap_open, gap_extend) -> int:
    a = list(a)
    b = list(b)
    return max(alignment_score(a, b, p, match, mismatch, gap_open, gap_extend)
               for p in alignments(len(a), len(b)))


def levenshtein_brute(a, b) -> int:
    a = tuple(a)
    b = tuple(b)

    @functools.lru_cache(maxsize=None)
    def d(i: int, j: int) -> int:
        if i == 0:
            return j
        if j == 0:
            return i
        return min(d(i - 1, j) + 1, d(i, j - 1) + 1, d(i - 1, j - 1) + (a[i - 1] != b[j - 1]))

    return d(len(a), len(b))
