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

Only for |a| <= 14 or so.
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
