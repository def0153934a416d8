"""Writes tests/golden/lcs_bruteforce.txt.

Every stored value comes from `oracle.brute.lcs_brute` (enumeration of all
subsequences of a); nothing here touches the two-row DP or the CUDA library.
Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import random
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.brute import lcs_brute  # noqa: E402


def main():
    rng = random.Random(20110144)
    lines = ["# a b LCS(a,b)  -- symbols are digits 0..9; '-' is the empty string",
             "# values by brute-force subsequence enumeration (oracle/brute.py)"]
    for _ in range(80):
        sigma = rng.choice([2, 3, 4, 10])
        a = [rng.randrange(sigma) for _ in range(rng.randint(0, 11))]
        b = [rng.randrange(sigma) for _ in range(rng.randint(0, 11))]
        enc = lambda s: "".join(map(str, s)) if s else "-"
        lines.append(f"{enc(a)} {enc(b)} {lcs_brute(a, b)}")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lcs_bruteforce.txt")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
