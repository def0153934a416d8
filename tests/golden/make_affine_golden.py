"""Writes affine_pair131072.txt: the oracle's affine-gap alignment of the
131072-square mutated pair (alphabet 20, 10% substitutions, 2.5% insertions,
2.5% deletions, seed 2) under scores match 2, mismatch 3, gap open 5, gap
extend 2.  Calls only the oracle (about a minute on one core).

    python tests/golden/make_affine_golden.py
"""
import hashlib
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2011_01441_gb300 import workloads as W  # noqa: E402

SCORES = (2, 3, 5, 2)
STRIDE = 4096


def main():
    pair = W.single_mutated()
    s, row, col = oracle.affine(pair.a, pair.b, *SCORES)
    row32 = row.astype(np.int32)
    col32 = col.astype(np.int32)
    assert np.array_equal(row32, row) and np.array_equal(col32, col)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "affine_pair131072.txt")
    with open(out, "w") as f:
        f.write("# oracle.affine(W.single_mutated(), match 2, mismatch 3, gap open 5, gap extend 2)\n")
        f.write("# written by tests/golden/make_affine_golden.py (oracle only)\n")
        f.write(f"n {pair.a.size}\nm {pair.b.size}\nscores {' '.join(map(str, SCORES))}\nscore {s}\n")
        f.write(f"bottom_row_sha256 {hashlib.sha256(row32.tobytes()).hexdigest()}\n")
        f.write(f"right_col_sha256 {hashlib.sha256(col32.tobytes()).hexdigest()}\n")
        f.write(f"stride {STRIDE}\n")
        f.write("bottom_row_samples " + " ".join(str(int(v)) for v in row32[::STRIDE]) + "\n")
        f.write("right_col_samples " + " ".join(str(int(v)) for v in col32[::STRIDE]) + "\n")
    print(out, s)


if __name__ == "__main__":
    main()
