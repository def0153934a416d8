"""Writes lws_n131072.txt: the oracle's D[0..131072] for the 1D problem
(Sec. "PACO 1D") with D[0] = 0 and the benchmark weight (T = 40, seed 6,
hashed byte on).  Calls only the oracle (about half a minute on one core).

    python tests/golden/make_lws_golden.py
"""
import hashlib
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

N, T, SEED, STRIDE = 131072, 40, 6, 1024


def main():
    D, _ = oracle.lws(N, 0, 0, T, SEED)
    D32 = D.astype(np.int32)
    assert np.array_equal(D32, D)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lws_n131072.txt")
    with open(out, "w") as f:
        f.write("# oracle.lws(131072, d0=0, kind=0, T=40, seed=6)\n")
        f.write("# written by tests/golden/make_lws_golden.py (oracle only)\n")
        f.write(f"n {N}\nT {T}\nseed {SEED}\nlast {int(D[-1])}\n")
        f.write(f"D_sha256 {hashlib.sha256(D32.tobytes()).hexdigest()}\n")
        f.write(f"stride {STRIDE}\n")
        f.write("D_samples " + " ".join(str(int(v)) for v in D32[::STRIDE]) + "\n")
    print(out, int(D[-1]))


if __name__ == "__main__":
    main()
