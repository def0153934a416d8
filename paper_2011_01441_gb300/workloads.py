"""Seeded synthetic inputs for the LCS workloads (no LCS arithmetic lives here).

This module is shared by the CUDA path's tests/bench and by the CPU oracle's
tests: it only produces byte strings, lengths and arrival times.  It imports
neither side.

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014; the
64-bit finaliser constants are the ones Vigna publishes for splitmix64):

    x_i = mix64(key + (i + 1) * 0x9E3779B97F4A7C15)            (mod 2**64)
    mix64(z): z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
              z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31

with `key = mix64(seed * 2**32 + stream)`.  Being counter based, any element
of any stream is computable on its own, so the whole module is vectorised
numpy and gives the same bytes on x86 and Arm.

The paper's LCS experiment prints no sizes or inputs (Sec. "LCS and Sorting"
shows only relative speedups), so the five workloads below are the synthetic
stand-ins: sizes, alphabets and mutation processes are stated per function.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, stream: int) -> np.uint64:
    base = np.array([((seed & 0xFFFFFFFF) << 32) | (stream & 0xFFFFFFFF)], dtype=np.uint64)
    return _mix64(base)[0]


def u64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Elements offset..offset+count-1 of the SplitMix64 stream (seed, stream)."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = stream_key(seed, stream) + idx * _GAMMA
        return _mix64(z)


def below(seed: int, stream: int, count: int, bound, offset: int = 0) -> np.ndarray:
    """Integers in [0, bound) by the multiply-shift map of the high 32 bits.

    `bound` may be a scalar or an array of per-element bounds (each < 2**32).
    """
    hi = u64(seed, stream, count, offset) >> np.uint64(32)
    b = np.asarray(bound, dtype=np.uint64)
    return ((hi * b) >> np.uint64(32)).astype(np.int64)


def unit(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles uniform in [0, 1) from the top 53 bits."""
    return (u64(seed, stream, count, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def symbols(seed: int, stream: int, count: int, sigma: int, offset: int = 0) -> np.ndarray:
    """`count` i.i.d. symbols uniform over 0..sigma-1, as uint8."""
    if not 1 <= sigma <= 256:
        raise ValueError("sigma must be in 1..256")
    return below(seed, stream, count, sigma, offset).astype(np.uint8)


# --------------------------------------------------------------------------
# mutation processes
# --------------------------------------------------------------------------

def mutate_exact(a: np.ndarray, sigma: int, n_sub: int, n_ins: int, n_del: int,
                 seed: int, stream: int) -> np.ndarray:
    """Exact-count mutation: `n_sub` substitutions, `n_ins` single-symbol
    insertions and `n_del` deletions at distinct positions of `a`.

    Positions come from one seeded permutation of range(len(a)) (sort by a
    random key): the first n_sub are substituted (new symbol uniform over the
    sigma-1 other symbols), the next n_del are deleted, the next n_ins get a
    uniform random symbol inserted in front of them.
    """
    n = a.size
    if n_sub + n_ins + n_del > n:
        raise ValueError("more mutations than positions")
    perm = np.argsort(u64(seed, stream, n), kind="stable")
    sub_pos = perm[:n_sub]
    del_pos = perm[n_sub:n_sub + n_del]
    ins_pos = perm[n_sub + n_del:n_sub + n_del + n_ins]
    out = a.astype(np.int64).copy()
    shift = 1 + below(seed, stream + 1, n_sub, sigma - 1)
    out[sub_pos] = (out[sub_pos] + shift) % sigma
    keep = np.ones(n, dtype=bool)
    keep[del_pos] = False
    ins_mark = np.zeros(n, dtype=bool)
    ins_mark[ins_pos] = True
    ins_sym = np.zeros(n, dtype=np.int64)
    ins_sym[ins_pos] = below(seed, stream + 2, n_ins, sigma)
    # interleave: [inserted symbol]? then [original or substituted]? per position
    reps = ins_mark.astype(np.int64) + keep.astype(np.int64)
    total = int(reps.sum())
    res = np.empty(total, dtype=np.int64)
    starts = np.cumsum(reps) - reps
    res[starts[ins_mark]] = ins_sym[ins_mark]
    res[(starts + ins_mark.astype(np.int64))[keep]] = out[keep]
    return res.astype(np.uint8)


def mutate_rate(a: np.ndarray, sigma: int, rate: float, seed: int, stream: int) -> np.ndarray:
    """Per-position mutation: each position mutates with probability `rate`;
    a mutation is a substitution (prob 1/2, new symbol uniform over the other
    sigma-1), a single-symbol insertion in front of it (1/4) or a deletion
    (1/4)."""
    n = a.size
    u = unit(seed, stream, n)
    kind = unit(seed, stream + 1, n)
    mut = u < rate
    sub = mut & (kind < 0.5)
    ins = mut & (kind >= 0.5) & (kind < 0.75)
    dele = mut & (kind >= 0.75)
    out = a.astype(np.int64).copy()
    if sigma > 1:
        shift = 1 + below(seed, stream + 2, n, sigma - 1)
        out[sub] = (out[sub] + shift[sub]) % sigma
    keep = ~dele
    new_sym = below(seed, stream + 3, n, sigma)
    reps = ins.astype(np.int64) + keep.astype(np.int64)
    res = np.empty(int(reps.sum()), dtype=np.int64)
    starts = np.cumsum(reps) - reps
    res[starts[ins]] = new_sym[ins]
    res[(starts + ins.astype(np.int64))[keep]] = out[keep]
    return res.astype(np.uint8)


def fit_length(s: np.ndarray, length: int, sigma: int, seed: int, stream: int) -> np.ndarray:
    """Truncate `s` to `length`, or extend it with i.i.d. uniform symbols."""
    if s.size >= length:
        return s[:length].copy()
    tail = symbols(seed, stream, length - s.size, sigma)
    return np.concatenate([s, tail])


def log_uniform_lengths(seed: int, stream: int, count: int, lo: int, hi: int) -> np.ndarray:
    """floor(exp(U[ln lo, ln(hi+1)))) : integers log-uniform in [lo, hi]."""
    u = unit(seed, stream, count)
    v = np.floor(np.exp(math.log(lo) + u * (math.log(hi + 1) - math.log(lo)))).astype(np.int64)
    return np.clip(v, lo, hi)


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

@dataclass
class Pair:
    a: np.ndarray
    b: np.ndarray
    name: str


def single_small(seed: int = 1, n: int = 4096, m: int = 4096, sigma: int = 4) -> Pair:
    """4096 x 4096, i.i.d. uniform over {0..3}, a and b independent."""
    return Pair(symbols(seed, 0, n, sigma), symbols(seed, 1, m, sigma),
                f"pair {n}x{m} sigma={sigma} iid")


def single_mutated(seed: int = 2, n: int = 131072, sigma: int = 20,
                   sub_frac: float = 0.10, indel_frac: float = 0.05) -> Pair:
    """n x n with alphabet 20: b is a with exactly round(0.10 n) substitutions,
    round(0.025 n) insertions and round(0.025 n) deletions (the 5% of single
    symbol indels split evenly), so |b| = |a|."""
    a = symbols(seed, 0, n, sigma)
    n_sub = int(round(sub_frac * n))
    n_ins = int(round(indel_frac * n / 2))
    b = mutate_exact(a, sigma, n_sub, n_ins, n_ins, seed, 10)
    return Pair(a, b, f"pair {n}x{b.size} sigma={sigma} mutated")


def single_skinny(seed: int = 3, n: int = 1048576, m: int = 16384, sigma: int = 256) -> Pair:
    """n rows x m columns, bytes uniform over 0..255, a and b independent."""
    return Pair(symbols(seed, 0, n, sigma), symbols(seed, 1, m, sigma),
                f"pair {n}x{m} sigma={sigma} iid")


@dataclass
class Batch:
    a_cat: np.ndarray   # uint8, all a strings concatenated
    a_off: np.ndarray   # int64[npairs+1]
    b_cat: np.ndarray
    b_off: np.ndarray
    name: str

    @property
    def npairs(self) -> int:
        return self.a_off.size - 1

    def pair(self, k: int):
        return (self.a_cat[self.a_off[k]:self.a_off[k + 1]],
                self.b_cat[self.b_off[k]:self.b_off[k + 1]])

    def cells(self) -> int:
        return int(np.sum(np.diff(self.a_off) * np.diff(self.b_off)))


def _concat(strings):
    off = np.zeros(len(strings) + 1, dtype=np.int64)
    off[1:] = np.cumsum([s.size for s in strings])
    cat = np.concatenate(strings) if strings else np.zeros(0, dtype=np.uint8)
    return cat.astype(np.uint8), off


def batch_pairs(seed: int = 4, npairs: int = 4096, lo: int = 64, hi: int = 8192,
                sigma: int = 4, rate: float = 0.15) -> Batch:
    """Uneven batch: len_a and len_b independently log-uniform in [lo, hi];
    a i.i.d. uniform; b = a mutated per position at `rate` (substitution 1/2,
    insertion 1/4, deletion 1/4), then fitted to len_b."""
    la = log_uniform_lengths(seed, 0, npairs, lo, hi)
    lb = log_uniform_lengths(seed, 1, npairs, lo, hi)
    a_list, b_list = [], []
    for k in range(npairs):
        a = symbols(seed, 1000 + 8 * k, int(la[k]), sigma)
        b = mutate_rate(a, sigma, rate, seed, 1000 + 8 * k + 1)
        b = fit_length(b, int(lb[k]), sigma, seed, 1000 + 8 * k + 6)
        a_list.append(a)
        b_list.append(b)
    a_cat, a_off = _concat(a_list)
    b_cat, b_off = _concat(b_list)
    return Batch(a_cat, a_off, b_cat, b_off,
                 f"batch {npairs} pairs len log-uniform [{lo},{hi}] sigma={sigma} mut={rate}")


@dataclass
class Request:
    index: int
    arrival_s: float
    a: np.ndarray
    b: np.ndarray


def serve_lengths(seed: int = 5, count: int = 100000, lo: int = 32, hi: int = 65536):
    return (log_uniform_lengths(seed, 0, count, lo, hi),
            log_uniform_lengths(seed, 1, count, lo, hi))


def serve_request(k: int, seed: int = 5, count: int = 100000, lo: int = 32, hi: int = 65536,
                  sigma: int = 20, rate: float = 0.20, arrival_s: float = 0.0) -> Request:
    """Request k of the serving stream: side lengths log-uniform in [lo, hi]
    independently; alphabet 20; with probability 1/2 b is a 20%-mutated copy
    of a (same 1/2, 1/4, 1/4 split, fitted to len_b), else independent."""
    ua = unit(seed, 0, 1, offset=k)[0]
    ub = unit(seed, 1, 1, offset=k)[0]
    la = int(min(max(math.floor(math.exp(math.log(lo) + ua * (math.log(hi + 1) - math.log(lo)))), lo), hi))
    lb = int(min(max(math.floor(math.exp(math.log(lo) + ub * (math.log(hi + 1) - math.log(lo)))), lo), hi))
    a = symbols(seed, 1000 + 8 * k, la, sigma)
    related = unit(seed, 2, 1, offset=k)[0] < 0.5
    if related:
        b = mutate_rate(a, sigma, rate, seed, 1000 + 8 * k + 1)
        b = fit_length(b, lb, sigma, seed, 1000 + 8 * k + 6)
    else:
        b = symbols(seed, 1000 + 8 * k + 7, lb, sigma)
    return Request(k, arrival_s, a, b)


def poisson_arrivals(seed: int, count: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (s) of a Poisson process: cumulative exponential gaps."""
    u = unit(seed, 3, count)
    gaps = -np.log1p(-u) / rate_per_s
    return np.cumsum(gaps)


def _serve_chunk(args):
    k0, k1, seed = args
    reqs = [serve_request(k, seed=seed) for k in range(k0, k1)]
    a_cat, a_off = _concat([r.a for r in reqs])
    b_cat, b_off = _concat([r.b for r in reqs])
    return k0, a_cat, a_off, b_cat, b_off


def serve_stream(count: int = 100000, seed: int = 5, workers: int = 0, chunk: int = 2000) -> Batch:
    """Requests 0..count-1 of the serving stream (the same bytes as
    serve_request(k) one by one), concatenated like a batch.  With workers > 1
    the chunks are made by a process pool started with `spawn` (safe in a
    process that already uses CUDA); the result does not depend on it."""
    jobs = [(k, min(count, k + chunk), seed) for k in range(0, count, chunk)]
    if workers > 1 and len(jobs) > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(workers, len(jobs))) as pool:
            parts = pool.map(_serve_chunk, jobs)
    else:
        parts = [_serve_chunk(j) for j in jobs]
    parts.sort(key=lambda x: x[0])
    a_cat = np.concatenate([p[1] for p in parts]) if parts else np.zeros(0, np.uint8)
    b_cat = np.concatenate([p[3] for p in parts]) if parts else np.zeros(0, np.uint8)
    a_off = np.zeros(count + 1, dtype=np.int64)
    b_off = np.zeros(count + 1, dtype=np.int64)
    k = 0
    for p in parts:
        n = p[2].size - 1
        a_off[k + 1:k + n + 1] = a_off[k] + p[2][1:]
        b_off[k + 1:k + n + 1] = b_off[k] + p[4][1:]
        k += n
    return Batch(a_cat, a_off, b_cat, b_off,
                 f"serving stream: {count} requests, lengths log-uniform [32, 65536], sigma 20, "
                 f"half 20%-mutated (seed {seed})")
