"""CPU oracle for the LCS table - TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The product library never calls it and
shares no code with it; it is built with plain gcc from `lcs_oracle.c`.

Functions (all follow Eq. (1) of the paper's Sec. "PACO LCS", generalised to
caller-given first row/column, see `lcs_oracle.c`):

* `lcs(a, b, top=None, left=None)` -> (L, bottom_row[m+1], right_col[n+1])
* `lcs_table(a, b, top=None, left=None)` -> full (n+1) x (m+1) table
* `lcs_batch(a_cat, a_off, b_cat, b_off, threads)` -> per-pair L, rows, cols
* `lcs_bitpar(a, b)` -> (L, bottom_row, right_col) by an independent method
  (the bit-vector LCS of Allison & Dix / Hyyro, `lcs_bitpar.c`), zero
  boundaries only: a cross-check of the DP on large inputs, not the
  definition
* `affine(a, b, match, mismatch, gap_open, gap_extend)` -> (score,
  bottom_row[m+1], right_col[n+1]): global alignment with affine gap costs,
  the variant the footnote to Eq. (1) names (Gotoh's recurrence,
  `affine_oracle.c`)
* `affine_batch(a_cat, a_off, b_cat, b_off, scores, threads)` -> per-pair
  scores
* `lws(n, d0, kind, T, seed)` -> (D[0..n], argmin[0..n]): the 1D problem of
  Sec. "PACO 1D" (least weight subsequence) with the weight families of
  `lws_oracle.c`; `lws_weight(kind, i, j, T, seed)` evaluates one weight

Pins that tie it to something other than itself live in
`tests/test_oracle_pins.py` (brute-force enumeration, indel distance,
closed forms, invariants, the CLRS worked example) and
`tests/test_oracle_affine_pins.py` (enumeration of every alignment, the
LCS, Levenshtein and indel special cases, gap-block closed forms,
symmetries) and `tests/test_oracle_lws_pins.py` (enumeration of every
subsequence path, Dijkstra of scipy on the same DAG, closed forms of the
test weight families).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lcs_oracle.c")
_SRC_BITPAR = os.path.join(_HERE, "lcs_bitpar.c")
_SRC_AFFINE = os.path.join(_HERE, "affine_oracle.c")
_SRC_LWS = os.path.join(_HERE, "lws_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no vector intrinsics)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_BITPAR), os.path.getmtime(_SRC_AFFINE),
                 os.path.getmtime(_SRC_LWS))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               _SRC, _SRC_BITPAR, _SRC_AFFINE, _SRC_LWS, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            lib.oracle_lcs.argtypes = [P, I64, P, I64, P, P, P, P, P]
            lib.oracle_lcs.restype = ctypes.c_int
            lib.oracle_lcs_table.argtypes = [P, I64, P, I64, P, P, P]
            lib.oracle_lcs_table.restype = ctypes.c_int
            lib.oracle_lcs_batch.argtypes = [P, P, P, P, I64, P, P, P, P, P, ctypes.c_int]
            lib.oracle_lcs_batch.restype = ctypes.c_int
            lib.oracle_lcs_bitpar.argtypes = [P, I64, P, I64, P, P, P]
            lib.oracle_lcs_bitpar.restype = ctypes.c_int
            lib.oracle_affine.argtypes = [P, I64, P, I64, I64, I64, I64, I64, P, P, P]
            lib.oracle_affine.restype = ctypes.c_int
            lib.oracle_affine_batch.argtypes = [P, P, P, P, I64, I64, I64, I64, I64, P, ctypes.c_int]
            lib.oracle_affine_batch.restype = ctypes.c_int
            lib.oracle_lws.argtypes = [I64, I64, ctypes.c_int, I64, ctypes.c_uint32, P, P]
            lib.oracle_lws.restype = ctypes.c_int
            lib.oracle_lws_weight.argtypes = [ctypes.c_int, I64, I64, I64, ctypes.c_uint32]
            lib.oracle_lws_weight.restype = I64
            _lib = lib
    return _lib


def _ptr(x):
    return None if x is None else x.ctypes.data_as(ctypes.c_void_p)


def _u8(x):
    if isinstance(x, (bytes, bytearray)):
        return np.frombuffer(bytes(x), dtype=np.uint8).copy()
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint8))


def _i32(x):
    return None if x is None else np.ascontiguousarray(np.asarray(x, dtype=np.int32))


def lcs(a, b, top=None, left=None):
    """(L, bottom_row, right_col) of the table of Eq. (1) with optional
    first row `top` (m+1 values) and first column `left` (n+1 values)."""
    lib = _load()
    a = _u8(a)
    b = _u8(b)
    n, m = a.size, b.size
    top = _i32(top)
    left = _i32(left)
    if top is not None and top.size != m + 1:
        raise ValueError("top must have m+1 entries")
    if left is not None and left.size != n + 1:
        raise ValueError("left must have n+1 entries")
    row = np.empty(m + 1, dtype=np.int32)
    col = np.empty(n + 1, dtype=np.int32)
    L = ctypes.c_int32(0)
    rc = lib.oracle_lcs(_ptr(a), n, _ptr(b), m, _ptr(top), _ptr(left), _ptr(row), _ptr(col),
                        ctypes.byref(L))
    if rc != 0:
        raise ValueError(f"oracle_lcs failed ({rc})")
    return int(L.value), row, col


def lcs_table(a, b, top=None, left=None):
    lib = _load()
    a = _u8(a)
    b = _u8(b)
    n, m = a.size, b.size
    H = np.empty((n + 1, m + 1), dtype=np.int32)
    rc = lib.oracle_lcs_table(_ptr(a), n, _ptr(b), m, _ptr(_i32(top)), _ptr(_i32(left)), _ptr(H))
    if rc != 0:
        raise ValueError(f"oracle_lcs_table failed ({rc})")
    return H


def lcs_batch(a_cat, a_off, b_cat, b_off, threads=None, boundaries=True):
    """Per-pair (L[npairs], rows_cat, row_off, cols_cat, col_off); pairs are
    spread over `threads` host threads (default: all cores)."""
    lib = _load()
    a_cat = _u8(a_cat)
    b_cat = _u8(b_cat)
    a_off = np.ascontiguousarray(a_off, dtype=np.int64)
    b_off = np.ascontiguousarray(b_off, dtype=np.int64)
    npairs = a_off.size - 1
    n = np.diff(a_off)
    m = np.diff(b_off)
    row_off = np.zeros(npairs + 1, dtype=np.int64)
    row_off[1:] = np.cumsum(m + 1)
    col_off = np.zeros(npairs + 1, dtype=np.int64)
    col_off[1:] = np.cumsum(n + 1)
    L = np.zeros(npairs, dtype=np.int32)
    rows = np.empty(int(row_off[-1]), dtype=np.int32) if boundaries else None
    cols = np.empty(int(col_off[-1]), dtype=np.int32) if boundaries else None
    if threads is None:
        threads = os.cpu_count() or 1
    rc = lib.oracle_lcs_batch(_ptr(a_cat), _ptr(a_off), _ptr(b_cat), _ptr(b_off), npairs,
                              _ptr(L), _ptr(rows), _ptr(row_off), _ptr(cols), _ptr(col_off),
                              int(threads))
    if rc != 0:
        raise ValueError(f"oracle_lcs_batch failed ({rc})")
    return L, rows, row_off, cols, col_off


def lcs_bitpar(a, b):
    """(L, bottom_row[m+1], right_col[n+1]) by the bit-vector method."""
    a = _u8(a)
    b = _u8(b)
    n, m = a.size, b.size
    L = ctypes.c_int32(0)
    row = np.zeros(m + 1, dtype=np.int32)
    col = np.zeros(n + 1, dtype=np.int32)
    vp = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    rc = _load().oracle_lcs_bitpar(vp(a) if n else None, n, vp(b) if m else None, m, ctypes.byref(L),
                                   vp(row), vp(col))
    if rc != 0:
        raise RuntimeError(f"oracle_lcs_bitpar failed ({rc})")
    return int(L.value), row, col


def affine(a, b, match, mismatch, gap_open, gap_extend):
    """(score, bottom_row[m+1], right_col[n+1]) of global alignment with
    affine gap costs: +match / -mismatch per aligned column, a gap run of k
    columns costs gap_open + k * gap_extend (all four >= 0)."""
    a = _u8(a)
    b = _u8(b)
    n, m = a.size, b.size
    score = ctypes.c_int64(0)
    row = np.empty(m + 1, dtype=np.int64)
    col = np.empty(n + 1, dtype=np.int64)
    rc = _load().oracle_affine(_ptr(a) if n else None, n, _ptr(b) if m else None, m, int(match), int(mismatch),
                               int(gap_open), int(gap_extend), ctypes.byref(score), _ptr(row), _ptr(col))
    if rc != 0:
        raise ValueError(f"oracle_affine failed ({rc})")
    return int(score.value), row, col


def affine_batch(a_cat, a_off, b_cat, b_off, scores, threads=None):
    """Per-pair scores (int64[npairs]); `scores` = (match, mismatch,
    gap_open, gap_extend); pairs spread over `threads` host threads."""
    a_cat = _u8(a_cat)
    b_cat = _u8(b_cat)
    a_off = np.ascontiguousarray(a_off, dtype=np.int64)
    b_off = np.ascontiguousarray(b_off, dtype=np.int64)
    npairs = a_off.size - 1
    out = np.zeros(npairs, dtype=np.int64)
    if threads is None:
        threads = os.cpu_count() or 1
    M, X, O, E = (int(v) for v in scores)
    rc = _load().oracle_affine_batch(_ptr(a_cat), _ptr(a_off), _ptr(b_cat), _ptr(b_off), npairs, M, X, O, E,
                                     _ptr(out), int(threads))
    if rc != 0:
        raise ValueError(f"oracle_affine_batch failed ({rc})")
    return out


def lws(n, d0=0, kind=0, T=40, seed=0):
    """(D[0..n], argmin[0..n]) of D[j] = min_{i<j} D[i] + w(i, j), D[0] = d0
    (int64 arrays; argmin = smallest minimising i, argmin[0] = -1)."""
    D = np.empty(int(n) + 1, dtype=np.int64)
    arg = np.empty(int(n) + 1, dtype=np.int64)
    rc = _load().oracle_lws(int(n), int(d0), int(kind), int(T), int(seed) & 0xFFFFFFFF, _ptr(D), _ptr(arg))
    if rc != 0:
        raise ValueError(f"oracle_lws failed ({rc})")
    return D, arg


def lws_weight(kind, i, j, T=40, seed=0):
    return int(_load().oracle_lws_weight(int(kind), int(i), int(j), int(T), int(seed) & 0xFFFFFFFF))
