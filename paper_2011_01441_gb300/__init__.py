"""Python binding of the GB300 LCS library (include/paco_lcs.h, include/paco_plan.h,
include/paco_affine.h, include/paco_lws.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libpaco_lcs.so.  Device buffers are torch CUDA tensors (torch is
used for device memory and streams); the functions keep the C names.  There
is no CPU fallback: if the library is missing or no GPU is present the calls
raise.

Table semantics (Eq. (1) of Tang & Gao, Sec. "PACO LCS"): a gives the rows,
b the columns; results are L = H[n][m], bottom_row = H[n][0..m] and
right_col = H[0..n][m].
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpaco_lcs.so")

PACO_OK = 0
PACO_PENDING = 1
PACO_EINVAL = -1
PACO_ENOMEM = -2
PACO_ETIMEOUT = -3
PACO_EDEVICE = -4
PACO_EBUSY = -5
PACO_ENOTFOUND = -6

OPT_ENGINE = 1
OPT_CHUNK = 2
OPT_WARPS = 3
OPT_WAIT_LIMIT_NS = 4
OPT_ORIENT = 5
OPT_SCHEDULE = 6
OPT_ALPHABET = 7
OPT_BATCH_CHUNKS = 8
OPT_WORDS_PER_LANE = 9
OPT_TILES = 10
OPT_TILE_BASE = 11
OPT_AFFINE_ROWS = 12
OPT_SERVE_CHUNKS = 13
OPT_TEST_STALL = 100

_lib = None


class PacoError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        super().__init__(f"paco status {status} ({_strerror(status)}){': ' + msg if msg else ''}")


class PacoTile(ctypes.Structure):
    _fields_ = [("r0", ctypes.c_int64), ("r1", ctypes.c_int64), ("c0", ctypes.c_int64),
                ("c1", ctypes.c_int64), ("label", ctypes.c_int32), ("owner", ctypes.c_int32),
                ("order", ctypes.c_int64)]


class PacoPairPlan(ctypes.Structure):
    _fields_ = [("transpose", ctypes.c_int32), ("chunk", ctypes.c_int32), ("warps", ctypes.c_int32),
                ("nstrips", ctypes.c_int32), ("words_per_lane", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("L", ctypes.c_int64), ("S", ctypes.c_int64)]


class PacoAffineScores(ctypes.Structure):
    _fields_ = [("match", ctypes.c_int32), ("mismatch", ctypes.c_int32), ("gap_open", ctypes.c_int32),
                ("gap_extend", ctypes.c_int32)]


class Paco1dTask(ctypes.Structure):
    _fields_ = [("j0", ctypes.c_int64), ("j1", ctypes.c_int64), ("i0", ctypes.c_int64), ("i1", ctypes.c_int64),
                ("proc", ctypes.c_int32), ("phase", ctypes.c_int32), ("merge_group", ctypes.c_int32),
                ("kind", ctypes.c_int32)]


class PacoLwsWeight(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int32), ("seed", ctypes.c_uint32), ("noise", ctypes.c_int32)]


class PacoServeStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in
                ("submitted", "completed", "cells_done", "queued_now", "inflight_now",
                 "batches_launched", "bytes_in_use", "bytes_budget", "host_launch_ns", "host_complete_ns",
                 "host_stage_ns", "host_batch_ns")]


def load():
    """Load libpaco_lcs.so (built by __graft_entry__.build()); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    P, I64, I32, INT = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
    sig = {
        "paco_ctx_create": ([INT, ctypes.c_size_t, ctypes.POINTER(P)], INT),
        "paco_ctx_destroy": ([P], None),
        "paco_strerror": ([INT], ctypes.c_char_p),
        "paco_last_error": ([P], ctypes.c_char_p),
        "paco_ctx_sync": ([P, P], INT),
        "paco_ctx_set_option": ([P, INT, I64], INT),
        "paco_ctx_get_option": ([P, INT, ctypes.POINTER(I64)], INT),
        "paco_lcs_length": ([P, P, I64, P, I64, P, P], INT),
        "paco_lcs_boundaries": ([P, P, I64, P, I64, P, P, P, P, P, P], INT),
        "paco_lcs_boundaries_host": ([P, P, I64, P, I64, P, P, P, P, P, P], INT),
        "paco_lcs_batch": ([P, P, P, P, P, I32, P, P, P, P, P, P], INT),
        "paco_lcs_boundaries_static": ([P, I64, P, I64, P, P, P, P], INT),
        "paco_lcs_submit": ([P, P, I64, P, I64, INT, ctypes.POINTER(ctypes.c_uint64)], INT),
        "paco_lcs_poll": ([P, ctypes.c_uint64, P, P, P], INT),
        "paco_lcs_submit_many": ([P, P, P, P, P, I64, P, P], INT),
        "paco_lcs_subsequence": ([P, P, I64, P, I64, P, P, P, P], INT),
        "paco_lcs_poll_many": ([P, P, I64, P, P, P], INT),
        "paco_serve_get_stats": ([P, ctypes.POINTER(PacoServeStats)], INT),
        "paco_measure_int_peak": ([P, INT, ctypes.POINTER(ctypes.c_double), P], INT),
        "paco_last_kernel_ms": ([P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_char_p)], INT),
        "paco_plan_partition": ([I64, I64, I32, I64, P, I64, ctypes.POINTER(I64)], INT),
        "paco_plan_partition_deps": ([I64, I64, I32, I64, P, P, I64, ctypes.POINTER(I64)], INT),
        "paco_plan_pair": ([I64, I64, I32, I32, I32, I32, I32, I32, ctypes.POINTER(PacoPairPlan), P, I64], INT),
        "paco_plan_tiles": ([I64, I64, I32, I32, I64, P, I64, P, P, P, I64, P, P], INT),
        "paco_affine_align": ([P, P, I64, P, I64, ctypes.POINTER(PacoAffineScores), P, P, P, P], INT),
        "paco_affine_align_host": ([P, P, I64, P, I64, ctypes.POINTER(PacoAffineScores), P, P, P, P], INT),
        "paco_affine_batch": ([P, P, P, P, P, I32, ctypes.POINTER(PacoAffineScores), P, P], INT),
        "paco_lws": ([P, I64, I32, ctypes.POINTER(PacoLwsWeight), P, P], INT),
        "paco_plan_1d": ([I64, I32, I64, P, I64, ctypes.POINTER(I64), ctypes.POINTER(I32), ctypes.POINTER(I64)], INT),
        "paco_plan_shard": ([P, P, I64, I32, P, P], INT),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _strerror(status: int) -> str:
    try:
        return load().paco_strerror(status).decode()
    except Exception:
        return "?"


def _check(rc: int, ctx=None):
    if rc < 0:
        msg = ""
        if ctx is not None and ctx.handle:
            msg = (load().paco_last_error(ctx.handle) or b"").decode()
        raise PacoError(rc, msg)
    return rc


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """Owns a paco_ctx (scratch, plans, serving loop) on one CUDA device."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        h = ctypes.c_void_p()
        _check(load().paco_ctx_create(device, mem_budget_bytes, ctypes.byref(h)))
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            load().paco_ctx_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, option: int, value: int):
        _check(load().paco_ctx_set_option(self.handle, option, int(value)), self)

    def get_option(self, option: int) -> int:
        v = ctypes.c_int64()
        _check(load().paco_ctx_get_option(self.handle, option, ctypes.byref(v)), self)
        return v.value

    def sync(self, stream=None) -> int:
        """Wait for enqueued work; raises on a sticky device error."""
        s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        return _check(load().paco_ctx_sync(self.handle, s), self)


def _u8(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.uint8 or not t.is_cuda or t.dim() != 1:
        raise TypeError(f"{name} must be a 1-D uint8 CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def paco_lcs_length(ctx: Context, a, b, out=None, stream=None):
    """L for device strings a (rows) and b (columns); returns an int32[1] tensor."""
    import torch
    a, b = _u8(a, "a"), _u8(b, "b")
    if out is None:
        out = torch.empty(1, dtype=torch.int32, device=a.device)
    _check(load().paco_lcs_length(ctx.handle, _ptr(a), a.numel(), _ptr(b), b.numel(), _ptr(out),
                                  _stream(stream)), ctx)
    return out


def paco_lcs_boundaries(ctx: Context, a, b, top=None, left=None, bottom_row=None, right_col=None,
                        length=None, stream=None, want_rows=True, want_cols=True):
    """(L int32[1], bottom_row int32[m+1], right_col int32[n+1]) for device strings."""
    import torch
    a, b = _u8(a, "a"), _u8(b, "b")
    n, m = a.numel(), b.numel()
    dev = a.device
    if want_rows and bottom_row is None:
        bottom_row = torch.empty(m + 1, dtype=torch.int32, device=dev)
    if want_cols and right_col is None:
        right_col = torch.empty(n + 1, dtype=torch.int32, device=dev)
    if length is None:
        length = torch.empty(1, dtype=torch.int32, device=dev)
    for t, k, name in ((top, m + 1, "top"), (left, n + 1, "left")):
        if t is not None and (t.dtype != torch.int32 or t.numel() != k or not t.is_cuda):
            raise ValueError(f"{name} must be int32[{k}] on the GPU")
    _check(load().paco_lcs_boundaries(ctx.handle, _ptr(a), n, _ptr(b), m, _ptr(top), _ptr(left),
                                      _ptr(bottom_row), _ptr(right_col), _ptr(length),
                                      _stream(stream)), ctx)
    return length, bottom_row, right_col


def paco_lcs_boundaries_static(a, b, bottom_row=None, right_col=None, length=None, stream=None,
                               want_rows=True, want_cols=True, checked=False):
    """The allocation-free variant (see include/paco_lcs.h): zero boundaries,
    scratch in the library's fixed device array.  Outputs are allocated here
    by torch only when not given; a caller that cannot allocate passes all
    three.  The call runs with a's device made current; every tensor must be
    on that device.

    A device wait that timed out shows up as a NEGATIVE value in `length` (a
    paco_status), not as an exception, because the call is stream ordered.
    With checked=True the stream is synchronised and a negative length
    raises PacoError."""
    import torch
    a, b = _u8(a, "a"), _u8(b, "b")
    n, m = a.numel(), b.numel()
    dev = a.device
    with torch.cuda.device(dev):
        if want_rows and bottom_row is None:
            bottom_row = torch.empty(m + 1, dtype=torch.int32, device=dev)
        if want_cols and right_col is None:
            right_col = torch.empty(n + 1, dtype=torch.int32, device=dev)
        if length is None:
            length = torch.empty(1, dtype=torch.int32, device=dev)
        for t, k, name in ((b, m, "b"), (bottom_row, m + 1, "bottom_row"), (right_col, n + 1, "right_col"),
                           (length, 1, "length")):
            if t is None:
                continue
            if t.device != dev:
                raise ValueError(f"{name} is on {t.device}, a is on {dev}: every buffer must share one device")
            if t is not b and (t.dtype != torch.int32 or t.numel() < k or not t.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous int32 tensor of at least {k} values")
        st = torch.cuda.current_stream(dev) if stream is None else stream
        _check(load().paco_lcs_boundaries_static(_ptr(a), n, _ptr(b), m, _ptr(bottom_row), _ptr(right_col),
                                                 _ptr(length), ctypes.c_void_p(st.cuda_stream)))
        if checked:
            st.synchronize()
            v = int(length[0].item())
            if v < 0:
                raise PacoError(v, "device-side failure in paco_lcs_boundaries_static")
    return length, bottom_row, right_col


def paco_lcs_boundaries_host(ctx: Context, a, b, top=None, left=None, want_rows=True,
                             want_cols=True):
    """Host-buffer variant: numpy uint8 in, numpy int32 out (copies inside the call)."""
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.uint8)
    b = np.ascontiguousarray(b, dtype=np.uint8)
    n, m = a.size, b.size
    row = np.empty(m + 1, dtype=np.int32) if want_rows else None
    col = np.empty(n + 1, dtype=np.int32) if want_cols else None
    top = None if top is None else np.ascontiguousarray(top, dtype=np.int32)
    left = None if left is None else np.ascontiguousarray(left, dtype=np.int32)
    L = ctypes.c_int32(0)
    p = lambda x: None if x is None else x.ctypes.data_as(ctypes.c_void_p)
    _check(load().paco_lcs_boundaries_host(ctx.handle, p(a), n, p(b), m, p(top), p(left), p(row), p(col),
                                           ctypes.byref(L), None), ctx)
    return int(L.value), row, col


def paco_lcs_boundaries_host_ptr(ctx: Context, a_ptr, n, b_ptr, m, row_ptr, col_ptr, len_ptr):
    """Raw host pointers (e.g. pinned torch tensors): for end-to-end timing."""
    _check(load().paco_lcs_boundaries_host(ctx.handle, a_ptr, n, b_ptr, m, None, None, row_ptr, col_ptr,
                                           len_ptr, None), ctx)


def paco_lcs_batch(ctx: Context, a_cat, b_cat, h_a_off, h_b_off, lengths=None, rows_cat=None,
                   h_row_off=None, cols_cat=None, h_col_off=None, stream=None):
    """Batch of independent pairs: device concatenations (uint8 tensors) and
    HOST int64 offsets.  Returns the int32[npairs] length tensor; optional
    device outputs rows_cat/cols_cat at the host offsets h_row_off/h_col_off."""
    import numpy as np
    import torch
    h_a_off = np.ascontiguousarray(h_a_off, dtype=np.int64)
    h_b_off = np.ascontiguousarray(h_b_off, dtype=np.int64)
    npairs = h_a_off.size - 1
    if lengths is None:
        lengths = torch.empty(max(npairs, 1), dtype=torch.int32, device=a_cat.device)
    ro = None if h_row_off is None else np.ascontiguousarray(h_row_off, dtype=np.int64)
    co = None if h_col_off is None else np.ascontiguousarray(h_col_off, dtype=np.int64)
    p = lambda x: None if x is None else x.ctypes.data_as(ctypes.c_void_p)
    _check(load().paco_lcs_batch(ctx.handle, _ptr(a_cat), _ptr(b_cat), p(h_a_off), p(h_b_off), npairs,
                                 _ptr(lengths), _ptr(rows_cat), p(ro), _ptr(cols_cat), p(co),
                                 _stream(stream)), ctx)
    return lengths


def _scores(scores):
    M, X, O, E = (int(v) for v in scores)
    return ctypes.byref(PacoAffineScores(M, X, O, E))


def paco_affine_align(ctx: Context, a, b, scores, score=None, bottom_row=None, right_col=None,
                      want_rows=False, want_cols=False, stream=None):
    """Global alignment with affine gap costs of device strings a (rows) and
    b (columns); scores = (match, mismatch, gap_open, gap_extend).  Returns
    (score int32[1], bottom_row int32[m+1] or None, right_col int32[n+1] or None)."""
    import torch
    a, b = _u8(a, "a"), _u8(b, "b")
    n, m = a.numel(), b.numel()
    if score is None:
        score = torch.empty(1, dtype=torch.int32, device=a.device)
    if want_rows and bottom_row is None:
        bottom_row = torch.empty(m + 1, dtype=torch.int32, device=a.device)
    if want_cols and right_col is None:
        right_col = torch.empty(n + 1, dtype=torch.int32, device=a.device)
    _check(load().paco_affine_align(ctx.handle, _ptr(a), n, _ptr(b), m, _scores(scores), _ptr(score),
                                    _ptr(bottom_row), _ptr(right_col), _stream(stream)), ctx)
    return score, bottom_row, right_col


def paco_affine_align_host_ptr(ctx: Context, a_ptr, n, b_ptr, m, scores, score_ptr, row_ptr=None, col_ptr=None):
    """Host-buffer variant on raw host pointers (e.g. pinned tensors)."""
    _check(load().paco_affine_align_host(ctx.handle, a_ptr, n, b_ptr, m, _scores(scores), score_ptr, row_ptr,
                                         col_ptr, None), ctx)


def paco_affine_batch(ctx: Context, a_cat, b_cat, h_a_off, h_b_off, scores, out=None, stream=None):
    """Scores of independent pairs: device concatenations, HOST int64 offsets;
    returns the int32[npairs] score tensor."""
    import numpy as np
    import torch
    h_a_off = np.ascontiguousarray(h_a_off, dtype=np.int64)
    h_b_off = np.ascontiguousarray(h_b_off, dtype=np.int64)
    npairs = h_a_off.size - 1
    if out is None:
        out = torch.empty(max(npairs, 1), dtype=torch.int32, device=a_cat.device)
    p = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    _check(load().paco_affine_batch(ctx.handle, _ptr(a_cat), p(h_a_off), _ptr(b_cat), p(h_b_off), npairs,
                                    _scores(scores), _ptr(out), _stream(stream)), ctx)
    return out


def paco_lws(ctx: Context, n: int, d0: int = 0, T: int = 40, seed: int = 0, noise: bool = True, out=None,
             stream=None):
    """D[0..n] of the 1D problem (Eq. 1D) with the weight of include/paco_lws.h;
    returns an int32[n+1] CUDA tensor."""
    import torch
    if out is None:
        out = torch.empty(int(n) + 1, dtype=torch.int32, device="cuda")
    w = PacoLwsWeight(int(T), int(seed) & 0xFFFFFFFF, int(bool(noise)))
    _check(load().paco_lws(ctx.handle, int(n), int(d0), ctypes.byref(w), _ptr(out), _stream(stream)), ctx)
    return out


def paco_plan_1d(n: int, p: int, base: int):
    """The PACO 1D partition (include/paco_plan.h): dict with `tasks` (list of
    dicts j0, j1, i0, i1, proc, phase, merge_group, kind), `phases`, `temp_words`."""
    L = load()
    cnt, ph, tw = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
    if L.paco_plan_1d(int(n), int(p), int(base), None, 0, ctypes.byref(cnt), ctypes.byref(ph), ctypes.byref(tw)) != 0:
        raise ValueError("paco_plan_1d failed")
    arr = (Paco1dTask * max(1, cnt.value))()
    L.paco_plan_1d(int(n), int(p), int(base), ctypes.cast(arr, ctypes.c_void_p), cnt.value, ctypes.byref(cnt),
                   ctypes.byref(ph), ctypes.byref(tw))
    tasks = [{f: getattr(arr[k], f) for f, _ in Paco1dTask._fields_} for k in range(cnt.value)]
    return {"tasks": tasks, "phases": ph.value, "temp_words": tw.value}


def paco_lcs_submit(ctx: Context, a, b, want_boundaries=False) -> int:
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.uint8)
    b = np.ascontiguousarray(b, dtype=np.uint8)
    t = ctypes.c_uint64(0)
    _check(load().paco_lcs_submit(ctx.handle, a.ctypes.data_as(ctypes.c_void_p), a.size,
                                  b.ctypes.data_as(ctypes.c_void_p), b.size, int(bool(want_boundaries)),
                                  ctypes.byref(t)), ctx)
    return t.value


def paco_lcs_poll(ctx: Context, ticket: int, n: int = 0, m: int = 0, want_boundaries=False):
    """None while pending; else (L, row or None, col or None)."""
    import numpy as np
    L = ctypes.c_int32(0)
    row = np.empty(m + 1, dtype=np.int32) if want_boundaries else None
    col = np.empty(n + 1, dtype=np.int32) if want_boundaries else None
    p = lambda x: None if x is None else x.ctypes.data_as(ctypes.c_void_p)
    rc = load().paco_lcs_poll(ctx.handle, ctypes.c_uint64(ticket), ctypes.byref(L), p(row), p(col))
    if rc == PACO_PENDING:
        return None
    _check(rc, ctx)
    return int(L.value), row, col


def paco_lcs_submit_many(ctx: Context, a_cat, a_off, b_cat, b_off, partial=False):
    """Submit len(a_off)-1 length-only requests (host arrays) in one call;
    returns their tickets (uint64 array).  With partial=True a full queue or
    arena (PACO_EBUSY) is not an error: the tickets of the first requests
    taken are returned and the caller submits the rest later."""
    import numpy as np
    a_cat = np.ascontiguousarray(a_cat, dtype=np.uint8)
    b_cat = np.ascontiguousarray(b_cat, dtype=np.uint8)
    a_off = np.ascontiguousarray(a_off, dtype=np.int64)
    b_off = np.ascontiguousarray(b_off, dtype=np.int64)
    count = a_off.size - 1
    t = np.zeros(max(count, 1), dtype=np.uint64)
    taken = ctypes.c_int64(0)
    vp = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    rc = load().paco_lcs_submit_many(ctx.handle, vp(a_cat), vp(a_off), vp(b_cat), vp(b_off), count, vp(t),
                                     ctypes.byref(taken))
    if not (partial and rc == PACO_EBUSY):
        _check(rc, ctx)
    return t[:taken.value]


def paco_lcs_poll_many(ctx: Context, tickets):
    """Poll length-only tickets: returns (status, lengths) int32 arrays;
    status PACO_PENDING for those still running (finished ones are released)."""
    import numpy as np
    tickets = np.ascontiguousarray(tickets, dtype=np.uint64)
    st = np.empty(max(tickets.size, 1), dtype=np.int32)
    ln = np.zeros(max(tickets.size, 1), dtype=np.int32)
    vp = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    _check(load().paco_lcs_poll_many(ctx.handle, vp(tickets), tickets.size, vp(ln), vp(st), None), ctx)
    return st[:tickets.size], ln[:tickets.size]


def paco_lcs_subsequence(ctx: Context, a, b, stream=None):
    """One LCS of device uint8 tensors a, b: returns (ai, bj) int32 device
    tensors of length L with a[ai] == b[bj], both strictly increasing."""
    import torch
    a, b = _u8(a, "a"), _u8(b, "b")
    n, m = a.numel(), b.numel()
    cap = max(1, min(n, m))
    ai = torch.empty(cap, dtype=torch.int32, device=a.device)
    bj = torch.empty(cap, dtype=torch.int32, device=a.device)
    ln = torch.zeros(1, dtype=torch.int32, device=a.device)
    _check(load().paco_lcs_subsequence(ctx.handle, _ptr(a), n, _ptr(b), m, _ptr(ai), _ptr(bj), _ptr(ln),
                                       _stream(stream)), ctx)
    L = int(ln.item())
    return ai[:L], bj[:L]


def paco_serve_get_stats(ctx: Context) -> dict:
    s = PacoServeStats()
    _check(load().paco_serve_get_stats(ctx.handle, ctypes.byref(s)), ctx)
    return {k: getattr(s, k) for k, _ in PacoServeStats._fields_}


def paco_measure_int_peak(ctx: Context, op: int) -> float:
    v = ctypes.c_double(0)
    _check(load().paco_measure_int_peak(ctx.handle, op, ctypes.byref(v), None), ctx)
    return v.value


def paco_last_kernel_ms(ctx: Context):
    v = ctypes.c_double(0)
    name = ctypes.c_char_p()
    _check(load().paco_last_kernel_ms(ctx.handle, ctypes.byref(v), ctypes.byref(name)), ctx)
    return v.value, (name.value or b"").decode()


# ---- planner (host only) --------------------------------------------------

def paco_plan_partition(n: int, m: int, p: int, base: int):
    """List of tile dicts (r0, r1, c0, c1, label, owner, order) in time-line order."""
    cnt = ctypes.c_int64(0)
    _check(load().paco_plan_partition(n, m, p, base, None, 0, ctypes.byref(cnt)))
    arr = (PacoTile * max(cnt.value, 1))()
    _check(load().paco_plan_partition(n, m, p, base, arr, cnt.value, ctypes.byref(cnt)))
    return [{k: getattr(arr[i], k) for k, _ in PacoTile._fields_} for i in range(cnt.value)]


def paco_plan_partition_deps(n: int, m: int, p: int, base: int):
    import numpy as np
    cnt = ctypes.c_int64(0)
    _check(load().paco_plan_partition(n, m, p, base, None, 0, ctypes.byref(cnt)))
    off = np.zeros(cnt.value + 1, dtype=np.int64)
    nidx = ctypes.c_int64(0)
    _check(load().paco_plan_partition_deps(n, m, p, base, off.ctypes.data_as(ctypes.c_void_p), None, 0,
                                           ctypes.byref(nidx)))
    idx = np.zeros(max(nidx.value, 1), dtype=np.int64)
    _check(load().paco_plan_partition_deps(n, m, p, base, off.ctypes.data_as(ctypes.c_void_p),
                                           idx.ctypes.data_as(ctypes.c_void_p), nidx.value,
                                           ctypes.byref(nidx)))
    return off, idx[:nidx.value]


TILES_PACO, TILES_PA, TILES_PO = 1, 2, 3


def paco_plan_tiles(n: int, m: int, p: int, kind: int, base: int):
    """Tile schedule (kind TILES_PACO / TILES_PA / TILES_PO): returns dict with
    tiles (list of dicts r0 r1 c0 c1), dep_off, dep_idx, critical_cells."""
    import numpy as np
    cnt, nidx, crit = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load().paco_plan_tiles(n, m, p, kind, base, None, 0, ctypes.byref(cnt), None, None, 0,
                                  ctypes.byref(nidx), ctypes.byref(crit)))
    arr = (PacoTile * max(1, cnt.value))()
    off = np.zeros(cnt.value + 1, dtype=np.int64)
    idx = np.zeros(max(1, nidx.value), dtype=np.int64)
    vp = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    _check(load().paco_plan_tiles(n, m, p, kind, base, arr, cnt.value, ctypes.byref(cnt), vp(off), vp(idx),
                                  idx.size, ctypes.byref(nidx), ctypes.byref(crit)))
    tiles = [{k: getattr(arr[i], k) for k in ("r0", "r1", "c0", "c1")} for i in range(cnt.value)]
    return {"tiles": tiles, "dep_off": off, "dep_idx": idx[:nidx.value], "critical_cells": crit.value}


def paco_plan_pair(n: int, m: int, sms: int, chunk=0, warps=0, orient=0, schedule=0, words_per_lane=0):
    import numpy as np
    pl = PacoPairPlan()
    rows = np.zeros(1 << 16, dtype=np.int64)
    _check(load().paco_plan_pair(n, m, sms, chunk, warps, orient, schedule, words_per_lane, ctypes.byref(pl),
                                 rows.ctypes.data_as(ctypes.c_void_p), rows.size))
    d = {k: getattr(pl, k) for k, _ in PacoPairPlan._fields_ if k != "pad"}
    d["row0"] = rows[:pl.nstrips + 1].copy()
    return d
