"""LCS GCUPS benchmark on GB300 (one JSON line on rank 0).

Default workload: one 131072 x 131072 pair (alphabet 20, b = a with exactly
10% substitutions and 5% single-symbol indels), LCS length plus the last row
and column, through paco_lcs_boundaries.  A step is one whole pass of the
path over that pair: boundary preparation, the strip-pipeline kernel, and the
two boundary prefixes.  Inputs are resident in HBM before timing; the 256 KB
of inputs fit in L2, so L2 is flushed (a 512 MiB write) between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W]
                 [--config mutated|small|skinny|batch|serve|recover|schedules|affine|affine_batch|lws]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Under torchrun each rank computes its own copy of the workload (independent
problems: weak scaling, no collective on the data path); the timed region is
bracketed by a barrier and synchronize and the max over ranks is reported.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2011_01441_gb300 import workloads as W  # noqa: E402

METRIC = "LCS GCUPS on 1 GB300, % of INT32 roofline; served p50/p99 latency vs plain"
# Algorithmic integer lane-ops of one bit-parallel column step of a 31-row
# word: X = V & M, the carry add V + X + c, V & ~M, and the final OR (the
# recurrence of Eq. 1 in the bit-vector form of Allison-Dix / Hyyro).
OPS_PER_WORD_STEP = 4
# The per-cell work the roofline is defined on: Eq. 1 evaluated cell by cell
# as h = max(max(up, left), diag + (a_i == b_j)) is 4 INT32 lane-ops (match,
# add, max, max).  The bit-parallel kernels need only OPS_PER_WORD_STEP per
# 31 cells, so they can exceed this cell-wise roofline; both are reported.
CELL_OPS = 4
# Affine-gap alignment (Gotoh's recurrence, the variant named beside Eq. 1):
# per cell H - (open + extend) once (shared by the gap to the right and the
# gap below), E and F each one subtract and one max, the match score one
# compare and one select, the diagonal add, and the three-way max as two
# maxes: 10 INT32 lane-ops.
AFFINE_CELL_OPS = 10
AFFINE_SCORES = (2, 3, 5, 2)   # match, mismatch, gap open, gap extend
# The 1D problem (Eq. 1D): one term D[i] + w(i, j) and its min is 20 INT32
# lane-ops with the benchmark weight: the jump deviation, the cap test (two
# compares) and select, the square, the hash (a multiply, the xor with j and
# the seed, three shift-xor rounds, two multiplies, the mask), the two adds
# and the min.
LWS_TERM_OPS = 20
LWS_N, LWS_T, LWS_SEED = 131072, 40, 6


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _init_dist(ws, local, backend="nccl"):
    """One process per GPU (torchrun): join the process group when ws > 1."""
    import torch
    import torch.distributed as dist
    if ws > 1 and not dist.is_initialized():
        if backend == "nccl":
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)


def _max_over_ranks(x, device=None):
    """The slowest rank's value (the timed region is the max over ranks)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def weak_scaling_value(cells_per_rank, ws, steps, max_ms):
    """Whole-job GCUPS: the cells all ranks processed over the slowest rank's time."""
    return cells_per_rank * ws * steps / (max_ms * 1e-3) / 1e9


def _workload(name):
    if name == "small":
        return W.single_small(), "pair 4096x4096 sigma=4 iid (seed 1)"
    if name == "mutated":
        return W.single_mutated(), "pair 131072x131072 sigma=20, b = a with 10% subs + 5% indels (seed 2)"
    if name == "skinny":
        return W.single_skinny(), "pair 1048576x16384 bytes uniform 0..255 (seed 3)"
    raise ValueError(name)


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region.

    nvidia-smi is started on entry and the region only begins once its first
    sample has arrived; each sample is stamped with its arrival time, and
    the summary keeps the samples that arrived inside the region (plus one
    sampling period after it, for the sample that covers the region's end).
    A region shorter than the sampling period may hold none: then the first
    sample after the region began stands in and `in_region` says so."""

    PERIOD_MS = 50

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []   # (arrival time, csv line)
        self.t_in = self.t_out = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.monotonic()
            while not self.lines and time.monotonic() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.005)
        except Exception:
            self.proc = None
        self.t_in = time.monotonic()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def __exit__(self, *exc):
        self.t_out = time.monotonic()
        if self.proc is not None:
            time.sleep(self.PERIOD_MS * 1.5e-3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    @staticmethod
    def _parse(line):
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            return None
        try:
            sm, mx = float(f[1]), float(f[2])
        except ValueError:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        return sm, mx, {nm for nm, v in zip(names, f[5:9]) if v.lower().startswith("active")}

    def summary(self):
        if self.t_in is None:
            return None
        t_end = (self.t_out if self.t_out is not None else time.monotonic()) + self.PERIOD_MS * 1e-3
        parsed = [(t, self._parse(ln)) for t, ln in self.lines]
        parsed = [(t, r) for t, r in parsed if r is not None]
        inside = [r for t, r in parsed if self.t_in <= t <= t_end]
        in_region = bool(inside)
        if not inside:
            after = [r for t, r in parsed if t >= self.t_in]
            inside = after[:1]
        if not inside:
            return None
        reasons = set().union(*(r[2] for r in inside))
        return {"sm_mhz": statistics.median(r[0] for r in inside), "sm_max_mhz": inside[-1][1],
                "reasons": sorted(reasons), "samples": len(inside), "in_region": in_region,
                "period_ms": self.PERIOD_MS,
                "region_ms": round(((self.t_out or time.monotonic()) - self.t_in) * 1e3, 1)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def _profiled_traffic(profile, sources):
    """Per-launch DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum)
    from a committed ncu summary under profiles/, only while the kernel's
    sources still hash to the ones that were profiled; else None."""
    import hashlib
    try:
        rec = {}
        with open(os.path.join(ROOT, "profiles", profile)) as f:
            for line in f:
                k, _, v = line.partition(":")
                if k.strip() in ("traffic_bytes_per_launch", "source_sha256"):
                    rec[k.strip()] = v.strip()
        h = hashlib.sha256()
        for src in sources:
            with open(os.path.join(ROOT, "paper_2011_01441_gb300", "csrc", src), "rb") as f:
                h.update(f.read())
        if rec.get("source_sha256") != h.hexdigest():
            return None
        return int(rec["traffic_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


# Dependency chain of one column of the bit-parallel step on a lane's critical
# path: one LOP3 (4.4 cycles) then the carry add (about 4 cycles), measured
# on GB300 with single-warp dependent chains.
CHAIN_CYCLES_PER_COLUMN = 8.4


def cpu_baseline_pair(a, b, budget_s=12.0):
    """The oracle as it stands, single thread, on the first rows of the same
    pair (a bounded sample), extrapolated to GCUPS."""
    import oracle
    oracle.build()
    probe = min(a.size, 512)
    t = time.perf_counter()
    oracle.lcs(a[:probe], b)
    dt = max(time.perf_counter() - t, 1e-6)
    rows = int(min(a.size, max(probe, probe * budget_s / dt)))
    t = time.perf_counter()
    oracle.lcs(a[:rows], b)
    dt = time.perf_counter() - t
    return {"value": rows * b.size / dt / 1e9, "unit": "GCUPS", "cores": 1, "kind": "oracle",
            "sample": f"first {rows} rows x all {b.size} columns of the same pair ({rows * b.size:.3e} cells, {dt:.1f} s)"}


def _reference_step(config, budget_s):
    """One bounded sample of the oracle on the host cores for `config`:
    (result dict like cpu_baseline, workload description, unit)."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    if config in ("mutated", "small", "skinny"):
        pair, desc = _workload(config)
        return cpu_baseline_pair(pair.a, pair.b, budget_s=budget_s), desc, "GCUPS"
    if config == "affine":
        pair = W.single_mutated()
        return (cpu_baseline_affine(pair.a, pair.b, AFFINE_SCORES, budget_s=budget_s),
                "affine-gap alignment, pair 131072x131072 sigma=20, 10% subs + 2.5% ins + 2.5% del (seed 2)", "GCUPS")
    if config == "lws":
        t0 = time.perf_counter()
        oracle.lws(4096, 0, 0, LWS_T, LWS_SEED)
        dt = max(time.perf_counter() - t0, 1e-6)
        m = int(min(LWS_N, 4096 * (budget_s / dt) ** 0.5))
        t0 = time.perf_counter()
        oracle.lws(m, 0, 0, LWS_T, LWS_SEED)
        dt = time.perf_counter() - t0
        return ({"value": m * (m + 1) / 2 / dt / 1e9, "unit": "GCUPS", "cores": 1, "kind": "oracle",
                 "sample": f"the first {m} outputs of the same problem ({m * (m + 1) / 2:.3e} terms, {dt:.1f} s)"},
                f"1D problem (least weight subsequence), n={LWS_N}, D[0]=0, weight T={LWS_T} seed={LWS_SEED}",
                "GCUPS (terms D[i] + w(i, j) of Eq. 1D per second)")
    # the batch workloads: the first k pairs, spread over the host cores
    bt = W.batch_pairs()
    affine = config == "affine_batch"
    k = min(bt.npairs, 4 * cores)
    while True:
        t0 = time.perf_counter()
        if affine:
            oracle.affine_batch(bt.a_cat, bt.a_off[:k + 1], bt.b_cat, bt.b_off[:k + 1], AFFINE_SCORES, threads=cores)
        else:
            oracle.lcs_batch(bt.a_cat, bt.a_off[:k + 1], bt.b_cat, bt.b_off[:k + 1], threads=cores, boundaries=False)
        dt = time.perf_counter() - t0
        if dt > budget_s / 2 or k == bt.npairs:
            break
        k = min(bt.npairs, int(k * max(2.0, budget_s / max(dt, 1e-3))))
    ck = float(np.sum(np.diff(bt.a_off[:k + 1]) * np.diff(bt.b_off[:k + 1])))
    desc = ("affine-gap alignment, " if affine else "") + bt.name + " (seed 4)"
    return ({"value": ck / dt / 1e9, "unit": "GCUPS", "cores": cores, "kind": "oracle",
             "sample": f"first {k} of {bt.npairs} pairs ({ck:.3e} cells, {dt:.1f} s)"}, desc, "GCUPS")


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    cfg = args.config if args.config in ("mutated", "small", "skinny", "affine", "affine_batch", "lws") else "batch"
    for _ in range(args.warmup):
        _reference_step(cfg, 1.0)
    vals = []
    t0 = time.perf_counter()
    last = desc = unit = None
    for _ in range(args.steps):
        last, desc, unit = _reference_step(cfg, max(2.0, 40.0 / max(1, args.steps)))
        vals.append(last["value"])
    el = time.perf_counter() - t0
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": desc, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": last["unit"], "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"]},
            "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _pair_timing(P, ctx, pair, steps, warmup, dev, stream, flush, rank_sync=False):
    """Timed steps of one pair through paco_lcs_boundaries (inputs resident,
    L2 flushed between steps): per-step CUDA-event times, the library's own
    event time of the kernel, the host time of each call, and the clocks."""
    import torch
    n, m = pair.a.size, pair.b.size
    da = torch.from_numpy(pair.a).to(dev)
    db = torch.from_numpy(pair.b).to(dev)
    row = torch.empty(m + 1, dtype=torch.int32, device=dev)
    col = torch.empty(n + 1, dtype=torch.int32, device=dev)
    L = torch.empty(1, dtype=torch.int32, device=dev)

    def step():
        P.paco_lcs_boundaries(ctx, da, db, bottom_row=row, right_col=col, length=L, stream=stream)

    h0 = time.perf_counter()
    step()  # the first call plans and sizes the context's scratch
    first_us = (time.perf_counter() - h0) * 1e6
    for _ in range(warmup - 1):
        step()
    ctx.sync()
    kernel_ms, step_ms, host_us = [], [], []
    if rank_sync:
        _barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index or 0) as clocks:
        for _ in range(steps):
            flush.fill_(1)  # evict the inputs from L2 between timed steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h0 = time.perf_counter()
            step()
            host_us.append((time.perf_counter() - h0) * 1e6)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            kernel_ms.append(P.paco_last_kernel_ms(ctx)[0])
        torch.cuda.synchronize()
    if rank_sync:
        _barrier()
    ctx.sync()
    return {"kernel_ms": kernel_ms, "step_ms": step_ms, "host_us": host_us, "first_us": first_us,
            "clocks": clocks.summary(), "L": L}


def _pair_model(plan, kmed, clk):
    """The critical-path model of the strip pipeline: every lane streams all S
    columns, and lane k starts skew x C columns after lane k-1 (skew 3
    chunks), at the column chain's latency."""
    sm_hz = (clk["sm_mhz"] if clk else 2070.0) * 1e6
    wpl = plan.get("words_per_lane", 1)
    lanes = (plan["L"] + 31 * wpl - 1) // (31 * wpl)
    cp_steps = plan["S"] + 3 * plan["chunk"] * lanes
    cp_ms = cp_steps * CHAIN_CYCLES_PER_COLUMN / sm_hz * 1e3
    return {"bound": "dependency chain", "model_ms": cp_ms, "measured_ms": kmed, "frac": cp_ms / kmed,
            "column_steps": cp_steps, "cycles_per_column": CHAIN_CYCLES_PER_COLUMN,
            "measured_cycles_per_column_step": kmed * 1e-3 * sm_hz / cp_steps,
            "note": "one lane streams all S columns; lanes trail by 3 chunks each"}


def pair_record(P, ctx, name, steps, warmup, dev, stream, flush, peak_ops, sms):
    """A nested record for another single-pair workload (the 4096 pair, the
    1048576 x 16384 pair): GCUPS, kernel and step times, launches per step,
    roofline fractions and its own clock record."""
    pair, desc = _workload(name)
    n, m = pair.a.size, pair.b.size
    t = _pair_timing(P, ctx, pair, steps, warmup, dev, stream, flush)
    cells = float(n) * m
    kmed = statistics.median(t["kernel_ms"])
    plan = P.paco_plan_pair(n, m, sms)
    word_steps = (plan["L"] + 30) // 31 * plan["S"]
    return {"value": cells * steps / (sum(t["step_ms"]) * 1e-3) / 1e9, "unit": "GCUPS", "steps": steps,
            "warmup": warmup, "ms_per_step": sum(t["step_ms"]) / steps,
            "config": {"workload": desc, "n": n, "m": m, "chunk": plan["chunk"], "warps_per_cta": plan["warps"],
                       "strips": plan["nstrips"], "words_per_lane": plan.get("words_per_lane", 1),
                       "l2": "flushed between timed steps (512 MiB write)"},
            "kernel_ms_median": kmed, "kernel_ms_min": min(t["kernel_ms"]),
            "host_call_us_median": statistics.median(t["host_us"]), "host_first_call_us": t["first_us"],
            "gpu_launches_per_step": 1,
            "roofline": {"bound": "alu", "frac": cells * CELL_OPS / (kmed * 1e-3) / peak_ops,
                         "achieved": cells * CELL_OPS / (kmed * 1e-3) / 1e12, "peak": peak_ops / 1e12,
                         "unit": "Tops/s (int32 lane-ops, 4 per cell)", "kernel": "k_pair_bp"},
            "roofline_bitparallel": {"frac": word_steps * OPS_PER_WORD_STEP / (kmed * 1e-3) / peak_ops},
            "critical_path": _pair_model(plan, kmed, t["clocks"]),
            "clocks": t["clocks"]}


def run_gpu(args):
    import torch
    import paper_2011_01441_gb300 as P

    ws, rank, local = _dist()
    _init_dist(ws, local)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P.load()
    ctx = P.Context(local)
    pair, desc = _workload(args.config)
    n, m = pair.a.size, pair.b.size
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    t = _pair_timing(P, ctx, pair, args.steps, args.warmup, dev, stream, flush, rank_sync=True)
    kernel_ms, step_ms, host_us, clk = t["kernel_ms"], t["step_ms"], t["host_us"], t["clocks"]
    tot_ms = _max_over_ranks(sum(step_ms), dev)
    cells = float(n) * m
    value = weak_scaling_value(cells, ws, args.steps, tot_ms)

    # end to end through the host-buffer entry point (pinned host memory)
    ha = torch.from_numpy(pair.a).pin_memory()
    hb = torch.from_numpy(pair.b).pin_memory()
    hrow = torch.empty(m + 1, dtype=torch.int32).pin_memory()
    hcol = torch.empty(n + 1, dtype=torch.int32).pin_memory()
    hlen = torch.empty(1, dtype=torch.int32)
    import ctypes
    vp = lambda x: ctypes.c_void_p(x.data_ptr())
    P.paco_lcs_boundaries_host_ptr(ctx, vp(ha), n, vp(hb), m, vp(hrow), vp(hcol), vp(hlen))
    e2e_t = []
    for _ in range(max(3, args.steps)):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P.paco_lcs_boundaries_host_ptr(ctx, vp(ha), n, vp(hb), m, vp(hrow), vp(hcol), vp(hlen))
        e2e_t.append(time.perf_counter() - t0)
    e2e_val = cells / statistics.median(e2e_t) / 1e9
    assert int(hlen.item()) == int(t["L"].item())

    # roofline of the dominant kernel: measured integer-ALU issue rate
    peak_ops = P.paco_measure_int_peak(ctx, 0)
    kmed = statistics.median(kernel_ms)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    plan = P.paco_plan_pair(n, m, sms)
    word_steps = (plan["L"] + 30) // 31 * plan["S"]
    achieved_bp = word_steps * OPS_PER_WORD_STEP / (kmed * 1e-3)
    achieved = cells * CELL_OPS / (kmed * 1e-3)
    peaks = _peaks()
    traffic = _profiled_traffic("k_pair_bp_pair131072_launches.md", ["pair_kernels.cu", "bp_device.cuh"]) \
        if args.config == "mutated" else None
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": desc, "n": n, "m": m, "engine": "bit-parallel strip pipeline, one launch",
                   "chunk": plan["chunk"], "warps_per_cta": plan["warps"], "strips": plan["nstrips"],
                   "words_per_lane": plan.get("words_per_lane", 1),
                   "l2": "flushed between timed steps (512 MiB write)"},
        "kernel_ms_median": kmed,
        "kernel_ms_min": min(kernel_ms),
        "host_call_us_median": statistics.median(host_us),
        "host_first_call_us": t["first_us"],
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                     "unit": "Tops/s (int32 lane-ops, 4 per cell)", "frac": achieved / peak_ops,
                     "traffic": traffic, "kernel": "k_pair_bp", "ops_per_cell": CELL_OPS,
                     "peak_source": "measured: paco_measure_int_peak(op=0), full-rate IADD3 on all SMs "
                                    "(152 SMs x 128 lanes x clock), this run"},
        "roofline_bitparallel": {"ops_per_cell": OPS_PER_WORD_STEP / 31, "achieved": achieved_bp / 1e12,
                                 "frac": achieved_bp / peak_ops,
                                 "note": "lane-ops the bit-parallel recurrence itself needs (4 per 31-row word "
                                         "and column) over the same peak"},
        "critical_path": _pair_model(plan, kmed, clk),
        "e2e": {"value": e2e_val, "unit": "GCUPS", "h2d_bytes_per_step": n + m,
                "d2h_bytes_per_step": 4 * (n + 1) + 4 * (m + 1) + 4},
        "gpu_launches": args.steps,  # k_pair_bp: the whole step is one launch
        "clocks": clk,
        "hbm_peak_gbs_measured": peaks.get("hbm_gbs"),
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_pair(pair.a, pair.b)
    if ws == 1 and args.config == "mutated" and not args.headline_only:
        # the other workloads of the metric, each with its own clock record
        line["small"] = pair_record(P, ctx, "small", DEFAULT_STEPS["small"], args.warmup, dev, stream, flush,
                                    peak_ops, sms)
        line["skinny"] = pair_record(P, ctx, "skinny", 100, args.warmup, dev, stream, flush, peak_ops, sms)
        ctx.close()
        del flush
        torch.cuda.empty_cache()
        line["batch"] = batch_record(200, max(3, args.warmup))
        line["served"] = served_record(100000)
    else:
        ctx.close()
    print(json.dumps(line), flush=True)


def _chunks_by_class(packed):
    """Chunk width per size class of the streamed side, as the batch ran."""
    names = ("S<256", "S<1024", "S<4096", "S>=4096")
    return {nm: (int(packed) >> (4 * k)) & 15 for k, nm in enumerate(names)}


def batch_record(steps, warmup, plain=True):
    """The 4096-pair batch through paco_lcs_batch (one graph replay per step),
    against the single-pair path called once per pair.  Returns the record."""
    import torch
    import paper_2011_01441_gb300 as P
    P.load()
    ctx = P.Context(0)
    bt = W.batch_pairs()
    ctx.set_option(P.OPT_ALPHABET, 4)  # the workload's symbols are 0..3
    da = torch.from_numpy(bt.a_cat).cuda()
    db = torch.from_numpy(bt.b_cat).cuda()
    L = torch.empty(bt.npairs, dtype=torch.int32, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    h0 = time.perf_counter()  # the first call plans, autotunes the chunk widths and captures the graph
    P.paco_lcs_batch(ctx, da, db, bt.a_off, bt.b_off, lengths=L)
    ctx.sync()
    first_ms = (time.perf_counter() - h0) * 1e3
    for _ in range(max(0, warmup - 1)):
        P.paco_lcs_batch(ctx, da, db, bt.a_off, bt.b_off, lengths=L)
    ctx.sync()
    ms = []
    with ClockSampler(0) as clocks:
        for _ in range(steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            P.paco_lcs_batch(ctx, da, db, bt.a_off, bt.b_off, lengths=L)
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
    ctx.sync()
    cells = bt.cells()
    value = cells * steps / (sum(ms) * 1e-3) / 1e9
    # plain: one pair per launch on one stream, same pairs
    plain_rec = None
    if plain:
        lens = torch.empty(1, dtype=torch.int32, device="cuda")
        views = [(da[bt.a_off[k]:bt.a_off[k + 1]], db[bt.b_off[k]:bt.b_off[k + 1]]) for k in range(bt.npairs)]
        for a, b in views[:64]:
            P.paco_lcs_length(ctx, a, b, out=lens)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for a, b in views:
            P.paco_lcs_length(ctx, a, b, out=lens)
        torch.cuda.synchronize()
        plain_s = time.perf_counter() - t0
        plain_rec = {"value": cells / plain_s / 1e9, "unit": "GCUPS", "seconds": plain_s,
                     "method": "paco_lcs_length once per pair on one stream (one launch each)"}
    peak_ops = P.paco_measure_int_peak(ctx, 0)
    med = statistics.median(ms)
    word_steps = sum(((max(n, m) + 30) // 31) * min(n, m) for n, m in zip(np.diff(bt.a_off), np.diff(bt.b_off)))
    achieved_bp = word_steps * OPS_PER_WORD_STEP / (med * 1e-3)
    achieved = cells * CELL_OPS / (med * 1e-3)
    rec = {"value": value, "unit": "GCUPS", "steps": steps, "warmup": warmup, "ms_per_step": sum(ms) / steps,
           "config": {"workload": bt.name + " (seed 4)", "pairs": bt.npairs, "cells": cells,
                      "engine": "batch graph, warp jobs", "alphabet": 4,
                      "chunk_by_class": _chunks_by_class(ctx.get_option(P.OPT_BATCH_CHUNKS)),
                      "l2": "flushed between timed steps"},
           "step_ms_median": med, "step_ms_min": min(ms), "first_call_host_ms": first_ms,
           "plain_one_pair_per_launch": plain_rec,
           "batch_over_plain": (value / plain_rec["value"]) if plain_rec else None,
           "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                        "unit": "Tops/s (int32 lane-ops, 4 per cell)", "frac": achieved / peak_ops,
                        "traffic": _profiled_traffic("k_batch_batch4096_full.md", ["batch.cu", "bp_device.cuh"]),
                        "duration": "whole step (column offsets + k_batch + prefixes), an upper bound on k_batch",
                        "kernel": "k_batch", "ops_per_cell": CELL_OPS,
                        "peak_source": "measured: paco_measure_int_peak(op=0), full-rate IADD3 on all SMs"},
           "roofline_bitparallel": {"ops_per_cell": OPS_PER_WORD_STEP / 31, "achieved": achieved_bp / 1e12,
                                    "frac": achieved_bp / peak_ops,
                                    "note": "the lane-ops the bit-parallel step needs (4 per 31-row word and "
                                            "column) over the same peak"},
           "clocks": clocks.summary()}
    ctx.close()
    return rec


def run_batch_bench(args):
    rec = batch_record(args.steps, args.warmup, plain=not args.no_plain)
    line = {"metric": METRIC, "value": rec["value"], "unit": "GCUPS", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic"}
    line.update({k: v for k, v in rec.items() if k not in line})
    print(json.dumps(line), flush=True)


def _serve_run(P, ctx, st, arr, cells, window=4096):
    """Submit the stream at its arrival times (every arrived request in one
    paco_lcs_submit_many call) from a thread, poll completions, and return
    per-request completion times (s from the start) and the wall time."""
    import threading as th
    nreq = st.npairs
    tickets = np.zeros(nreq, dtype=np.uint64)
    done_t = np.full(nreq, np.nan)
    submitted = [0]
    t_start = time.perf_counter()

    def submitter():
        k = 0
        while k < nreq:
            now = time.perf_counter() - t_start
            j = int(np.searchsorted(arr, now, side="right"))
            if j <= k:
                time.sleep(max(0.0, min(arr[k] - now, 0.0005)))
                continue
            got = P.paco_lcs_submit_many(ctx, st.a_cat, st.a_off[k:j + 1], st.b_cat, st.b_off[k:j + 1],
                                         partial=True)
            tickets[k:k + got.size] = got
            k += got.size
            submitted[0] = k
            if got.size < j - (k - got.size):
                time.sleep(0.0002)  # the engine's queue or host arena is full: retry shortly
    thr = th.Thread(target=submitter)
    thr.start()
    lo = 0  # every request before lo is done
    while lo < nreq:
        hi = min(submitted[0], lo + window)
        if hi > lo:
            idx = np.arange(lo, hi)
            idx = idx[np.isnan(done_t[lo:hi])]
            if idx.size:
                status, _ = P.paco_lcs_poll_many(ctx, tickets[idx])
                fin = idx[status != P.PACO_PENDING]
                if fin.size:
                    done_t[fin] = time.perf_counter() - t_start
            while lo < hi and not np.isnan(done_t[lo]):
                lo += 1
        time.sleep(0.0003)
    thr.join()
    return done_t, float(np.nanmax(done_t) - arr[0])


def served_record(nreq=100000, plain_prefix=5000, fracs=(0.5, 0.9, 1.0)):
    """The serving stream through paco_lcs_submit_many / paco_lcs_poll_many at
    fractions of the saturating rate (the batch path's rate on the same mix):
    GCUPS, p50/p99 latency and host time per micro-batch; the plain path (one
    pair per launch through the host-buffer entry point, FIFO) really served
    on the first `plain_prefix` requests at 0.9 of the saturating rate."""
    import torch
    import paper_2011_01441_gb300 as P
    P.load()
    t0 = time.perf_counter()
    st = W.serve_stream(nreq, workers=min(16, os.cpu_count() or 1))
    gen_s = time.perf_counter() - t0
    cells = (np.diff(st.a_off) * np.diff(st.b_off)).astype(np.float64)
    ctx = P.Context(0, mem_budget_bytes=8 << 30)
    ctx.set_option(P.OPT_ALPHABET, 20)  # the serving mix uses symbols 0..19
    # saturating rate: the batch path on the whole mix (autotuned once)
    da, db = torch.from_numpy(st.a_cat).cuda(), torch.from_numpy(st.b_cat).cuda()
    P.paco_lcs_batch(ctx, da, db, st.a_off, st.b_off)
    ctx.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(); P.paco_lcs_batch(ctx, da, db, st.a_off, st.b_off); e1.record(); e1.synchronize()
    sat_gcups = cells.sum() / (e0.elapsed_time(e1) * 1e-3) / 1e9
    tuned = ctx.get_option(P.OPT_BATCH_CHUNKS)
    ctx.set_option(P.OPT_SERVE_CHUNKS, tuned)  # the micro-batches use the batch autotuner's widths
    del da, db
    torch.cuda.empty_cache()
    lam_sat = sat_gcups * 1e9 / cells.mean()
    # warm-up (not recorded): the first requests of the stream through the
    # engine, so its streams, pools and buffers exist before the timed runs
    k_w = min(3000, nreq)
    wst = W.Batch(st.a_cat, st.a_off[:k_w + 1], st.b_cat, st.b_off[:k_w + 1], "warm-up")
    _serve_run(P, ctx, wst, W.poisson_arrivals(8, k_w, 0.5 * lam_sat), cells[:k_w])
    results = {}
    for frac in fracs:
        lam = frac * lam_sat
        arr = W.poisson_arrivals(7, nreq, lam)
        s0 = P.paco_serve_get_stats(ctx)
        with ClockSampler(0) as clocks:
            done_t, wall = _serve_run(P, ctx, st, arr, cells)
        s1 = P.paco_serve_get_stats(ctx)
        lat = done_t - arr
        nb = max(1, s1["batches_launched"] - s0["batches_launched"])
        results[f"{frac:.1f}"] = {
            "rate_per_s": lam, "requests": nreq, "gcups": cells.sum() / wall / 1e9, "wall_s": wall,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "micro_batches": nb,
            "host_launch_us_per_batch": (s1["host_launch_ns"] - s0["host_launch_ns"]) / nb / 1e3,
            "host_complete_us_per_batch": (s1["host_complete_ns"] - s0["host_complete_ns"]) / nb / 1e3,
            "host_stage_us_per_batch": (s1["host_stage_ns"] - s0["host_stage_ns"]) / nb / 1e3,
            "host_batch_us_per_batch": (s1["host_batch_ns"] - s0["host_batch_ns"]) / nb / 1e3,
            "clocks": clocks.summary()}
    # plain: FIFO, one pair per launch through the host-buffer entry point, same arrivals at 0.9
    k_plain = min(plain_prefix, nreq)
    arr = W.poisson_arrivals(7, nreq, 0.9 * lam_sat)[:k_plain]
    fin_t = np.zeros(k_plain)
    t_start = time.perf_counter()
    for k in range(k_plain):
        now = time.perf_counter() - t_start
        if arr[k] > now:
            time.sleep(arr[k] - now)
        a = st.a_cat[st.a_off[k]:st.a_off[k + 1]]
        b = st.b_cat[st.b_off[k]:st.b_off[k + 1]]
        P.paco_lcs_boundaries_host(ctx, a, b, want_rows=False, want_cols=False)
        fin_t[k] = time.perf_counter() - t_start
    lat_plain = fin_t - arr
    plain_wall = fin_t[-1] - arr[0]
    ctx.close()
    return {"value": results[f"{fracs[-1]:.1f}"]["gcups"], "unit": "GCUPS",
            "config": {"workload": st.name, "requests": nreq, "budget_bytes": 8 << 30,
                       "saturating_rate_per_s": lam_sat, "batch_gcups_on_mix": sat_gcups,
                       "serve_chunks_by_class": _chunks_by_class(tuned), "stream_generation_s": gen_s},
            "served": results,
            "served_over_batch_at_1.0": results.get("1.0", {}).get("gcups", float("nan")) / sat_gcups,
            "plain_fifo_one_pair_per_launch_at_0.9": {
                "measured": "real: the first %d requests of the same arrival schedule, served one at a time "
                            "(paco_lcs_boundaries_host: copy in, one launch, copy out)" % k_plain,
                "requests": k_plain, "gcups": cells[:k_plain].sum() / plain_wall / 1e9,
                "p50_ms": float(np.percentile(lat_plain, 50) * 1e3),
                "p99_ms": float(np.percentile(lat_plain, 99) * 1e3)}}


def run_serve_bench(args):
    rec = served_record(args.requests)
    line = {"metric": METRIC, "value": rec["value"], "unit": "GCUPS", "n_gpus": 1, "steps": 1, "warmup": 0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic"}
    line.update({k: v for k, v in rec.items() if k not in line})
    print(json.dumps(line), flush=True)


def run_recover_bench(args):
    """One longest common subsequence of the 131072-square mutated pair
    (Hirschberg levels on the batch engine): time per recovery, reported as
    n*m / time beside the pair path's length-only figure."""
    import torch
    import paper_2011_01441_gb300 as P
    P.load()
    ctx = P.Context(0)
    pair = W.single_mutated()
    da, db = torch.from_numpy(pair.a).cuda(), torch.from_numpy(pair.b).cuda()
    for _ in range(max(1, args.warmup)):
        ai, bj = P.paco_lcs_subsequence(ctx, da, db)
    torch.cuda.synchronize()
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        ai, bj = P.paco_lcs_subsequence(ctx, da, db)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    L = int(P.paco_lcs_length(ctx, da, db).item())
    a_np, b_np = ai.cpu().numpy(), bj.cpu().numpy()
    valid = (a_np.size == L and bool(np.all(np.diff(a_np) > 0)) and bool(np.all(np.diff(b_np) > 0))
             and bool(np.array_equal(pair.a[a_np], pair.b[b_np])))
    med = statistics.median(ts)
    cells = float(pair.a.size) * pair.b.size
    line = {"metric": METRIC, "value": cells / med / 1e9, "unit": "GCUPS (n*m per recovery)", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": med * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "LCS recovery, pair 131072x131072 sigma=20 mutated (seed 2)",
                       "method": "Hirschberg levels, each one batch launch", "L": L, "valid": valid}}
    print(json.dumps(line), flush=True)
    ctx.close()


def cpu_baseline_affine(a, b, scores, budget_s=12.0):
    """The affine oracle as it stands, single thread, on the first rows of the
    same pair (a bounded sample), extrapolated to GCUPS."""
    import oracle
    oracle.build()
    probe = min(a.size, 256)
    t = time.perf_counter()
    oracle.affine(a[:probe], b, *scores)
    dt = max(time.perf_counter() - t, 1e-6)
    rows = int(min(a.size, max(probe, probe * budget_s / dt)))
    t = time.perf_counter()
    oracle.affine(a[:rows], b, *scores)
    dt = time.perf_counter() - t
    return {"value": rows * b.size / dt / 1e9, "unit": "GCUPS", "cores": 1, "kind": "oracle",
            "sample": f"first {rows} rows x all {b.size} columns of the same pair ({rows * b.size:.3e} cells, {dt:.1f} s)"}


def run_affine_bench(args):
    """Affine-gap alignment (include/paco_affine.h): the 131072-square mutated
    pair (config affine) or the 4096-pair batch (config affine_batch), scores
    match 2, mismatch 3, gap open 5, gap extend 2."""
    import ctypes
    import torch
    import paper_2011_01441_gb300 as P
    P.load()
    ctx = P.Context(0)
    batch = args.config == "affine_batch"
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    S = AFFINE_SCORES
    if batch:
        bt = W.batch_pairs()
        da = torch.from_numpy(bt.a_cat).cuda()
        db = torch.from_numpy(bt.b_cat).cuda()
        out = torch.empty(bt.npairs, dtype=torch.int32, device="cuda")
        cells = bt.cells()
        desc = "affine-gap alignment, " + bt.name + " (seed 4)"

        def step():
            P.paco_affine_batch(ctx, da, db, bt.a_off, bt.b_off, S, out=out)
    else:
        pair = W.single_mutated()
        n, m = pair.a.size, pair.b.size
        da = torch.from_numpy(pair.a).cuda()
        db = torch.from_numpy(pair.b).cuda()
        sc = torch.empty(1, dtype=torch.int32, device="cuda")
        row = torch.empty(m + 1, dtype=torch.int32, device="cuda")
        col = torch.empty(n + 1, dtype=torch.int32, device="cuda")
        cells = float(n) * m
        desc = "affine-gap alignment, pair 131072x131072 sigma=20, 10% subs + 2.5% ins + 2.5% del (seed 2)"

        def step():
            P.paco_affine_align(ctx, da, db, S, score=sc, bottom_row=row, right_col=col)
    for _ in range(args.warmup):
        step()
    ctx.sync()
    step_ms, kernel_ms = [], []
    with ClockSampler(0) as clocks:
        for _ in range(args.steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            step()
            e1.record()
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            kernel_ms.append(P.paco_last_kernel_ms(ctx)[0])
    ctx.sync()
    value = cells * args.steps / (sum(step_ms) * 1e-3) / 1e9
    peak_ops = P.paco_measure_int_peak(ctx, 0)
    kmed = statistics.median(kernel_ms)
    achieved = cells * AFFINE_CELL_OPS / (kmed * 1e-3)
    rows = ctx.get_option(P.OPT_AFFINE_ROWS) or 4
    line = {"metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sum(step_ms) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": desc, "cells": cells, "scores": dict(zip(("match", "mismatch", "gap_open",
                                                                             "gap_extend"), S)),
                       "engine": f"row bands of 32 lanes x {rows} rows, tagged hand-off words",
                       "l2": "flushed between timed steps (512 MiB write)"},
            "kernel_ms_median": kmed, "kernel_ms_min": min(kernel_ms),
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                         "unit": f"Tops/s (int32 lane-ops, {AFFINE_CELL_OPS} per cell)", "frac": achieved / peak_ops,
                         "traffic": _profiled_traffic("k_affine_batch4096_full.md" if batch else "k_affine_pair131072_launches.md",
                                                      ["affine.cu", "bp_device.cuh"]),
                         "kernel": "k_affine", "ops_per_cell": AFFINE_CELL_OPS,
                         "peak_source": "measured: paco_measure_int_peak(op=0), full-rate IADD3 on all SMs"},
            "gpu_launches": args.steps,
            "clocks": clocks.summary()}
    if batch:
        line["config"]["pairs"] = bt.npairs
        if not args.no_cpu_baseline:
            import oracle
            oracle.build()
            cores = os.cpu_count() or 1
            k = min(bt.npairs, 4 * cores)
            while True:   # grow the sample of pairs until it takes ~10 s on all host cores
                t0 = time.perf_counter()
                oracle.affine_batch(bt.a_cat, bt.a_off[:k + 1], bt.b_cat, bt.b_off[:k + 1], S, threads=cores)
                dt = time.perf_counter() - t0
                if dt > 5.0 or k == bt.npairs:
                    break
                k = min(bt.npairs, int(k * max(2.0, 10.0 / max(dt, 1e-3))))
            ck = float(np.sum(np.diff(bt.a_off[:k + 1]) * np.diff(bt.b_off[:k + 1])))
            line["cpu_baseline"] = {"value": ck / dt / 1e9, "unit": "GCUPS", "cores": cores, "kind": "oracle",
                                    "sample": f"first {k} of {bt.npairs} pairs ({ck:.3e} cells, {dt:.1f} s)"}
    else:
        ha = torch.from_numpy(pair.a).pin_memory()
        hb = torch.from_numpy(pair.b).pin_memory()
        hrow = torch.empty(m + 1, dtype=torch.int32).pin_memory()
        hcol = torch.empty(n + 1, dtype=torch.int32).pin_memory()
        hs = ctypes.c_int32(0)
        vp = lambda t: ctypes.c_void_p(t.data_ptr())
        P.paco_affine_align_host_ptr(ctx, vp(ha), n, vp(hb), m, S, ctypes.byref(hs), vp(hrow), vp(hcol))
        e2e_t = []
        for _ in range(max(3, args.steps)):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            P.paco_affine_align_host_ptr(ctx, vp(ha), n, vp(hb), m, S, ctypes.byref(hs), vp(hrow), vp(hcol))
            e2e_t.append(time.perf_counter() - t0)
        assert hs.value == int(sc.item())
        line["e2e"] = {"value": cells / statistics.median(e2e_t) / 1e9, "unit": "GCUPS", "h2d_bytes_per_step": n + m,
                       "d2h_bytes_per_step": 4 * (n + 1) + 4 * (m + 1) + 4}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_affine(pair.a, pair.b, S)
    print(json.dumps(line), flush=True)
    ctx.close()


def run_lws_bench(args):
    """The 1D problem (include/paco_lws.h) for n = 131072, D[0] = 0, weight
    T = 40, seed 6: every term D[i] + w(i, j), i < j, is one cell."""
    import torch
    import paper_2011_01441_gb300 as P
    P.load()
    ctx = P.Context(0)
    n = LWS_N
    out = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        P.paco_lws(ctx, n, 0, LWS_T, LWS_SEED, out=out)
    ctx.sync()
    step_ms, kernel_ms = [], []
    with ClockSampler(0) as clocks:
        for _ in range(args.steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            P.paco_lws(ctx, n, 0, LWS_T, LWS_SEED, out=out)
            e1.record()
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            kernel_ms.append(P.paco_last_kernel_ms(ctx)[0])
    ctx.sync()
    cells = n * (n + 1) / 2
    value = cells * args.steps / (sum(step_ms) * 1e-3) / 1e9
    peak_ops = P.paco_measure_int_peak(ctx, 0)
    kmed = statistics.median(kernel_ms)
    achieved = cells * LWS_TERM_OPS / (kmed * 1e-3)
    line = {"metric": METRIC, "value": value, "unit": "GCUPS (terms D[i] + w(i, j) of Eq. 1D per second)",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(step_ms) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"1D problem (least weight subsequence), n={n}, D[0]=0, weight T={LWS_T} seed={LWS_SEED}",
                       "cells": cells, "engine": "blocks of 256: squares as jobs (atomicMin into running minima), triangles by warp sweeps, tagged words between blocks",
                       "l2": "flushed between timed steps (512 MiB write)"},
            "kernel_ms_median": kmed, "kernel_ms_min": min(kernel_ms),
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                         "unit": f"Tops/s (int32 lane-ops, {LWS_TERM_OPS} per term)", "frac": achieved / peak_ops,
                         "traffic": _profiled_traffic("k_lws_n131072_full.md", ["lws.cu", "bp_device.cuh"]),
                         "kernel": "k_lws", "ops_per_cell": LWS_TERM_OPS,
                         "peak_source": "measured: paco_measure_int_peak(op=0), full-rate IADD3 on all SMs"},
            "gpu_launches": args.steps,
            "clocks": clocks.summary()}
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        oracle.lws(8192, 0, 0, LWS_T, LWS_SEED)
        dt = max(time.perf_counter() - t0, 1e-6)
        m = int(min(n, 8192 * (10.0 / dt) ** 0.5))
        t0 = time.perf_counter()
        oracle.lws(m, 0, 0, LWS_T, LWS_SEED)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": m * (m + 1) / 2 / dt / 1e9, "unit": "GCUPS", "cores": 1, "kind": "oracle",
                                "sample": f"the first {m} outputs of the same problem ({m * (m + 1) / 2:.3e} terms, {dt:.1f} s)"}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_schedules_bench(args):
    """The paper's comparison on one GB300: the 131072-square mutated pair
    under the strip pipeline and under the PACO, PA and PO tile schedules
    (all on the same warp kernel), with each schedule's critical path from
    the planner in units of n*m/p."""
    import torch
    import paper_2011_01441_gb300 as P
    P.load()
    ctx = P.Context(0)
    pair = W.single_mutated()
    n, m = pair.a.size, pair.b.size
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    da, db = torch.from_numpy(pair.a).cuda(), torch.from_numpy(pair.b).cuda()
    L_ref = None
    rows = {}
    for name, kind, base in (("strips (PACO p-way rows)", 0, 0), ("PACO tiles", P.TILES_PACO, 4),
                             ("PACO tiles base 2", P.TILES_PACO, 2), ("PA p x p", P.TILES_PA, 4),
                             ("PO 2-way D&C", P.TILES_PO, 16)):
        ctx.set_option(P.OPT_TILES, kind)
        ctx.set_option(P.OPT_TILE_BASE, base)
        for _ in range(max(1, args.warmup)):
            L, _, _ = P.paco_lcs_boundaries(ctx, da, db)
        ctx.sync()
        ks = []
        for _ in range(args.steps):
            P.paco_lcs_boundaries(ctx, da, db)
            ctx.sync()
            ks.append(P.paco_last_kernel_ms(ctx)[0])
        Lv = int(L.item())
        L_ref = Lv if L_ref is None else L_ref
        crit = None
        if kind:
            t = P.paco_plan_tiles(n, m, sms, kind, base)
            crit = t["critical_cells"] / (n * m / sms)
            ntiles = len(t["tiles"])
        else:
            ntiles = P.paco_plan_pair(n, m, sms)["nstrips"]
        med = statistics.median(ks)
        rows[name] = {"kernel_ms": med, "gcups": n * m / (med * 1e-3) / 1e9, "tiles": ntiles,
                      "critical_path_nm_over_p": crit, "L_matches": Lv == L_ref}
    ctx.set_option(P.OPT_TILES, 0)
    ctx.set_option(P.OPT_TILE_BASE, 0)
    best = max(rows.values(), key=lambda r: r["gcups"])
    line = {"metric": METRIC, "value": best["gcups"], "unit": "GCUPS", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": "schedule comparison, pair 131072x131072 sigma=20 mutated (seed 2)", "p": sms},
            "schedules": rows}
    print(json.dumps(line), flush=True)
    ctx.close()


# Default timed steps per workload: about half a second of GPU work, so that
# the clock sampler sees several samples inside the timed region.
DEFAULT_STEPS = {"mutated": 200, "small": 2000, "skinny": 200, "batch": 1000, "affine": 20,
                 "affine_batch": 60, "lws": 60}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: about half a second of GPU work per workload; 10 for the reference arm)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="mutated", choices=["mutated", "small", "skinny", "batch", "serve", "recover", "schedules",
                                                               "affine", "affine_batch", "lws"])
    ap.add_argument("--requests", type=int, default=100000, help="serving: requests taken from the stream")
    ap.add_argument("--headline-only", action="store_true",
                    help="default workload: skip the nested small / skinny / batch / served records")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="batch: skip the one-pair-per-launch comparison")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 10 if args.impl == "reference" else DEFAULT_STEPS.get(args.config, 10)
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "batch":
        run_batch_bench(args)
    elif args.config == "serve":
        run_serve_bench(args)
    elif args.config == "recover":
        run_recover_bench(args)
    elif args.config == "schedules":
        run_schedules_bench(args)
    elif args.config in ("affine", "affine_batch"):
        run_affine_bench(args)
    elif args.config == "lws":
        run_lws_bench(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
