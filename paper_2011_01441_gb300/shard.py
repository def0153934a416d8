"""A batch of independent pairs over several GPUs, one process per GPU.

The pairs of a batch share nothing, so the multi-GPU form needs no exchange
of intermediate data: the native planner (paco_plan_shard in
include/paco_plan.h) assigns each pair to a rank by size-balanced greedy
assignment, every rank runs its own pairs (paco_lcs_batch on its GPU), and
one gather returns the lengths in the batch's order.  The gather is the only
collective; it carries 12 bytes per pair.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _check, load


def paco_plan_shard(a_off, b_off, ranks: int):
    """(owner int32[npairs], cells per rank int64[ranks]) from the native planner."""
    a_off = np.ascontiguousarray(a_off, dtype=np.int64)
    b_off = np.ascontiguousarray(b_off, dtype=np.int64)
    npairs = a_off.size - 1
    if b_off.size != a_off.size:
        raise ValueError("a_off and b_off must have the same length")
    owner = np.zeros(max(npairs, 1), dtype=np.int32)
    cells = np.zeros(max(int(ranks), 1), dtype=np.int64)
    vp = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    _check(load().paco_plan_shard(vp(a_off), vp(b_off), npairs, int(ranks), vp(owner), vp(cells)))
    return owner[:npairs], cells


def sub_batch(a_cat, a_off, b_cat, b_off, idx):
    """The pairs `idx` of a concatenated batch as a batch of their own."""
    a_off = np.asarray(a_off, dtype=np.int64)
    b_off = np.asarray(b_off, dtype=np.int64)
    la = a_off[idx + 1] - a_off[idx]
    lb = b_off[idx + 1] - b_off[idx]
    sa = np.zeros(idx.size + 1, dtype=np.int64)
    sb = np.zeros(idx.size + 1, dtype=np.int64)
    np.cumsum(la, out=sa[1:])
    np.cumsum(lb, out=sb[1:])
    ca = np.concatenate([a_cat[a_off[k]:a_off[k + 1]] for k in idx]) if idx.size else np.zeros(0, np.uint8)
    cb = np.concatenate([b_cat[b_off[k]:b_off[k + 1]] for k in idx]) if idx.size else np.zeros(0, np.uint8)
    return ca.astype(np.uint8), sa, cb.astype(np.uint8), sb


def run_sharded_batch(a_cat, a_off, b_cat, b_off, compute, group=None, device="cpu"):
    """Run this rank's share of the batch and gather every pair's length.

    `compute(a_cat, a_off, b_cat, b_off)` returns the int32 lengths of a
    (sub-)batch; on a GPU it is paco_lcs_batch on this rank's device.  All
    ranks must call this with the same batch.  `device` is where the gather
    tensors live (a CUDA device for NCCL, "cpu" for gloo).  Returns
    (lengths int32[npairs] in batch order, this rank's pair indices)."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    npairs = len(a_off) - 1
    owner, _ = paco_plan_shard(a_off, b_off, ws)
    mine = np.nonzero(owner == rank)[0].astype(np.int64)
    ca, sa, cb, sb = sub_batch(a_cat, a_off, b_cat, b_off, mine)
    lens = np.asarray(compute(ca, sa, cb, sb), dtype=np.int32).reshape(-1)[:mine.size]
    if ws == 1:
        out = np.zeros(npairs, dtype=np.int32)
        out[mine] = lens
        return out, mine
    counts = [int((owner == r).sum()) for r in range(ws)]
    width = max(counts) if counts else 0
    send = torch.full((width, 2), -1, dtype=torch.int64, device=device)
    if mine.size:
        send[:mine.size, 0] = torch.from_numpy(mine).to(device)
        send[:mine.size, 1] = torch.from_numpy(lens.astype(np.int64)).to(device)
    recv = [torch.empty_like(send) for _ in range(ws)]
    dist.all_gather(recv, send, group=group)
    out = np.zeros(npairs, dtype=np.int32)
    for r in range(ws):
        part = recv[r][:counts[r]].cpu().numpy()
        out[part[:, 0]] = part[:, 1].astype(np.int32)
    return out, mine


def batch_on_device(ctx, alphabet: int = 0):
    """The per-rank computation on GPUs: paco_lcs_batch of the rank's
    sub-batch on the context's device (strings copied in, lengths copied
    out).  `alphabet` > 0 declares the symbols' range (PACO_OPT_ALPHABET)."""
    from . import OPT_ALPHABET, paco_lcs_batch

    def compute(a_cat, a_off, b_cat, b_off):
        import torch
        if len(a_off) <= 1:
            return np.zeros(0, dtype=np.int32)
        if alphabet:
            ctx.set_option(OPT_ALPHABET, alphabet)
        dev = torch.device("cuda", ctx.device)
        da = torch.from_numpy(np.ascontiguousarray(a_cat)).to(dev)
        db = torch.from_numpy(np.ascontiguousarray(b_cat)).to(dev)
        with torch.cuda.device(dev):
            lens = paco_lcs_batch(ctx, da, db, a_off, b_off)
            ctx.sync()
        return lens.cpu().numpy()[:len(a_off) - 1]
    return compute
