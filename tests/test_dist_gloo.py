"""The multi-rank host logic of bench.py on CPU: two gloo ranks (world size
2) join the group, time-reduce to the slowest rank, and compute the
whole-job weak-scaling value from the same per-rank workload; a non-zero
rank of the reference arm exits without work or output."""
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    try:
        import bench
        from paper_2011_01441_gb300 import workloads as W
        got_ws, got_rank, _ = bench._dist()
        bench._init_dist(got_ws, got_rank, backend="gloo")
        bench._barrier()
        local_ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
        max_ms = bench._max_over_ranks(local_ms)
        pair = W.single_small()
        digest = int(np.frombuffer(pair.a.tobytes() + pair.b.tobytes(), dtype=np.uint8).astype(np.uint64).sum())
        value = bench.weak_scaling_value(float(pair.a.size) * pair.b.size, got_ws, 4, max_ms)
        bench._barrier()
        import torch.distributed as dist
        dist.destroy_process_group()
        q.put((rank, got_ws, max_ms, digest, value, None))
    except Exception as e:  # reported to the parent
        q.put((rank, None, None, None, None, repr(e)))


def test_two_gloo_ranks_reduce_to_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, ws, max_ms, digest, value, err in res:
        assert err is None, err
        assert ws == 2
        assert max_ms == 15.0           # the slowest rank's time on every rank
    assert res[0][3] == res[1][3]       # every rank processes the same workload (weak scaling)
    cells = 4096.0 * 4096.0
    assert res[0][4] == pytest.approx(cells * 2 * 4 / 15e-3 / 1e9)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env,
                       timeout=120, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_single_rank_helpers_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(3.5) == 3.5
    bench._barrier()
    assert bench.weak_scaling_value(1e9, 1, 2, 1000.0) == pytest.approx(2.0)
