"""The benchmark's multi-rank path on CPU: two gloo ranks (127.0.0.1) exercise the barrier,
the max-over-ranks timing reduction and the weak-scaling aggregate, and a non-zero rank of
the reference arm exits quietly."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    r, ws, dist = bench._dist("gloo")
    bench._barrier(dist)
    ms = 10.0 + 5.0 * r  # rank 1 is the slow one
    ms_max = bench._max_over_ranks(ms, dist)
    value = bench.weak_scaling_value(ws, 1000.0, ms_max / 1e3)
    bench._barrier(dist)
    dist.destroy_process_group()
    q.put((r, ws, ms_max, value))


def test_two_gloo_ranks_max_timing_and_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for _, ws, ms_max, value in res:
        assert ws == 2 and ms_max == 15.0
        # 2 ranks x 1000 units in 15 ms = 0.1333 M units/s
        assert value == pytest.approx(2 * 1000.0 / 0.015 / 1e6)


def test_reference_arm_non_zero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
