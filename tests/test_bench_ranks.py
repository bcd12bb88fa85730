"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

bench.py runs one replica of the workload per GPU; the job time is the
maximum over ranks and the job throughput counts every rank's units.  These
tests exercise that reduction and the reference arm's rank handling with
two CPU processes, without a GPU.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, times, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.rank_max(times[rank], world, "cpu")
        q.put((rank, t, bench.job_rate(1000, world, t)))
    finally:
        dist.destroy_process_group()


def test_rank_max_and_job_rate_two_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [12.5, 20.0]                  # ms per rank: rank 1 is the slow one
    ps = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == 20.0                  # every rank sees the slowest rank's time
        assert v == pytest.approx(2 * 1000 / 0.020)   # units of both ranks over that time


def test_job_rate_single_rank():
    import bench
    assert bench.rank_max(3.0, 1, "cpu") == 3.0
    assert bench.job_rate(500, 1, 250.0) == pytest.approx(2000.0)


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
