"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

The path does not shard: N GPUs run N independent replicas of the same workload.  What the
ranks share is the reduction of the timings: every rank takes the slowest rank's time, and
the job rate is the units of all ranks over that time.  The reference leg runs on rank 0
only; the other ranks exit at once.
"""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t = 0.5 + 0.25 * rank                      # rank 1 is the slow one
    t_max = bench.max_over_ranks(t, ws, "cpu")
    q.put((rank, t_max, bench.whole_job_rate(1000.0, t_max, ws)))
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
        assert p.exitcode == 0
    for rank, t_max, rate in out:
        assert t_max == pytest.approx(0.75)
        assert rate == pytest.approx(2 * 1000.0 / 0.75)


def test_one_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.3, 1) == 0.3
    assert bench.whole_job_rate(10.0, 2.0, 1) == 5.0


def test_reference_leg_runs_on_rank_zero_only():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
