"""The bench's multi-rank path on CPU: world_size 2 over gloo.  Each rank times
its own replica; the job's step time is the slowest rank's and the job rate
counts every rank's sweeps.  The reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(1.0 + 2.0 * rank, world, "cpu")     # rank 0: 1 ms, rank 1: 3 ms
    out[rank] = (ms, bench.job_rate(world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_step_time_is_the_slowest_rank_and_rate_counts_all_ranks():
    world, port = 2, _free_port()
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == 3.0 and out[1][0] == 3.0
    assert out[0][1] == pytest.approx(2 * 1e3 / 3.0)


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1, "cpu") == 2.5
    assert bench.job_rate(1, 2.5) == pytest.approx(400.0)


def test_reference_arm_runs_on_rank_0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
