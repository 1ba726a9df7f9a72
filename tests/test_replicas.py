"""The N > 1 path of bench.py on CPU: every rank advances its own grid
(replicas, no collective on the data path), the timed region's length is the
maximum over ranks, the reported value is the whole job's cell updates over
that time, and the reference arm runs on rank 0 only.  Two gloo ranks on
127.0.0.1 stand in for two GPUs."""
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


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) * 10 ms for its steps: the job's time is the slowest rank's
        t = bench.max_over_ranks(0.010 * (rank + 1), world, "cpu")
        out[rank] = (t, bench.whole_job_rate(1000, 50, t, world))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_two_gloo_ranks():
    world = 2
    out = mp.get_context("spawn").Manager().dict()  # no fork of this multi-threaded process
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        t, rate = out[r]
        assert t == pytest.approx(0.020)
        assert rate == pytest.approx(2 * 1000 * 50 / 0.020 / 1e9)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.5, 1, "cpu") == 0.5
    assert bench.whole_job_rate(100, 10, 2.0, 1) == pytest.approx(500 / 1e9)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm's other ranks exit 0 without work or
    output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "3",
                        "--warmup", "3"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
