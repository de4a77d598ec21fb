"""The multi-rank logic of bench.py on CPU: world_size 2 over gloo (127.0.0.1).
The path does not shard, so N GPUs run N replicas; the job value is all
ranks' units over the slowest rank's time, and the reference arm runs on
rank 0 alone."""
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


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        # rank r processed 100 (r + 1) units in 2 (r + 1) seconds
        v = bench.replica_throughput(100.0 * (rank + 1), 2.0 * (rank + 1), ws)
        mx = bench._max_over_ranks(float(rank), ws)
        bench._barrier(ws)
        out[rank] = (v, mx)
    finally:
        dist.destroy_process_group()


def test_replica_throughput_two_ranks():
    ws = 2
    port = _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_worker, args=(ws, port, out), nprocs=ws, start_method="spawn", join=True)
    # (100 + 200) units over the slowest rank's 4 s, on every rank
    assert out[0] == out[1] == (75.0, 1.0)


def test_single_rank_is_plain_ratio():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_throughput(300.0, 4.0, 1) == 75.0


@pytest.mark.parametrize("rank", ["1"])
def test_reference_arm_other_ranks_exit_without_work(rank):
    env = dict(os.environ, RANK=rank, WORLD_SIZE="2", LOCAL_RANK=rank)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
