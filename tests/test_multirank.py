"""The multi-rank logic of bench.py on CPU: world_size 2 over gloo (127.0.0.1).
A single graph does not shard, so N GPUs run N replicas of it; the job value
is all ranks' units over the slowest rank's time, and the reference arm runs
on rank 0 alone.  Batched work shards by graph: contiguous, cost-balanced
graph ranges per rank, results gathered in graph order."""
import json
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


def test_reference_arm_rank_zero_prints_one_contract_line():
    """Rank 0 (or a single process) times the oracle on its bounded sample
    and prints exactly one JSON line carrying the keys the driver reads."""
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=env, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["n_gpus"] == 1 and line["steps"] == 1 and line["warmup"] == 1
    assert line["value"] > 0 and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = line["e2e"]
    assert (e2e["value"], e2e["unit"]) == (line["value"], line["unit"])
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


# ---- batched work sharded by graph (contiguous, cost-balanced ranges)

def _shard_worker(rank, ws, port, costs, out):
    import numpy as np
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2311_04333_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        lo, hi = shard.my_range(costs, rank, ws)
        # each rank's per-graph result rows: (graph index, cost, rank)
        rows = np.array([[g, costs[g], rank] for g in range(lo, hi)], dtype=np.int64).reshape(-1, 3)
        out[rank] = (lo, hi, shard.gather_rows(rows, ws).tolist())
    finally:
        dist.destroy_process_group()


def test_batch_shards_gathered_over_two_ranks():
    import numpy as np
    rng = np.random.default_rng(3)
    costs = [int(x) for x in rng.integers(1, 10_000, size=37)]
    ws = 2
    port = _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_shard_worker, args=(ws, port, costs, out), nprocs=ws, start_method="spawn", join=True)
    (lo0, hi0, rows0), (lo1, hi1, rows1) = out[0], out[1]
    assert (lo0, hi1) == (0, len(costs)) and hi0 == lo1          # disjoint, contiguous, complete
    assert rows0 == rows1                                        # every rank holds all results
    assert [r[0] for r in rows0] == list(range(len(costs)))     # in graph order
    assert [r[2] for r in rows0] == [0] * hi0 + [1] * (len(costs) - hi0)
    share = [sum(costs[lo0:hi0]), sum(costs[lo1:hi1])]
    assert abs(share[0] - sum(costs) / 2) <= max(costs)


def test_graph_ranges_balance_and_cover():
    import numpy as np
    sys.path.insert(0, ROOT)
    from paper_2311_04333_gb300 import shard
    rng = np.random.default_rng(4)
    for ws in (1, 2, 3, 4, 8):
        for G in (0, 1, 5, 64, 4096):
            costs = rng.integers(0, 1_000_000, size=G)
            rs = shard.graph_ranges(costs, ws)
            assert len(rs) == ws and rs[0][0] == 0 and rs[-1][1] == G
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            assert all(lo <= hi for lo, hi in rs)
            tot = int(costs.sum())
            cmax = int(costs.max()) if G else 0
            for lo, hi in rs:
                assert abs(int(costs[lo:hi].sum()) - tot / ws) <= cmax
    # one graph per rank when costs are equal and the count divides
    assert shard.graph_ranges([5] * 8, 4) == [(0, 2), (2, 4), (4, 6), (6, 8)]
    # the cost of a graph is its arcs plus its vertices
    assert shard.graph_cost(10, 20) == 50
