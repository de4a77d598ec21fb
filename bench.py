"""Benchmark: GTEPS per PaRSorting++ iteration on R-MAT scale 27 (+ 10 planted
G(s, 1/2) blocks, s = 200..2000), T = 20 iterations per step, one GB300.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

A step is one dsg_run of T iterations (all of: load sort, edge scan, fused
densest-suffix scan, best-set materialisation) on the graph resident in HBM.
value = m * T * K * N / (max over ranks of the timed region) / 1e9 (GTEPS).
e2e   = the same metric through the C ABI with host buffers: each step
        uploads the CSR from pinned host memory, runs, and reads back the
        loads and the best set.
The line also carries the batched form (4,096 small graphs in one persistent
launch against one dsg_run per graph) and serving (Poisson arrivals through
the native request loop: p50/p99 latency and throughput).
Multi-GPU: a single graph does not shard (replicas only): each rank runs its
own replica of the headline workload and value aggregates the replicas.  The
batched form shards by graph: each rank runs a contiguous, cost-balanced
range of the 4,096 graphs and the per-graph results are gathered.
--impl reference times the CPU oracle (the only reference this build has)
on a bounded sample of the workload (same recipe at a smaller scale).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SCALE = 27
EDGE_FACTOR = 16
SEED = 3
BLOCKS = [200 * (i + 1) for i in range(10)]
T_ITERS = 20
SAMPLE_SCALE = 21          # CPU baseline sample: same recipe, smaller scale
METRIC = "GTEPS per Greedy++ iteration (HBM roofline %); batched graphs/s vs one-per-launch"
BATCH_G = 4096
BATCH_SEED = 4
BATCH_T = 32
BATCH_T_PEEL = 16
SERVE_POOL = 48        # request graphs of the serving workload
SERVE_SEED = 5
SERVE_SLOTS = 4
SERVE_RATE = 200.0     # Poisson arrival rate of the serving workload, req/s
UNIT = "GTEPS"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def replica_throughput(units_local: float, seconds_local: float, ws: int) -> float:
    """Whole-job throughput of ws independent replicas: the units all ranks
    processed over the slowest rank's time (every rank gets the same value)."""
    return _sum_over_ranks(units_local, ws) / _max_over_ranks(seconds_local, ws)


def _barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peak_hbm() -> tuple[float, str]:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current source of the kernel's file (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel]
        src = os.path.join(ROOT, rec["source"])
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if sha != rec["source_sha"] or rec.get("workload") != workload:
            return None
        return rec["dram_bytes_per_launch"]
    except (OSError, KeyError, ValueError):
        return None


def cpu_baseline(budget_s: float = 20.0) -> dict:
    """The oracle as it stands (sequential C, one core) on a bounded sample:
    the same R-MAT recipe at scale SAMPLE_SCALE, PaRSorting++ iterations until
    about budget_s seconds have been spent."""
    import graphgen as gg
    import oracle as orc
    g = gg.rmat(SAMPLE_SCALE, EDGE_FACTOR, SEED)
    t0 = time.perf_counter()
    r = orc.run(g, orc.SORTING, 1)
    one = time.perf_counter() - t0
    T = max(1, min(T_ITERS, int(budget_s / max(one, 1e-3))))
    t0 = time.perf_counter()
    r = orc.run(g, orc.SORTING, T)
    dt = time.perf_counter() - t0
    return {"value": g.m * T / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"R-MAT scale {SAMPLE_SCALE} (same recipe, no planted blocks), n={g.n}, "
                      f"m={g.m}, PaRSorting++ T={T}, {dt:.1f} s, sequential C oracle"}


def cpu_parallel_baseline(T: int = 10, reps: int = 3) -> dict:
    """A separately written OpenMP PaRSorting++ (exact, parity-tested
    against the oracle) on all host cores, on the same bounded sample; the
    fastest of a few runs, since one run is well under a second."""
    import cpu_baseline as cb
    import graphgen as gg
    g = gg.rmat(SAMPLE_SCALE, EDGE_FACTOR, SEED)
    nt = cb.threads()
    cb.run(g, 1, nt)
    dts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        cb.run(g, T, nt)
        dts.append(time.perf_counter() - t0)
    dt = min(dts)
    return {"value": g.m * T / dt / 1e9, "unit": UNIT, "cores": nt, "kind": "openmp",
            "sample": f"R-MAT scale {SAMPLE_SCALE}, n={g.n}, m={g.m}, PaRSorting++ T={T}, "
                      f"fastest of {reps} runs: {dt:.2f} s (slowest {max(dts):.2f} s)"}


def bench_batch(dsg, ctx, graphs, args, ws: int = 1, rank: int = 0) -> dict:
    """Graphs/s of the batched launch (autotuned block size) against one
    dsg_run per graph on the same GPU, with identical per-graph results.
    With N ranks the batch is sharded by graph: rank r runs its contiguous,
    cost-balanced range (shard.graph_ranges), the job's graphs/s is all G
    graphs over the slowest rank's time, and the per-graph results are
    gathered on every rank (no collective on the data path)."""
    import numpy as np
    import torch
    from paper_2311_04333_gb300 import shard, tune
    G = len(graphs)
    lo, hi = shard.my_range([shard.graph_cost(g.n, g.m) for g in graphs], rank, ws)
    mine = graphs[lo:hi]
    Gl = len(mine)
    T = np.full(Gl, BATCH_T, np.int32)
    b = dsg.dsg_upload_batch(ctx, [(g.n, g.off, g.adj) for g in mine], 0)
    Gb, N, M = dsg.dsg_batch_info(b)
    rec = tune.tune_batch(ctx, b, T, force=True)
    th = rec["threads"]
    best_b = np.zeros(4 * Gl, np.int64)
    dsg.dsg_run_batch(ctx, b, dsg.DSG_SORTING, T, th, best_b)
    torch.cuda.synchronize()
    _barrier(ws)
    t0 = time.perf_counter()
    for _ in range(args.batch_steps):
        dsg.dsg_run_batch(ctx, b, dsg.DSG_SORTING, T, th, best_b)
    tb = _max_over_ranks((time.perf_counter() - t0) / args.batch_steps, ws)
    dsg.dsg_free_batch(b)
    # one graph per launch (graphs resident, outputs: the best triple)
    hs = [dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj, 0) for g in mine]
    best_1 = np.zeros((Gl, 4), np.int64)
    dsg.dsg_run(ctx, hs[0], dsg.DSG_SORTING, BATCH_T)
    torch.cuda.synchronize()
    _barrier(ws)
    t0 = time.perf_counter()
    for i, h in enumerate(hs):
        r = dsg.dsg_run(ctx, h, dsg.DSG_SORTING, BATCH_T)
        best_1[i] = (r["best_edges"], r["best_vertices"], r["best_iter"], r["best_set_size"])
    t1 = _max_over_ranks(time.perf_counter() - t0, ws)
    for h in hs:
        dsg.dsg_free_graph(h)
    all_b = shard.gather_rows(best_b.reshape(Gl, 4), ws)
    all_1 = shard.gather_rows(best_1, ws)
    same = bool(all_b.shape == (G, 4) and np.array_equal(all_b, all_1))
    Mtot = int(_sum_over_ranks(float(M), ws))
    Ntot = int(_sum_over_ranks(float(N), ws))
    out = {"workload": f"{G} graphs, n log-uniform in [50, 50000] (ER / R-MAT / planted clique), "
                       f"N={Ntot}, M={Mtot}, PaRSorting++ T={BATCH_T} each",
           "graphs_per_s": G / tb, "ms_per_batch": tb * 1e3, "threads_per_graph": th,
           "autotune": {"threads": th, "thread_degree": rec.get("thread_degree"), "ms": rec["ms"]},
           "one_per_launch_graphs_per_s": G / t1,
           "one_per_launch_ms": t1 * 1e3, "speedup": t1 / tb, "identical_results": same,
           "gteps_batched": Mtot * BATCH_T / tb / 1e9,
           "roofline": _batch_roofline(Mtot, Ntot, BATCH_T, tb),
           "sharding": {"ranks": ws, "split": "contiguous graph ranges balanced by 2m + n",
                        "rank0_range": [lo, hi] if rank == 0 else None}}
    out["peeling"] = bench_batch_peeling(dsg, ctx, graphs, args, ws, rank)
    return out


def _batch_roofline(M: int, N: int, T: int, seconds: float) -> dict:
    """The batch against HBM by the symmetric-CSR edge-scan model of one
    iteration, 16m + 16n bytes per graph (each of the 2m arcs read once and
    its target's load gathered once; offsets, own load and count per
    vertex), times T iterations: the bytes one batched launch would move if
    every access went to DRAM.  Each block keeps its graph in L2, so the
    fraction shows how far the latency-bound blocks are from that rate."""
    peak, kind = _peak_hbm()
    by = (16 * M + 16 * N) * T
    ach = by / seconds / 1e9
    return {"bound": "hbm", "model": "(16m + 16n) per graph and iteration", "bytes_per_batch": by,
            "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "peak_kind": kind}


def bench_batch_peeling(dsg, ctx, graphs, args, ws: int = 1, rank: int = 0) -> dict:
    """Batched PaRGreedy++ (eps = 1/10, T = BATCH_T_PEEL) on the same batch,
    sharded by graph as above; one dsg_run per graph is timed on a seeded
    sample of the graphs (it takes minutes on all of them; each rank runs the
    sampled graphs of its range) and compared with the batch's results there."""
    import numpy as np
    import torch
    from paper_2311_04333_gb300 import shard, tune
    G = len(graphs)
    lo, hi = shard.my_range([shard.graph_cost(g.n, g.m) for g in graphs], rank, ws)
    mine = graphs[lo:hi]
    Gl = len(mine)
    T = np.full(Gl, BATCH_T_PEEL, np.int32)
    p = np.ones(Gl, np.int64)
    q = np.full(Gl, 10, np.int64)
    b = dsg.dsg_upload_batch(ctx, [(g.n, g.off, g.adj) for g in mine], 0)
    Gb, N, M = dsg.dsg_batch_info(b)
    rec = tune.tune_batch(ctx, b, T, force=True, variant=dsg.DSG_PEELING, eps_num=p, eps_den=q)
    th = rec["threads"]
    best_b = np.zeros(4 * Gl, np.int64)
    torch.cuda.synchronize()
    _barrier(ws)
    t0 = time.perf_counter()
    for _ in range(args.batch_steps):
        dsg.dsg_run_batch(ctx, b, dsg.DSG_PEELING, T, th, best_b, eps_num=p, eps_den=q)
    tb = _max_over_ranks((time.perf_counter() - t0) / args.batch_steps, ws)
    dsg.dsg_free_batch(b)
    sample = np.sort(np.random.default_rng(BATCH_SEED).choice(G, size=min(G, 128), replace=False))
    local = [int(i) for i in sample if lo <= i < hi]
    hs = [dsg.dsg_upload_csr(ctx, graphs[i].n, graphs[i].off, graphs[i].adj, 0) for i in local]
    if hs:
        dsg.dsg_run(ctx, hs[0], dsg.DSG_PEELING, BATCH_T_PEEL, 1, 10)
    best_1 = np.zeros((len(local), 4), np.int64)
    torch.cuda.synchronize()
    _barrier(ws)
    t0 = time.perf_counter()
    for k, h in enumerate(hs):
        r = dsg.dsg_run(ctx, h, dsg.DSG_PEELING, BATCH_T_PEEL, 1, 10)
        best_1[k] = (r["best_edges"], r["best_vertices"], r["best_iter"], r["best_set_size"])
    t1 = _max_over_ranks(time.perf_counter() - t0, ws)
    for h in hs:
        dsg.dsg_free_graph(h)
    m_sample = sum(graphs[i].m for i in sample)
    got = shard.gather_rows(best_b.reshape(Gl, 4)[[i - lo for i in local]], ws)
    want = shard.gather_rows(best_1, ws)
    same = bool(got.shape == (len(sample), 4) and np.array_equal(got, want))
    Mtot = int(_sum_over_ranks(float(M), ws))
    return {"workload": f"same {G} graphs, PaRGreedy++ eps=1/10, T={BATCH_T_PEEL} each",
            "graphs_per_s": G / tb, "ms_per_batch": tb * 1e3, "threads_per_graph": th,
            "autotune": {"threads": th, "block_degree": rec.get("block_degree"), "ms": rec["ms"]},
            "gteps_batched": Mtot * BATCH_T_PEEL / tb / 1e9,
            "one_per_launch_sample": len(sample),
            "one_per_launch_graphs_per_s": len(sample) / t1,
            "one_per_launch_gteps": m_sample * BATCH_T_PEEL / t1 / 1e9,
            "identical_results_on_sample": same}


def bench_pruned(dsg, g, ctx, stream, T, plain_ms, plain_r) -> dict:
    """dsg_run_pruned (k_max, the ceil(k_max/2)-core, T refine iterations with
    re-pruning) against plain dsg_run, at T and at 5 T iterations."""
    import torch

    def timed(fn):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        out = fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1), out

    ms, r = timed(lambda: dsg.dsg_run_pruned(ctx, g, dsg.DSG_SORTING, T))
    ms5, r5 = timed(lambda: dsg.dsg_run_pruned(ctx, g, dsg.DSG_SORTING, 5 * T))
    plain5, p5 = timed(lambda: dsg.dsg_run(ctx, g, dsg.DSG_SORTING, 5 * T))
    # PaRApxSorting++: pruning by the 1.5-approximate core numbers
    msa, ra = timed(lambda: dsg.dsg_run_pruned(ctx, g, dsg.DSG_SORTING, T, c=(3, 2)))
    msa5, ra5 = timed(lambda: dsg.dsg_run_pruned(ctx, g, dsg.DSG_SORTING, 5 * T, c=(3, 2)))
    apx = {"variant": "PaRApxSorting++ (approximate pruning, c = 3/2)", "ms": msa, "ms_T5": msa5,
           "speedup_vs_plain": plain_ms / msa, "speedup_vs_plain_T5": plain5 / msa5,
           "k_hat_max": ra["k_max"], "core_vertices": ra["core_vertices"], "core_edges": ra["core_edges"],
           "final_vertices": ra["final_vertices"], "best": [ra["best_edges"], ra["best_vertices"], ra["best_iter"]],
           "best_T5": [ra5["best_edges"], ra5["best_vertices"], ra5["best_iter"]]}
    # PaRGreedy++ (eps = 1/10) with exact pruning, and PaRApxGreedy++
    # (approximate pruning followed by exact pruning): identical outputs
    msg, rg = timed(lambda: dsg.dsg_run_pruned(ctx, g, dsg.DSG_PEELING, T, 1, 10))
    msga, rga = timed(lambda: dsg.dsg_run_pruned_apx_exact(ctx, g, dsg.DSG_PEELING, T, 1, 10, 3, 2))
    greedy = {"variant": "PaRGreedy++ eps=1/10 with exact pruning; PaRApxGreedy++ (c = 3/2, then exact)",
              "T": T, "ms_exact_pruning": msg, "ms_apx_then_exact": msga, "k_max": rga["k_max"],
              "core_vertices": rga["core_vertices"], "core_edges": rga["core_edges"],
              "best": [rg["best_edges"], rg["best_vertices"], rg["best_iter"]],
              "identical": (rg["best_edges"], rg["best_vertices"], rg["best_iter"], rg["core_vertices"]) ==
                           (rga["best_edges"], rga["best_vertices"], rga["best_iter"], rga["core_vertices"])}
    return {"variant": "PaRSorting++ with exact pruning (Alg. 1)", "T": T, "ms": ms, "plain_ms": plain_ms,
            "speedup_vs_plain": plain_ms / ms, "k_max": r["k_max"], "core_vertices": r["core_vertices"],
            "core_edges": r["core_edges"], "final_vertices": r["final_vertices"],
            "best": [r["best_edges"], r["best_vertices"], r["best_iter"]],
            "plain_best": [plain_r["best_edges"], plain_r["best_vertices"], plain_r["best_iter"]],
            "T5": 5 * T, "ms_T5": ms5, "plain_ms_T5": plain5, "speedup_vs_plain_T5": plain5 / ms5,
            "best_T5": [r5["best_edges"], r5["best_vertices"], r5["best_iter"]],
            "plain_best_T5": [p5["best_edges"], p5["best_vertices"], p5["best_iter"]], "approximate": apx,
            "greedy": greedy}


def peel_bytes(m: int, n: int, rounds_per_iter: float, alive_per_iter: float) -> float:
    """Algorithmic bytes of one PaRGreedy++ iteration (the byte model of the
    round peel): 8m (each arc's neighbour id read once when its F vertex is
    peeled) + 4m (the neighbour's state word) + 8m (at most one atomic
    decrement per arc, read and write) + 8 per alive vertex per round (key
    read and snapshot write) + the (round, id) sort with the fused suffix
    scan over n (12n for one radix pass, 20n + 16n(P - 2) + 8n for P >= 2)."""
    bits = max(1, math.ceil(math.log2(max(rounds_per_iter, 2))))
    P = (bits + 7) // 8
    sort = 12 * n if P == 1 else (20 + 16 * (P - 2) + 8) * n
    return 20 * m + 8 * alive_per_iter + sort


def bench_peeling(dsg, ctx, g, n, m, stream, T, eps=(1, 10), steps=1) -> dict:
    """PaRGreedy++ (whole-GPU round peel) on a resident graph: GTEPS per
    iteration, rounds per iteration, microseconds per round, and the
    fraction of the measured HBM bandwidth by the byte model above."""
    import torch
    loads = torch.empty(n, dtype=torch.int64, device="cuda")
    dsg.dsg_run(ctx, g, dsg.DSG_PEELING, 1, eps[0], eps[1], None, loads, None, None, dsg.DSG_PATH_GRID)
    dsg.dsg_get_peel_stats(ctx, reset=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        r = dsg.dsg_run(ctx, g, dsg.DSG_PEELING, T, eps[0], eps[1], None, loads, None, None, dsg.DSG_PATH_GRID)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_it = ev0.elapsed_time(ev1) / (steps * T)
    st = dsg.dsg_get_peel_stats(ctx, reset=True)
    rounds = st["rounds"] / max(st["iterations"], 1)
    alive = st["alive_sum"] / max(st["iterations"], 1)
    by = peel_bytes(m, n, rounds, alive)
    peak, kind = _peak_hbm()
    return {"eps": f"{eps[0]}/{eps[1]}", "T": T, "gteps": m / (ms_it * 1e-3) / 1e9, "ms_per_iteration": ms_it,
            "rounds_per_iteration": rounds, "us_per_round": ms_it * 1e3 / max(rounds, 1),
            "alive_per_round": alive / max(rounds, 1),
            "roofline": {"bytes_per_iteration": by, "achieved_gbs": by / (ms_it * 1e-3) / 1e9, "peak": peak,
                         "frac": by / (ms_it * 1e-3) / 1e9 / peak, "peak_kind": kind,
                         "model": "20m + 8 (alive vertices summed over rounds) + radix bytes of the (round, id) sort"},
            "best": [r["best_edges"], r["best_vertices"], r["best_iter"]]}


def bench_rmat20(dsg, ctx, gg, stream, args) -> dict:
    """The R-MAT scale-20 workload (edge factor 16, seed 2) with both
    variants, T = 20, eps = 1/10 for PaRGreedy++: GTEPS per iteration with the
    graph resident (whole-GPU path)."""
    import torch
    n, off, adj = gg.rmat_cuda(20, 16, 2)
    g = dsg.dsg_upload_csr(ctx, n, off, adj, dsg.DSG_SRC_DEVICE)
    _, m, _ = dsg.dsg_graph_info(g)
    T = 20
    loads = torch.empty(n, dtype=torch.int64, device="cuda")
    bset = torch.empty(n, dtype=torch.int32, device="cuda")
    out = {"workload": f"rmat20_ef16_seed2, n={n}, m={m}, T={T}"}
    try:
        for name, variant, p, q in (("sorting", dsg.DSG_SORTING, 0, 1),):
            for _ in range(2):
                dsg.dsg_run(ctx, g, variant, T, p, q, None, loads, bset, None, dsg.DSG_PATH_GRID)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            steps = max(1, args.steps)
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(steps):
                r = dsg.dsg_run(ctx, g, variant, T, p, q, None, loads, bset, None, dsg.DSG_PATH_GRID)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms_it = ev0.elapsed_time(ev1) / (steps * T)
            out[name] = {"gteps": m / (ms_it * 1e-3) / 1e9, "ms_per_iteration": ms_it,
                         "best": [r["best_edges"], r["best_vertices"], r["best_iter"]]}
        out["peeling_eps_1_10"] = bench_peeling(dsg, ctx, g, n, m, stream, T, (1, 10), max(1, args.steps // 2))
        out["peeling_eps_1_100"] = bench_peeling(dsg, ctx, g, n, m, stream, 4, (1, 100), 1)
    finally:
        dsg.dsg_free_graph(g)
    return out


def bench_serving(dsg, pool, device, args) -> dict:
    """The native request loop under Poisson arrivals: capacity from a
    closed burst of four rounds of the request pool, then an open-loop run at
    the configured rate (SERVE_RATE req/s) for args.serve_seconds after a
    warm-up; latency percentiles are per request, submit to results on the
    host.  When the offered rate is above capacity the queue grows during the
    run and the line reports that queueing (mean / p99 queue delay, the drain
    time after the last arrival) and each worker's occupancy."""
    import numpy as np
    from paper_2311_04333_gb300 import serve
    srv = dsg.dsg_server_create(device, args.serve_slots, 0)
    try:
        rng = np.random.default_rng(SERVE_SEED)
        burst = []
        t0 = time.perf_counter()
        # a closed burst of 4 rounds of the pool, so that the slowest request
        # does not set the capacity alone
        for _ in range(4):
            for g in pool:
                burst.append(dsg.dsg_server_submit(srv, g.n, g.off, g.adj, int(rng.integers(2)),
                                                   int(rng.choice([8, 16, 32])), 1, int(rng.choice([10, 100]))))
        ok = all(dsg.dsg_server_wait(srv, tk)["status"] == 0 for tk in burst)
        cap = len(burst) / (time.perf_counter() - t0)
        rate = args.serve_rate
        res = serve.poisson_run(srv, pool, rate, args.serve_seconds, warmup=args.serve_warmup, seed=SERVE_SEED)
    finally:
        dsg.dsg_server_destroy(srv)
    ms = [g.m for g in pool]
    res.update({"workload": f"pool of {len(pool)} graphs, m log-uniform in [1e3, 1e7] "
                            f"(R-MAT ef 8 / Chung-Lu gamma 2.1 avg degree 16, m {min(ms)}..{max(ms)}), "
                            "T in {8,16,32}, eps in {1/10,1/100}, PaRSorting++ / PaRGreedy++ 50/50, "
                            "host CSR in, loads and best set out",
                "slots": args.serve_slots, "burst_capacity_req_s": cap, "burst_ok": ok,
                "offered_vs_capacity": rate / cap if cap else None,
                "workers": f"occupancy keys 0..{args.serve_slots - 1} are slots, {args.serve_slots} the batch worker"})
    return res


def profile_case(name: str) -> int:
    """One small run of a kernel for profilers (nothing is timed):
    edge_scan_rmat25: PaRSorting++ T = 3 on R-MAT 25 (k_edge_scan launches 2 and 3);
    edge_scan_rmat27: the same on the benchmarked R-MAT 27 workload (for
      single-pass counters only: it holds about 30 GB on the device);
    peel_rmat20: PaRGreedy++ eps = 1/10, T = 2, whole-GPU path, on R-MAT 20;
    batch_1024: batched PaRSorting++ T = 8 on 1,024 graphs of the batch recipe."""
    import numpy as np
    import torch
    import graphgen as gg
    import paper_2311_04333_gb300 as dsg
    ctx = dsg.dsg_create(0, torch.cuda.current_stream().cuda_stream)
    if name in ("edge_scan_rmat25", "edge_scan_rmat27"):
        if name == "edge_scan_rmat25":
            n, off, adj = gg.rmat_cuda(25, 16, 3)
        else:
            n, off, adj = gg.rmat_cuda(SCALE, EDGE_FACTOR, SEED, blocks=BLOCKS)
        g = dsg.dsg_upload_csr(ctx, n, off, adj, dsg.DSG_SRC_DEVICE)
        dsg.dsg_run(ctx, g, dsg.DSG_SORTING, 3, 0, 1, None, torch.empty(n, dtype=torch.int64, device="cuda"))
        dsg.dsg_free_graph(g)
    elif name == "peel_rmat20":
        n, off, adj = gg.rmat_cuda(20, 16, 2)
        g = dsg.dsg_upload_csr(ctx, n, off, adj, dsg.DSG_SRC_DEVICE)
        dsg.dsg_run(ctx, g, dsg.DSG_PEELING, 2, 1, 10, None, torch.empty(n, dtype=torch.int64, device="cuda"),
                    path=dsg.DSG_PATH_GRID)
        dsg.dsg_free_graph(g)
    else:
        graphs = gg.batch_mix(G=1024, seed=BATCH_SEED)
        b = dsg.dsg_upload_batch(ctx, [(x.n, x.off, x.adj) for x in graphs], 0)
        best = np.zeros(4 * len(graphs), np.int64)
        dsg.dsg_run_batch(ctx, b, dsg.DSG_SORTING, np.full(len(graphs), 8, np.int32), 1024, best)
        dsg.dsg_free_batch(b)
    torch.cuda.synchronize()
    dsg.dsg_destroy(ctx)
    print(f"profile case {name}: done")
    return 0


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import graphgen as gg
    import oracle as orc
    g = gg.rmat(SAMPLE_SCALE - 1, EDGE_FACTOR, SEED)
    T = 2
    for _ in range(args.warmup):
        orc.run(g, orc.SORTING, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orc.run(g, orc.SORTING, T)
    dt = time.perf_counter() - t0
    v = g.m * T * args.steps / dt / 1e9
    sample = (f"R-MAT scale {SAMPLE_SCALE - 1} (same recipe as the GPU workload, no planted blocks), "
              f"n={g.n}, m={g.m}, PaRSorting++ T={T} per step, sequential C oracle")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i64",
        "data": "synthetic",
        "config": {"workload": f"rmat{SCALE}_ef{EDGE_FACTOR}_seed{SEED}+10blocks({BLOCKS[0]}..{BLOCKS[-1]},p=1/2)",
                   "variant": "PaRSorting++", "T": T_ITERS,
                   "sample": f"each step: rmat{SAMPLE_SCALE - 1}_ef{EDGE_FACTOR}, PaRSorting++ T={T} "
                             "(the same recipe, bounded to run on the host cores)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--scale", type=int, default=SCALE)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-warmup", type=float, default=2.0)
    ap.add_argument("--serve-rate", type=float, default=SERVE_RATE)
    ap.add_argument("--serve-slots", type=int, default=SERVE_SLOTS)
    ap.add_argument("--profile-case", choices=["edge_scan_rmat25", "edge_scan_rmat27", "peel_rmat20", "batch_1024"],
                    help="run one small case for a profiler instead of the benchmark")
    args = ap.parse_args()
    if args.profile_case:
        return profile_case(args.profile_case)
    if args.impl == "reference":
        return run_reference(args)

    # the batched workload is generated before CUDA starts (process pool)
    graphs_batch = None
    if not args.no_batch:
        import graphgen as gg
        t0 = time.perf_counter()
        graphs_batch = gg.batch_mix(BATCH_G, BATCH_SEED, processes=max(1, min(16, os.cpu_count() or 1)))
        print(f"batch generated in {time.perf_counter() - t0:.1f} s", file=sys.stderr)
    serve_pool = None
    if not args.no_serve:
        from paper_2311_04333_gb300 import serve
        t0 = time.perf_counter()
        serve_pool = serve.request_pool(SERVE_POOL, SERVE_SEED,
                                        processes=max(1, min(16, os.cpu_count() or 1)))
        print(f"request pool generated in {time.perf_counter() - t0:.1f} s", file=sys.stderr)

    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import graphgen as gg
    import paper_2311_04333_gb300 as dsg

    stream = torch.cuda.current_stream()
    ctx = dsg.dsg_create(local, stream.cuda_stream)
    blocks = BLOCKS if args.scale == SCALE else [max(4, s >> (SCALE - args.scale)) for s in BLOCKS]
    workload = f"rmat{args.scale}_ef{EDGE_FACTOR}_seed{SEED}+10blocks({blocks[0]}..{blocks[-1]},p=1/2)"
    n, off, adj = gg.rmat_cuda(args.scale, EDGE_FACTOR, SEED, blocks=blocks)
    g = dsg.dsg_upload_csr(ctx, n, off, adj, 0)
    _, m, maxdeg = dsg.dsg_graph_info(g)
    T = T_ITERS
    loads = torch.empty(n, dtype=torch.int64, device="cuda")
    bset = torch.empty(n, dtype=torch.int32, device="cuda")
    trace = torch.empty(3 * T, dtype=torch.int64, device="cuda")

    def step():
        return dsg.dsg_run(ctx, g, dsg.DSG_SORTING, T, 0, 1, None, loads, bset, trace)

    for _ in range(args.warmup):
        r = step()
    # ---- timed region: device-resident inputs
    dsg.dsg_get_stats(ctx, reset=True)
    dsg.dsg_set_profiling(ctx, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    _barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            r = step()
        ev1.record(stream)
        torch.cuda.synchronize()
    _barrier(ws)
    dsg.dsg_set_profiling(ctx, False)
    ms_local = ev0.elapsed_time(ev1)
    value = replica_throughput(m * T * args.steps, ms_local * 1e-3, ws) / 1e9
    ms_total = _max_over_ranks(ms_local, ws)
    st = dsg.dsg_get_stats(ctx, reset=True)
    launches = sum(v["launches"] for v in st.values())
    es_ms = st["edge_scan"]["ms"] / (args.steps * T)
    # algorithmic bytes of one edge scan over the symmetric CSR: 8m adjacency
    # + 8m neighbour-load gathers (4 B each) + 8(n+1) offsets + 4n own loads
    # + 4n counts A.  The kernel reads the degree-oriented copy (each edge
    # once), whose own minimum is 8m + 16n.
    es_bytes = 16 * m + 16 * n + 8
    es_bytes_oriented = 8 * m + 16 * n
    peak, peak_kind = _peak_hbm()
    achieved = es_bytes / (es_ms * 1e-3) / 1e9
    sort_ms = st["sort"]["ms"] / (args.steps * T)
    sort_bytes = st["sort"]["bytes"] / (args.steps * T)
    ms_iter = ms_total / (args.steps * T)
    # per-iteration algorithmic bytes of the whole PaRSorting++ iteration:
    # 16m + (16P + 40)n with P the radix passes of the iteration (the
    # counted sort bytes are (16P - 4)n, which gives the mean P)
    mean_passes = (sort_bytes / n + 4) / 16
    it_bytes = 16 * m + (16 * mean_passes + 40) * n

    # ---- Pruning-and-Refining (Alg. 1) on the same resident graph
    pruned = bench_pruned(dsg, g, ctx, stream, T, ms_total / args.steps, r)
    # ---- PaRGreedy++ on the same resident graph (a few iterations)
    peeling27 = bench_peeling(dsg, ctx, g, n, m, stream, 3, (1, 10), 1)

    # ---- end to end through the C ABI with host buffers
    off_h = torch.empty(off.numel(), dtype=torch.int64, pin_memory=True)
    adj_h = torch.empty(adj.numel(), dtype=torch.int32, pin_memory=True)
    off_h.copy_(off)
    adj_h.copy_(adj)
    loads_h = torch.empty(n, dtype=torch.int64, pin_memory=True)
    bset_h = torch.empty(n, dtype=torch.int32, pin_memory=True)
    dsg.dsg_free_graph(g)
    del off, adj, loads, bset
    torch.cuda.empty_cache()

    # both calls return after their work is done: host clocks split each step
    # into the upload (host-to-device copy + oriented copy) and the run (T
    # iterations + read-back)
    e2e_split = {"upload_ms": [], "run_ms": []}

    def e2e_step():
        ta = time.perf_counter()
        gh = dsg.dsg_upload_csr(ctx, n, off_h, adj_h, 0)
        tb = time.perf_counter()
        try:
            rr = dsg.dsg_run(ctx, gh, dsg.DSG_SORTING, T, 0, 1, None, loads_h, bset_h)
            e2e_split["upload_ms"].append(round(1e3 * (tb - ta), 1))
            e2e_split["run_ms"].append(round(1e3 * (time.perf_counter() - tb), 1))
            return rr
        finally:
            dsg.dsg_free_graph(gh)

    re = e2e_step()
    e2e_split = {"upload_ms": [], "run_ms": []}
    assert (re["best_edges"], re["best_vertices"]) == (r["best_edges"], r["best_vertices"])
    _barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        re = e2e_step()
    torch.cuda.synchronize()
    e2e_value = replica_throughput(m * T * args.e2e_steps, time.perf_counter() - t0, ws) / 1e9
    h2d = 8 * (n + 1) + 4 * 2 * m
    d2h = 8 * n + 4 * re["best_set_size"]

    # ---- batched form: 4,096 graphs, one persistent launch vs one graph per launch
    batched = None
    if not args.no_batch:
        batched = bench_batch(dsg, ctx, graphs_batch, args, ws, rank)

    # ---- R-MAT scale 20: both variants
    rmat20 = bench_rmat20(dsg, ctx, gg, stream, args)

    # ---- serving: Poisson arrivals through the native request loop
    serving = None
    if not args.no_serve:
        serving = bench_serving(dsg, serve_pool, local, args)

    cpu = cpu_par = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline()
        cpu_par = cpu_parallel_baseline()
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": workload, "variant": "PaRSorting++", "T": T, "n": n, "m": m,
                       "max_degree": maxdeg, "step": f"one dsg_run of T={T} iterations",
                       "l2": "inputs larger than L2 (adjacency %.1f GB)" % (8 * m / 1e9),
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "best": [r["best_edges"], r["best_vertices"], r["best_iter"]]},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "kernel": "k_edge_scan", "ms_per_launch": es_ms,
                         "algorithmic_bytes_per_launch": es_bytes,
                         "oriented_min_bytes_per_launch": es_bytes_oriented,
                         "traffic": _traffic("k_edge_scan", workload)},
            "iteration_roofline": {"bytes": it_bytes, "achieved": it_bytes / (ms_iter * 1e-3) / 1e9,
                                   "peak": peak, "unit": "GB/s",
                                   "frac": it_bytes / (ms_iter * 1e-3) / 1e9 / peak, "ms": ms_iter,
                                   "model": "16m + (16P + 40)n per iteration", "mean_radix_passes": mean_passes},
            "phases": {"edge_scan_ms": es_ms, "sort_ms": sort_ms,
                       "sort_gbs": sort_bytes / (sort_ms * 1e-3) / 1e9 if sort_ms else None,
                       "other_ms": st["other"]["ms"] / (args.steps * T)},
            "cpu_baseline": cpu,
            "cpu_parallel_baseline": cpu_par,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
                    "upload_ms_per_step": e2e_split["upload_ms"], "run_ms_per_step": e2e_split["run_ms"]},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "batched": batched,
            "rmat20": rmat20,
            "pruned": pruned,
            "peeling_rmat27": peeling27,
            "serving": serving,
        }
        print(json.dumps(out))
    dsg.dsg_destroy(ctx)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
