"""Serving workload driver over the native request loop (dsg_server_*):
Poisson arrivals of densest-subgraph requests, each drawn from a pool of
graphs with edge counts log-uniform in [1e3, 1e7] (R-MAT with edge factor 8,
or Chung-Lu with exponent 2.1 and average degree 16), T in {8, 16, 32},
eps in {1/10, 1/100}, variant PaRSorting++ or PaRGreedy++ at random.
Reports p50 / p99 latency and throughput."""
from __future__ import annotations

import math
import threading
import time

import numpy as np

from . import _dsg


def request_pool(size: int, seed: int = 5, m_lo: float = 1e3, m_hi: float = 1e7, processes: int = 1):
    """`size` request graphs (graphgen), log-uniform edge counts."""
    import graphgen as gg
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(size):
        m = float(np.exp(rng.uniform(math.log(m_lo), math.log(m_hi))))
        kind = "rmat" if rng.random() < 0.5 else "chung_lu"
        specs.append((i, kind, m, seed))
    if processes > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            return pool.map(_make_graph, specs, chunksize=1)
    return [_make_graph(sp) for sp in specs]


def _make_graph(spec):
    import graphgen as gg
    i, kind, m, seed = spec
    if kind == "rmat":
        scale = max(4, math.ceil(math.log2(max(m / 8, 16))))
        return gg.rmat(scale, 8, seed * 10_000 + i)
    n = max(16, int(m / 8))
    return gg.chung_lu(n, 16, 2.1, seed * 10_000 + i)


def poisson_run(server, pool, rate: float, seconds: float, warmup: float = 0.0, seed: int = 5,
                variants=(_dsg.DSG_SORTING, _dsg.DSG_PEELING)) -> dict:
    """Submit requests with exponential inter-arrival times for warmup+seconds
    and wait for all of them; statistics cover the requests submitted after
    the warm-up."""
    rng = np.random.default_rng(seed + 1)
    tickets = []
    lock = threading.Lock()
    results = {}

    def collector():
        while True:
            with lock:
                pending = [t for t in tickets if t[0] not in results]
                finished = submitting_done[0] and not pending
            if finished:
                return
            for tk, *_ in pending[:64]:
                r = _dsg.dsg_server_wait(server, tk, 5)
                if r is not None:
                    with lock:
                        results[tk] = r
            time.sleep(0.001)

    submitting_done = [False]
    th = threading.Thread(target=collector, daemon=True)
    th.start()
    t0 = time.perf_counter()
    t_next = t0
    while True:
        now = time.perf_counter()
        if now - t0 >= warmup + seconds:
            break
        if now < t_next:
            time.sleep(min(t_next - now, 0.002))
            continue
        g = pool[int(rng.integers(len(pool)))]
        T = int(rng.choice([8, 16, 32]))
        q = int(rng.choice([10, 100]))
        variant = int(rng.choice(variants))
        tk = _dsg.dsg_server_submit(server, g.n, g.off, g.adj, variant, T, 1, q)
        with lock:
            tickets.append((tk, now - t0 >= warmup, g.m, T, now - t0))
        t_next += rng.exponential(1.0 / rate)
    t_submit_end = time.perf_counter()
    submitting_done[0] = True
    th.join()
    t_end = time.perf_counter()
    meas = [(tk, m, T) for tk, w, m, T, _ in tickets if w]
    lat = np.array([results[tk]["latency_ms"] for tk, _, _ in meas])
    q_ms = np.array([results[tk]["queue_ms"] for tk, _, _ in meas])
    ok = all(results[tk]["status"] == 0 for tk, _, _ in meas)
    edges_iter = sum(m * T for _, m, T in meas)
    span = t_end - (t0 + warmup)
    # busy time of each worker (slots 0..K-1, then the batch worker) over the
    # measured span: the union of its requests' [start, end) intervals
    # (requests of one batch share theirs)
    busy = {}
    for tk, w, _, _, t_sub in tickets:
        r = results[tk]
        a = t_sub + r["queue_ms"] / 1e3
        busy.setdefault(int(r["slot"]), []).append((a, a + r["run_ms"] / 1e3))
    occ = {}
    for slot, iv in sorted(busy.items()):
        iv.sort()
        tot, cur_a, cur_b = 0.0, None, None
        for a, b in iv:
            a, b = max(a, warmup), max(b, warmup)
            if cur_b is None or a > cur_b:
                if cur_b is not None:
                    tot += cur_b - cur_a
                cur_a, cur_b = a, b
            else:
                cur_b = max(cur_b, b)
        if cur_b is not None:
            tot += cur_b - cur_a
        occ[slot] = round(tot / span, 3) if span > 0 else None
    return {"requests": len(meas), "rate_req_s": rate, "seconds": seconds, "warmup_s": warmup,
            "all_ok": ok,
            "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
            "mean_queue_ms": float(q_ms.mean()) if len(q_ms) else None,
            "p99_queue_ms": float(np.percentile(q_ms, 99)) if len(q_ms) else None,
            "throughput_req_s": len(meas) / span if span > 0 else None,
            "gteps": edges_iter / span / 1e9 if span > 0 else None,
            "submit_span_s": t_submit_end - t0, "drain_s": t_end - t_submit_end,
            "worker_occupancy": occ}
