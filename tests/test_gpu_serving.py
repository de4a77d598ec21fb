"""The native request loop (dsg_server_*): every request served in a mix of
concurrent requests gives exactly what the oracle gives on it alone; the
HBM budget bounds what runs at once; bad requests fail alone."""
import threading

import numpy as np
import pytest

import graphgen as gg
import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dsg():
    import torch
    torch.cuda.init()
    import paper_2311_04333_gb300 as m
    return m


def _mix():
    graphs = [gg.er_m(400, 6, 1), gg.complete(30), gg.star(300), gg.rmat(12, 8, 7),
              gg.er_planted_clique(n=900, p=(1, 100), k=25, seed=2), gg.chung_lu(3000, 16, 2.1, 5),
              gg.from_edges(1, []), gg.path(100), gg.rmat(14, 8, 9), gg.chung_lu(20000, 16, 2.1, 6)]
    reqs = []
    rng = np.random.default_rng(11)
    for i in range(24):
        g = graphs[i % len(graphs)]
        variant = int(rng.integers(2))
        reqs.append((g, variant, int(rng.choice([1, 4, 8])), 1, int(rng.choice([10, 100]))))
    return reqs


def _expect(g, variant, T, p, q):
    o = orc.run(g, orc.SORTING if variant == 0 else orc.PEELING, T, p, q)
    return o


@pytest.mark.parametrize("slots", [1, 4])
def test_mix_matches_oracle(dsg, slots):
    reqs = _mix()
    srv = dsg.dsg_server_create(0, slots, 0)
    try:
        tickets = [dsg.dsg_server_submit(srv, g.n, g.off, g.adj, v, T, p, q) for g, v, T, p, q in reqs]
        for (g, v, T, p, q), tk in zip(reqs, tickets):
            loads = np.zeros(g.n, np.int64)
            bset = np.zeros(g.n, np.int32)
            r = dsg.dsg_server_wait(srv, tk, -1, loads, bset)
            assert r["status"] == 0, r["error"]
            o = _expect(g, v, T, p, q)
            assert (r["best_edges"], r["best_vertices"], r["best_iter"]) == \
                (o.best_edges, o.best_vertices, o.best_iter), (g.name, v, T, q)
            assert r["best_set_size"] == len(o.best_set)
            assert np.array_equal(np.sort(bset[:r["best_set_size"]]).astype(np.int64), np.sort(o.best_set))
            assert np.array_equal(loads, o.loads), (g.name, v, T, q)
            assert r["n"] == g.n and r["m"] == g.m and 0 <= r["slot"] <= slots
            compact = g.n <= 32768 and 2 * g.m <= 1 << 20
            assert (r["slot"] == slots) == compact        # compact graphs: the batch worker
            assert r["latency_ms"] >= r["run_ms"] >= 0 and r["queue_ms"] >= 0
        st = dsg.dsg_server_stats(srv)
        assert st["queued"] == 0 and st["running"] == 0 and st["done"] == len(reqs) and st["bytes_in_use"] == 0
    finally:
        dsg.dsg_server_destroy(srv)


def test_budget_bounds_concurrency(dsg):
    """With a budget that holds one of these graphs but not two, requests
    run one at a time whatever the number of slots."""
    g = gg.rmat(15, 8, 3)
    est = 24 * g.m + 128 * g.n + (4 << 20)
    srv = dsg.dsg_server_create(0, 4, int(est * 1.5))
    seen = []
    stop = threading.Event()

    def sampler():
        while not stop.is_set():
            seen.append(dsg.dsg_server_stats(srv))

    th = threading.Thread(target=sampler)
    th.start()
    try:
        tickets = [dsg.dsg_server_submit(srv, g.n, g.off, g.adj, 0, 4, 0, 1) for _ in range(6)]
        res = [dsg.dsg_server_wait(srv, tk) for tk in tickets]
    finally:
        stop.set()
        th.join()
    try:
        assert all(r["status"] == 0 for r in res)
        assert len({(r["best_edges"], r["best_vertices"], r["best_iter"]) for r in res}) == 1
        assert max(s["running"] for s in seen) <= 1
        assert max(s["bytes_in_use"] for s in seen) <= est * 1.5
        # a request larger than the whole budget is refused at submission
        big = gg.rmat(17, 8, 3)
        with pytest.raises(dsg.DsgError):
            dsg.dsg_server_submit(srv, big.n, big.off, big.adj, 0, 1, 0, 1)
    finally:
        dsg.dsg_server_destroy(srv)


def test_bad_request_fails_alone(dsg):
    good = gg.er_m(500, 8, 4)
    bad_adj = good.adj.copy()
    bad_adj[3] = good.n + 5                       # neighbour id out of range
    srv = dsg.dsg_server_create(0, 2, 0)
    try:
        t1 = dsg.dsg_server_submit(srv, good.n, good.off, good.adj, 0, 3, 0, 1)
        t2 = dsg.dsg_server_submit(srv, good.n, good.off, bad_adj, 0, 3, 0, 1)
        t3 = dsg.dsg_server_submit(srv, good.n, good.off, good.adj, 1, 3, 1, 10)
        r1, r2, r3 = (dsg.dsg_server_wait(srv, t) for t in (t1, t2, t3))
        assert r1["status"] == 0 and r3["status"] == 0
        assert r2["status"] == dsg.DSG_ERR_INVALID and "out of" in r2["error"]
        o = orc.run(good, orc.SORTING, 3)
        assert (r1["best_edges"], r1["best_vertices"]) == (o.best_edges, o.best_vertices)
        with pytest.raises(dsg.DsgError):
            dsg.dsg_server_wait(srv, t1)              # ticket already released
        with pytest.raises(dsg.DsgError):
            dsg.dsg_server_submit(srv, good.n, good.off, good.adj, 7, 3, 0, 1)
    finally:
        dsg.dsg_server_destroy(srv)
