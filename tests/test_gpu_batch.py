"""Batched PaRSorting++ and PaRGreedy++ (one persistent launch over a packed
batch of graphs) against the oracle run on each graph alone, and against
dsg_run per graph."""
import numpy as np
import pytest

import graphgen as gg
import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2311_04333_gb300 as dsg
    ctx = dsg.dsg_create(0, torch.cuda.current_stream().cuda_stream)
    yield dsg, ctx
    dsg.dsg_destroy(ctx)


def _run_batch(dsg, ctx, graphs, T, threads=0, variant=0, p=None, q=None):
    b = dsg.dsg_upload_batch(ctx, [(g.n, g.off, g.adj) for g in graphs], dsg.DSG_VALIDATE)
    try:
        G, N, M = dsg.dsg_batch_info(b)
        assert G == len(graphs) and N == sum(g.n for g in graphs) and M == sum(g.m for g in graphs)
        Tmax = int(max(T))
        best = np.zeros(4 * G, np.int64)
        loads = np.zeros(N, np.int64)
        sets = np.zeros(N, np.int32)
        trace = np.zeros(3 * G * Tmax, np.int64)
        dsg.dsg_run_batch(ctx, b, variant, T, threads, best, loads, sets, trace, p, q)
    finally:
        dsg.dsg_free_batch(b)
    return best.reshape(G, 4), loads, sets, trace.reshape(G, Tmax, 3)


def _check(graphs, T, best, loads, sets, trace, variant=0, p=None, q=None):
    base = 0
    for i, g in enumerate(graphs):
        if variant == 0:
            o = orc.run(g, orc.SORTING, int(T[i]))
        else:
            o = orc.run(g, orc.PEELING, int(T[i]), int(p[i]), int(q[i]))
        assert tuple(best[i, :3]) == (o.best_edges, o.best_vertices, o.best_iter), f"graph {i}"
        assert best[i, 3] == len(o.best_set)
        assert np.array_equal(loads[base:base + g.n], o.loads), f"graph {i} loads"
        assert np.array_equal(sets[base:base + best[i, 3]].astype(np.int64), o.best_set), f"graph {i} set"
        assert np.array_equal(trace[i, :T[i]], o.trace), f"graph {i} trace"
        base += g.n


@pytest.mark.parametrize("threads", [256, 512, 1024])
def test_batch_mixed_graphs(env, threads):
    dsg, ctx = env
    graphs = [gg.er_m(300, 6, 1), gg.complete(40), gg.from_edges(1, []), gg.star(500),
              gg.er_planted_clique(n=700, p=(1, 100), k=20, seed=3), gg.rmat(11, 8, 5),
              gg.from_edges(9, [(0, 1), (2, 3)]), gg.chung_lu(2000, 10, 2.1, 4), gg.path(257)]
    T = np.array([5, 3, 2, 4, 8, 6, 1, 7, 3], np.int32)
    _check(graphs, T, *_run_batch(dsg, ctx, graphs, T, threads))


def test_batch_mix_recipe_sample(env):
    dsg, ctx = env
    graphs = gg.batch_mix(G=48, seed=4, n_hi=5000)
    T = np.full(len(graphs), 32, np.int32)
    _check(graphs, T, *_run_batch(dsg, ctx, graphs, T))


def test_batch_equals_one_graph_per_launch(env):
    dsg, ctx = env
    graphs = gg.batch_mix(G=24, seed=9, n_hi=20000)
    T = np.full(len(graphs), 12, np.int32)
    best, loads, sets, trace = _run_batch(dsg, ctx, graphs, T)
    base = 0
    for i, g in enumerate(graphs):
        r = dsg.densest(ctx, g.n, g.off, g.adj, dsg.DSG_SORTING, 12)
        assert (r.best_edges, r.best_vertices, r.best_iter) == tuple(best[i, :3])
        assert np.array_equal(r.loads, loads[base:base + g.n])
        base += g.n


def test_batch_rejects_bad_input(env):
    dsg, ctx = env
    with pytest.raises(dsg.DsgError, match="INVALID"):
        dsg.dsg_upload_batch(ctx, [(2, np.array([0, 1, 2], np.int64), np.array([1, 5], np.int32))])
    b = dsg.dsg_upload_batch(ctx, [(3, gg.path(3).off, gg.path(3).adj)])
    try:
        with pytest.raises(dsg.DsgError, match="INVALID"):
            dsg.dsg_run_batch(ctx, b, 7, [3], 0, np.zeros(4, np.int64))
        with pytest.raises(dsg.DsgError, match="INVALID"):
            dsg.dsg_run_batch(ctx, b, dsg.DSG_PEELING, [3], 0, np.zeros(4, np.int64), eps_num=[1], eps_den=[0])
        with pytest.raises(dsg.DsgError, match="OVERFLOW"):
            dsg.dsg_run_batch(ctx, b, dsg.DSG_PEELING, [3], 0, np.zeros(4, np.int64), eps_num=[1 << 31],
                              eps_den=[1])
        with pytest.raises(dsg.DsgError, match="INVALID"):
            dsg.dsg_run_batch(ctx, b, dsg.DSG_SORTING, [0], 0, np.zeros(4, np.int64))
    finally:
        dsg.dsg_free_batch(b)


def _mixed_graphs():
    return [gg.er_m(300, 6, 1), gg.complete(40), gg.from_edges(1, []), gg.star(500),
            gg.er_planted_clique(n=700, p=(1, 100), k=20, seed=3), gg.rmat(11, 8, 5),
            gg.from_edges(9, [(0, 1), (2, 3)]), gg.chung_lu(2000, 10, 2.1, 4), gg.path(257),
            gg.chung_lu(3000, 30, 2.1, 8)]


@pytest.mark.parametrize("threads", [256, 512, 1024])
def test_batch_peeling_mixed_graphs(env, threads):
    """PaRGreedy++ per graph, eps from 0 to 1, against the oracle."""
    dsg, ctx = env
    graphs = _mixed_graphs()
    T = np.array([5, 3, 2, 4, 8, 6, 1, 7, 3, 5], np.int32)
    p = np.array([1, 1, 0, 1, 1, 1, 1, 0, 1, 1], np.int64)
    q = np.array([10, 100, 1, 2, 10, 100, 1, 1, 10, 1000], np.int64)
    _check(graphs, T, *_run_batch(dsg, ctx, graphs, T, threads, 1, p, q), variant=1, p=p, q=q)


def test_batch_peeling_recipe_sample(env):
    dsg, ctx = env
    graphs = gg.batch_mix(G=40, seed=6, n_hi=5000)
    G = len(graphs)
    T = np.full(G, 8, np.int32)
    p = np.ones(G, np.int64)
    q = np.where(np.arange(G) % 2 == 0, 10, 100).astype(np.int64)
    _check(graphs, T, *_run_batch(dsg, ctx, graphs, T, 0, 1, p, q), variant=1, p=p, q=q)


def test_batch_peeling_equals_one_graph_per_launch(env):
    dsg, ctx = env
    graphs = gg.batch_mix(G=12, seed=10, n_hi=20000)
    G = len(graphs)
    T = np.full(G, 6, np.int32)
    best, loads, sets, trace = _run_batch(dsg, ctx, graphs, T, 1024, 1, np.ones(G, np.int64),
                                          np.full(G, 20, np.int64))
    base = 0
    for i, g in enumerate(graphs):
        r = dsg.densest(ctx, g.n, g.off, g.adj, dsg.DSG_PEELING, 6, eps=(1, 20))
        assert (r.best_edges, r.best_vertices, r.best_iter) == tuple(best[i, :3])
        assert np.array_equal(r.loads, loads[base:base + g.n])
        assert np.array_equal(r.best_set, sets[base:base + best[i, 3]])
        base += g.n


def _check_full(graphs, T, best, loads, sets, trace, sample):
    """Every graph: its loads sum to T m (each iteration charges every edge
    once) and its best set has the reported size and induced edge count;
    the sampled graphs: every output equals the oracle's."""
    bases = np.concatenate([[0], np.cumsum([g.n for g in graphs])])
    for i, g in enumerate(graphs):
        b = int(bases[i])
        assert int(loads[b:b + g.n].sum()) == int(T[i]) * g.m, f"graph {i} load sum"
        k = int(best[i, 3])
        assert k == best[i, 1] and 0 < k <= g.n, f"graph {i} set size"
        s = sets[b:b + k].astype(np.int64)
        assert np.all(np.diff(s) > 0) and s[0] >= 0 and s[-1] < g.n, f"graph {i} set order"
        inside = np.zeros(g.n, bool)
        inside[s] = True
        c = np.concatenate([[0], np.cumsum(inside[g.adj].astype(np.int64))])
        deg_in = c[g.off[1:]] - c[g.off[:-1]]          # neighbours inside the set
        assert int(deg_in[s].sum()) == 2 * int(best[i, 0]), f"graph {i} set edges"
    for i in sample:
        g, b = graphs[i], int(bases[i])
        o = orc.run(g, orc.SORTING, int(T[i]))
        assert tuple(best[i, :3]) == (o.best_edges, o.best_vertices, o.best_iter), f"graph {i}"
        assert np.array_equal(loads[b:b + g.n], o.loads), f"graph {i} loads"
        assert np.array_equal(sets[b:b + len(o.best_set)].astype(np.int64), o.best_set), f"graph {i} set"
        assert np.array_equal(trace[i, :T[i]], o.trace), f"graph {i} trace"


def test_batch_full_config(env):
    """The batched configuration at full size: 4,096 graphs of the batch
    recipe (n log-uniform in [50, 50,000]; ER, R-MAT and planted cliques),
    T = 32 each, in one launch; all graphs checked by their invariants, the
    8 largest and 24 random ones against the oracle output for output."""
    import os
    dsg, ctx = env
    graphs = gg.batch_mix(G=4096, seed=4, processes=max(1, min(16, os.cpu_count() or 1)))
    T = np.full(len(graphs), 32, np.int32)
    best, loads, sets, trace = _run_batch(dsg, ctx, graphs, T)
    rng = np.random.default_rng(21)
    largest = sorted(range(len(graphs)), key=lambda i: -graphs[i].m)[:8]
    sample = sorted(set(largest) | set(rng.choice(len(graphs), 24, replace=False).tolist()))
    _check_full(graphs, T, best, loads, sets, trace, sample)


@pytest.mark.parametrize("variant", [0, 1])
def test_batch_tuning_knobs_do_not_change_results(env, variant):
    """dsg_set_batch_tuning moves the thread-versus-warp list length and the
    whole-block degree; every setting gives the oracle's results."""
    dsg, ctx = env
    graphs = [gg.er_m(300, 6, 1), gg.complete(40), gg.star(500), gg.rmat(11, 8, 5), gg.chung_lu(2000, 10, 2.1, 4),
              gg.er_planted_clique(n=700, p=(1, 100), k=20, seed=3)]
    T = np.array([5, 3, 4, 6, 7, 8], np.int32)
    p = np.ones(len(graphs), np.int64)
    q = np.full(len(graphs), 10, np.int64)
    b = dsg.dsg_upload_batch(ctx, [(g.n, g.off, g.adj) for g in graphs], 0)
    try:
        G, N, _ = dsg.dsg_batch_info(b)
        for td, bd in ((1, 1), (8, 100000), (1000, 64), (0, 0)):
            dsg.dsg_set_batch_tuning(ctx, b, td, bd)
            best = np.zeros(4 * G, np.int64)
            loads = np.zeros(N, np.int64)
            sets = np.zeros(N, np.int32)
            trace = np.zeros(3 * G * int(T.max()), np.int64)
            dsg.dsg_run_batch(ctx, b, variant, T, 512, best, loads, sets, trace, p, q)
            _check(graphs, T, best.reshape(G, 4), loads, sets, trace.reshape(G, int(T.max()), 3), variant, p, q)
        with pytest.raises(dsg.DsgError, match="INVALID"):
            dsg.dsg_set_batch_tuning(ctx, b, -1, 0)
    finally:
        dsg.dsg_free_batch(b)
