"""Parity of the CUDA PaRGreedy++ round peel (through the C ABI) with the
oracle: loads, best, best set and trace must be identical."""
import numpy as np
import pytest

import graphgen as gg
import oracle as orc

from test_gpu_sorting import check, path  # noqa: F401  (shared exact comparison, both paths)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dsg():
    import paper_2311_04333_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(dsg):
    import torch
    c = dsg.dsg_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    dsg.dsg_destroy(c)


def test_planted_clique_config(dsg, ctx):
    r, _ = check(dsg, ctx, gg.er_planted_clique(), orc.PEELING, 10, 1, 10)
    assert (r.best_edges, r.best_vertices) == (435, 30)


@pytest.mark.parametrize("p,q", [(0, 1), (1, 10), (1, 100), (3, 1)])
def test_eps_values(dsg, ctx, p, q):
    check(dsg, ctx, gg.er_m(6000, 12, 3), orc.PEELING, 5, p, q)


@pytest.mark.parametrize("n,d,seed", [(20000, 8, 1), (4097, 3, 4), (30000, 20, 5)])
def test_random_graphs(dsg, ctx, n, d, seed):
    check(dsg, ctx, gg.er_m(n, d, seed), orc.PEELING, 6, 1, 10)


def test_power_law_and_heavy(dsg, ctx):
    check(dsg, ctx, gg.chung_lu(20000, 16, 2.1, 7), orc.PEELING, 6, 1, 10)
    g = gg.disjoint_union(gg.er_m(3000, 10, 9), gg.star(5000), gg.complete(60), gg.star(2049))
    check(dsg, ctx, g, orc.PEELING, 5, 1, 10)


def test_rmat_small(dsg, ctx):
    check(dsg, ctx, gg.rmat(16, 16, 11), orc.PEELING, 8, 1, 10)


def test_complete_and_degenerate(dsg, ctx):
    check(dsg, ctx, gg.complete(200), orc.PEELING, 4, 1, 10)
    check(dsg, ctx, gg.from_edges(1, []), orc.PEELING, 2, 1, 10)
    check(dsg, ctx, gg.path(500), orc.PEELING, 2, 0, 1)      # many rounds
    check(dsg, ctx, gg.from_edges(9000, [(i, i + 3) for i in range(0, 8990, 7)]), orc.PEELING, 3, 1, 10)


def test_resume(dsg, ctx, path):
    g = gg.er_m(8000, 10, 31)
    full = dsg.densest(ctx, g.n, g.off, g.adj, dsg.DSG_PEELING, 7, (1, 10), path=path)
    a = dsg.densest(ctx, g.n, g.off, g.adj, dsg.DSG_PEELING, 3, (1, 10), path=path)
    b = dsg.densest(ctx, g.n, g.off, g.adj, dsg.DSG_PEELING, 4, (1, 10), init_loads=a.loads, path=path)
    assert np.array_equal(b.loads, full.loads)


@pytest.mark.slow
def test_rmat20_config(dsg, ctx):
    """R-MAT scale 20, eps = 1/10, T = 20 (the second workload, PaRGreedy++)."""
    check(dsg, ctx, gg.rmat(20, 16, 2), orc.PEELING, 20, 1, 10)


def test_round_telemetry_matches_the_oracle(dsg, ctx):
    """dsg_get_peel_stats: rounds per iteration and alive vertices summed over
    the rounds of the whole-GPU peel equal the oracle's round structure."""
    g = gg.rmat(14, 8, 3)
    T, p, q = 3, 1, 10
    loads = np.zeros(g.n, np.int64)
    rounds = alive = 0
    for _ in range(T):
        order, rof, rmin = orc.round_order(g, loads, p, q)
        R = len(rmin)
        sizes = np.bincount(rof, minlength=R)
        rounds += R
        alive += int((g.n - np.concatenate([[0], np.cumsum(sizes)[:-1]])).sum())
        loads = orc.iteration(g, order, loads)["loads"]
    h = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj, 0)
    try:
        dsg.dsg_get_peel_stats(ctx, reset=True)
        dsg.dsg_run(ctx, h, dsg.DSG_PEELING, T, p, q, path=dsg.DSG_PATH_GRID)
        st = dsg.dsg_get_peel_stats(ctx, reset=True)
    finally:
        dsg.dsg_free_graph(h)
    assert st == {"iterations": T, "rounds": rounds, "alive_sum": alive}


@pytest.mark.parametrize("blocks", [1, 4, 38])
def test_capped_grid_matches_oracle(dsg, ctx, blocks):
    """The round kernel with its grid capped to 1, 4 and 38 SMs' worth of
    blocks (as each server slot caps it): every block carries a long share
    of the alive list and long queues of peeled vertices."""
    g = gg.rmat(16, 16, 4)
    dsg.dsg_debug_set(ctx, dsg.DSG_DEBUG_PEEL_BLOCKS, blocks)
    try:
        for p, q in ((1, 10), (1, 100)):
            loads = np.zeros(g.n, np.int64)
            bset = np.zeros(g.n, np.int32)
            trace = np.zeros(3 * 4, np.int64)
            h = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj, 0)
            try:
                r = dsg.dsg_run(ctx, h, dsg.DSG_PEELING, 4, p, q, None, loads, bset, trace, dsg.DSG_PATH_GRID)
            finally:
                dsg.dsg_free_graph(h)
            o = orc.run(g, orc.PEELING, 4, p, q)
            assert np.array_equal(loads, o.loads)
            assert (r["best_edges"], r["best_vertices"], r["best_iter"]) == (o.best_edges, o.best_vertices, o.best_iter)
            assert np.array_equal(bset[: r["best_set_size"]].astype(np.int64), o.best_set)
            assert np.array_equal(trace.reshape(4, 3), o.trace)
    finally:
        dsg.dsg_debug_set(ctx, dsg.DSG_DEBUG_PEEL_BLOCKS, 0)
