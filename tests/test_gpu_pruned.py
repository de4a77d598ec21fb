"""The Pruning-and-Refining run (Alg. 1) and the core numbers through the C
ABI, against the oracle: every output exact."""
import numpy as np
import pytest

import graphgen as gg
import oracle as orc

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


def _graphs():
    return {
        "planted": gg.er_planted_clique(),
        "dense_and_sparse": gg.disjoint_union(gg.er_m(60, 40, 8), gg.er_m(150, 20, 9)),
        "clique_star": gg.disjoint_union(gg.complete(6), gg.star(30)),
        "chung_lu": gg.chung_lu(20000, 16, 2.1, 6),
        "rmat14": gg.rmat(14, 8, 7),
        "blocks": gg.disjoint_union(gg.er_m(80, 50, 1), gg.er_m(300, 24, 2), gg.er_m(3000, 6, 3)),
        "cycle": gg.cycle(64),
        "single": gg.from_edges(1, []),
    }


@pytest.mark.parametrize("name", list(_graphs()))
def test_coreness(dsg, ctx, name):
    g = _graphs()[name]
    h = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj, 0)
    try:
        core, kmax = dsg.dsg_coreness(ctx, h)
    finally:
        dsg.dsg_free_graph(h)
    exp = orc.coreness(g)
    assert np.array_equal(core.astype(np.int64), exp)
    assert kmax == int(exp.max())


def test_coreness_large(dsg, ctx):
    """R-MAT 18 (whole-GPU peel with many rounds)."""
    g = gg.rmat(18, 16, 5)
    h = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj, 0)
    try:
        core, kmax = dsg.dsg_coreness(ctx, h)
    finally:
        dsg.dsg_free_graph(h)
    assert np.array_equal(core.astype(np.int64), orc.coreness(g))


@pytest.mark.parametrize("name", list(_graphs()))
@pytest.mark.parametrize("variant,p,q,T", [(0, 0, 1, 8), (1, 1, 10, 6), (1, 1, 100, 4)])
def test_pruned_run(dsg, ctx, name, variant, p, q, T):
    g = _graphs()[name]
    h = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj, 0)
    loads = np.zeros(g.n, np.int64)
    bset = np.zeros(g.n, np.int32)
    trace = np.zeros(3 * T, np.int64)
    try:
        r = dsg.dsg_run_pruned(ctx, h, variant, T, p, q, loads, bset, trace)
    finally:
        dsg.dsg_free_graph(h)
    o = orc.run_pruned(g, variant, T, p, q)
    assert (r["best_edges"], r["best_vertices"], r["best_iter"]) == (o.best_edges, o.best_vertices, o.best_iter)
    assert np.array_equal(bset[:r["best_set_size"]].astype(np.int64), o.best_set)
    assert np.array_equal(loads, o.loads)
    assert np.array_equal(trace.reshape(T, 3), o.trace)
    assert (r["k_max"], r["core_vertices"], r["core_edges"], r["final_vertices"]) == \
        (o.k_max, o.core_vertices, o.core_edges, o.final_vertices)
    assert (r["L_num"], r["L_den"]) == o.L


def test_pruned_run_device_buffers(dsg, ctx):
    import torch
    g = gg.disjoint_union(gg.er_m(60, 40, 8), gg.er_m(150, 20, 9))
    T = 6
    h = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj, 0)
    loads = torch.empty(g.n, dtype=torch.int64, device="cuda")
    bset = torch.empty(g.n, dtype=torch.int32, device="cuda")
    trace = torch.empty(3 * T, dtype=torch.int64, device="cuda")
    try:
        r = dsg.dsg_run_pruned(ctx, h, 0, T, 0, 1, loads, bset, trace)
        with pytest.raises(dsg.DsgError):
            dsg.dsg_run_pruned(ctx, h, 0, 0)
    finally:
        dsg.dsg_free_graph(h)
    o = orc.run_pruned(g, 0, T)
    assert np.array_equal(loads.cpu().numpy(), o.loads)
    assert np.array_equal(bset[:r["best_set_size"]].cpu().numpy().astype(np.int64), o.best_set)
    assert np.array_equal(trace.cpu().numpy().reshape(T, 3), o.trace)


@pytest.mark.parametrize("name", list(_graphs()))
@pytest.mark.parametrize("c", [(3, 2), (2, 1)])
def test_apx_coreness(dsg, ctx, name, c):
    """c-approximate core numbers (level-by-level peels) equal the oracle's."""
    g = _graphs()[name]
    h = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj, 0)
    try:
        core, khat = dsg.dsg_apx_coreness(ctx, h, c)
    finally:
        dsg.dsg_free_graph(h)
    exp = orc.apx_coreness(g, c)
    assert np.array_equal(core.astype(np.int64), exp)
    assert khat == int(exp.max())


@pytest.mark.parametrize("name", list(_graphs()))
@pytest.mark.parametrize("variant,p,q,T,c", [(0, 0, 1, 8, (3, 2)), (1, 1, 10, 6, (3, 2)), (0, 0, 1, 6, (2, 1)),
                                             (0, 0, 1, 5, (10001, 10000))])
def test_apx_pruned_run(dsg, ctx, name, variant, p, q, T, c):
    """Alg. 1 with approximate pruning: every output equals the oracle's."""
    g = _graphs()[name]
    h = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj, 0)
    loads = np.zeros(g.n, np.int64)
    bset = np.zeros(g.n, np.int32)
    trace = np.zeros(3 * T, np.int64)
    try:
        r = dsg.dsg_run_pruned(ctx, h, variant, T, p, q, loads, bset, trace, c=c)
    finally:
        dsg.dsg_free_graph(h)
    o = orc.run_pruned(g, variant, T, p, q, c=c)
    assert (r["best_edges"], r["best_vertices"], r["best_iter"]) == (o.best_edges, o.best_vertices, o.best_iter)
    assert np.array_equal(bset[:r["best_set_size"]].astype(np.int64), o.best_set)
    assert np.array_equal(loads, o.loads)
    assert np.array_equal(trace.reshape(T, 3), o.trace)
    assert (r["k_max"], r["core_vertices"], r["core_edges"], r["final_vertices"]) == \
        (o.k_max, o.core_vertices, o.core_edges, o.final_vertices)
    assert (r["L_num"], r["L_den"]) == o.L


def test_apx_large(dsg, ctx):
    """R-MAT 18: the approximate decomposition and the approximately pruned
    PaRSorting++ run (whole-GPU k-core peels on the larger cores)."""
    g = gg.rmat(18, 16, 5)
    T = 4
    h = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj, 0)
    loads = np.zeros(g.n, np.int64)
    bset = np.zeros(g.n, np.int32)
    try:
        core, khat = dsg.dsg_apx_coreness(ctx, h, (3, 2))
        r = dsg.dsg_run_pruned(ctx, h, 0, T, 0, 1, loads, bset, None, c=(3, 2))
    finally:
        dsg.dsg_free_graph(h)
    exp = orc.apx_coreness(g, (3, 2))
    assert np.array_equal(core.astype(np.int64), exp) and khat == int(exp.max())
    o = orc.run_pruned(g, 0, T, c=(3, 2))
    assert (r["best_edges"], r["best_vertices"], r["best_iter"]) == (o.best_edges, o.best_vertices, o.best_iter)
    assert np.array_equal(bset[:r["best_set_size"]].astype(np.int64), o.best_set)
    assert np.array_equal(loads, o.loads)
    assert (r["k_max"], r["core_vertices"], r["final_vertices"]) == (o.k_max, o.core_vertices, o.final_vertices)


def test_apx_invalid(dsg, ctx):
    g = gg.complete(5)
    h = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj, 0)
    try:
        for c in [(1, 1), (2, 3), (3, 0), (1 << 31, 2)]:
            with pytest.raises(dsg.DsgError, match="INVALID"):
                dsg.dsg_apx_coreness(ctx, h, c)
            with pytest.raises(dsg.DsgError, match="INVALID"):
                dsg.dsg_run_pruned(ctx, h, 0, 2, c=c)
        with pytest.raises(dsg.DsgError, match="INVALID"):
            dsg.dsg_run_pruned(ctx, h, 0, 2, c=(0, 1))
    finally:
        dsg.dsg_free_graph(h)


@pytest.mark.parametrize("name", list(_graphs()))
@pytest.mark.parametrize("variant,p,q,T,c", [(1, 1, 10, 6, (3, 2)), (1, 1, 100, 4, (2, 1)), (0, 0, 1, 6, (3, 2)),
                                             (1, 0, 1, 4, (5, 4))])
def test_apx_exact_pruned_run(dsg, ctx, name, variant, p, q, T, c):
    """PaRApxGreedy++'s pruning (approximate, then exact): every output equals
    the oracle's run of that reading (which equals exact pruning)."""
    g = _graphs()[name]
    h = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj, 0)
    loads = np.zeros(g.n, np.int64)
    bset = np.zeros(g.n, np.int32)
    trace = np.zeros(3 * T, np.int64)
    try:
        r = dsg.dsg_run_pruned_apx_exact(ctx, h, variant, T, p, q, c[0], c[1], loads, bset, trace)
    finally:
        dsg.dsg_free_graph(h)
    o, _, _, _ = orc.run_pruned_apx_exact(g, variant, T, p, q, c)
    assert (r["best_edges"], r["best_vertices"], r["best_iter"]) == (o.best_edges, o.best_vertices, o.best_iter)
    assert np.array_equal(bset[:r["best_set_size"]].astype(np.int64), o.best_set)
    assert np.array_equal(loads, o.loads)
    assert np.array_equal(trace.reshape(T, 3), o.trace)
    assert (r["k_max"], r["core_vertices"], r["core_edges"], r["final_vertices"]) == \
        (o.k_max, o.core_vertices, o.core_edges, o.final_vertices)
    assert (r["L_num"], r["L_den"]) == o.L


def test_apx_exact_large(dsg, ctx):
    """R-MAT 18, PaRApxGreedy++ (eps = 1/10): the exact stage inside the
    approximate bracket on the whole-GPU k-core peels."""
    g = gg.rmat(18, 16, 5)
    T = 3
    h = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj, 0)
    loads = np.zeros(g.n, np.int64)
    bset = np.zeros(g.n, np.int32)
    try:
        r = dsg.dsg_run_pruned_apx_exact(ctx, h, 1, T, 1, 10, 3, 2, loads, bset, None)
    finally:
        dsg.dsg_free_graph(h)
    o, _, _, _ = orc.run_pruned_apx_exact(g, 1, T, 1, 10, (3, 2))
    assert (r["best_edges"], r["best_vertices"], r["best_iter"]) == (o.best_edges, o.best_vertices, o.best_iter)
    assert np.array_equal(bset[:r["best_set_size"]].astype(np.int64), o.best_set)
    assert np.array_equal(loads, o.loads)
    assert (r["k_max"], r["core_vertices"], r["final_vertices"]) == (o.k_max, o.core_vertices, o.final_vertices)
