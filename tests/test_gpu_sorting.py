"""Parity of the CUDA PaRSorting++ path (through the C ABI) with the oracle.

Every comparison is exact: final loads, best (edges, vertices, iteration),
best vertex set and the per-iteration trace must be identical.  Each test
runs on both execution paths of dsg_run: the whole-GPU kernels and the
single-block kernel (the default for compact graphs).
"""
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


PATHS = {"grid": 0x4, "block": 0x8}
_CUR = {"path": 0x4}
BLOCK_PATH_MAX_N = 300_000      # larger graphs take the block path only in dedicated tests


@pytest.fixture(params=["grid", "block"], autouse=True)
def path(request):
    _CUR["path"] = PATHS[request.param]
    yield _CUR["path"]


def check(dsg, ctx, g, variant=orc.SORTING, T=10, p=1, q=10, init=None):
    if _CUR["path"] == PATHS["block"] and g.n > BLOCK_PATH_MAX_N:
        pytest.skip("single-block path: covered on smaller graphs")
    r = dsg.densest(ctx, g.n, g.off, g.adj, variant, T, (p, q), init, path=_CUR["path"])
    o = orc.run(g, variant, T, p, q, init)
    assert (r.best_edges, r.best_vertices, r.best_iter) == (o.best_edges, o.best_vertices, o.best_iter)
    bad = np.flatnonzero(r.loads != o.loads)
    assert bad.size == 0, f"{bad.size} loads differ, first at {bad[:5]}"
    assert np.array_equal(r.best_set.astype(np.int64), o.best_set)
    assert np.array_equal(r.trace, o.trace)
    return r, o


def test_planted_clique_config(dsg, ctx):
    """ER(2000, 0.005) + K_30, T = 10."""
    g = gg.er_planted_clique()
    r, _ = check(dsg, ctx, g, T=10)
    assert (r.best_edges, r.best_vertices) == (435, 30)


@pytest.mark.parametrize("n,d,seed", [(20000, 8, 1), (9001, 30, 2), (4096, 5, 3), (4097, 3, 4),
                                      (50000, 12, 5)])
def test_random_graphs_several_tiles(dsg, ctx, n, d, seed):
    check(dsg, ctx, gg.er_m(n, d, seed), T=7)


def test_power_law(dsg, ctx):
    check(dsg, ctx, gg.chung_lu(30000, 16, 2.1, 7), T=12)


def test_heavy_vertices(dsg, ctx):
    """Stars of degree > 4096 are processed as heavy chunks."""
    big = gg.star(10000)
    g = gg.disjoint_union(gg.er_m(3000, 10, 9), big, gg.complete(40), gg.star(4096), gg.star(4097))
    check(dsg, ctx, g, T=6)


def test_rmat_small(dsg, ctx):
    check(dsg, ctx, gg.rmat(16, 16, 11), T=10)


def test_complete_graph_closed_form(dsg, ctx):
    n = 300
    g = gg.complete(n)
    for T in (1, 2, 5):
        r, _ = check(dsg, ctx, g, T=T)
        k = np.arange(n)
        exp = ((T - 1) // 2) * (n - 1) + (n - 1 - k) if T % 2 else np.full(n, (T // 2) * (n - 1))
        assert np.array_equal(r.loads, exp)
        assert (r.best_edges, r.best_vertices, r.best_iter) == (n * (n - 1) // 2, n, 0)


def test_single_vertex_and_isolated(dsg, ctx):
    check(dsg, ctx, gg.from_edges(1, []), T=3)
    check(dsg, ctx, gg.from_edges(7, []), T=2)
    # zero-degree vertices interleaved with edges, ragged tail
    g = gg.from_edges(9000, [(i, i + 3) for i in range(0, 8990, 7)])
    check(dsg, ctx, g, T=5)


def test_many_ties_and_large_loads(dsg, ctx):
    g = gg.er_m(12000, 10, 21)
    rng = np.random.default_rng(0)
    init = rng.integers(0, 4, size=g.n).astype(np.int64)          # many ties
    check(dsg, ctx, g, T=4, init=init)
    init = rng.integers(0, 2**31, size=g.n).astype(np.int64)      # four radix passes
    check(dsg, ctx, g, T=4, init=init)


def test_resume_equals_one_run(dsg, ctx, path):
    g = gg.er_m(15000, 9, 31)
    full = dsg.densest(ctx, g.n, g.off, g.adj, dsg.DSG_SORTING, 9, path=path)
    a = dsg.densest(ctx, g.n, g.off, g.adj, dsg.DSG_SORTING, 4, path=path)
    b = dsg.densest(ctx, g.n, g.off, g.adj, dsg.DSG_SORTING, 5, init_loads=a.loads, path=path)
    assert np.array_equal(b.loads, full.loads)
    assert np.array_equal(np.concatenate([a.trace, b.trace]), full.trace)


def test_rmat20_config(dsg, ctx):
    """R-MAT scale 20, edge factor 16, T = 20 (the full second workload)."""
    g = gg.rmat(20, 16, 2)
    check(dsg, ctx, g, T=20)


def test_device_buffers(dsg, ctx, path):
    import torch
    g = gg.er_m(30000, 10, 41)
    off = torch.from_numpy(g.off).cuda()
    adj = torch.from_numpy(g.adj).cuda()
    gr = dsg.dsg_upload_csr(ctx, g.n, off, adj, dsg.DSG_VALIDATE)
    try:
        T = 6
        init = torch.arange(g.n, dtype=torch.int64, device="cuda") % 5
        loads = torch.empty(g.n, dtype=torch.int64, device="cuda")
        bset = torch.empty(g.n, dtype=torch.int32, device="cuda")
        trace = torch.empty(3 * T, dtype=torch.int64, device="cuda")
        r = dsg.dsg_run(ctx, gr, dsg.DSG_SORTING, T, 0, 1, init, loads, bset, trace, path)
    finally:
        dsg.dsg_free_graph(gr)
    o = orc.run(g, orc.SORTING, T, 0, 1, init.cpu().numpy())
    assert np.array_equal(loads.cpu().numpy(), o.loads)
    assert (r["best_edges"], r["best_vertices"], r["best_iter"]) == (o.best_edges, o.best_vertices, o.best_iter)
    assert np.array_equal(bset[: r["best_set_size"]].cpu().numpy().astype(np.int64), o.best_set)
    assert np.array_equal(trace.cpu().numpy().reshape(T, 3), o.trace)


def test_grid_path_of_a_compact_graph_after_an_invalid_upload(dsg, ctx):
    """A compact graph builds its degree-oriented copy on its first grid run,
    with the adjacency checks of that copy's count pass; flags that an
    invalid graph's upload raised in between belong to that graph alone."""
    g = gg.er_m(2_000, 6, 24)
    gr = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj)
    try:
        with pytest.raises(dsg.DsgError, match="self-loop"):
            dsg.dsg_upload_csr(ctx, 2, np.array([0, 2, 2], np.int64), np.array([0, 1], np.int32), 0)
        T = 3
        loads = np.zeros(g.n, np.int64)
        bset = np.zeros(g.n, np.int32)
        trace = np.zeros(3 * T, np.int64)
        r = dsg.dsg_run(ctx, gr, dsg.DSG_SORTING, T, 0, 1, None, loads, bset, trace, dsg.DSG_PATH_GRID)
    finally:
        dsg.dsg_free_graph(gr)
    o = orc.run(g, orc.SORTING, T)
    assert np.array_equal(loads, o.loads)
    assert (r["best_edges"], r["best_vertices"], r["best_iter"]) == (o.best_edges, o.best_vertices, o.best_iter)
    assert np.array_equal(bset[: r["best_set_size"]].astype(np.int64), o.best_set)
    assert np.array_equal(trace.reshape(T, 3), o.trace)


def test_invalid_inputs(dsg, ctx, path):
    ok = gg.complete(4)
    with pytest.raises(dsg.DsgError, match="INVALID"):
        dsg.dsg_upload_csr(ctx, 0, np.zeros(1, np.int64), np.zeros(0, np.int32))
    # odd arc count
    with pytest.raises(dsg.DsgError, match="even"):
        dsg.dsg_upload_csr(ctx, 2, np.array([0, 1, 1], np.int64), np.array([1], np.int32))
    # asymmetric (0->1, 1->2)
    with pytest.raises(dsg.DsgError, match="symmetric"):
        dsg.dsg_upload_csr(ctx, 3, np.array([0, 1, 2, 2], np.int64), np.array([1, 2], np.int32),
                           dsg.DSG_VALIDATE)
    # self-loop (checked even without DSG_VALIDATE)
    with pytest.raises(dsg.DsgError, match="self-loop"):
        dsg.dsg_upload_csr(ctx, 2, np.array([0, 2, 2], np.int64), np.array([0, 1], np.int32), 0)
    # out of range
    with pytest.raises(dsg.DsgError, match="out of"):
        dsg.dsg_upload_csr(ctx, 2, np.array([0, 1, 2], np.int64), np.array([5, 0], np.int32), 0)
    # duplicate neighbour
    with pytest.raises(dsg.DsgError, match="ascending"):
        dsg.dsg_upload_csr(ctx, 2, np.array([0, 2, 4], np.int64), np.array([1, 1, 0, 0], np.int32),
                           dsg.DSG_VALIDATE)
    g = dsg.dsg_upload_csr(ctx, ok.n, ok.off, ok.adj, dsg.DSG_VALIDATE)
    try:
        with pytest.raises(dsg.DsgError, match="INVALID"):
            dsg.dsg_run(ctx, g, dsg.DSG_SORTING, 0, path=path)
        with pytest.raises(dsg.DsgError, match="INVALID"):
            dsg.dsg_run(ctx, g, 7, 3, path=path)
        with pytest.raises(dsg.DsgError, match="INVALID"):
            dsg.dsg_run(ctx, g, dsg.DSG_SORTING, 3, path=0xC)
        with pytest.raises(dsg.DsgError, match="OVERFLOW"):
            dsg.dsg_run(ctx, g, dsg.DSG_SORTING, 2, init_loads=np.full(4, 2**32 - 3, np.int64), path=path)
        with pytest.raises(dsg.DsgError, match="INVALID"):
            dsg.dsg_run(ctx, g, dsg.DSG_SORTING, 2, init_loads=np.array([0, -1, 0, 0], np.int64), path=path)
        # the context still works after the errors
        r = dsg.dsg_run(ctx, g, dsg.DSG_SORTING, 2, path=path)
        assert (r["best_edges"], r["best_vertices"]) == (6, 4)
    finally:
        dsg.dsg_free_graph(g)


def test_profiling_stats(dsg, ctx, path):
    if path != PATHS["grid"]:
        pytest.skip("phase statistics of the whole-GPU kernels")
    g = gg.er_m(20000, 8, 51)
    dsg.dsg_get_stats(ctx, reset=True)
    dsg.dsg_set_profiling(ctx, True)
    try:
        dsg.densest(ctx, g.n, g.off, g.adj, dsg.DSG_SORTING, 3, path=path)
    finally:
        dsg.dsg_set_profiling(ctx, False)
    st = dsg.dsg_get_stats(ctx, reset=True)
    # two edge-scan launches per iteration (one exits at once), two more with a hot tier
    assert st["edge_scan"]["launches"] in (6, 12) and st["sort"]["launches"] == 15
    assert st["edge_scan"]["ms"] > 0 and st["sort"]["ms"] > 0
    assert st["edge_scan"]["bytes"] == 3 * (8 * g.m + 16 * g.n)


def test_unsorted_adjacency_lists(dsg, ctx, path):
    """Lists need not be sorted without DSG_VALIDATE: the equal-loads shortcut
    (binary search in a sorted list) is then off and the general scan runs."""
    g = gg.er_m(20000, 10, 71)
    rng = np.random.default_rng(1)
    adj = g.adj.copy()
    for u in range(0, g.n, 3):
        a, b = g.off[u], g.off[u + 1]
        adj[a:b] = rng.permutation(adj[a:b])
    gr = dsg.dsg_upload_csr(ctx, g.n, g.off, adj, 0)
    try:
        T = 5
        loads = np.zeros(g.n, np.int64)
        bset = np.zeros(g.n, np.int32)
        trace = np.zeros(3 * T, np.int64)
        r = dsg.dsg_run(ctx, gr, dsg.DSG_SORTING, T, 0, 1, None, loads, bset, trace, path)
    finally:
        dsg.dsg_free_graph(gr)
    o = orc.run(g, orc.SORTING, T)
    assert np.array_equal(loads, o.loads)
    assert (r["best_edges"], r["best_vertices"], r["best_iter"]) == (o.best_edges, o.best_vertices, o.best_iter)
    assert np.array_equal(bset[: r["best_set_size"]].astype(np.int64), o.best_set)
    assert np.array_equal(trace.reshape(T, 3), o.trace)


def test_default_path_by_size(dsg, ctx, path):
    """Without a path flag, graphs up to 16,384 vertices take the single-block
    kernel (one launch per run) and larger ones the whole-GPU kernels, which a
    compact upload (up to 32,768 vertices) builds on first use."""
    if path != PATHS["grid"]:
        pytest.skip("checked once")
    cases = [(gg.er_m(10000, 8, 3), orc.SORTING, True), (gg.er_m(20000, 8, 3), orc.SORTING, False),
             (gg.er_m(10000, 8, 3), orc.PEELING, True), (gg.er_m(20000, 8, 3), orc.PEELING, False),
             (gg.er_m(70000, 4, 3), orc.PEELING, False)]
    for g, variant, one_launch in cases:
        gr = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj, 0)
        try:
            dsg.dsg_get_stats(ctx, reset=True)
            r = dsg.dsg_run(ctx, gr, variant, 3, 1, 10)
            st = dsg.dsg_get_stats(ctx, reset=True)
        finally:
            dsg.dsg_free_graph(gr)
        launches = sum(v["launches"] for v in st.values())
        assert (launches == 2) == one_launch, (g.n, variant, launches)   # block path: reset + kernel
        o = orc.run(g, variant, 3, 1, 10)
        assert (r["best_edges"], r["best_vertices"], r["best_iter"]) == (o.best_edges, o.best_vertices, o.best_iter)


def test_block_path_on_a_large_graph(dsg, ctx, path):
    """The single-block kernel forced on a graph above the compact size."""
    if path != PATHS["block"]:
        pytest.skip("checked once")
    check(dsg, ctx, gg.chung_lu(120000, 12, 2.1, 17), orc.SORTING, 4)
    check(dsg, ctx, gg.chung_lu(120000, 12, 2.1, 17), orc.PEELING, 3, 1, 10)


def test_chunked_host_upload(dsg, ctx, path):
    """A host graph of at least 2^24 arcs arrives in vertex-range chunks on a
    copy stream, overlapped with the preparation of the oriented copy; without
    DSG_VALIDATE each chunk's oriented counts start as soon as it is in place
    (with it, after the last chunk: test_rmat20_config)."""
    if path != PATHS["grid"]:
        pytest.skip("checked once")
    g = gg.rmat(20, 16, 2)
    assert 2 * g.m >= 1 << 24
    T = 3
    gr = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj, 0)
    try:
        loads = np.zeros(g.n, np.int64)
        bset = np.zeros(g.n, np.int32)
        r = dsg.dsg_run(ctx, gr, dsg.DSG_SORTING, T, 0, 1, None, loads, bset)
    finally:
        dsg.dsg_free_graph(gr)
    o = orc.run(g, orc.SORTING, T)
    assert (r["best_edges"], r["best_vertices"], r["best_iter"]) == (o.best_edges, o.best_vertices, o.best_iter)
    assert np.array_equal(loads, o.loads)
    assert np.array_equal(bset[: r["best_set_size"]].astype(np.int64), o.best_set)
    # a self-loop in the last chunk is still found
    deg = np.diff(g.off)
    u = int(np.flatnonzero(deg > 0)[-1])
    adj = g.adj.copy()
    adj[g.off[u]] = u
    with pytest.raises(dsg.DsgError, match="INVALID"):
        dsg.dsg_upload_csr(ctx, g.n, g.off, adj, 0)


def test_chunked_upload_of_asymmetric_lists_without_validation(dsg, ctx, path):
    """Without DSG_VALIDATE the lists are taken as given, symmetric or not.
    A host upload in chunks fills the oriented arcs into m slots as the
    chunks land, which is exact for a symmetric graph; here two arcs have no
    reverse and both are kept by the orientation, m + 1 oriented arcs in all,
    so the upload counts and fills again at that size.  The run equals the
    one on the same arrays uploaded from device memory in one pass."""
    if path != PATHS["grid"]:
        pytest.skip("checked once")
    import torch
    g = gg.rmat(20, 16, 2)
    off, adj = g.off.astype(np.int64), g.adj.astype(np.int32)
    deg = np.diff(off)
    a = int(np.argmax(deg))
    nb_a = adj[off[a]:off[a + 1]]
    x = int(nb_a[np.argmin(deg[nb_a])])             # a's neighbour of least degree
    others = np.flatnonzero((deg > 0) & (np.arange(g.n) != a) & (np.arange(g.n) != x))
    b = int(others[np.argmin(deg[others])])         # a vertex of least degree, not next to a
    assert a not in set(adj[off[b]:off[b + 1]].tolist())
    lists = [adj[off[u]:off[u + 1]] for u in range(g.n)]
    lists[a] = lists[a][lists[a] != x]              # x -> a stays, a -> x goes
    lists[b] = np.sort(np.append(lists[b], a))      # b -> a without a -> b
    off2 = np.zeros(g.n + 1, np.int64)
    off2[1:] = np.cumsum([len(l) for l in lists])
    adj2 = np.concatenate(lists).astype(np.int32)
    assert off2[-1] == off[-1] and off2[-1] >= 1 << 24
    T = 3
    outs = []
    for src in ("host", "device"):
        if src == "host":
            gr = dsg.dsg_upload_csr(ctx, g.n, off2, adj2, 0)
        else:
            gr = dsg.dsg_upload_csr(ctx, g.n, torch.from_numpy(off2).cuda(), torch.from_numpy(adj2).cuda(),
                                    dsg.DSG_SRC_DEVICE)
        try:
            loads = np.zeros(g.n, np.int64)
            trace = np.zeros(3 * T, np.int64)
            r = dsg.dsg_run(ctx, gr, dsg.DSG_SORTING, T, 0, 1, None, loads, None, trace)
        finally:
            dsg.dsg_free_graph(gr)
        outs.append(((r["best_edges"], r["best_vertices"], r["best_iter"]), loads, trace))
    assert outs[0][0] == outs[1][0]
    assert np.array_equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][2], outs[1][2])


def test_graphs_of_one_size_back_to_back(dsg, ctx):
    """Graphs of one size, uploaded and freed one after the other, get device
    memory the previous graph just gave back; the look-back words left there
    (whose epochs repeat, since every graph's count restarts) must not be
    taken for the new graph's."""
    for seed in range(6):
        g = gg.er_m(60000, 10, 100 + seed)
        if seed % 2:
            check(dsg, ctx, g, orc.PEELING, T=3, p=1, q=10)
        else:
            check(dsg, ctx, g, orc.SORTING, T=3)
