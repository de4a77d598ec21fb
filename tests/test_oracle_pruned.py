"""Pins of the oracle's Pruning-and-Refining run (Alg. 1, exact pruning).

They check it against what Sec. 2.1 and Alg. 1 (Sec. 3) fix: the ceil(k_max/2)-core keeps the
densest subgraph (Lemma on cores and Corollary on k_max, via exact max-flow
on both graphs), the closed forms of graphs the pruning leaves whole or cuts
to a clique, the lower bound rho >= k_max/2, the self-consistency of the
returned set, and the size of the final core against the core numbers."""
import numpy as np
import pytest

import graphgen as gg
import oracle as orc


def _induced(g, keep):
    """CSR of the subgraph induced on the vertices with keep[v], relabelled."""
    new = -np.ones(g.n, np.int64)
    new[keep] = np.arange(int(keep.sum()))
    edges = []
    for u in np.flatnonzero(keep):
        for w in g.adj[g.off[u]:g.off[u + 1]]:
            if keep[w] and u < w:
                edges.append((int(new[u]), int(new[w])))
    return gg.from_edges(int(keep.sum()), edges)


def _set_density(g, s):
    inside = np.zeros(g.n, bool)
    inside[s] = True
    e = sum(int(inside[g.adj[g.off[u]:g.off[u + 1]]].sum()) for u in s) // 2
    return e, len(s)


def _gt(a, b):
    return a[0] * b[1] > b[0] * a[1]


def _graphs():
    return [gg.er_planted_clique(),
            gg.disjoint_union(gg.complete(12), gg.er_m(200, 6, 3), gg.star(40)),
            gg.er_m(300, 10, 5),
            gg.chung_lu(400, 12, 2.1, 6),
            gg.rmat(9, 8, 7),
            gg.disjoint_union(gg.er_m(60, 40, 8), gg.er_m(500, 4, 9))]


@pytest.mark.parametrize("gi", range(6))
def test_core_keeps_the_densest_subgraph(gi):
    """rho*(G) = rho*(ceil(k_max/2)-core) by exact max-flow on both."""
    g = _graphs()[gi]
    core = orc.coreness(g)
    kmax = int(core.max())
    keep = core >= (kmax + 1) // 2
    sub = _induced(g, keep)
    assert orc.core_subgraph_size(g, core, (kmax + 1) // 2) == (sub.n, sub.m)
    e1, v1 = orc.maxflow_densest(g)[0]
    e2, v2 = orc.maxflow_densest(sub)[0]
    assert e1 * v2 == e2 * v1


@pytest.mark.parametrize("gi", range(6))
@pytest.mark.parametrize("variant,p,q", [(orc.SORTING, 0, 1), (orc.PEELING, 1, 10)])
def test_bounds_and_consistency(gi, variant, p, q):
    g = _graphs()[gi]
    T = 8
    r = orc.run_pruned(g, variant, T, p, q)
    core = orc.coreness(g)
    kmax = int(core.max())
    assert r.k_max == kmax
    # rho(S) >= rho(first core) >= k_max / 2, and rho(S) <= rho*
    assert 2 * r.best_edges >= kmax * r.best_vertices
    assert (r.core_vertices, r.core_edges) == orc.core_subgraph_size(g, core, (kmax + 1) // 2)
    assert r.best_edges * r.core_vertices >= r.core_edges * r.best_vertices
    e_opt, v_opt = orc.maxflow_densest(g)[0]
    assert r.best_edges * v_opt <= e_opt * r.best_vertices
    # the returned set has the returned density, inside the first core
    assert _set_density(g, r.best_set) == (r.best_edges, r.best_vertices)
    assert np.all(core[r.best_set] >= (kmax + 1) // 2)
    assert np.all(np.diff(r.best_set) > 0)
    # L = max(ceil(k_max/2), rho(S)) once a refine result replaced S (Alg. 1
    # raises L only on an improvement); the final G is the ceil(L)-core
    L = (-(-kmax // 2), 1)
    if r.best_iter > 0 and _gt((r.best_edges, r.best_vertices), L):
        L = (r.best_edges, r.best_vertices)
    assert L[0] * r.L[1] == r.L[0] * L[1]
    lev = -(-r.L[0] // r.L[1])
    assert r.final_vertices == orc.core_subgraph_size(g, core, lev)[0]
    # every iteration ran on a core no larger than the previous one
    assert np.all(np.diff(r.trace[:, 2]) <= 0)
    # the best is the first strict maximum over the iterations' results
    best = (r.core_edges, r.core_vertices)
    it = 0
    for t, (e, v, _) in enumerate(r.trace, 1):
        if _gt((e, v), best):
            best, it = (e, v), t
    assert (best, it) == ((r.best_edges, r.best_vertices), r.best_iter)


@pytest.mark.parametrize("variant,p,q", [(orc.SORTING, 0, 1), (orc.PEELING, 1, 10), (orc.PEELING, 0, 1)])
def test_nothing_pruned_equals_plain_run(variant, p, q):
    """Graphs whose ceil(k_max/2)-core is the whole graph and that no suffix
    can beat (K_n, C_n): the pruned run is the plain run."""
    for g in (gg.complete(25), gg.cycle(40)):
        r = orc.run_pruned(g, variant, 6, p, q)
        o = orc.run(g, variant, 6, p, q)
        assert r.core_vertices == g.n and r.final_vertices == g.n
        assert np.array_equal(r.loads, o.loads)
        assert (r.best_edges, r.best_vertices, r.best_iter) == (g.m, g.n, 0)
        assert np.array_equal(r.trace[:, :2], o.trace[:, :2])


def test_clique_and_star_closed_form():
    """K_6 plus a star: k_max = 5, the 3-core is the K_6 alone; its loads
    follow the K_n closed form, the star's stay 0."""
    g = gg.disjoint_union(gg.complete(6), gg.star(30))
    T = 5
    r = orc.run_pruned(g, orc.SORTING, T)
    assert (r.k_max, r.core_vertices, r.core_edges) == (5, 6, 15)
    assert (r.best_edges, r.best_vertices, r.best_iter) == (15, 6, 0)
    k = np.arange(6)
    exp = ((T - 1) // 2) * 5 + (5 - k) if T % 2 else np.full(6, (T // 2) * 5)
    assert np.array_equal(r.loads[:6], exp)
    assert np.all(r.loads[6:] == 0)


def test_re_pruning_freezes_loads():
    """A dense block (rho above half its core number) next to a sparser one
    inside the first core: once the refine finds the block, L rises above
    the sparser block's core numbers and the re-prune drops it; the vertices
    that leave keep the load they had, the others continue."""
    g = gg.disjoint_union(gg.er_m(60, 40, 8), gg.er_m(150, 20, 9))
    r = orc.run_pruned(g, orc.SORTING, 8)
    assert (r.k_max, r.core_vertices, r.final_vertices) == (24, 203, 60)
    assert (r.best_edges, r.best_vertices) == (875, 60) and r.best_iter > 0
    assert np.array_equal(r.best_set, np.arange(60))
    # the bookkeeping (relabelling, carried and frozen loads, re-pruning)
    # against single plain iterations on the cores it names
    core = orc.coreness(g)
    L, level = (12, 1), 12
    cur = core >= level
    loads = np.zeros(g.n, np.int64)
    S = (int(_induced(g, cur).m), int(cur.sum()))
    for t in range(8):
        ids = np.flatnonzero(cur)
        o = orc.run(_induced(g, cur), orc.SORTING, 1, init_loads=loads[ids])
        loads[ids] = o.loads
        assert tuple(r.trace[t]) == (o.best_edges, o.best_vertices, len(ids))
        if _gt((o.best_edges, o.best_vertices), S):
            S = (o.best_edges, o.best_vertices)
            if _gt(S, L):
                L = S
            if -(-L[0] // L[1]) > level:
                level = -(-L[0] // L[1])
                cur = core >= level
    assert np.array_equal(r.loads, loads)
    assert r.L == L and level == 15
