"""Pins of the oracle's approximate pruning (Sec. 2 definition of a
c-approximate k-core decomposition; Sec. 2.1 corollary on the approximate
k_max; Sec. 4 approximate variants).

They check the decomposition against hand-computed level lists, the
definition's bounds, a direct simulation of threshold peeling, and cores by
repeated deletion; and the pruned run against exact max-flow (the first
approximate core keeps the densest subgraph, the bound L never passes
ceil(rho*)), its own bookkeeping, and the exact variant it reduces to when
the levels are consecutive integers."""
import numpy as np
import pytest

import graphgen as gg
import oracle as orc

# levels tau_0 = 1, tau_{i+1} = ceil(tau_i * c), written out by hand
LEVELS = {
    (3, 2): [1, 2, 3, 5, 8, 12, 18, 27, 41, 62, 93, 140, 210, 315, 473, 710],
    (2, 1): [1, 2, 4, 8, 16, 32, 64, 128, 256],
    (5, 4): [1, 2, 3, 4, 5, 7, 9, 12, 15, 19, 24, 30, 38, 48],
}


def _graphs():
    return [gg.er_planted_clique(),
            gg.disjoint_union(gg.complete(12), gg.er_m(200, 6, 3), gg.star(40)),
            gg.er_m(300, 10, 5),
            gg.chung_lu(400, 12, 2.1, 6),
            gg.rmat(9, 8, 7),
            gg.disjoint_union(gg.er_m(60, 40, 8), gg.er_m(500, 4, 9))]


def _ceil_div(a, b):
    return -(-a // b)


def _set_density(g, s):
    inside = np.zeros(g.n, bool)
    inside[s] = True
    e = sum(int(inside[g.adj[g.off[u]:g.off[u + 1]]].sum()) for u in s) // 2
    return e, len(s)


def _gt(a, b):
    return a[0] * b[1] > b[0] * a[1]


def _threshold_peel(g, levels):
    """The procedure the definition is computed by, simulated directly: at
    level i remove, until none is left, every vertex whose degree among the
    remaining ones is <= tau_i; those removed get tau_i (degree-0 vertices
    of the input get 0)."""
    alive = np.ones(g.n, bool)
    deg = np.diff(g.off).astype(np.int64)
    out = np.zeros(g.n, np.int64)
    zero = deg == 0
    alive[zero] = False
    for tau in levels:
        while True:
            drop = np.flatnonzero(alive & (deg <= tau))
            if drop.size == 0:
                break
            alive[drop] = False
            out[drop] = tau
            for u in drop:
                for w in g.adj[g.off[u]:g.off[u + 1]]:
                    deg[w] -= 1
        if not alive.any():
            break
    assert not alive.any()
    return out


@pytest.mark.parametrize("c", sorted(LEVELS))
def test_levels_on_cliques(c):
    """Every vertex of K_{k+1} has core number k; its approximate core
    number is the smallest level >= k."""
    lev = LEVELS[c]
    for k in range(1, min(lev[-1], 75) + 1):
        a = orc.apx_coreness(gg.complete(k + 1), c)
        assert np.all(a == min(t for t in lev if t >= k)), (c, k)


@pytest.mark.parametrize("gi", range(6))
@pytest.mark.parametrize("c", [(3, 2), (2, 1), (5, 4)])
def test_definition_bounds_and_threshold_peeling(gi, c):
    g = _graphs()[gi]
    k = orc.coreness(g)
    a = orc.apx_coreness(g, c)
    # k / c <= k-hat <= c k (the definition), here with k <= k-hat < c k
    pos = k > 0
    assert np.all(a[~pos] == 0)
    assert np.all(a[pos] >= k[pos])
    assert np.all(a[pos] * c[1] < k[pos] * c[0])
    # exactly what peeling level by level gives
    assert np.array_equal(a, _threshold_peel(g, LEVELS[c]))
    # {k-hat >= tau_{i+1}} is the (tau_i + 1)-core by repeated deletion
    kd = orc.coreness_by_deletion(g)
    lev = LEVELS[c]
    for t0, t1 in zip(lev, lev[1:]):
        assert np.array_equal(a >= t1, kd >= t0 + 1)


@pytest.mark.parametrize("gi", range(6))
@pytest.mark.parametrize("variant,p,q", [(orc.SORTING, 0, 1), (orc.PEELING, 1, 10)])
@pytest.mark.parametrize("c", [(3, 2), (2, 1)])
def test_apx_pruned_bounds_and_consistency(gi, variant, p, q, c):
    g = _graphs()[gi]
    T = 8
    r = orc.run_pruned(g, variant, T, p, q, c=c)
    a = orc.apx_coreness(g, c)
    khat = int(a.max())
    assert r.k_max == khat
    (e_opt, v_opt), mask = orc.maxflow_densest(g)
    # Cor. on the approximate k_max: rho* >= k-hat_max / (2c), so the first
    # approximate core keeps S*, and ceil(L) never passes ceil(rho*)
    assert khat * c[1] * v_opt <= 2 * c[0] * e_opt
    L0 = _ceil_div(khat * c[1], 2 * c[0])
    first = a >= L0
    assert np.all(first[mask])
    assert (r.core_vertices, r.core_edges) == orc.core_subgraph_size(g, a, L0)
    assert _ceil_div(r.L[0], r.L[1]) <= _ceil_div(e_opt, v_opt)
    # rho(S) <= rho*, the set has the returned density, inside the first core
    assert r.best_edges * v_opt <= e_opt * r.best_vertices
    assert _set_density(g, r.best_set) == (r.best_edges, r.best_vertices)
    assert np.all(first[r.best_set]) and np.all(np.diff(r.best_set) > 0)
    # L = max(L0, rho(S)) once a refine result replaced S; the final G keeps
    # {k-hat >= ceil(L)}, and it never grows
    L = (L0, 1)
    if r.best_iter > 0 and _gt((r.best_edges, r.best_vertices), L):
        L = (r.best_edges, r.best_vertices)
    assert L[0] * r.L[1] == r.L[0] * L[1]
    assert r.final_vertices == orc.core_subgraph_size(g, a, _ceil_div(r.L[0], r.L[1]))[0]
    assert np.all(np.diff(r.trace[:, 2]) <= 0)
    best, it = (r.core_edges, r.core_vertices), 0
    for t, (e, v, _) in enumerate(r.trace, 1):
        if _gt((e, v), best):
            best, it = (e, v), t
    assert (best, it) == ((r.best_edges, r.best_vertices), r.best_iter)


@pytest.mark.parametrize("gi", range(6))
@pytest.mark.parametrize("variant,p,q", [(orc.SORTING, 0, 1), (orc.PEELING, 1, 10)])
def test_consecutive_levels_reduce_to_exact_pruning(gi, variant, p, q):
    """With c = (D + 1) / D and D above k_max every level up to k_max is an
    integer step, so k-hat = k, and ceil(k_max D / (2 (D + 1))) = ceil(k_max / 2):
    the approximate run is the exact one."""
    g = _graphs()[gi]
    D = 10 * int(orc.coreness(g).max()) + 10
    r = orc.run_pruned(g, variant, 6, p, q, c=(D + 1, D))
    x = orc.run_pruned(g, variant, 6, p, q)
    assert np.array_equal(orc.apx_coreness(g, (D + 1, D)), orc.coreness(g))
    assert (r.k_max, r.core_vertices, r.core_edges, r.final_vertices, r.L) == \
        (x.k_max, x.core_vertices, x.core_edges, x.final_vertices, x.L)
    assert (r.best_edges, r.best_vertices, r.best_iter) == (x.best_edges, x.best_vertices, x.best_iter)
    assert np.array_equal(r.best_set, x.best_set)
    assert np.array_equal(r.loads, x.loads)
    assert np.array_equal(r.trace, x.trace)


def test_clique_and_star_closed_form():
    """K_6 plus a star, c = 3/2: k-hat = 5 on the K_6 (5 is a level) and 1
    on the star; L = ceil(5 / 3) = 2, so the first approximate core is the
    K_6 alone, as with exact pruning. K_5, c = 3/2: k = 4, k-hat = 5, L =
    ceil(5 / 3) = 2 = ceil(rho*)."""
    g = gg.disjoint_union(gg.complete(6), gg.star(30))
    r = orc.run_pruned(g, orc.SORTING, 5, c=(3, 2))
    assert (r.k_max, r.core_vertices, r.core_edges) == (5, 6, 15)
    assert (r.best_edges, r.best_vertices, r.best_iter) == (15, 6, 0)
    assert np.all(r.loads[6:] == 0)
    r5 = orc.run_pruned(gg.complete(5), orc.SORTING, 3, c=(3, 2))
    assert (r5.k_max, r5.core_vertices, r5.L) == (5, 5, (2, 1))


def test_invalid_c():
    g = gg.complete(4)
    for c in [(1, 1), (2, 3), (3, 0)]:
        with pytest.raises(ValueError):
            orc.apx_coreness(g, c)
        with pytest.raises(ValueError):
            orc.run_pruned(g, orc.SORTING, 1, c=c)


def test_isolated_vertices_get_zero():
    """Core number 0 (no edge) stays 0; K_4's vertices (core 3, a level of
    c = 3/2) get 3; pruning never keeps the isolated vertices."""
    edges = [(u, w) for u in range(4) for w in range(u + 1, 4)]
    g = gg.from_edges(7, edges)
    a = orc.apx_coreness(g, (3, 2))
    assert list(a) == [3, 3, 3, 3, 0, 0, 0]
    assert np.array_equal(a, _threshold_peel(g, LEVELS[(3, 2)]))
    r = orc.run_pruned(g, orc.SORTING, 2, c=(3, 2))
    assert (r.k_max, r.core_vertices, r.core_edges, r.best_edges, r.best_vertices) == (3, 4, 6, 6, 4)
