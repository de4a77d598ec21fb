"""Pins of the CPU oracle against facts that do not come from the oracle.

Each check ties one part of the oracle to something the paper or the
mathematics fixes: closed forms, brute force over all subsets, an exact
max-flow, the textbook k-core, the invariants of Alg. 3 and the ordering
properties of Sec. 3.2 / 3.3.
"""
from fractions import Fraction
from itertools import combinations

import numpy as np
import pytest

import graphgen as gg
import oracle as orc


def _edges(g):
    return [(u, int(w)) for u in range(g.n) for w in g.adj[g.off[u]:g.off[u + 1]] if w > u]


def _random_graph(n, p, seed):
    rng = np.random.default_rng(seed)
    e = [(i, j) for i, j in combinations(range(n), 2) if rng.random() < p]
    return gg.from_edges(n, e)


def _frac(ev):
    return Fraction(ev[0], ev[1])


# ---------------------------------------------------------------- densities

@pytest.mark.parametrize("n", range(2, 9))
def test_brute_force_complete(n):
    # rho(K_n) = (n-1)/2 and K_n itself is the densest subgraph (Sec. 2 definition)
    e, v, mask = orc.brute_force(gg.complete(n))
    assert (e, v) == (n * (n - 1) // 2, n) and mask == (1 << n) - 1


@pytest.mark.parametrize("g,expect", [
    (gg.star(5), (5, 6)), (gg.star(1), (1, 2)),
    (gg.complete_bipartite(3, 4), (12, 7)), (gg.complete_bipartite(2, 5), (10, 7)),
    (gg.cycle(7), (7, 7)), (gg.path(6), (5, 6)),
])
def test_brute_force_closed_forms(g, expect):
    e, v, _ = orc.brute_force(g)
    assert Fraction(e, v) == Fraction(*expect) and (e, v) == expect


def test_brute_force_disjoint_union():
    g = gg.disjoint_union(gg.complete(3), gg.complete(5), gg.cycle(4))
    e, v, mask = orc.brute_force(g)
    assert (e, v) == (10, 5) and mask == 0b11111000


@pytest.mark.parametrize("seed", range(12))
def test_maxflow_matches_brute_force(seed):
    n = 6 + seed % 9
    g = _random_graph(n, [0.2, 0.35, 0.5, 0.7][seed % 4], seed)
    if g.m == 0:
        return
    bf = orc.brute_force(g)
    (e, v), side = orc.maxflow_densest(g)
    assert Fraction(e, v) == Fraction(bf[0], bf[1])
    # the returned set really has that density
    idx = np.flatnonzero(side)
    sub = sum(1 for a, b in _edges(g) if side[a] and side[b])
    assert (sub, len(idx)) == (e, v)


@pytest.mark.parametrize("g,expect", [
    (gg.complete(12), (66, 12)), (gg.complete_bipartite(5, 9), (45, 14)),
    (gg.cycle(40), (40, 40)), (gg.star(30), (30, 31)),
])
def test_maxflow_closed_forms(g, expect):
    assert _frac(orc.maxflow_densest(g)[0]) == Fraction(*expect)


def test_maxflow_planted_clique():
    # a 30-clique (435 edges) in ER(2000, 0.005): rho* >= 435/30 and the
    # min cut certifies it is the optimum
    g = gg.er_planted_clique()
    (e, v), side = orc.maxflow_densest(g)
    assert (e, v) == (435, 30)


# ---------------------------------------------------------------- coreness

@pytest.mark.parametrize("g,expect", [
    (gg.complete(7), 6), (gg.cycle(9), 2), (gg.path(9), 1), (gg.star(8), 1),
])
def test_coreness_closed_forms(g, expect):
    assert (orc.coreness(g) == expect).all()
    assert (orc.coreness_by_deletion(g) == expect).all()


def test_coreness_bipartite():
    g = gg.complete_bipartite(3, 6)
    assert (orc.coreness(g) == 3).all()


@pytest.mark.parametrize("seed", range(8))
def test_coreness_bz_matches_definition(seed):
    g = _random_graph(30 + 5 * seed, 0.15, 100 + seed)
    assert (orc.coreness(g) == orc.coreness_by_deletion(g)).all()


# ---------------------------------------------------------------- orderings

@pytest.mark.parametrize("seed", range(5))
def test_sorting_order_is_load_then_id(seed):
    rng = np.random.default_rng(seed)
    loads = rng.integers(0, 5, size=200)
    order = orc.sorting_order(loads)
    assert list(order) == sorted(range(200), key=lambda v: (int(loads[v]), v))


def _check_iteration(g, order, loads_in, out):
    pos = np.empty(g.n, dtype=np.int64)
    pos[order] = np.arange(g.n)
    # deg*_H(v_j) = number of neighbours later in the order (Alg. 3, counts)
    later = np.zeros(g.n, dtype=np.int64)
    for a, b in _edges(g):
        later[min(pos[a], pos[b])] += 1
    assert (out["degstar"] == later).all()
    assert int(out["degstar"].sum()) == g.m
    # loads: l(v_j) += A[j]  (Alg. 3, load update)
    exp = np.array(loads_in, dtype=np.int64).copy()
    exp[order] += later
    assert (out["loads"] == exp).all()
    # densest suffix by enumeration: B[i] = sum_{j>=i} A[j], rho_i = B[i]/(n-i)
    best, bi = None, -1
    for i in range(g.n):
        r = Fraction(int(later[i:].sum()), g.n - i)
        if best is None or r > best:
            best, bi = r, i
    e, v, p = out["it_best"]
    assert Fraction(e, v) == best and p == bi and v == g.n - bi


@pytest.mark.parametrize("seed", range(6))
def test_iteration_against_enumeration(seed):
    g = _random_graph(40 + 7 * seed, 0.12, 200 + seed)
    rng = np.random.default_rng(seed)
    loads = rng.integers(0, 8, size=g.n)
    order = orc.sorting_order(loads)
    out = orc.iteration(g, order, loads)
    _check_iteration(g, order, loads, out)


@pytest.mark.parametrize("p,q", [(0, 1), (1, 10), (1, 2), (3, 1)])
def test_round_order_rule(p, q):
    """Each round peels exactly {alive v : (l(v)+deg_H(v))*q <= min*(p+q)}
    with deg_H recomputed from the alive set, listed by ascending id."""
    g = _random_graph(60, 0.1, 7)
    rng = np.random.default_rng(3)
    loads = rng.integers(0, 6, size=g.n)
    order, rnd, rmin = orc.round_order(g, loads, p, q)
    assert sorted(order.tolist()) == list(range(g.n))
    alive = set(range(g.n))
    nbr = [set(int(w) for w in g.adj[g.off[u]:g.off[u + 1]]) for u in range(g.n)]
    k = 0
    for r in range(len(rmin)):
        key = {v: int(loads[v]) + len(nbr[v] & alive) for v in alive}
        mn = min(key.values())
        assert mn == rmin[r]
        F = sorted(v for v in alive if key[v] * q <= mn * (p + q))
        assert order[k:k + len(F)].tolist() == F
        assert all(rnd[v] == r for v in F)
        k += len(F)
        alive -= set(F)
    assert k == g.n and not alive
    out = orc.iteration(g, order, loads)
    _check_iteration(g, order, loads, out)


@pytest.mark.parametrize("seed", range(4))
def test_round_order_eps0_gives_coreness(seed):
    """With l = 0 and eps = 0 the running maximum of the round minima is the
    core number of the vertices peeled in that round (Sec. 2, Coreness)."""
    g = _random_graph(80, 0.08 + 0.03 * seed, 300 + seed)
    order, rnd, rmin = orc.round_order(g, np.zeros(g.n, dtype=np.int64), 0, 1)
    run = np.maximum.accumulate(rmin)
    assert (run[rnd] == orc.coreness_by_deletion(g)).all()


@pytest.mark.parametrize("seed", range(3))
def test_round_order_eps0_load_property(seed):
    """Sec. 3.3: i < j implies l(v_i) <= l(v_j) + Delta for the round order."""
    g = _random_graph(70, 0.1, 400 + seed)
    loads = np.random.default_rng(seed).integers(0, 30, size=g.n)
    order, _, _ = orc.round_order(g, loads, 0, 1)
    delta = g.max_degree
    lo = loads[order]
    suffix_min = np.minimum.accumulate(lo[::-1])[::-1]
    assert all(lo[i] <= suffix_min[i + 1] + delta for i in range(g.n - 1))


def test_load_order_first_iteration_is_min_degree_peel():
    """Greedy++ iteration 1 (l = 0) is Charikar's peel: every step removes a
    vertex of minimum current degree (smallest id on ties)."""
    g = _random_graph(50, 0.15, 11)
    order = orc.load_order(g, np.zeros(g.n, dtype=np.int64))
    alive = set(range(g.n))
    nbr = [set(int(w) for w in g.adj[g.off[u]:g.off[u + 1]]) for u in range(g.n)]
    for v in order:
        d = {u: len(nbr[u] & alive) for u in alive}
        mn = min(d.values())
        assert int(v) == min(u for u in alive if d[u] == mn)
        alive.remove(int(v))


# ---------------------------------------------------------------- full runs

@pytest.mark.parametrize("n", [2, 5, 8, 13])
def test_sorting_complete_graph_loads(n):
    """K_n under the load sort with id ties: after odd t,
    l(k) = ((t-1)/2)(n-1) + (n-1-k); after even t, l = (t/2)(n-1).
    The best never beats S = G: (n(n-1)/2, n), iteration 0."""
    g = gg.complete(n)
    for t in range(1, 6):
        r = orc.run(g, orc.SORTING, t)
        k = np.arange(n)
        exp = ((t - 1) // 2) * (n - 1) + (n - 1 - k) if t % 2 else np.full(n, (t // 2) * (n - 1))
        assert (r.loads == exp).all()
        assert (r.best_edges, r.best_vertices, r.best_iter) == (n * (n - 1) // 2, n, 0)
        assert r.best_set.tolist() == list(range(n))


@pytest.mark.parametrize("variant", [orc.SORTING, orc.PEELING, orc.GREEDY])
@pytest.mark.parametrize("seed", range(4))
def test_run_invariants(variant, seed):
    g = _random_graph(16, 0.3, 500 + seed)
    if g.m == 0:
        return
    T = 6
    r = orc.run(g, variant, T, 1, 10)
    # each edge charges exactly one endpoint per iteration
    assert int(r.loads.sum()) == T * g.m
    rho_star = Fraction(*orc.brute_force(g)[:2])
    best = Fraction(r.best_edges, r.best_vertices)
    assert Fraction(g.m, g.n) <= best <= rho_star
    # the best set has exactly the reported density
    s = set(r.best_set.tolist())
    assert len(s) == r.best_vertices
    assert sum(1 for a, b in _edges(g) if a in s and b in s) == r.best_edges
    assert r.best_set.tolist() == sorted(s)
    # trace: every iteration's densest suffix is no better than the best
    for e, v, w in r.trace:
        assert Fraction(int(e), int(v)) <= best and w <= g.max_degree


@pytest.mark.parametrize("seed", range(5))
def test_first_iteration_two_approximation(seed):
    """Iteration 1 of Greedy++ and of the eps = 0 round peel are 2-approximate
    (Charikar; Sec. 3.2), and the eps > 0 round peel is 2(1+eps)-approximate."""
    g = _random_graph(18, 0.25 + 0.05 * seed, 600 + seed)
    if g.m == 0:
        return
    rho = Fraction(*orc.brute_force(g)[:2])
    for variant, p, q, bound in [(orc.GREEDY, 0, 1, 2), (orc.PEELING, 0, 1, 2),
                                 (orc.PEELING, 1, 10, Fraction(22, 10))]:
        r = orc.run(g, variant, 1, p, q)
        assert Fraction(r.best_edges, r.best_vertices) * bound >= rho


def test_resume_equals_one_run():
    g = gg.er_planted_clique(n=300, p=(3, 100), k=12, seed=9)
    for variant in (orc.SORTING, orc.PEELING):
        full = orc.run(g, variant, 7, 1, 10)
        a = orc.run(g, variant, 3, 1, 10)
        b = orc.run(g, variant, 4, 1, 10, init_loads=a.loads)
        assert (b.loads == full.loads).all()
        assert (np.concatenate([a.trace, b.trace]) == full.trace).all()


def test_disjoint_union_finds_larger_clique():
    # K_5 on ids 0..4, K_10 on ids 5..14: iteration 1 of the sort peels by id,
    # so the suffix after the K_5 is the K_10 (density 4.5 > 55/15)
    g = gg.disjoint_union(gg.complete(5), gg.complete(10))
    r = orc.run(g, orc.SORTING, 1)
    assert (r.best_edges, r.best_vertices, r.best_iter) == (45, 10, 1)
    assert r.best_set.tolist() == list(range(5, 15))


@pytest.mark.parametrize("variant", [orc.SORTING, orc.PEELING])
def test_planted_clique_config(variant):
    """ER(2000, 0.005) + K_30, eps = 1/10, T = 10: the result never exceeds
    rho* = 435/30 (max-flow) and stays within 2x of it from iteration 1."""
    g = gg.er_planted_clique()
    r = orc.run(g, variant, 10, 1, 10)
    best = Fraction(r.best_edges, r.best_vertices)
    assert best <= Fraction(435, 30) and 2 * best >= Fraction(435, 30)
    assert int(r.loads.sum()) == 10 * g.m


def test_iteration_ties_keep_first_suffix():
    """K_4 + K_4 in id order: the whole graph (12/8) and the second K_4 (6/4)
    tie at 3/2; the iteration's densest suffix is the first one (position 0),
    and the running best S = G is not replaced (strict comparison, Alg. 2)."""
    g = gg.disjoint_union(gg.complete(4), gg.complete(4))
    loads = np.zeros(g.n, dtype=np.int64)
    order = orc.sorting_order(loads)
    out = orc.iteration(g, order, loads)
    _check_iteration(g, order, loads, out)
    assert out["it_best"] == (12, 8, 0) and out["improved_at"] == -1
    r = orc.run(g, orc.SORTING, 1)
    assert (r.best_edges, r.best_vertices, r.best_iter) == (12, 8, 0)
