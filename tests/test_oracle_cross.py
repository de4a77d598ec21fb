"""A second, independent statement of the refine loop in plain Python
(lists, sets and Fractions; nothing shared with oracle.c), run for several
iterations on small graphs and compared with the C oracle output by output:
final loads, best density, iteration and set, and the per-iteration trace.

It restates Alg. 2 with the three orderings the oracle offers: the load sort
of GreedySorting++ (Sec. 3.2), the simultaneous rounds of ParallelGreedy++
(Sec. 3.3; a round takes every alive v with (l(v) + deg_H(v)) q <= min (p + q),
in ascending id, and its degree decrements land after the round), and
Greedy++'s one-vertex-at-a-time load ordering (Sec. 2)."""
from fractions import Fraction
from itertools import combinations

import numpy as np
import pytest

import graphgen as gg
import oracle as orc


def _lists(g):
    return [sorted(int(w) for w in g.adj[g.off[u]:g.off[u + 1]]) for u in range(g.n)]


def _sorting_order(n, loads):
    return sorted(range(n), key=lambda v: (loads[v], v))


def _round_order(nbrs, loads, p, q):
    alive = set(range(len(nbrs)))
    deg = [len(x) for x in nbrs]
    order = []
    while alive:
        key = {v: loads[v] + deg[v] for v in alive}
        mn = min(key.values())
        F = sorted(v for v in alive if key[v] * q <= mn * (p + q))
        order.extend(F)
        fs = set(F)
        for v in F:
            for w in nbrs[v]:
                if w in alive and w not in fs:
                    deg[w] -= 1
        alive -= fs
    return order


def _greedy_order(nbrs, loads):
    alive = set(range(len(nbrs)))
    deg = [len(x) for x in nbrs]
    order = []
    while alive:
        v = min(alive, key=lambda x: (loads[x] + deg[x], x))
        order.append(v)
        alive.remove(v)
        for w in nbrs[v]:
            if w in alive:
                deg[w] -= 1
    return order


def _py_run(g, variant, T, p, q, init):
    nbrs = _lists(g)
    n, m = g.n, g.m
    loads = [int(x) for x in init]
    best, best_iter, best_set = Fraction(m, n), 0, list(range(n))
    best_ev = (m, n)
    trace = []
    for t in range(1, T + 1):
        if variant == orc.SORTING:
            order = _sorting_order(n, loads)
        elif variant == orc.PEELING:
            order = _round_order(nbrs, loads, p, q)
        else:
            order = _greedy_order(nbrs, loads)
        pos = {v: i for i, v in enumerate(order)}
        # each vertex is charged the neighbours that come after it
        A = [sum(1 for w in nbrs[v] if pos[w] > i) for i, v in enumerate(order)]
        # the iteration's densest suffix: the first maximum going forward
        it, it_ev, it_i = None, None, -1
        edges_left = m
        for i in range(n):
            r = Fraction(edges_left, n - i)
            if it is None or r > it:
                it, it_ev, it_i = r, (edges_left, n - i), i
            edges_left -= A[i]
        trace.append((it_ev[0], it_ev[1], max(A)))
        if it > best:
            best, best_ev, best_iter, best_set = it, it_ev, t, sorted(order[it_i:])
        for i, v in enumerate(order):
            loads[v] += A[i]
    return loads, best_ev, best_iter, best_set, trace


def _random_graph(n, p, seed):
    rng = np.random.default_rng(seed)
    e = [(i, j) for i, j in combinations(range(n), 2) if rng.random() < p]
    return gg.from_edges(n, e)


def _cases():
    return [("er60", _random_graph(60, 0.1, 1)),
            ("er120", _random_graph(120, 0.05, 2)),
            ("dense40", _random_graph(40, 0.4, 3)),
            ("clique_in_sparse", gg.disjoint_union(gg.complete(9), _random_graph(80, 0.04, 4))),
            ("star_cycle", gg.disjoint_union(gg.star(15), gg.cycle(20))),
            ("chung_lu", gg.chung_lu(150, 6, 2.1, 5))]


@pytest.mark.parametrize("ci", range(6))
@pytest.mark.parametrize("variant,p,q", [(orc.SORTING, 0, 1), (orc.PEELING, 0, 1), (orc.PEELING, 1, 10),
                                         (orc.PEELING, 1, 2), (orc.PEELING, 3, 2), (orc.PEELING, 5, 1),
                                         (orc.GREEDY, 0, 1)])
@pytest.mark.parametrize("seeded_init", [False, True])
def test_c_oracle_equals_python_restatement(ci, variant, p, q, seeded_init):
    name, g = _cases()[ci]
    T = 7
    init = np.random.default_rng(ci).integers(0, 9, size=g.n) if seeded_init else np.zeros(g.n, np.int64)
    loads, (be, bv), bit, bset, trace = _py_run(g, variant, T, p, q, init)
    o = orc.run(g, variant, T, p, q, init if seeded_init else None)
    assert np.array_equal(o.loads, np.array(loads, np.int64)), name
    assert (o.best_edges, o.best_vertices, o.best_iter) == (be, bv, bit), name
    assert o.best_set.tolist() == bset, name
    assert o.trace.tolist() == [list(x) for x in trace], name
    # each iteration charges every edge to exactly one endpoint
    assert sum(loads) == sum(int(x) for x in init) + T * g.m


def test_c_oracle_equals_python_restatement_on_random_cases():
    """300 seeded random cases: G(n, p) of 2..69 vertices, T of 1..8, every
    ordering (ParallelGreedy++ rounds at eps = 0, 1/10, 3/2 and 5), zero or
    seeded initial loads."""
    rng = np.random.default_rng(123)
    orders = [(orc.SORTING, 0, 1), (orc.PEELING, 0, 1), (orc.PEELING, 1, 10), (orc.PEELING, 3, 2),
              (orc.PEELING, 5, 1), (orc.GREEDY, 0, 1)]
    for i in range(300):
        n = int(rng.integers(2, 70))
        g = _random_graph(n, float(rng.choice([0.03, 0.08, 0.2, 0.5])), 1000 + i)
        variant, p, q = orders[i % len(orders)]
        T = int(rng.integers(1, 9))
        init = rng.integers(0, 6, size=g.n) if i % 2 else np.zeros(g.n, np.int64)
        loads, (be, bv), bit, bset, trace = _py_run(g, variant, T, p, q, init)
        o = orc.run(g, variant, T, p, q, init if i % 2 else None)
        assert np.array_equal(o.loads, np.array(loads, np.int64)), i
        assert (o.best_edges, o.best_vertices, o.best_iter) == (be, bv, bit), i
        assert o.best_set.tolist() == bset, i
        assert o.trace.tolist() == [list(x) for x in trace], i
