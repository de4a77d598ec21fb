"""Pins of the oracle's PaRApxGreedy++ pruning (Sec. 4, the approximate
variants: approximate k-core pruning followed by exact k-core pruning),
read as: prune G by the c-approximate decomposition to
G1 = {k-hat >= ceil(k-hat_max / (2c))} (Sec. 2.1, the corollary on the
approximate k_max), then run Alg. 1 with exact pruning on G1.

The paper reports the same approximation ratios for PaRApxGreedy++ as for
PaRGreedy++ (its approximation-ratio tables omit PaRApxGreedy++ for that
reason): under this reading the two give the same outputs, because every
core Alg. 1 takes has order >= ceil(k_max / 2) >= the approximate bound and
lies inside G1 with the same core numbers.  So the run is pinned to the
exact pruned run output for output, and its approximate stage to the
bounds and cores it must respect (by exact max-flow and by Batagelj-Zaversnik
cores of G and of G1)."""
import numpy as np
import pytest

import graphgen as gg
import oracle as orc


def _graphs():
    return [gg.er_planted_clique(),
            gg.disjoint_union(gg.complete(12), gg.er_m(200, 6, 3), gg.star(40)),
            gg.er_m(300, 10, 5),
            gg.chung_lu(400, 12, 2.1, 6),
            gg.rmat(9, 8, 7),
            gg.disjoint_union(gg.er_m(60, 40, 8), gg.er_m(500, 4, 9)),
            gg.rmat(12, 16, 3, blocks=[30, 60]),
            gg.path(50)]


def _same(a, b):
    assert np.array_equal(a.loads, b.loads)
    assert (a.best_edges, a.best_vertices, a.best_iter) == (b.best_edges, b.best_vertices, b.best_iter)
    assert np.array_equal(a.best_set, b.best_set)
    assert np.array_equal(a.trace, b.trace)
    assert (a.k_max, a.core_vertices, a.core_edges, a.final_vertices, a.L) == \
        (b.k_max, b.core_vertices, b.core_edges, b.final_vertices, b.L)


@pytest.mark.parametrize("variant,p,q", [(orc.PEELING, 1, 10), (orc.PEELING, 0, 1), (orc.SORTING, 0, 1)])
@pytest.mark.parametrize("c", [(3, 2), (2, 1), (5, 4)])
def test_equals_exact_pruning(variant, p, q, c):
    for g in _graphs():
        ax, _, _, _ = orc.run_pruned_apx_exact(g, variant, 8, p, q, c)
        _same(ax, orc.run_pruned(g, variant, 8, p, q))


def test_equals_exact_pruning_on_random_graphs():
    """The same equality on 150 seeded random graphs (G(n, p) of 5..90
    vertices, half of them beside a clique of 3..11), T of 1..7, each
    variant and each c in turn; and each run's best set has the reported
    density, at most rho* by exact max-flow."""
    rng = np.random.default_rng(7)
    for i in range(150):
        n = int(rng.integers(5, 90))
        pr = float(rng.choice([0.05, 0.1, 0.3]))
        keep = rng.random((n, n)) < pr
        g = gg.from_edges(n, [(u, w) for u in range(n) for w in range(u + 1, n) if keep[u, w]])
        if rng.random() < 0.5:
            g = gg.disjoint_union(g, gg.complete(int(rng.integers(3, 12))))
        if g.m == 0:
            continue
        variant, p, q = [(orc.SORTING, 0, 1), (orc.PEELING, 1, 10), (orc.PEELING, 0, 1)][i % 3]
        T = int(rng.integers(1, 8))
        ex = orc.run_pruned(g, variant, T, p, q)
        ax, _, _, _ = orc.run_pruned_apx_exact(g, variant, T, p, q, [(3, 2), (2, 1), (5, 4)][i % 3])
        _same(ax, ex)
        s = set(ex.best_set.tolist())
        e_in = sum(1 for u in s for j in range(g.off[u], g.off[u + 1]) if int(g.adj[j]) in s) // 2
        assert (e_in, len(s)) == (ex.best_edges, ex.best_vertices)
        (re, rv), _ = orc.maxflow_densest(g)
        assert ex.best_edges * rv <= re * ex.best_vertices


@pytest.mark.parametrize("c", [(3, 2), (2, 1), (5, 4)])
def test_approximate_stage_bounds(c):
    for g in _graphs():
        _, khat_max, n1, m1 = orc.run_pruned_apx_exact(g, orc.PEELING, 1, 1, 10, c)
        core = orc.coreness(g)
        kmax = int(core.max())
        # k-hat_max in [k_max, c k_max) (the decomposition's bounds)
        assert kmax <= khat_max and khat_max * c[1] < c[0] * kmax + (kmax == 0) * c[0]
        La = -(-khat_max * c[1] // (2 * c[0]))
        assert La <= -(-kmax // 2)                     # the approximate bound never passes Alg. 1's L
        khat = orc.apx_coreness(g, c)
        assert (n1, m1) == orc.core_subgraph_size(g, khat, La)
        # G1 holds the ceil(k_max/2)-core of G, with the same core numbers there
        n_half, m_half = orc.core_subgraph_size(g, core, -(-kmax // 2))
        assert n1 >= n_half and m1 >= m_half
        keep = np.flatnonzero(khat >= La)
        sub = gg.from_edges(len(keep), _induced_edges(g, keep))
        c1 = orc.coreness(sub)
        hi = core[keep] >= -(-kmax // 2)
        assert np.array_equal(c1[hi], core[keep][hi])
        assert int(c1.max()) == kmax


def _induced_edges(g, keep):
    new = -np.ones(g.n, np.int64)
    new[keep] = np.arange(len(keep))
    out = []
    for u in keep:
        for w in g.adj[g.off[u]:g.off[u + 1]]:
            if w > u and new[w] >= 0:
                out.append((int(new[u]), int(new[w])))
    return out


def test_first_stage_keeps_the_densest_subgraph():
    """By exact max-flow: rho*(G1) = rho*(G) (G1 holds S*)."""
    for g in _graphs()[:6]:
        _, khat_max, n1, _ = orc.run_pruned_apx_exact(g, orc.PEELING, 1, 1, 10, (3, 2))
        khat = orc.apx_coreness(g, (3, 2))
        La = -(-khat_max * 2 // 6)
        keep = np.flatnonzero(khat >= La)
        (e, v), _ = orc.maxflow_densest(g)
        (e1, v1), _ = orc.maxflow_densest(gg.from_edges(len(keep), _induced_edges(g, keep)))
        assert e * v1 == e1 * v


def test_differs_from_approximate_only_pruning():
    """The exact stage matters: pruning by the approximate cores alone gives a
    different first core on some of these graphs (so the pins above would
    catch an implementation that skipped it)."""
    differ = 0
    for g in _graphs():
        ax, _, _, _ = orc.run_pruned_apx_exact(g, orc.PEELING, 4, 1, 10, (3, 2))
        ap = orc.run_pruned(g, orc.PEELING, 4, 1, 10, c=(3, 2))
        differ += (ax.core_vertices, ax.k_max) != (ap.core_vertices, ap.k_max)
    assert differ >= 3
