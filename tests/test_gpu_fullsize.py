"""Parity at full size: the benchmarked workload (R-MAT scale 27, edge
factor 16, seed 3, ten planted G(s, 1/2) blocks of s = 200 .. 2000 vertices;
n = 63.1M, m = 2.1G) on the whole-GPU path that bench.py times.

The oracle cannot run this graph, so every iteration is checked on outputs
that can be recomputed from their definitions (Alg. 3): each edge charges one
endpoint (sum A = m); A[u] of sampled vertices (random ones and the
largest-degree hubs) counted from u's adjacency list on the CPU; the
iteration's densest suffix recomputed from the (load, id) order with a
library sort and prefix sums and compared exactly; and, for the T-iteration
run, the resume property, the best over the iterations (strict, S = G first)
and the best set as the suffix of its iteration's order, with its induced
edge count."""
import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu

SCALE, EDGE_FACTOR, SEED = 27, 16, 3
BLOCKS = [200 * (i + 1) for i in range(10)]


def _sampled_counts(off, adj, loads_cpu, sample):
    """A[u] = #{w in N(u) : (l[w], w) > (l[u], u)} for each sampled u."""
    out = []
    for u in sample:
        s, e = int(off[u]), int(off[u + 1])
        nb = adj[s:e].cpu().numpy().astype(np.int64)
        lw, lu = loads_cpu[nb], loads_cpu[u]
        out.append(int(np.count_nonzero((lw > lu) | ((lw == lu) & (nb > u)))))
    return out


def _densest_suffix(torch, loads, A, n):
    """First maximum of (sum of A over the suffix) / (suffix length) over the
    suffixes of the order by (load, id): (edges, vertices, start, order)."""
    ids = torch.arange(n, device=loads.device, dtype=torch.int64)
    assert int(loads.max()) < (1 << 36) and n < (1 << 27)
    order = torch.sort((loads << 27) | ids).indices
    E = torch.flip(torch.cumsum(torch.flip(A[order], [0]), 0), [0])
    V = n - ids
    r = E.double() / V.double()
    # rounding is monotone: the exact maximum has the largest rounded ratio,
    # and exact ties round alike; the candidates are then compared exactly
    cand = torch.nonzero(r == r.max()).flatten()
    ce, cv, ci = E[cand].tolist(), V[cand].tolist(), cand.tolist()
    b = 0
    for k in range(1, len(ci)):
        if ce[k] * cv[b] > ce[b] * cv[k]:
            b = k
    return ce[b], cv[b], ci[b], order


def _induced_edges(torch, off, adj, vs, n, arcs_per_chunk=1 << 27):
    """Edges of the subgraph induced on the vertex ids vs (int64 tensor),
    over the lists of vs in chunks of about arcs_per_chunk arcs."""
    mask = torch.zeros(n, dtype=torch.bool, device=adj.device)
    mask[vs] = True
    lens_all = (off[vs + 1] - off[vs]).tolist()
    inside, a = 0, 0
    while a < len(lens_all):
        b, tot = a, 0
        while b < len(lens_all) and (b == a or tot + lens_all[b] <= arcs_per_chunk):
            tot += lens_all[b]
            b += 1
        part = vs[a:b]
        s = off[part]
        lens = off[part + 1] - s
        seg = torch.repeat_interleave(torch.arange(part.numel(), device=adj.device), lens)
        starts = torch.cumsum(lens, 0) - lens
        idx = torch.arange(tot, device=adj.device) - starts[seg] + s[seg]
        inside += int(mask[adj[idx].long()].sum())
        a = b
    assert inside % 2 == 0
    return inside // 2


def test_bench_workload_iterations():
    import torch
    import paper_2311_04333_gb300 as dsg
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    ctx = dsg.dsg_create(0, torch.cuda.current_stream().cuda_stream)
    n, off, adj = gg.rmat_cuda(SCALE, EDGE_FACTOR, SEED, blocks=BLOCKS)
    g = dsg.dsg_upload_csr(ctx, n, off, adj, dsg.DSG_SRC_DEVICE)
    try:
        _, m, _ = dsg.dsg_graph_info(g)
        assert m == int(off[-1]) // 2
        T = 3
        rng = np.random.default_rng(11)
        deg = off[1:] - off[:-1]
        sample = sorted(set(rng.integers(0, n, 400).tolist()) | set(torch.topk(deg, 16).indices.tolist()))
        ell = torch.zeros(n, dtype=torch.int64, device=dev)
        traces, suffixes = [], []
        for _ in range(T):
            nxt = torch.empty_like(ell)
            bset = torch.empty(n, dtype=torch.int32, device=dev)
            tr = torch.empty(3, dtype=torch.int64, device=dev)
            dsg.dsg_run(ctx, g, dsg.DSG_SORTING, 1, 0, 1, ell, nxt, bset, tr, dsg.DSG_PATH_GRID)
            A = nxt - ell
            assert int(A.min()) >= 0 and int(A.sum()) == m
            got = A[torch.tensor(sample, device=dev)].tolist()
            assert got == _sampled_counts(off, adj, ell.cpu().numpy(), sample)
            e, v, i, order = _densest_suffix(torch, ell, A, n)
            assert tr.tolist() == [e, v, int(A.max())]
            traces.append((e, v))
            suffixes.append(torch.sort(order[i:]).values)
            del order
            ell = nxt
        # one run of T iterations from zero loads
        loads = torch.empty_like(ell)
        bset = torch.empty(n, dtype=torch.int32, device=dev)
        trace = torch.empty(3 * T, dtype=torch.int64, device=dev)
        r = dsg.dsg_run(ctx, g, dsg.DSG_SORTING, T, 0, 1, None, loads, bset, trace, dsg.DSG_PATH_GRID)
        assert torch.equal(loads, ell)
        assert [tuple(x) for x in trace.view(T, 3)[:, :2].tolist()] == traces
        best, it = (m, n), 0
        for t, (e, v) in enumerate(traces, 1):
            if e * best[1] > best[0] * v:
                best, it = (e, v), t
        assert (r["best_edges"], r["best_vertices"], r["best_iter"]) == (best[0], best[1], it)
        k = r["best_set_size"]
        assert k == best[1]
        got = bset[:k].long()
        if it == 0:
            assert k == n          # S = G was never beaten: the whole graph
        else:
            assert torch.equal(got, suffixes[it - 1])
            assert _induced_edges(torch, off, adj, got, n) == best[0]
    finally:
        dsg.dsg_free_graph(g)
        dsg.dsg_destroy(ctx)
