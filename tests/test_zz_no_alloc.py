"""The allocation-free densest-suffix entry point (dsg_densest_suffix_noalloc)
against the regular entry point dsg_run.

Some callers cannot call cudaMalloc (code running during CUDA-graph capture,
processes confined to a fixed memory arena, callers without a context); this
entry point keeps all its scratch in a static device array instead.  One
PaRSorting++ iteration of dsg_run from loads L gives the loads L + A and, in
its trace, the densest suffix of the (L, id) order; the allocation-free call
on (L, A) must return the same suffix.  Calls follow one another on the same
scratch: different graphs and sizes, load ranges that need one to four radix
passes, a call at the largest accepted n, and a call after sixteen thousand
smaller ones (enough for the radix passes' 16-bit look-back epoch to come
round again), so a word left behind by an earlier call must never be read.
"""
import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2311_04333_gb300 as dsg
    ctx = dsg.dsg_create(0, torch.cuda.current_stream().cuda_stream)
    yield dsg, ctx
    dsg.dsg_destroy(ctx)


class Case:
    """A graph with start loads L, its later-neighbour counts A and the
    densest suffix that dsg_run reports for them."""

    def __init__(self, dsg, ctx, g, L):
        import torch
        gr = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj, dsg.DSG_VALIDATE)
        try:
            loads = np.zeros(g.n, np.int64)
            self.bset = np.zeros(g.n, np.int32)
            self.trace = np.zeros(3, np.int64)
            self.r = dsg.dsg_run(ctx, gr, dsg.DSG_SORTING, 1, 0, 1, L, loads, self.bset, self.trace)
        finally:
            dsg.dsg_free_graph(gr)
        A = loads - L
        assert int(A.sum()) == g.m
        self.g, self.L = g, L
        self.Ld = torch.from_numpy(L.astype(np.uint32).view(np.int32)).cuda()
        self.Ad = torch.from_numpy(A.astype(np.uint32).view(np.int32)).cuda()
        self.res = torch.full((5,), -1, dtype=torch.int64, device="cuda")

    def call(self, dsg, stream):
        dsg.dsg_densest_suffix_noalloc(self.Ld, self.Ad, self.g.n, self.g.m, self.res, stream)

    def check(self):
        import torch
        torch.cuda.synchronize()
        g, L = self.g, self.L
        e, v, pos, key, status = self.res.cpu().tolist()
        assert status == 0
        assert (e, v) == (int(self.trace[0]), int(self.trace[1]))
        assert v == g.n - pos
        order = np.lexsort((np.arange(g.n), L))
        assert key == int(L[order[pos]])
        if self.r["best_iter"] == 1:   # dsg_run replaced S = G by this suffix
            assert np.array_equal(np.sort(order[pos:]), self.bset[: self.r["best_set_size"]])


def _passes(L):
    r = int(L.max() - L.min())
    return max(1, (r.bit_length() + 7) // 8)


def test_noalloc_matches_dsg_run_two_calls(env):
    import torch
    dsg, ctx = env
    rng = np.random.default_rng(5)
    graphs = [gg.er_m(30000, 9, 61), gg.chung_lu(12000, 12, 2.1, 62)]
    loads0 = [rng.integers(0, 50, size=graphs[0].n).astype(np.int64),
              rng.integers(0, 3, size=graphs[1].n).astype(np.int64)]
    stream = torch.cuda.current_stream().cuda_stream
    for g, L in zip(graphs, loads0):
        c = Case(dsg, ctx, g, L)
        c.call(dsg, stream)
        c.check()


def test_noalloc_multipass_and_largest_n(env):
    """One pass, then four passes at the largest accepted n (43 tiles), then
    three and two passes on other sizes, back to back."""
    import torch
    dsg, ctx = env
    rng = np.random.default_rng(7)
    nmax = dsg.DSG_NOALLOC_MAX_VERTICES
    specs = [(gg.er_m(50000, 8, 71), 1 << 6), (gg.er_m(nmax, 8, 72, drop_isolated=False), 1 << 28),
             (gg.chung_lu(200000, 10, 2.1, 73), 1 << 20), (gg.er_m(100000, 6, 74), 1 << 12)]
    stream = torch.cuda.current_stream().cuda_stream
    seen = []
    for g, hi in specs:
        L = rng.integers(0, hi, size=g.n).astype(np.int64)
        seen.append((g.n, _passes(L)))
        c = Case(dsg, ctx, g, L)
        c.call(dsg, stream)
        c.check()
    assert seen[1] == (nmax, 4)
    assert sorted(p for _, p in seen) == [1, 2, 3, 4]


def test_noalloc_after_epoch_wrap(env):
    """A 4-tile call, 16,383 one-tile calls, then a 4-tile call again with new
    loads: the last call's radix passes reuse the look-back epochs of the
    first call's, whose words for tiles 1-3 nothing overwrote in between."""
    import torch
    dsg, ctx = env
    rng = np.random.default_rng(9)
    g = gg.er_m(20000, 8, 81, drop_isolated=False)
    small = gg.er_m(6000, 8, 82, drop_isolated=False)
    stream = torch.cuda.current_stream().cuda_stream
    first = Case(dsg, ctx, g, rng.integers(0, 1 << 16, size=g.n).astype(np.int64))
    filler = Case(dsg, ctx, small, rng.integers(0, 1 << 16, size=small.n).astype(np.int64))
    again = Case(dsg, ctx, g, rng.integers(0, 1 << 16, size=g.n).astype(np.int64))
    first.call(dsg, stream)
    first.check()
    for _ in range(16383):
        filler.call(dsg, stream)
    filler.check()
    again.call(dsg, stream)
    again.check()


def test_noalloc_rejects_bad_sizes(env):
    import torch
    dsg, _ = env
    n = dsg.DSG_NOALLOC_MAX_VERTICES + 1
    x = torch.zeros(n, dtype=torch.int32, device="cuda")
    res = torch.zeros(5, dtype=torch.int64, device="cuda")
    with pytest.raises(dsg.DsgError, match="INVALID"):
        dsg.dsg_densest_suffix_noalloc(x, x, n, 0, res)
    with pytest.raises(dsg.DsgError, match="INVALID"):
        dsg.dsg_densest_suffix_noalloc(x, x, 10, 1 << 48, res)
    with pytest.raises(dsg.DsgError, match="INVALID"):
        dsg.dsg_densest_suffix_noalloc(x, x, 0, 0, res)
