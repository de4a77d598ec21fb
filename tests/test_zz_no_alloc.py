"""The allocation-free densest-suffix entry point (dsg_densest_suffix_noalloc)
against the regular entry point dsg_run.

Some callers cannot call cudaMalloc (code running during CUDA-graph capture,
processes confined to a fixed memory arena, callers without a context); this
entry point keeps all its scratch in a static device array instead.  One
PaRSorting++ iteration of dsg_run from loads L gives the loads L + A and, in
its trace, the densest suffix of the (L, id) order; the allocation-free call
on (L, A) must return the same suffix.  Two calls in a row, on different
graphs and sizes, check that the shared scratch is reset between calls.
"""
import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu


def _case(dsg, ctx, g, L):
    import torch
    gr = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj, dsg.DSG_VALIDATE)
    try:
        loads = np.zeros(g.n, np.int64)
        bset = np.zeros(g.n, np.int32)
        trace = np.zeros(3, np.int64)
        r = dsg.dsg_run(ctx, gr, dsg.DSG_SORTING, 1, 0, 1, L, loads, bset, trace)
    finally:
        dsg.dsg_free_graph(gr)
    A = loads - L
    assert int(A.sum()) == g.m
    Ld = torch.from_numpy(L.astype(np.uint32).view(np.int32)).cuda()
    Ad = torch.from_numpy(A.astype(np.uint32).view(np.int32)).cuda()
    res = torch.full((5,), -1, dtype=torch.int64, device="cuda")
    return r, trace, bset, Ld, Ad, res


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2311_04333_gb300 as dsg
    ctx = dsg.dsg_create(0, torch.cuda.current_stream().cuda_stream)
    yield dsg, ctx
    dsg.dsg_destroy(ctx)


def test_noalloc_matches_dsg_run_two_calls(env):
    import torch
    dsg, ctx = env
    rng = np.random.default_rng(5)
    graphs = [gg.er_m(30000, 9, 61), gg.chung_lu(12000, 12, 2.1, 62)]
    loads0 = [rng.integers(0, 50, size=graphs[0].n).astype(np.int64),
              rng.integers(0, 3, size=graphs[1].n).astype(np.int64)]
    stream = torch.cuda.current_stream().cuda_stream
    for g, L in zip(graphs, loads0):
        r, trace, bset, Ld, Ad, res = _case(dsg, ctx, g, L)
        dsg.dsg_densest_suffix_noalloc(Ld, Ad, g.n, g.m, res, stream)
        torch.cuda.synchronize()
        e, v, pos, key, status = res.cpu().tolist()
        assert status == 0
        assert (e, v) == (int(trace[0]), int(trace[1]))
        assert v == g.n - pos
        order = np.lexsort((np.arange(g.n), L))
        assert key == int(L[order[pos]])
        if r["best_iter"] == 1:   # dsg_run replaced S = G by this suffix
            assert np.array_equal(np.sort(order[pos:]), bset[: r["best_set_size"]])


def test_noalloc_rejects_oversize(env):
    import torch
    dsg, _ = env
    n = dsg.DSG_NOALLOC_MAX_VERTICES + 1
    x = torch.zeros(n, dtype=torch.int32, device="cuda")
    res = torch.zeros(5, dtype=torch.int64, device="cuda")
    with pytest.raises(dsg.DsgError, match="INVALID"):
        dsg.dsg_densest_suffix_noalloc(x, x, n, 0, res)
