"""Failure detection on the GPU without a GPU fault.

Every device-side wait of the whole-GPU path is bounded: the radix passes'
decoupled look-back and the PaRGreedy++ grid barrier give up after a poll
limit, record DSG_ERR_TIMEOUT and return.  These tests make those waits run
out on purpose through the test-only knobs of dsg_debug_set (a short poll
limit, and a look-back word or a barrier arrival that is withheld, so the
wait is on something nothing sets), check that the run reports
DSG_ERR_TIMEOUT, and then that a normal run on the same context and graph
still matches the oracle output for output.  Host-side failures (an
allocation that reports exhausted memory, an upload copy that fails) are
injected the same way: the call fails with its status, leaves no device
memory of its own behind, and the next call works."""
import numpy as np
import pytest

import graphgen as gg
import oracle as orc

pytestmark = pytest.mark.gpu

SHORT = 4096       # polls before a wait gives up (a few milliseconds)


@pytest.fixture(scope="module")
def dsg():
    import paper_2311_04333_gb300 as m
    return m


@pytest.fixture()
def ctx(dsg):
    import torch
    c = dsg.dsg_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    dsg.dsg_debug_set(None, dsg.DSG_DEBUG_FAIL_ALLOC, 0)
    dsg.dsg_debug_set(None, dsg.DSG_DEBUG_FAIL_UPLOAD, 0)
    dsg.dsg_destroy(c)


@pytest.fixture(scope="module")
def graph():
    return gg.er_m(100_000, 8, 21)


def _pool_used():
    """Bytes in use from device 0's default stream-ordered memory pool (the
    pool the library allocates from), after the device is idle; read through
    the driver API's CU_MEMPOOL_ATTR_USED_MEM_CURRENT (= 7)."""
    import ctypes
    import torch
    torch.cuda.synchronize()
    cu = ctypes.CDLL("libcuda.so.1")
    dev = ctypes.c_int()
    assert cu.cuDeviceGet(ctypes.byref(dev), 0) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    used = ctypes.c_uint64()
    assert cu.cuMemPoolGetAttribute(pool, 7, ctypes.byref(used)) == 0
    return used.value


def _fail_each_allocation(dsg, ctx, call, limit):
    """Makes the 1st, 2nd, ... device allocation of `call` fail until one
    call runs through; each failed call must report DSG_ERR_NOMEM and leave
    the pool as it found it.  Returns (allocations failed, the result)."""
    base = _pool_used()
    for nth in range(1, limit):
        dsg.dsg_debug_set(None, dsg.DSG_DEBUG_FAIL_ALLOC, nth)
        try:
            out = call()
        except dsg.DsgError as ex:
            assert ex.status == dsg.DSG_ERR_NOMEM, (nth, dsg.dsg_last_error(ctx))
            assert _pool_used() == base, (nth, dsg.dsg_last_error(ctx))
            continue
        dsg.dsg_debug_set(None, dsg.DSG_DEBUG_FAIL_ALLOC, 0)
        return nth - 1, out
    raise AssertionError(f"every call up to the {limit}th allocation failed")


def _run(dsg, ctx, gr, g, variant, T, p, q):
    loads = np.zeros(g.n, np.int64)
    bset = np.zeros(g.n, np.int32)
    trace = np.zeros(3 * T, np.int64)
    r = dsg.dsg_run(ctx, gr, variant, T, p, q, None, loads, bset, trace, dsg.DSG_PATH_GRID)
    return r, loads, bset[: r["best_set_size"]], trace.reshape(T, 3)


def _matches_oracle(dsg, ctx, gr, g, variant, T, p, q):
    r, loads, bset, trace = _run(dsg, ctx, gr, g, variant, T, p, q)
    o = orc.run(g, variant, T, p, q)
    assert np.array_equal(loads, o.loads)
    assert (r["best_edges"], r["best_vertices"], r["best_iter"]) == (o.best_edges, o.best_vertices, o.best_iter)
    assert np.array_equal(bset.astype(np.int64), o.best_set)
    assert np.array_equal(trace, o.trace)


@pytest.mark.parametrize("stall,variant", [(1, 0), (1, 1), (2, 1)],
                         ids=["lookback-sorting", "lookback-peeling", "grid-barrier-peeling"])
def test_bounded_wait_runs_out_then_context_still_exact(dsg, ctx, graph, stall, variant):
    g = graph
    p, q = (1, 10) if variant == 1 else (0, 1)
    gr = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj)
    try:
        dsg.dsg_debug_set(ctx, dsg.DSG_DEBUG_SPIN_LIMIT, SHORT)
        dsg.dsg_debug_set(ctx, dsg.DSG_DEBUG_STALL, stall)
        with pytest.raises(dsg.DsgError) as ei:
            _run(dsg, ctx, gr, g, variant, 3, p, q)
        assert ei.value.status == dsg.DSG_ERR_TIMEOUT
        assert "bounded wait" in dsg.dsg_last_error(ctx)
        dsg.dsg_debug_set(ctx, dsg.DSG_DEBUG_STALL, 0)
        dsg.dsg_debug_set(ctx, dsg.DSG_DEBUG_SPIN_LIMIT, 0)
        _matches_oracle(dsg, ctx, gr, g, variant, 3, p, q)
    finally:
        dsg.dsg_free_graph(gr)


def test_short_spin_limit_alone_changes_nothing(dsg, ctx, graph):
    """Without a withheld word the waits end long before even a short limit."""
    g = graph
    gr = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj)
    try:
        dsg.dsg_debug_set(ctx, dsg.DSG_DEBUG_SPIN_LIMIT, 1 << 16)
        _matches_oracle(dsg, ctx, gr, g, 0, 3, 0, 1)
        _matches_oracle(dsg, ctx, gr, g, 1, 2, 1, 10)
    finally:
        dsg.dsg_debug_set(ctx, dsg.DSG_DEBUG_SPIN_LIMIT, 0)
        dsg.dsg_free_graph(gr)


@pytest.mark.parametrize("nth", [1, 2], ids=["offsets", "adjacency"])
def test_upload_allocation_fails_then_works(dsg, ctx, graph, nth):
    g = graph
    dsg.dsg_debug_set(None, dsg.DSG_DEBUG_FAIL_ALLOC, nth)
    with pytest.raises(dsg.DsgError) as ei:
        dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj)
    assert ei.value.status == dsg.DSG_ERR_NOMEM
    gr = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj)
    try:
        _matches_oracle(dsg, ctx, gr, g, 0, 2, 0, 1)
    finally:
        dsg.dsg_free_graph(gr)


def test_run_buffer_allocation_fails_then_works(dsg, ctx, graph):
    g = graph
    gr = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj)
    try:
        dsg.dsg_debug_set(None, dsg.DSG_DEBUG_FAIL_ALLOC, 1)
        with pytest.raises(dsg.DsgError) as ei:
            _run(dsg, ctx, gr, g, 0, 2, 0, 1)
        assert ei.value.status == dsg.DSG_ERR_NOMEM
        _matches_oracle(dsg, ctx, gr, g, 0, 2, 0, 1)
    finally:
        dsg.dsg_free_graph(gr)


def test_each_allocation_of_an_upload_fails_in_turn(dsg, ctx, graph):
    """The copies, the oriented copy with its hub and hot tiers and its
    scratch, and the work schedule: each allocation fails in turn, and each
    such upload returns DSG_ERR_NOMEM with every buffer it took freed."""
    g = graph
    dsg.dsg_free_graph(dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj))
    base = _pool_used()
    failed, gr = _fail_each_allocation(dsg, ctx, lambda: dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj), 64)
    assert failed >= 15
    try:
        _matches_oracle(dsg, ctx, gr, g, 0, 2, 0, 1)
    finally:
        dsg.dsg_free_graph(gr)
    assert _pool_used() == base


def test_each_allocation_of_a_first_grid_run_fails_in_turn(dsg, ctx):
    """A compact graph builds its grid path (the oriented copy, its tiers,
    the schedule, the run buffers) on its first grid run.  Each allocation of
    that run fails in turn and the call reports DSG_ERR_NOMEM; what a failed
    call built is either kept by the graph for the next call or freed, so
    once the graph is freed the pool holds what it held before the upload."""
    g = gg.er_m(3_000, 6, 23)            # compact: 3,000 vertices, 18,000 arcs
    gr = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj)
    _run(dsg, ctx, gr, g, 0, 3, 0, 1)
    dsg.dsg_free_graph(gr)
    base = _pool_used()
    gr = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj)
    try:
        failed = 0
        for nth in range(1, 64):
            dsg.dsg_debug_set(None, dsg.DSG_DEBUG_FAIL_ALLOC, nth)
            try:
                out = _run(dsg, ctx, gr, g, 0, 3, 0, 1)
            except dsg.DsgError as ex:
                assert ex.status == dsg.DSG_ERR_NOMEM, (nth, dsg.dsg_last_error(ctx))
                failed += 1
                continue
            break
        dsg.dsg_debug_set(None, dsg.DSG_DEBUG_FAIL_ALLOC, 0)
        assert failed >= 15
        r, loads, bset, trace = out
        o = orc.run(g, 0, 3)
        assert np.array_equal(loads, o.loads)
        assert (r["best_edges"], r["best_vertices"], r["best_iter"]) == (o.best_edges, o.best_vertices, o.best_iter)
        assert np.array_equal(bset.astype(np.int64), o.best_set)
        assert np.array_equal(trace, o.trace)
    finally:
        dsg.dsg_free_graph(gr)
    assert _pool_used() == base


def test_each_allocation_of_a_pruned_run_fails_in_turn(dsg, ctx, graph):
    """Alg. 1 with exact pruning allocates its buffers, each extracted core
    and the refine step's graph: each allocation fails in turn, and each such
    run returns DSG_ERR_NOMEM with every buffer it took freed; then the run
    matches the oracle."""
    g = graph
    T = 3
    gr = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj)

    def run():
        loads = np.zeros(g.n, np.int64)
        bset = np.zeros(g.n, np.int32)
        trace = np.zeros(3 * T, np.int64)
        r = dsg.dsg_run_pruned(ctx, gr, 0, T, 0, 1, loads, bset, trace)
        return r, loads, bset[: r["best_set_size"]], trace.reshape(T, 3)

    try:
        run()       # the graph's own run buffers stay with it from here on
        failed, (r, loads, bset, trace) = _fail_each_allocation(dsg, ctx, run, 400)
        assert failed >= 10
    finally:
        dsg.dsg_free_graph(gr)
    o = orc.run_pruned(g, 0, T)
    assert (r["best_edges"], r["best_vertices"], r["best_iter"]) == (o.best_edges, o.best_vertices, o.best_iter)
    assert np.array_equal(bset.astype(np.int64), o.best_set)
    assert np.array_equal(loads, o.loads)
    assert np.array_equal(trace, o.trace)


@pytest.mark.parametrize("nth", [1, 2], ids=["offsets", "adjacency"])
def test_upload_copy_fails_then_works(dsg, ctx, graph, nth):
    g = graph
    dsg.dsg_debug_set(None, dsg.DSG_DEBUG_FAIL_UPLOAD, nth)
    with pytest.raises(dsg.DsgError) as ei:
        dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj)
    assert ei.value.status == dsg.DSG_ERR_CUDA
    assert "injected upload failure" in dsg.dsg_last_error(ctx)
    gr = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj)
    try:
        _matches_oracle(dsg, ctx, gr, g, 1, 2, 1, 10)
    finally:
        dsg.dsg_free_graph(gr)


def test_batch_upload_copy_fails_then_works(dsg, ctx):
    graphs = [gg.er_m(300 + 50 * i, 6, 30 + i) for i in range(6)]
    dsg.dsg_debug_set(None, dsg.DSG_DEBUG_FAIL_UPLOAD, 1)
    with pytest.raises(dsg.DsgError) as ei:
        dsg.dsg_upload_batch(ctx, [(x.n, x.off, x.adj) for x in graphs], 0)
    assert ei.value.status == dsg.DSG_ERR_CUDA
    b = dsg.dsg_upload_batch(ctx, [(x.n, x.off, x.adj) for x in graphs], 0)
    try:
        best = np.zeros(4 * len(graphs), np.int64)
        dsg.dsg_run_batch(ctx, b, dsg.DSG_SORTING, np.full(len(graphs), 4, np.int32), 0, best)
        for i, x in enumerate(graphs):
            o = orc.run(x, orc.SORTING, 4)
            assert list(best[4 * i: 4 * i + 3]) == [o.best_edges, o.best_vertices, o.best_iter]
    finally:
        dsg.dsg_free_batch(b)


def test_server_request_fails_alone_on_allocation_failure(dsg):
    """A whole-GPU request whose device allocation fails gets DSG_ERR_NOMEM;
    the requests after it are served exactly."""
    import torch
    torch.cuda.init()
    srv = dsg.dsg_server_create(0, 2, 0)
    big = gg.er_m(60_000, 8, 41)           # above the compact size: runs in a slot
    small = gg.er_m(2_000, 6, 42)
    try:
        dsg.dsg_debug_set(None, dsg.DSG_DEBUG_FAIL_ALLOC, 1)
        t0 = dsg.dsg_server_submit(srv, big.n, big.off, big.adj, 0, 4, 0, 1)
        r0 = dsg.dsg_server_wait(srv, t0)
        assert r0["status"] == dsg.DSG_ERR_NOMEM
        dsg.dsg_debug_set(None, dsg.DSG_DEBUG_FAIL_ALLOC, 0)
        for g, variant, p, q in ((big, 0, 0, 1), (small, 1, 1, 10), (big, 1, 1, 100)):
            tk = dsg.dsg_server_submit(srv, g.n, g.off, g.adj, variant, 4, p, q)
            r = dsg.dsg_server_wait(srv, tk)
            o = orc.run(g, variant, 4, p, q)
            assert r["status"] == 0
            assert (r["best_edges"], r["best_vertices"], r["best_iter"]) == (o.best_edges, o.best_vertices, o.best_iter)
    finally:
        dsg.dsg_debug_set(None, dsg.DSG_DEBUG_FAIL_ALLOC, 0)
        dsg.dsg_server_destroy(srv)
