"""Oracle parity at full size, on the whole-GPU path that bench.py times.

The oracle's results for these cases are stored under tests/golden/ by
make_golden_fullsize.py (graphgen and the oracle only; the single-threaded
oracle needs tens of minutes for the benchmarked graph).  Every output is
compared exactly: the final loads, the best density as an (edges, vertices)
pair with its iteration, the best vertex set and the per-iteration trace
(Alg. 2 with the orderings of Sec. 3.3).  The input CSR is compared with the
one the oracle ran on first, so that a generator mismatch is not reported as
a kernel mismatch.

  * cold tier: 12M-vertex random graph, above the 8,388,608 vertices the
    edge scan keeps in its L2 tier, so the plain gather / atomic path of
    the cold targets and about two thousand look-back tiles per radix pass
    are compared with the oracle; PaRSorting++ and PaRGreedy++ (eps = 1/10);
  * the benchmarked R-MAT 27 workload (63.1M vertices, 2.1G edges),
    PaRSorting++, T = 20, generated on the GPU as bench.py does."""
import hashlib
import json
import os
import sys

import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden_fullsize as mg  # noqa: E402


def _stored(name):
    path = os.path.join(HERE, "golden", f"fullsize_{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"{path} not written")
    with open(path) as f:
        return json.load(f)


def _digest_tensor(t, dtype):
    """SHA-256 of a device tensor's values as little-endian `dtype`, copied to
    the host in chunks."""
    h = hashlib.sha256()
    step = 1 << 28
    for s in range(0, t.numel(), step):
        h.update(np.ascontiguousarray(t[s:s + step].cpu().numpy(), dtype=dtype).tobytes())
    return h.hexdigest()


def _compare(r, loads, bset, trace, rec, T):
    got = dict(best=[r["best_edges"], r["best_vertices"], r["best_iter"]],
               best_set_size=r["best_set_size"], trace=trace.reshape(T, 3).tolist(),
               loads_sum=int(loads.sum()), loads_max=int(loads.max()))
    want = {k: rec[k] for k in got}
    assert got == want
    assert mg.digest(loads) == rec["loads_sha256"]
    assert mg.digest(bset[: r["best_set_size"]]) == rec["best_set_sha256"]


@pytest.mark.parametrize("case", ["sorting", "peeling_eps_1_10"])
def test_cold_tier_graph_matches_oracle(case):
    import paper_2311_04333_gb300 as dsg
    stored = _stored("cold_tier")
    c = mg.COLD_TIER
    g = gg.er_m(c["n"], c["avg_degree"], c["seed"])
    assert (g.n, g.m) == (stored["graph"]["n"], stored["graph"]["m"])
    assert mg.digest(g.off) == stored["graph"]["offsets_sha256"]
    assert mg.digest(g.adj, "<i4") == stored["graph"]["adjacency_sha256"]
    assert g.n > 8_388_608
    rec = stored[case]
    ctx = dsg.dsg_create(0)
    gr = dsg.dsg_upload_csr(ctx, g.n, g.off, g.adj)
    try:
        T = rec["T"]
        loads = np.zeros(g.n, dtype=np.int64)
        bset = np.zeros(g.n, dtype=np.int32)
        trace = np.zeros(3 * T, dtype=np.int64)
        r = dsg.dsg_run(ctx, gr, rec["variant"], T, rec["p"], rec["q"], None, loads, bset, trace,
                        dsg.DSG_PATH_GRID)
        _compare(r, loads, bset, trace, rec, T)
    finally:
        dsg.dsg_free_graph(gr)
        dsg.dsg_destroy(ctx)


def test_benchmarked_rmat27_T20_matches_oracle():
    import torch
    import paper_2311_04333_gb300 as dsg
    stored = _stored("rmat27")
    c = mg.RMAT27
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    ctx = dsg.dsg_create(0, torch.cuda.current_stream().cuda_stream)
    n, off, adj = gg.rmat_cuda(c["scale"], c["edge_factor"], c["seed"], blocks=c["blocks"])
    assert (n, int(off[-1]) // 2) == (stored["graph"]["n"], stored["graph"]["m"])
    assert _digest_tensor(off, "<i8") == stored["graph"]["offsets_sha256"]
    assert _digest_tensor(adj, "<i4") == stored["graph"]["adjacency_sha256"]
    g = dsg.dsg_upload_csr(ctx, n, off, adj, dsg.DSG_SRC_DEVICE)
    del off, adj
    try:
        rec = stored["sorting"]
        T = rec["T"]
        loads = torch.empty(n, dtype=torch.int64, device=dev)
        bset = torch.empty(n, dtype=torch.int32, device=dev)
        trace = torch.empty(3 * T, dtype=torch.int64, device=dev)
        r = dsg.dsg_run(ctx, g, dsg.DSG_SORTING, T, 0, 1, None, loads, bset, trace, dsg.DSG_PATH_GRID)
        _compare(r, loads.cpu().numpy(), bset.cpu().numpy(), trace.cpu().numpy(), rec, T)
    finally:
        dsg.dsg_free_graph(g)
        dsg.dsg_destroy(ctx)


@pytest.mark.parametrize("shift", [0, 1], ids=["aligned", "misaligned"])
def test_cold_tier_from_pinned_host_memory(shift):
    """The same graph uploaded from pinned (page-locked) host buffers, which
    the SMs copy in chunks; `shift` offsets the adjacency by one word inside
    its buffer so that host and device addresses differ mod 16 (word copies).
    The loads and the best set come back into pinned buffers, which the
    kernels write directly."""
    import torch
    import paper_2311_04333_gb300 as dsg
    stored = _stored("cold_tier")
    c = mg.COLD_TIER
    g = gg.er_m(c["n"], c["avg_degree"], c["seed"])
    off_h = torch.from_numpy(g.off).pin_memory()
    buf = torch.empty(g.adj.size + shift, dtype=torch.int32).pin_memory()
    adj_h = buf[shift:]
    adj_h.copy_(torch.from_numpy(g.adj))
    rec = stored["sorting"]
    ctx = dsg.dsg_create(0)
    gr = dsg.dsg_upload_csr(ctx, g.n, off_h.numpy(), adj_h.numpy())
    try:
        T = rec["T"]
        loads = torch.full((g.n,), -1, dtype=torch.int64).pin_memory().numpy()
        bset = torch.full((g.n,), -1, dtype=torch.int32).pin_memory().numpy()
        trace = np.zeros(3 * T, dtype=np.int64)
        r = dsg.dsg_run(ctx, gr, 0, T, 0, 1, None, loads, bset, trace, dsg.DSG_PATH_GRID)
        _compare(r, loads, bset, trace, rec, T)
    finally:
        dsg.dsg_free_graph(gr)
        dsg.dsg_destroy(ctx)
