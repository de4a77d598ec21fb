"""Writes the stored oracle results of the full-size parity cases from the
oracle alone (graphgen builds the inputs on the CPU; nothing here touches the
CUDA library).  The GPU tests run the same seeded recipes through the CUDA
path and compare every output with these records.

Cases:
  * ``cold_tier``: a G(n, M)-style random graph with n = 12,000,000 and
    average degree 6 (seed 6), above the 8,388,608 vertices that the
    whole-GPU edge scan keeps in its L2 tier, so that part of its targets take
    the plain gather-and-atomic path; PaRSorting++ and PaRGreedy++
    (eps = 1/10), T = 4 (Alg. 2 with the orderings of Sec. 3.3);
  * ``rmat27``: the benchmarked workload -- R-MAT scale 27, edge factor 16,
    seed 3, with ten planted G(s, 1/2) blocks of s = 200 .. 2000 vertices --
    PaRSorting++, T = 20.  Its CSR is built bucket by bucket
    (``graphgen.rmat_large``, about 40 GB of host memory) and the oracle runs
    single-threaded (tens of minutes).

Arrays are stored as SHA-256 digests of their little-endian bytes: the
final loads and the best vertex set (ascending ids) as int64, and the CSR
itself (offsets as int64, adjacency as int32), so that a GPU test can also
tell a generator mismatch from a kernel mismatch.

    python tests/golden/make_golden_fullsize.py cold_tier
    python tests/golden/make_golden_fullsize.py rmat27
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import graphgen as gg  # noqa: E402
import oracle as orc  # noqa: E402

COLD_TIER = dict(n=12_000_000, avg_degree=6, seed=6, T=4)
RMAT27 = dict(scale=27, edge_factor=16, seed=3, blocks=[200 * (i + 1) for i in range(10)], T=20)


def digest(a, dtype="<i8") -> str:
    """SHA-256 of the array's bytes as `dtype` (little-endian int64 unless
    stated), hashed in chunks."""
    h = hashlib.sha256()
    a = np.asarray(a)
    step = 1 << 26
    for s in range(0, a.shape[0], step):
        h.update(np.ascontiguousarray(a[s:s + step], dtype=dtype).tobytes())
    return h.hexdigest()


def _log(msg):
    print(f"[{time.strftime('%H:%M:%S')}] {msg}", flush=True)


def _record(g, variant, T, p, q):
    t0 = time.time()
    r = orc.run(g, variant, T, p, q)
    _log(f"oracle variant {variant} T={T}: {time.time() - t0:.1f} s")
    return {"variant": variant, "T": T, "p": p, "q": q,
            "best": [r.best_edges, r.best_vertices, r.best_iter],
            "best_set_size": int(r.best_set.shape[0]), "best_set_sha256": digest(r.best_set),
            "loads_sha256": digest(r.loads), "loads_sum": int(r.loads.sum()),
            "loads_max": int(r.loads.max()), "trace": r.trace.tolist(),
            "oracle_seconds": round(time.time() - t0, 1)}


def _graph_record(g, recipe):
    return {"recipe": recipe, "n": int(g.n), "m": int(g.m),
            "offsets_sha256": digest(g.off), "adjacency_sha256": digest(g.adj, "<i4")}


def cold_tier() -> dict:
    c = COLD_TIER
    g = gg.er_m(c["n"], c["avg_degree"], c["seed"])
    _log(f"graph n={g.n} m={g.m}")
    return {"graph": _graph_record(g, f"graphgen.er_m({c['n']}, {c['avg_degree']}, seed={c['seed']})"),
            "sorting": _record(g, orc.SORTING, c["T"], 0, 1),
            "peeling_eps_1_10": _record(g, orc.PEELING, c["T"], 1, 10)}


def rmat27() -> dict:
    c = RMAT27
    t0 = time.time()
    g = gg.rmat_large(c["scale"], c["edge_factor"], c["seed"], blocks=c["blocks"], log=_log)
    _log(f"graph n={g.n} m={g.m} built in {time.time() - t0:.0f} s")
    rec = {"graph": _graph_record(g, f"graphgen.rmat({c['scale']}, {c['edge_factor']}, seed={c['seed']}, "
                                     f"blocks={c['blocks']})")}
    _log("graph digests done")
    rec["sorting"] = _record(g, orc.SORTING, c["T"], 0, 1)
    return rec


if __name__ == "__main__":
    which = sys.argv[1]
    rec = {"cold_tier": cold_tier, "rmat27": rmat27}[which]()
    path = os.path.join(HERE, f"fullsize_{which}.json")
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    _log(path)
