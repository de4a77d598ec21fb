"""Writes the stored expected values under tests/golden/ from the oracle
alone (graphgen builds the inputs; nothing here touches the CUDA library).

The paper prints no worked example with numbers, so these files are not the
paper's values: they freeze the oracle's outputs on the small benchmark
configuration (ER G(2000, 0.005) plus a planted 30-clique, seed 1; T = 10;
PaRSorting++ and PaRGreedy++ with eps = 1/10) and on the approximate and
exact pruned runs, so that any later change to the oracle's arithmetic shows
up as a failing test and has to be justified by the passage it follows.

    python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import graphgen as gg  # noqa: E402
import oracle as orc  # noqa: E402


def _digest(a) -> str:
    import numpy as np
    return hashlib.sha256(np.ascontiguousarray(a, dtype=np.int64).tobytes()).hexdigest()


def records() -> dict:
    g = gg.er_planted_clique()
    out = {"graph": {"recipe": "er_planted_clique(): ER G(2000, 0.005) + planted 30-clique, seed 1",
                     "n": g.n, "m": g.m, "adjacency_sha256": _digest(g.adj)}}
    for name, variant, p, q in (("sorting", orc.SORTING, 0, 1), ("peeling_eps_1_10", orc.PEELING, 1, 10),
                                ("greedy", orc.GREEDY, 0, 1)):
        r = orc.run(g, variant, 10, p, q)
        out[name] = {"T": 10, "p": p, "q": q, "best": [r.best_edges, r.best_vertices, r.best_iter],
                     "best_set": r.best_set.tolist(), "trace": r.trace.tolist(),
                     "loads_sha256": _digest(r.loads), "loads_sum": int(r.loads.sum())}
    for name, c in (("pruned_exact", None), ("pruned_apx_3_2", (3, 2))):
        r = orc.run_pruned(g, orc.SORTING, 10, c=c)
        out[name] = {"T": 10, "best": [r.best_edges, r.best_vertices, r.best_iter], "k_max": r.k_max,
                     "core": [r.core_vertices, r.core_edges], "final_vertices": r.final_vertices,
                     "L": list(r.L), "trace": r.trace.tolist(), "loads_sha256": _digest(r.loads)}
    return out


if __name__ == "__main__":
    path = os.path.join(HERE, "planted_clique_T10.json")
    with open(path, "w") as f:
        json.dump(records(), f, indent=1)
        f.write("\n")
    print(path)
