"""The parallel CPU baseline gives exactly what the oracle gives."""
import numpy as np
import pytest

import cpu_baseline as cb
import graphgen as gg
import oracle as orc


@pytest.mark.parametrize("g", [gg.er_planted_clique(), gg.er_m(5000, 8, 3), gg.chung_lu(4000, 12, 2.1, 5),
                               gg.rmat(12, 8, 7), gg.complete(30), gg.from_edges(1, [])],
                         ids=["planted", "er", "chung_lu", "rmat12", "k30", "single"])
@pytest.mark.parametrize("threads", [1, 4])
def test_matches_oracle(g, threads):
    T = 7
    loads, best = cb.run(g, T, threads)
    o = orc.run(g, orc.SORTING, T)
    assert np.array_equal(loads, o.loads)
    assert best == (o.best_edges, o.best_vertices, o.best_iter)
