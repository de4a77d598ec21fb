"""The bucketed CSR build of the R-MAT recipe (graphgen.rmat_large, used to
build the benchmarked scale-27 graph for the oracle in bounded host memory)
gives exactly the CSR of the pair-list build (graphgen.rmat), whatever the
bucket size."""
import numpy as np
import pytest

import graphgen as gg


@pytest.mark.parametrize("scale,ef,blocks,bucket", [(10, 16, None, 1 << 9), (12, 8, [20, 40, 60], 1 << 12),
                                                    (14, 16, [100, 200], 1 << 40), (13, 16, None, 1)])
def test_rmat_large_equals_rmat(scale, ef, blocks, bucket):
    a = gg.rmat(scale, ef, 3, blocks=blocks)
    b = gg.rmat_large(scale, ef, 3, blocks=blocks, bucket_arcs=bucket)
    assert a.n == b.n
    assert np.array_equal(a.off, b.off)
    assert np.array_equal(a.adj, b.adj)
