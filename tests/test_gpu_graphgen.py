"""The GPU R-MAT generator builds exactly the CSR of the CPU generator."""
import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scale,ef,blocks", [(12, 16, None), (14, 8, [30, 60, 90])])
def test_gpu_generator_matches_cpu(scale, ef, blocks):
    cpu = gg.rmat(scale, ef, 3, blocks=blocks)
    n, off, adj = gg.rmat_cuda(scale, ef, 3, blocks=blocks, chunk_arcs=1 << 12)
    assert n == cpu.n
    assert np.array_equal(off.cpu().numpy(), cpu.off)
    assert np.array_equal(adj.cpu().numpy(), cpu.adj)
