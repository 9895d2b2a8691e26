"""Block-row parts of one H-matrix on the GPU (hmat_build_tree_part), run
one after another on one device: every part's product is zero outside its
rows, the parts' products add up to the product of the whole matrix (each
row from exactly one part, with the same blocks in the same order, so
bitwise), the parts hold every block exactly once, and the whole product
still matches the oracle's dense product."""
import numpy as np
import pytest

import oracle
from paper_1711_01897_gb300 import bem, meshes

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("parts", [2, 3, 4])
@pytest.mark.parametrize("k", [0.0, 2.0])
def test_parts_add_up_to_the_whole(parts, k):
    import torch
    torch.cuda.init()
    V, T = meshes.icosphere_level(4)
    V = meshes.jitter(V, T, 0.05, 88)
    n = T.shape[0]
    m = bem.Mesh(V, T)
    x = np.random.default_rng(4).normal(size=n) + (1j * np.random.default_rng(5).normal(size=n) if k else 0)
    whole = bem.HMatrix(m, 32, 1.2)
    whole.assemble(bem.SLP, k, 1e-5, bem.MIXED)
    y_whole = whole.matvec(x)
    sw = whole.stats()
    blocks, perm = whole.blocks()
    bounds = bem.bem_partition_rows(blocks, n, parts)
    y_sum = np.zeros_like(y_whole)
    nfar = nnear = 0
    for p in range(parts):
        h = bem.HMatrix(m, 32, 1.2, parts=parts, part=p)
        rb, re = h.part_rows()
        assert (rb, re) == (bounds[p], bounds[p + 1])
        h.assemble(bem.SLP, k, 1e-5, bem.MIXED)
        y = h.matvec(x)
        outside = np.ones(n, bool)
        outside[perm[rb:re]] = False
        assert np.all(y[outside] == 0)
        y_sum[~outside] = y[~outside]
        st = h.stats()
        nfar += st["n_blocks_far"]
        nnear += st["n_blocks_near"]
        h.close()
    assert nfar == sw["n_blocks_far"] and nnear == sw["n_blocks_near"]
    assert np.array_equal(y_sum, y_whole)
    rows = np.random.default_rng(6).choice(n, 16, replace=False).astype(np.int32)
    A = oracle.entries(V, T, oracle.SLP, k, rows, np.arange(n, dtype=np.int32))
    if k == 0:
        A = A.real
    assert np.linalg.norm(y_sum[rows] - A @ x) / np.linalg.norm(A @ x) <= 2e-5
