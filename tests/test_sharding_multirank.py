"""Block-row sharding of one H-matrix (paper Sec. 4.1's split of the block
list between GPUs, generalised to cost-balanced block rows) with two and four
gloo ranks on CPU.  The partition comes from the library's host-only
partitioner; each rank's part of the matrix is the oracle's H-matrix
restricted to the blocks of its rows (the GPU path assembles the same blocks
with hmat_build_tree_part).  Checked: the bounds cut no block row and
balance the estimated cost; x gathered from the ranks' row segments is the
whole x; the rows of y gathered from the ranks equal the one-rank product."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_1711_01897_gb300 import bem, meshes, sharding  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    V, T = meshes.icosphere_level(3)
    V = meshes.jitter(V, T, 0.05, 77)
    ct = oracle.cluster_tree(V, T, 32)
    blocks = oracle.block_list(ct, oracle.block_tree(ct, 1.2))
    return V, T, ct.perm, blocks


def _cost(blocks, rows, rank_est=10.0):
    m = blocks[:, 1] - blocks[:, 0]
    n = blocks[:, 3] - blocks[:, 2]
    c = np.where(blocks[:, 4] == 1, (m + n) * rank_est, m * n).astype(float)
    inside = (blocks[:, 0] >= rows[0]) & (blocks[:, 1] <= rows[1])
    return c[inside].sum()


def _part_matvec(hm, ids, x):
    """The oracle H-matrix product over the blocks `ids` only (in block
    order, as the oracle's own product sums them)."""
    xt = x[hm.perm]
    yt = np.zeros(hm.n, dtype=np.complex128)
    for b in ids:
        tb, te, sb, se, adm = hm.blocks[b]
        if adm:
            U, Vv = hm.far[b]
            if U.shape[1]:
                yt[tb:te] += U @ (Vv.T @ xt[sb:se])
        else:
            yt[tb:te] += hm.near[b] @ xt[sb:se]
    y = np.zeros_like(yt)
    y[hm.perm] = yt
    return y


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bem.load()
        V, T, perm, blocks = _problem()
        n = T.shape[0]
        bounds = sharding.part_bounds(blocks, n, world)
        rb, re = int(bounds[rank]), int(bounds[rank + 1])
        mine = np.nonzero((blocks[:, 0] >= rb) & (blocks[:, 1] <= re))[0]
        hm = oracle.hmat_assemble(V, T, oracle.SLP, 0.0, 32, 1.2, 1e-4, block_ids=mine, nthreads=1)
        x = np.random.default_rng(3).normal(size=n)
        # each rank holds only its rows of x (cluster order); gather the rest
        xc = torch.from_numpy(sharding.to_cluster_order(x, perm)[rb:re].copy())
        x_full = sharding.from_cluster_order(sharding.gather_segments(xc, bounds, dist).numpy(), perm)
        y = _part_matvec(hm, mine, x_full).real
        yc = torch.from_numpy(sharding.to_cluster_order(y, perm)[rb:re].copy())
        y_full = sharding.from_cluster_order(sharding.gather_segments(yc, bounds, dist).numpy(), perm)
        # rows outside the part are untouched by its blocks
        outside = np.ones(n, bool)
        outside[perm[rb:re]] = False
        q.put((rank, bounds.tolist(), np.array_equal(x_full, x), y_full, float(np.abs(y[outside]).max(initial=0.0))))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_block_row_sharding_gloo(world):
    V, T, perm, blocks = _problem()
    n = T.shape[0]
    bounds = bem.bem_partition_rows(blocks, n, world)
    assert bounds[0] == 0 and bounds[-1] == n and np.all(np.diff(bounds) >= 0)
    for r in bounds[1:-1]:                       # no block row is cut
        assert not np.any((blocks[:, 0] < r) & (r < blocks[:, 1]))
    costs = [_cost(blocks, (bounds[p], bounds[p + 1])) for p in range(world)]
    total = _cost(blocks, (0, n))
    assert abs(sum(costs) - total) < 1e-6 * total   # every block in exactly one part
    assert max(costs) < 1.5 * total / world, costs

    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    got = sorted((q.get() for _ in range(world)), key=lambda t: t[0])
    full = oracle.hmat_assemble(V, T, oracle.SLP, 0.0, 32, 1.2, 1e-4, nthreads=1)
    x = np.random.default_rng(3).normal(size=n)
    y_ref = full.matvec(x).real
    for rank, b, x_ok, y_full, out_max in got:
        assert b == bounds.tolist()
        assert x_ok
        assert out_max == 0.0
        assert np.allclose(y_full, y_ref, rtol=0, atol=1e-14 * np.abs(y_ref).max())


def test_partition_edge_cases():
    V, T, perm, blocks = _problem()
    n = T.shape[0]
    one = bem.bem_partition_rows(blocks, n, 1)
    assert one.tolist() == [0, n]
    # more parts than block rows: some parts are empty, the bounds stay valid
    many = bem.bem_partition_rows(blocks, n, 200)
    assert many[0] == 0 and many[-1] == n and np.all(np.diff(many) >= 0)
    with pytest.raises(bem.BemError):
        bem.bem_partition_rows(blocks, n - 1, 2)      # a block outside the rows
