"""Block-row sharding of one H-matrix over the ranks of a torch.distributed
process group.

The paper assembles one H-matrix on two GPUs by dividing its block list
evenly between them (Sec. 4.1).  Here each rank owns whole block rows: the
library cuts the cluster-order rows where no block's rows are cut, balanced
by estimated cost (bem_partition_rows), and each rank assembles only its
part (hmat_build_tree_part).  A product then needs no reduction: the full
x is gathered from the ranks' row segments, each rank applies its part,
and the rows of y are gathered the same way.  Collectives are plain
all_gathers (NCCL on GPUs, gloo on CPU); this module does no arithmetic of
the method.
"""
from __future__ import annotations

import numpy as np


def part_bounds(blocks, n_rows: int, world: int, rank_est: float = 10.0) -> np.ndarray:
    """Cluster-order row bounds [world + 1] of the partition (see
    bem_partition_rows in include/bem.h)."""
    from . import bem
    return bem.bem_partition_rows(blocks, n_rows, world, rank_est)


def gather_segments(local, bounds, dist, group=None):
    """All ranks' row segments of a vector, concatenated in rank order:
    rank r contributes rows [bounds[r], bounds[r + 1]).  `local` is a torch
    tensor (1-D) on the backend's device; the segments are padded to the
    longest one for the all_gather and trimmed after."""
    import torch
    world = len(bounds) - 1
    lens = [int(bounds[r + 1] - bounds[r]) for r in range(world)]
    longest = max(max(lens), 1)
    pad = torch.zeros(longest, dtype=local.dtype, device=local.device)
    pad[:local.numel()] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:n] for p, n in zip(parts, lens)])


def to_cluster_order(v, perm):
    """v (original triangle order) -> cluster order (position p holds
    triangle perm[p])."""
    return v[perm]


def from_cluster_order(vc, perm):
    """Inverse of to_cluster_order."""
    out = vc.new_empty(vc.shape) if hasattr(vc, "new_empty") else np.empty_like(vc)
    out[perm] = vc
    return out
