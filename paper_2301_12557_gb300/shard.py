"""Multi-GPU helpers: one process per GPU, block shards, one histogram sum.

The count of one catalogue splits into independent i-blocks; rank r of N
counts the blocks with index % N == r (``pc_opts.shard_index/shard_count``),
and the int64 histograms of all ranks sum to the full count exactly.  This is
the distributed design of Sect. 4.3: no communication while counting, one
gather of the histograms at the end.  Independent catalogues (mocks) need no
collective at all: each rank counts its own.
"""

from __future__ import annotations

import numpy as np


def shard_opts(opts, rank: int, world: int):
    """Set the shard fields of a pc_opts for this rank (no-op for world 1)."""
    if world > 1:
        opts.shard_index = int(rank)
        opts.shard_count = int(world)
    return opts


def shard_units(n_units: int, rank: int, world: int) -> list[int]:
    """Round-robin assignment of independent units (e.g. mocks) to ranks."""
    return list(range(rank, int(n_units), int(world)))


def sum_histograms(counts, group=None):
    """Sum int64 (or float64) histograms over all ranks of torch.distributed.

    Works with the gloo backend on CPU tensors/arrays and with NCCL on CUDA
    tensors.  Integer sums are exact, so sharded totals equal unsharded ones.
    """
    import torch
    import torch.distributed as dist

    is_np = isinstance(counts, np.ndarray)
    t = torch.from_numpy(np.ascontiguousarray(counts)) if is_np else counts
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        t = t.clone()
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.numpy() if is_np else t
