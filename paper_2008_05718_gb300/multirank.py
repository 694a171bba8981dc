"""Sharding sources over ranks and combining their BC exactly.

Sources are independent (Eq. 2: BC is a sum over sources), so each rank runs
bc_compute on its own share of the source list over its own replica of the
graph, and only the final BC vectors are combined: one exchange step.  The
library keeps BC as 128-bit unsigned fixed point (units 2^-64); each rank
reads its partial in that form into device memory (bc_read_fixed), the
partials are all-gathered over the process group (NCCL between GPUs: each
rank receives copies in its own memory, no peer loads and no multicast), and
each rank adds the other ranks' partials into its handle with bc_add_fixed,
the library's exact integer adds.  Any split of the sources therefore gives
the bits one GPU over all of them would give; bc_read rounds to FP64 once.
"""
from __future__ import annotations

import numpy as np


def shard(sources, rank: int, world: int):
    """Contiguous share of rank `rank` (sizes differ by at most one)."""
    S = np.asarray(sources)
    k = len(S)
    lo = (k * rank) // world
    hi = (k * (rank + 1)) // world
    return S[lo:hi]


def allgather_fixed(local, group=None):
    """Every rank's fixed-point vector (a torch int64 tensor of 2n words,
    on the rank's device for NCCL or on the host for gloo), in rank order."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [torch.empty_like(local) for _ in range(world)]
    dist.all_gather(parts, local.contiguous(), group=group)
    return parts


def reduce_bc(bc, group=None, stream=None, device=None):
    """Add every other rank's partial BC into `bc` (a gbbc.BC handle) so that
    each rank's handle holds the sum over all ranks' sources; returns the
    gathered partials (rank order)."""
    import torch
    import torch.distributed as dist
    rank = dist.get_rank(group)
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    mine = torch.empty(2 * bc.n, dtype=torch.int64, device=dev)
    bc.read_fixed_into(mine, stream=stream)
    parts = allgather_fixed(mine, group)
    for r, p in enumerate(parts):
        if r != rank:
            bc.add_fixed(p, stream=stream)
    return parts
