"""Sharding sources over ranks and combining their BC exactly.

Sources are independent (Eq. 2: BC is a sum over sources), so each rank runs
bc_compute on its own share and only the final BC vectors are combined.  The
library keeps BC as 128-bit unsigned fixed point (units 2^-64, bc_read_fixed);
adding those integers is exact and order-free, so any split of the sources
gives the same bits as one GPU over all of them.  Rounding to FP64 happens
once, after the sum.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1


def shard(sources, rank: int, world: int):
    """Contiguous share of rank `rank` (sizes differ by at most one)."""
    S = np.asarray(sources)
    k = len(S)
    lo = (k * rank) // world
    hi = (k * (rank + 1)) // world
    return S[lo:hi]


def add_fixed(a, b):
    """Exact sum of two [n, 2] uint64 (low, high) fixed-point vectors."""
    a = np.asarray(a, np.uint64)
    b = np.asarray(b, np.uint64)
    lo = a[:, 0] + b[:, 0]
    carry = (lo < a[:, 0]).astype(np.uint64)
    hi = a[:, 1] + b[:, 1] + carry
    return np.stack([lo, hi], axis=1)


def sum_fixed(parts):
    out = np.zeros_like(np.asarray(parts[0], np.uint64))
    for p in parts:
        out = add_fixed(out, p)
    return out


def fixed_to_double(f):
    """Correctly rounded FP64 of 128-bit fixed point (units 2^-64)."""
    f = np.asarray(f, np.uint64)
    return np.array([float((int(h) << 64) | int(l)) / 18446744073709551616.0 for l, h in f], np.float64)


def allreduce_fixed(fixed, group=None):
    """Exact sum over the ranks of a torch.distributed group (any backend):
    gather every rank's vector, add in rank order with carries."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    t = torch.from_numpy(np.ascontiguousarray(fixed, np.uint64).view(np.int64))
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    return sum_fixed([p.numpy().view(np.uint64) for p in parts])
