"""Multi-rank host path on CPU: sources sharded over world_size-2 gloo ranks,
partial BC combined exactly in 128-bit fixed point, equal to one run."""
import os
import socket

import numpy as np
import pytest

from paper_2008_05718_gb300 import graphgen as gg, multirank as mr


def test_shard_covers_sources_once():
    S = np.arange(1001)
    parts = [mr.shard(S, r, 3) for r in range(3)]
    assert np.array_equal(np.concatenate(parts), S)
    assert max(map(len, parts)) - min(map(len, parts)) <= 1


def test_fixed_point_sum_is_exact_and_order_free():
    r = np.random.default_rng(0)
    parts = [np.stack([r.integers(0, 2**64, 50, dtype=np.uint64), r.integers(0, 2**40, 50, dtype=np.uint64)], 1)
             for _ in range(5)]
    a = mr.sum_fixed(parts)
    b = mr.sum_fixed(parts[::-1])
    assert np.array_equal(a, b)
    want = [sum((int(p[i, 1]) << 64) | int(p[i, 0]) for p in parts) for i in range(50)]
    assert [(int(a[i, 1]) << 64) | int(a[i, 0]) for i in range(50)] == want
    assert np.allclose(mr.fixed_to_double(a), [w / 2**64 for w in want], rtol=0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = gg.rmat(10, 16, seed=51)
        S = gg.sample_sources(g.n, 120, seed=51)
        mine = mr.shard(S, rank, world)
        part, _ = oracle.bc_graph(g, mine)
        # oracle partials are FP64: exchange them with an ordered sum
        import torch
        t = torch.from_numpy(part)
        parts = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(parts, t)
        total = sum(p.numpy() for p in parts)
        # the exact fixed-point exchange of the product path, on synthetic partials
        fx = np.stack([np.full(g.n, 2**63 + rank, np.uint64), np.full(g.n, rank, np.uint64)], 1)
        fsum = mr.allreduce_fixed(fx)
        if rank == 0:
            q.put((total, fsum[:3].tolist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import multiprocessing as mp
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    total, fsum = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = gg.rmat(10, 16, seed=51)
    S = gg.sample_sources(g.n, 120, seed=51)
    want, _ = oracle.bc_graph(g, S)
    assert np.allclose(total, want, rtol=1e-12, atol=1e-15)
    # (2^63 + 0) + (2^63 + 1) carries into the high word: 1 + (0 + 1 + carry)
    assert fsum[0] == [1, 2]
