"""Multi-rank host path on CPU: sources sharded over world_size-2 gloo ranks,
partial BC exchanged in 128-bit fixed point and combined exactly.

Without a GPU the library cannot run, so each rank's partial is the oracle's
BC over its shard, converted to fixed point by the oracle's reference helper
(oracle/fixed.py); the exchange and the reduction's orchestration are the
product's (multirank.allgather_fixed, multirank.reduce_bc), the latter
driving a stand-in handle whose exact add is the reference helper's.
"""
import os
import socket
from fractions import Fraction

import numpy as np
import pytest

from oracle import fixed as fx
from paper_2008_05718_gb300 import graphgen as gg, multirank as mr


def test_shard_covers_sources_once():
    S = np.arange(1001)
    parts = [mr.shard(S, r, 3) for r in range(3)]
    assert np.array_equal(np.concatenate(parts), S)
    assert max(map(len, parts)) - min(map(len, parts)) <= 1


def test_reference_fixed_point_helpers():
    # exact conversions: dyadic values and 1/3 rounded to 53 bits
    x = np.array([0.0, 0.5, 3.0, 1.0 / 3.0, 2.0**40 + 0.25, 2.0**-64, 2.0**-65 * 3], np.float64)
    f = fx.from_double(x)
    ints = fx.to_int(f)
    assert ints[:3] == [0, 1 << 63, 3 << 64]
    assert Fraction(ints[3], 1 << 64) == Fraction(1.0 / 3.0)
    assert ints[4] == (1 << 104) + (1 << 62)
    assert ints[5] == 1 and ints[6] == 2  # 1.5 ulps of 2^-64 rounds to even
    assert np.array_equal(fx.to_double(ints[:5]), x[:5])
    # order-free exact sums, carries into the high word
    r = np.random.default_rng(0)
    parts = [np.stack([r.integers(0, 2**64, 50, dtype=np.uint64), r.integers(0, 2**40, 50, dtype=np.uint64)], 1)
             for _ in range(5)]
    a, b = fx.sum_parts(parts), fx.sum_parts(parts[::-1])
    assert a == b
    assert a == [sum((int(p[i, 1]) << 64) | int(p[i, 0]) for p in parts) for i in range(50)]
    assert np.array_equal(fx.to_int(fx.from_int(a)), a)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _HostHandle:
    """Stand-in for gbbc.BC on the CPU: holds an exact fixed-point BC vector
    and adds partials with the reference helper."""

    def __init__(self, fixed_vec):
        self.n = len(fixed_vec)
        self.vals = fx.to_int(fixed_vec)

    def read_fixed_into(self, out, stream=None):
        out.copy_(__import__("torch").from_numpy(fx.from_int(self.vals).reshape(-1).view(np.int64)))
        return out

    def add_fixed(self, partial, stream=None):
        self.vals = [a + b for a, b in zip(self.vals, fx.to_int(partial.numpy()))]


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = gg.rmat(10, 16, seed=51)
        S = gg.sample_sources(g.n, 120, seed=51)
        part, _ = oracle.bc_graph(g, mr.shard(S, rank, world))
        mine = fx.from_double(part)
        # the exchange step of the product path
        parts = mr.allgather_fixed(torch.from_numpy(mine.reshape(-1).view(np.int64).copy()))
        total = fx.sum_parts([p.numpy() for p in parts])
        # the reduction's orchestration: every rank ends with the full sum
        h = _HostHandle(mine)
        mr.reduce_bc(h, device=torch.device("cpu"))
        q.put((rank, total, h.vals))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce_exactly():
    import multiprocessing as mp
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict((r, (t, v)) for r, t, v in (q.get(timeout=180) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = gg.rmat(10, 16, seed=51)
    S = gg.sample_sources(g.n, 120, seed=51)
    # the same partials summed in one process: identical integers on both ranks
    want_int = fx.sum_parts([fx.from_double(oracle.bc_graph(g, mr.shard(S, r, 2))[0]) for r in range(2)])
    for r in range(2):
        assert got[r][0] == want_int and got[r][1] == want_int
    whole, _ = oracle.bc_graph(g, S)
    assert np.allclose(fx.to_double(want_int), whole, rtol=1e-12, atol=1e-15)
