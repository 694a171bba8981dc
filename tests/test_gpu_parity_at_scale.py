"""GPU parity at full size, in the benchmark's launch configuration.

The CUDA path runs through the C ABI exactly as bench.py runs it (shipped
direction and grouping networks, automatic schedule, the grid schedule's
concurrent batches); the oracle runs over the same sources on every host
core (oracle/pool.py, the unmodified single-threaded oracle per process).
BC must agree within 1e-12 relative with a 1e-15 absolute floor; kept dist,
sigma mod 2^64 and overflow flags bit for bit.

  R-MAT 22: 512 sources of the 16,384-source list (8 batches, so all eight
            concurrent batches of the grid schedule run), and the kept
            state of 4 sources
  the 256-graph mix: every graph, all sources on graphs of at most 4096
            vertices and 16 sources on each larger one
  1024^2 grid: 256 sources (the pair schedule the autotuner picks)
"""
import numpy as np
import pytest

from oracle.pool import OraclePool, map_graphs
from paper_2008_05718_gb300 import graphgen as gg

pytestmark = [pytest.mark.gpu, pytest.mark.scale]

REL, ABS = 1e-12, 1e-15


def assert_bc_close(got, want, what=""):
    excess = np.abs(np.asarray(got) - want) - (REL * np.abs(want) + ABS)
    i = int(np.argmax(excess))
    assert excess[i] <= 0, f"{what} vertex {i}: gpu {got[i]!r} oracle {want[i]!r}"


def bench_handle(gb, make):
    from paper_2008_05718_gb300 import grouping, policy
    bc = make()
    bc.load_policy(policy.shipped_weights())
    bc.load_grouping(grouping.shipped_weights())
    return bc


def test_rmat22_bench_configuration_512_sources(gb):
    g, S = gg.workload("rmat22")
    pick = np.sort(gg.sample_sources(len(S), 512, seed=2205))
    src = S[pick]
    with bench_handle(gb, lambda: gb.BC.from_graph(g)) as bc:
        bc.compute(src)
        got = bc.read()
        st = bc.stats()
    assert st["schedule"] == 1 and st["batches"] == 8  # grid schedule, 8 batches at once
    keep = src[[0, 100, 300, 511]]
    with gb.BC.from_graph(g, flags=gb.GBBC_KEEP_STATE) as bc:
        bc.compute(keep)
        states = [bc.source_state(i) for i in range(len(keep))]
    with OraclePool(g) as pool:
        want, _ = pool.bc(src, shares_per_proc=2)
        ost = pool.states(keep)
    assert_bc_close(got, want, "rmat22")
    for i, ((d, s, o), (od, os_, oo)) in enumerate(zip(states, ost)):
        assert np.array_equal(d, od), f"dist of kept source #{i}"
        assert np.array_equal(s, os_), f"sigma of kept source #{i}"
        assert np.array_equal(o, oo), f"overflow flags of kept source #{i}"


def test_multi_workload_every_graph(gb):
    mw = gg.multi_workload()
    gid, loc, per_graph = [], [], []
    for i, (g, s) in enumerate(zip(mw.graphs, mw.sources)):
        s = np.arange(g.n, dtype=np.int32) if g.n <= 4096 else s[:16]
        per_graph.append(s)
        gid.append(np.full(len(s), i, np.int32))
        loc.append(s)
    with bench_handle(gb, lambda: gb.BC.from_graphs(mw.graphs)) as bc:
        bc.compute_multi(np.concatenate(gid), np.concatenate(loc))
        got = [bc.read(graph_id=i) for i in range(len(mw.graphs))]
    want = map_graphs([(g.n, g.row_ptr, g.col, s) for g, s in zip(mw.graphs, per_graph)])
    for i, (a, b) in enumerate(zip(got, want)):
        assert_bc_close(a, b, f"graph {i} {mw.kinds[i]}")


def test_grid1024_256_sources(gb):
    g, S = gg.workload("grid1024")
    src = S[:256]
    with bench_handle(gb, lambda: gb.BC.from_graph(g)) as bc:
        bc.compute(src)
        got = bc.read()
        st = bc.stats()
    assert st["wide_batches"] > 0  # path counts far beyond 2^64
    with OraclePool(g) as pool:
        want, _ = pool.bc(src, shares_per_proc=2)
    assert_bc_close(got, want, "grid1024")
