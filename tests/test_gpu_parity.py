"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

dist and sigma (mod 2^64) and the overflow flag must be bit-exact; BC must
agree within 1e-12 relative with a 1e-15 absolute floor (FP64 sums in a
different order: the oracle pushes in reverse BFS order and sums sources in
list order, the GPU pulls in CSR order and sums lanes in a fixed tree).
"""
import numpy as np
import pytest

import oracle
from paper_2008_05718_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

REL, ABS = 1e-12, 1e-15



def assert_bc_close(got, want):
    got = np.asarray(got)
    want = np.asarray(want)
    assert got.shape == want.shape
    excess = np.abs(got - want) - (REL * np.abs(want) + ABS)
    i = int(np.argmax(excess))
    assert excess[i] <= 0, f"vertex {i}: gpu {got[i]!r} oracle {want[i]!r}"


def run_gpu(gb, g, sources, keep=(), **opts):
    flags = gb.GBBC_KEEP_STATE if keep else 0
    with gb.BC.from_graph(g, flags=flags, **opts) as bc:
        bc.compute(np.asarray(sources, np.int32))
        out = bc.read()
        states = {i: bc.source_state(i) for i in keep}
        stats = bc.stats()
    return out, states, stats


def check(gb, g, sources, keep=(), **opts):
    want, ost = oracle.bc_graph(g, sources, dump=keep)
    got, st, stats = run_gpu(gb, g, sources, keep, **opts)
    assert_bc_close(got, want)
    for i in keep:
        d, s, o = st[i]
        assert np.array_equal(d, ost[i].dist), f"dist of source #{i}"
        assert np.array_equal(s, ost[i].sigma), f"sigma of source #{i}"
        assert np.array_equal(o, ost[i].ovf), f"overflow flag of source #{i}"
    return got, stats


CLOSED = [gg.path(17), gg.star(40), gg.cycle(31), gg.cycle(64), gg.complete(12), gg.complete_bipartite(5, 9),
          gg.diamond_chain(20), gg.full_grid(9, 11)]


@pytest.mark.parametrize("idx", range(len(CLOSED)))
def test_closed_form_graphs_all_sources(gb, idx):
    g = CLOSED[idx]
    S = np.arange(g.n, dtype=np.int32)
    check(gb, g, S, keep=(0, g.n - 1))


@pytest.mark.parametrize("policy", ["push", "pull", "beamer", "auto"])
def test_er4096_policies(gb, policy):
    g, S = gg.workload("er4096")
    # 300 sources: five batches, the last one ragged (44 lanes)
    check(gb, g, S[:300], keep=(0, 63, 64, 299), policy=policy)


def test_er4096_all_sources(gb):
    g, S = gg.workload("er4096")
    got, stats = check(gb, g, S, keep=(0, 4095))
    assert stats["batches"] == 64


@pytest.mark.parametrize("policy", ["push", "pull", "beamer"])
@pytest.mark.parametrize("heavy", [0, 32])
def test_rmat_heavy_rows_and_policies(gb, policy, heavy):
    g = gg.rmat(13, 16, seed=31)
    S = gg.sample_sources(g.n, 150, seed=31)
    check(gb, g, S, keep=(0, 149), policy=policy, heavy_degree=heavy)


def test_rmat18_full_size_sampled(gb):
    # the benchmark graph at full size, one batch of 64 sources in the
    # benchmark's launch configuration (width 64, auto policy)
    g, S = gg.workload("rmat18")
    check(gb, g, S[:64], keep=(0, 31, 63), batch_width=64, policy="auto")


def _bench_handle(gb, g, **opts):
    from paper_2008_05718_gb300 import grouping, policy
    bc = gb.BC.from_graph(g, **opts)
    bc.load_policy(policy.shipped_weights())
    bc.load_grouping(grouping.shipped_weights())
    return bc


@pytest.mark.parametrize("name,k", [("rmat18", None), ("rmat22", 512)])
def test_bench_configuration_gives_the_bits_of_one_batch_at_a_time(gb, name, k):
    # the benchmark's launch configuration (learned direction and grouping, 8
    # batches at once on their own streams) at full size against one batch at
    # a time in list order under the threshold rule: the same integer BC
    g, S = gg.workload(name)
    S = S if k is None else S[:k]
    with _bench_handle(gb, g) as bc:
        bc.compute(S)
        fast = bc.read_fixed()
        st = bc.stats()
    # every source once; the autotuner's trial blocks may add batches of 32
    assert st["schedule"] == 1 and st["sources"] == len(S) and st["batches"] >= (len(S) + 63) // 64
    with gb.BC.from_graph(g, policy="beamer", schedule="grid", streams=1) as bc:
        bc.compute(S)
        assert np.array_equal(bc.read_fixed(), fast)


def test_rmat18_bench_configuration_against_the_oracle(gb):
    g, S = gg.workload("rmat18")
    S = S[:96]  # two batches, so two workers
    with _bench_handle(gb, g) as bc:
        bc.compute(S)
        got = bc.read()
    want, _ = oracle.bc_graph(g, S)
    assert_bc_close(got, want)


def test_disconnected_isolated_and_duplicate_sources(gb):
    g = gg.from_edges(12, [(0, 1), (1, 2), (2, 3), (4, 5), (5, 6), (6, 4), (8, 9)])  # 7, 10, 11 isolated
    S = np.array([0, 7, 0, 4, 11, 9, 9, 3], np.int32)
    check(gb, g, S, keep=tuple(range(len(S))), policy="pull")
    check(gb, g, S, keep=tuple(range(len(S))), policy="push")


def test_empty_source_list_and_single_vertex(gb):
    g = gg.path(5)
    got, _, _ = run_gpu(gb, g, np.zeros(0, np.int32))
    assert np.all(got == 0)
    one = gg.from_edges(1, np.zeros((0, 2), np.int32))
    got, st, _ = run_gpu(gb, one, [0, 0], keep=(0,))
    assert got[0] == 0 and st[0][0][0] == 0 and st[0][1][0] == 1


def test_accumulates_across_calls_and_reset(gb):
    g = gg.er(500, "0.012", seed=4)
    S = gg.sample_sources(g.n, 100, seed=4)
    want, _ = oracle.bc_graph(g, S)
    with gb.BC.from_graph(g) as bc:
        bc.compute(S[:37]).compute(S[37:])
        assert_bc_close(bc.read(), want)
        bc.reset()
        assert np.all(bc.read() == 0)


def test_deterministic_reruns(gb):
    g = gg.rmat(12, 16, seed=8)
    S = gg.sample_sources(g.n, 200, seed=8)
    a, _, _ = run_gpu(gb, g, S)
    b, _, _ = run_gpu(gb, g, S)
    assert np.array_equal(a, b)


def test_multi_graph_union(gb):
    graphs = [gg.rmat(9, 16, seed=100 + i) for i in range(3)] + [gg.grid(20, "0.03", seed=200 + i)
                                                                 for i in range(2)] + [gg.path(70)]
    gids, locs, per = [], [], []
    for i, g in enumerate(graphs):
        S = np.arange(g.n, dtype=np.int32) if g.n <= 400 else gg.sample_sources(g.n, 90, seed=i)
        per.append(S)
        gids += [i] * len(S)
        locs += list(S)
    with gb.BC.from_graphs(graphs) as bc:
        bc.compute_multi(np.array(gids, np.int32), np.array(locs, np.int32))
        for i, g in enumerate(graphs):
            want, _ = oracle.bc_graph(g, per[i])
            assert_bc_close(bc.read(graph_id=i), want)


def test_device_pointers(gb):
    import torch
    g = gg.rmat(11, 16, seed=3)
    S = gg.sample_sources(g.n, 70, seed=3)
    want, _ = oracle.bc_graph(g, S)
    dev = torch.device("cuda:0")
    with gb.BC.from_csr(g.n, torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev)) as bc:
        bc.compute(torch.from_numpy(S).to(dev))
        out = torch.zeros(g.n, dtype=torch.float64, device=dev)
        bc.read(out)
        assert_bc_close(out.cpu().numpy(), want)


def test_invalid_inputs_rejected(gb):
    g = gg.path(6)
    bad = [
        (np.array([0, 1, 2], np.int32), np.array([1, 1], np.int32)),        # 0-1 ok, 1->1 self-loop
        (np.array([0, 2, 2, 2], np.int32), np.array([1, 2], np.int32)),     # asymmetric
        (np.array([0, 2, 4, 4], np.int32), np.array([1, 1, 0, 0], np.int32)),  # duplicates
        (np.array([0, 2, 3, 4], np.int32), np.array([2, 1, 0, 0], np.int32)),  # unsorted row
    ]
    for rp, col in bad:
        with pytest.raises(gb.GbbcError) as e:
            gb.bc_graph_create(len(rp) - 1, int(rp[-1]), rp, col, gb.options(validate=True))
        assert e.value.status == gb.GBBC_ERR_INVALID
        assert "validation" in e.value.detail
    with pytest.raises(gb.GbbcError) as e:
        gb.bc_graph_create(3, 5, np.array([0, 1, 2, 4], np.int32), np.array([1, 0, 2, 1], np.int32))
    assert e.value.status == gb.GBBC_ERR_INVALID
    with gb.BC.from_graph(g) as bc:
        with pytest.raises(gb.GbbcError) as e:
            bc.compute([0, 6])
        assert e.value.status == gb.GBBC_ERR_INVALID
        with pytest.raises(gb.GbbcError) as e:
            bc.source_state(0)
        assert e.value.status == gb.GBBC_ERR_STATE


def test_memory_limit_reports_oom(gb):
    g = gg.rmat(12, 16, seed=2)
    with gb.BC.from_graph(g, mem_limit_bytes=2 << 20) as bc:
        with pytest.raises(gb.GbbcError) as e:
            bc.compute([0, 1, 2])
        assert e.value.status == gb.GBBC_ERR_OOM


def test_trace_both_directions_keeps_results(gb):
    g = gg.rmat(12, 16, seed=12)
    S = gg.sample_sources(g.n, 100, seed=12)
    want, ost = oracle.bc_graph(g, S, dump=(0, 99))
    flags = gb.GBBC_KEEP_STATE | gb.GBBC_TRACE | gb.GBBC_TRACE_BOTH
    with gb.BC.from_graph(g, flags=flags) as bc:
        bc.compute(S)
        assert_bc_close(bc.read(), want)
        for i in (0, 99):
            d, s, o = bc.source_state(i)
            assert np.array_equal(d, ost[i].dist) and np.array_equal(s, ost[i].sigma)
        tr = bc.trace()
        prof = bc.profile()
    assert len(tr["level"]) == bc_levels(ost, S, g) and np.all(tr["ms_push"] > 0) and np.all(tr["ms_pull"] > 0)
    assert np.all(tr["ms_gather"][tr["next_vertices"] > 0] > 0)
    for k in ("gather", "backward"):
        assert prof[k]["launches"] > 0 and prof[k]["ms"] > 0 and prof[k]["bytes"] > 0


def bc_levels(ost, S, g):
    # forward steps = sum over batches of (deepest level + 1); recompute
    # each batch's deepest level from the oracle
    depths = []
    for b in range(0, len(S), 64):
        _, st = oracle.bc_graph(g, S[b:b + 64], dump=range(len(S[b:b + 64])))
        depths.append(max(int(st[i].dist.max()) for i in st))
    return sum(d + 1 for d in depths)


# ---- the wide sigma format (counts >= 2^64) ---------------------------------

@pytest.mark.parametrize("k", [63, 64, 65, 100])
def test_wide_sigma_diamond_chain(gb, k):
    g = gg.diamond_chain(k)
    S = np.arange(g.n, dtype=np.int32)
    got, stats = check(gb, g, S, keep=(0, g.n - 1, 3 * (k // 2)))
    assert (stats["wide_batches"] > 0) == (k >= 64)
    # every sigma in a diamond chain is a power of two: BC is exact
    from test_oracle_pins import diamond_closed_form
    assert np.array_equal(got, diamond_closed_form(k))


def test_wide_sigma_full_grid(gb):
    g = gg.full_grid(40, 40)  # sigma up to C(78, 39) ~ 2^75
    S = np.arange(g.n, dtype=np.int32)
    _, stats = check(gb, g, S, keep=(0, 39, 820, 1599))
    assert stats["wide_batches"] > 0


@pytest.mark.parametrize("policy", ["push", "auto"])
def test_wide_sigma_grid_with_removed_edges(gb, policy):
    g = gg.grid(96, "0.05", seed=17)
    S = gg.sample_sources(g.n, 130, seed=17)
    check(gb, g, S, keep=(0, 64, 129), policy=policy)


def test_grid1024_full_size_sampled(gb):
    # the high-diameter workload at full size: one batch of 64 sources;
    # sigma exceeds the double range (~2^2000), dist/sigma mod 2^64 exact
    g, S = gg.workload("grid1024")
    got, stats = check(gb, g, S[:64], keep=(0, 63), batch_width=64)
    assert stats["wide_batches"] >= 1 and stats["levels_fwd"] > 1500
    # the same sources in the bitset schedules: one 64-lane batch, rerun wide
    got2, stats2 = check(gb, g, S[:64], keep=(0, 63), batch_width=64, schedule="grid")
    assert stats2["wide_batches"] == 1
    assert np.allclose(got, got2, rtol=1e-12, atol=1e-15)


def test_bc_bit_identical_across_schedules(gb):
    # integer fixed-point accumulation: the schedule cannot change a bit
    g = gg.rmat(12, 16, seed=19)
    S = gg.sample_sources(g.n, 300, seed=19)
    runs = [run_gpu(gb, g, S, policy=p, heavy_degree=h)[0]
            for p, h in [("push", 0), ("pull", 0), ("beamer", 32), ("auto", 64)]]
    runs.append(run_gpu(gb, g, S[::-1].copy())[0])  # other batch composition
    for r in runs[1:]:
        assert np.array_equal(r, runs[0])


# ---- the plain one-source-at-a-time path (batch width 1) ---------------------

@pytest.mark.parametrize("make", [lambda: gg.workload("er4096")[0], lambda: gg.rmat(12, 16, seed=23),
                                  lambda: gg.from_edges(9, [(0, 1), (1, 2), (4, 5), (5, 6), (6, 4)])])
def test_plain_path_parity_and_identical_bits(gb, make):
    g = make()
    S = gg.sample_sources(g.n, min(g.n, 97), seed=23)
    got, _ = check(gb, g, S, keep=(0, len(S) - 1), batch_width=1)
    batched, _, _ = run_gpu(gb, g, S, batch_width=64)
    assert np.array_equal(got, batched)  # same integer arithmetic, same bits


def test_plain_path_rejects_wide_counts(gb):
    g = gg.diamond_chain(70)
    with gb.BC.from_graph(g, batch_width=1) as bc:
        with pytest.raises(gb.GbbcError) as e:
            bc.compute([0])
        assert e.value.status == gb.GBBC_ERR_CAPACITY


# ---- batch width 1 on the block schedule: a source per thread block ----------

PLAIN_BLOCK_CASES = [
    ("er4096", lambda: gg.workload("er4096")[0], 300, 0),  # every source on a block of its own
    ("rmat14", lambda: gg.rmat(14, 16, seed=24), 700, 0),  # more sources than resident blocks
    ("rmat12_few_blocks", lambda: gg.rmat(12, 16, seed=25), 257, 2 << 20),  # a dozen blocks: many sources each
    ("components", lambda: gg.from_edges(9, [(0, 1), (1, 2), (4, 5), (5, 6), (6, 4)]), 9, 0),
]


@pytest.mark.parametrize("name,make,k,limit", PLAIN_BLOCK_CASES, ids=[c[0] for c in PLAIN_BLOCK_CASES])
def test_plain_blocks_parity_and_identical_bits(gb, name, make, k, limit):
    g = make()
    S = gg.sample_sources(g.n, min(g.n, k), seed=24)
    opts = {"mem_limit_bytes": limit} if limit else {}
    with gb.BC.from_graph(g, batch_width=1, schedule="block", **opts) as bc:
        bc.compute(S)
        fx, got, st = bc.read_fixed(), bc.read(), bc.stats()
    assert st["sources"] == len(S) and st["schedule"] == gb.SCHEDULE["block"]
    want, _ = oracle.bc_graph(g, S)
    assert_bc_close(got, want)
    with gb.BC.from_graph(g, batch_width=64) as bc:
        bc.compute(S)
        assert np.array_equal(fx, bc.read_fixed())  # same integer sums, same bits


def test_plain_blocks_multi_graph_and_wide_counts(gb):
    graphs = [gg.rmat(10, 8, seed=26), gg.cycle(50), gg.full_grid(6, 7)]
    gid = np.repeat(np.arange(3, dtype=np.int32), 40)
    local = np.concatenate([gg.sample_sources(h.n, 40, seed=27 + i) for i, h in enumerate(graphs)]).astype(np.int32)
    out = []
    for opts in ({"batch_width": 1, "schedule": "block"}, {"batch_width": 64}):
        with gb.BC.from_graphs(graphs, **opts) as bc:
            bc.compute_multi(gid, local)
            out.append(bc.read_fixed())
    assert np.array_equal(out[0], out[1])
    with gb.BC.from_graph(gg.diamond_chain(70), batch_width=1, schedule="block") as bc:
        with pytest.raises(gb.GbbcError) as e:
            bc.compute([0, 1])
        assert e.value.status == gb.GBBC_ERR_CAPACITY


# ---- the block-per-batch schedule and the autotuner --------------------------

@pytest.mark.parametrize("make,k", [(lambda: gg.workload("er4096")[0], 300), (lambda: gg.rmat(12, 16, seed=61), 300),
                                    (lambda: gg.grid(64, "0.05", seed=62), 200), (lambda: gg.diamond_chain(70), 211),
                                    (lambda: gg.from_edges(7, [(0, 1), (1, 2), (4, 5)]), 7)])
@pytest.mark.parametrize("policy", ["push", "beamer"])
def test_block_schedule_parity_and_identical_bits(gb, make, k, policy):
    g = make()
    S = gg.sample_sources(g.n, min(k, g.n), seed=63)
    want, _ = oracle.bc_graph(g, S)
    blk, _, st = run_gpu(gb, g, S, schedule="block", policy=policy)
    assert st["schedule"] == 2 and st["block_slots"] >= 1
    assert_bc_close(blk, want)
    grid, _, _ = run_gpu(gb, g, S, schedule="grid", policy=policy)
    assert np.array_equal(blk, grid)


def test_block_schedule_with_idle_slots(gb):
    # one long batch (a path) and many one-level batches (isolated vertices):
    # clusters that start late find the work list empty and run no batch; their
    # slots' counters must not be read as errors.  Device memory is dirtied
    # first by a handle that is then destroyed, so fresh allocations may hold
    # old bytes.
    n_path, n_iso = 3000, 64 * 15
    g = gg.from_edges(n_path + n_iso, [(i, i + 1) for i in range(n_path - 1)])
    S = np.concatenate([gg.sample_sources(n_path, 64, seed=91), np.arange(n_path, n_path + n_iso)]).astype(np.int32)
    want, _ = oracle.bc_graph(g, S)
    for rep in range(3):
        h = gg.rmat(12, 16, seed=92 + rep)
        with gb.BC.from_graph(h, schedule="block") as bc:
            bc.compute(gg.sample_sources(h.n, 512, seed=93))
            bc.sync()
        got, _, st = run_gpu(gb, g, S, schedule="block")
        assert st["schedule"] == 2
        assert_bc_close(got, want)


@pytest.mark.parametrize("schedule", ["block", "grid"])
def test_wide_format_is_chosen_per_graph(gb, schedule):
    # the grid's batches pass 2^64 and are rerun wide; the R-MAT graph's are
    # not, in this call or the next (where the grid's batches start wide)
    graphs = [gg.rmat(10, 16, seed=95), gg.grid(64, "0.03", seed=96)]
    per = [gg.sample_sources(g.n, 128, seed=97) for g in graphs]
    gids = np.repeat(np.arange(2, dtype=np.int32), 128)
    locs = np.concatenate(per).astype(np.int32)
    with gb.BC.from_graphs(graphs, schedule=schedule) as bc:
        bc.compute_multi(gids, locs)
        assert bc.stats()["wide_batches"] == 2
        first = [bc.read_fixed(i) for i in range(2)]
        bc.reset()
        bc.compute_multi(gids, locs)
        assert bc.stats()["wide_batches"] == 4
        assert all(np.array_equal(bc.read_fixed(i), first[i]) for i in range(2))
        for i, g in enumerate(graphs):
            want, _ = oracle.bc_graph(g, per[i])
            assert_bc_close(bc.read(graph_id=i), want)


def test_block_schedule_large_sparse_graph_with_leftover_batches(gb):
    # 16 batches of a road-like graph above 65,536 vertices: the batches that
    # do not fill a round of resident 8-CTA clusters run in the grid schedule
    g = gg.grid(300, "0.05", seed=98)
    S = gg.sample_sources(g.n, 1024, seed=99)
    blk, _, st = run_gpu(gb, g, S, schedule="block")
    assert st["batches"] == 16 and st["wide_batches"] == 16
    grid, _, _ = run_gpu(gb, g, S, schedule="grid")
    assert np.array_equal(blk, grid)
    want, _ = oracle.bc_graph(g, S)
    assert_bc_close(blk, want)


@pytest.mark.parametrize("make,k", [(lambda: gg.tri(48, seed=101), 200), (lambda: gg.rgg(3000, 10.0, seed=102), 200),
                                    (lambda: gg.mesh27(12), 200)])
@pytest.mark.parametrize("schedule", ["grid", "block"])
def test_planar_geometric_and_mesh_classes(gb, make, k, schedule):
    # the Delaunay-like, random geometric and KKT-like mesh classes: dist and
    # sigma bit-exact, BC within tolerance, the same bits in both schedules
    g = make()
    S = gg.sample_sources(g.n, k, seed=103)
    got, _ = check(gb, g, S, keep=(0, k - 1), schedule=schedule)
    other, _, _ = run_gpu(gb, g, S, schedule="block" if schedule == "grid" else "grid")
    assert np.array_equal(got, other)


@pytest.mark.parametrize("name,nsrc", [("tri1024", 16), ("rgg20", 16), ("mesh100", 8)])
def test_planar_geometric_and_mesh_full_size_sampled(gb, name, nsrc):
    g, S = gg.workload(name)
    check(gb, g, S[:nsrc], keep=(0, nsrc - 1))


@pytest.mark.parametrize("make,k", [(lambda: gg.rmat(12, 16, seed=250), 1000), (lambda: gg.grid(64, "0.05", seed=251), 400),
                                    (lambda: gg.diamond_chain(70), 211)])
def test_concurrent_grid_batches_give_identical_bits(gb, make, k):
    # the grid schedule with 1, 2 and 4 batches at once (own streams, slots and
    # BC accumulators, summed exactly): the same bits, and the oracle's BC
    g = make()
    S = gg.sample_sources(g.n, min(k, g.n), seed=252)
    ref = None
    for streams in (1, 2, 4):
        with gb.BC.from_graph(g, schedule="grid", streams=streams) as bc:
            bc.compute(S)
            fixed = bc.read_fixed()
            got = bc.read()
            st = bc.stats()
        assert st["batches"] == (len(S) + 63) // 64
        if ref is None:
            ref = fixed
            want, _ = oracle.bc_graph(g, S)
            assert_bc_close(got, want)
        assert np.array_equal(fixed, ref)


def test_released_pool_memory_is_taken_again(gb):
    # handles draw on the library's pool; releasing its unused part between
    # handles changes nothing in the results
    g = gg.rmat(11, 16, seed=260)
    S = gg.sample_sources(g.n, 300, seed=261)
    outs = []
    for release in (False, True, False):
        if release:
            gb.bc_release_memory()
        with gb.BC.from_graph(g) as bc:
            bc.compute(S)
            outs.append(bc.read_fixed())
    gb.bc_release_memory(-1)
    assert all(np.array_equal(o, outs[0]) for o in outs)


def test_block_schedule_multi_graph_and_width32(gb):
    graphs = [gg.rmat(10, 16, seed=71), gg.grid(40, "0.03", seed=72), gg.path(50), gg.rmat(11, 16, seed=73)]
    gids, locs, per = [], [], []
    for i, g in enumerate(graphs):
        S = gg.sample_sources(g.n, min(g.n, 150), seed=74 + i)
        per.append(S)
        gids += [i] * len(S)
        locs += list(S)
    for width in (64, 32):
        with gb.BC.from_graphs(graphs, schedule="block", batch_width=width) as bc:
            bc.compute_multi(np.array(gids, np.int32), np.array(locs, np.int32))
            for i, g in enumerate(graphs):
                want, _ = oracle.bc_graph(g, per[i])
                assert_bc_close(bc.read(graph_id=i), want)


def test_autotuned_schedule_gives_identical_bits(gb):
    g = gg.grid(80, "0.05", seed=81)
    S = gg.sample_sources(g.n, 400, seed=81)
    auto, _, st = run_gpu(gb, g, S, schedule="auto")
    assert st["schedule"] in (1, 2)
    grid, _, _ = run_gpu(gb, g, S, schedule="grid")
    assert np.array_equal(auto, grid)


def test_autotuner_takes_block_schedule_when_batches_fill_the_gpu(gb):
    # 38 batches of a small graph (each source three times): block schedule
    # without a timed trial
    g = gg.rmat(12, 16, seed=82)
    S1 = gg.sample_sources(g.n, 810, seed=82)
    S = np.tile(S1, 3)
    auto, _, st = run_gpu(gb, g, S, schedule="auto")
    assert st["schedule"] == 2 and st["batches"] == 38
    grid, _, _ = run_gpu(gb, g, S, schedule="grid")
    assert np.array_equal(auto, grid)
    want, _ = oracle.bc_graph(g, S1)
    assert_bc_close(auto, 3.0 * want)


def test_fixed_point_partials_add_to_identical_bits(gb):
    # three shards on three handles (grid and block schedules), their exact
    # partials added into the first handle by the library (bc_add_fixed, one
    # partial from host memory and one from device memory): the bits of one
    # handle over all sources, and the reference helper's exact sum
    import torch
    from oracle import fixed as fx
    from paper_2008_05718_gb300 import multirank as mr
    g = gg.rmat(12, 16, seed=91)
    S = gg.sample_sources(g.n, 300, seed=91)
    with gb.BC.from_graph(g) as bc:
        bc.compute(S)
        whole_fixed, whole = bc.read_fixed(), bc.read()
    hs = [gb.BC.from_graph(g, schedule="block" if r % 2 else "grid") for r in range(3)]
    try:
        parts = []
        for r, h in enumerate(hs):
            h.compute(mr.shard(S, r, 3))
            parts.append(h.read_fixed())
        dev = torch.empty(2 * g.n, dtype=torch.int64, device="cuda")
        hs[2].read_fixed_into(dev)
        hs[0].add_fixed(parts[1])  # host numpy
        hs[0].add_fixed(dev)       # device tensor
        assert np.array_equal(hs[0].read_fixed(), whole_fixed)
        assert np.array_equal(hs[0].read(), whole)
        assert fx.sum_parts(parts) == fx.to_int(whole_fixed)
        assert np.array_equal(fx.to_double(fx.to_int(whole_fixed)), whole)
        with pytest.raises(gb.GbbcError):
            hs[1].add_fixed(parts[1], graph_id=3)
    finally:
        for h in hs:
            h.close()


# ---- the remaining workloads at full size (sampled sources) ------------------

def test_multi_workload_full_size_sampled(gb):
    # the 256-graph mix in one handle; two sources per graph, checked graph by graph
    mw = gg.multi_workload()
    assert len(mw.graphs) == 256
    gids, locs, per = [], [], []
    for i, (g, S) in enumerate(zip(mw.graphs, mw.sources)):
        sel = S[:2]
        per.append(sel)
        gids += [i] * len(sel)
        locs += list(sel)
    with gb.BC.from_graphs(mw.graphs) as bc:
        bc.compute_multi(np.array(gids, np.int32), np.array(locs, np.int32))
        st = bc.stats()
        for i in range(0, 256, 15):
            want, _ = oracle.bc_graph(mw.graphs[i], per[i])
            assert_bc_close(bc.read(graph_id=i), want)
    # one bitset batch per graph, or one pair batch per source (L = 1 here) for
    # the large grids the auto schedule sends to the pair kernel (144 sources)
    assert st["batches"] >= 256 and st["wide_batches"] > 0


def test_rmat22_full_size_sampled(gb):
    # the largest workload (4.2M vertices, ~128M entries): one batch of 8 sources
    g, S = gg.workload("rmat22")
    check(gb, g, S[:8], keep=(0, 7), batch_width=64)
