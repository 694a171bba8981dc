"""The weighted path on the GPU against the weighted oracle: dist and sigma
bit-exact (kept per-source state), BC within 1e-12 relative; unit weights
give the unweighted path's exact bits; overflow and bad weights are errors."""
import numpy as np
import pytest

import oracle
from paper_2008_05718_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def assert_bc_close(got, want):
    assert np.allclose(got, want, rtol=1e-12, atol=1e-15), np.max(np.abs(got - want))


def run_w(gb, g, w, S, keep=(), **opts):
    flags = gb.GBBC_KEEP_STATE if keep else 0
    with gb.BC.from_weighted(g.n, g.row_ptr, g.col, w, flags=flags, **opts) as bc:
        bc.compute(np.asarray(S, np.int32))
        out = bc.read()
        fixed = bc.read_fixed()
        states = {i: bc.source_state(i) for i in keep}
        stats = bc.stats()
    return out, fixed, states, stats


def check_w(gb, g, w, S, keep=(), **opts):
    want, ost = oracle.bc_graph_weighted(g, w, S, dump=keep)
    got, fixed, st, stats = run_w(gb, g, w, S, keep, **opts)
    assert_bc_close(got, want)
    for i in keep:
        d, s, o = st[i]
        assert np.array_equal(d, ost[i].dist), f"dist of source #{i}"
        assert np.array_equal(s, ost[i].sigma), f"sigma of source #{i}"
        assert np.array_equal(o, ost[i].ovf), f"overflow flags of source #{i}"
    return got, fixed, stats


CASES = [
    ("rmat10_w4", lambda: gg.rmat(10, 16, seed=201), 4, 150),
    ("grid40_w8", lambda: gg.grid(40, "0.05", seed=202), 8, 130),
    ("er800_w16", lambda: gg.er(800, "8/799", seed=203), 16, 200),
    ("tri30_w64", lambda: gg.tri(30, seed=204), 64, 100),
    ("rgg_w3", lambda: gg.rgg(2000, 10.0, seed=205), 3, 64),
    ("er800_all_w16", lambda: gg.er(800, "8/799", seed=208), 16, 800),  # 6 lanes per batch
    ("rmat12_w2", lambda: gg.rmat(12, 16, seed=209), 2, 4000),  # 27 lanes per batch, many ties
]


@pytest.mark.parametrize("name,make,maxw,k", CASES, ids=[c[0] for c in CASES])
def test_weighted_parity(gb, name, make, maxw, k):
    g = make()
    w = gg.edge_weights(g, maxw, seed=206)
    S = gg.sample_sources(g.n, min(k, g.n), seed=207)
    _, fixed, stats = check_w(gb, g, w, S, keep=(0, len(S) - 1))
    lanes = max(1, min(64, -(-len(S) // 152)))
    assert stats["batches"] >= (len(S) + lanes - 1) // lanes
    # rerun: the same bits
    _, fixed2, _, _ = run_w(gb, g, w, S)
    assert np.array_equal(fixed, fixed2)


def test_weighted_hand_example(gb):
    g = gg.from_edges(4, [(0, 1), (1, 3), (0, 2), (2, 3)])
    u = np.repeat(np.arange(4), np.diff(g.row_ptr))
    wt = {(0, 1): 1, (1, 3): 1, (0, 2): 1, (2, 3): 2}
    w = np.array([wt[(min(a, b), max(a, b))] for a, b in zip(u, g.col)], np.int32)
    got, _, _, _ = run_w(gb, g, w, np.arange(4))
    assert np.array_equal(got, [2.0, 2.0, 0.0, 0.0])


@pytest.mark.parametrize("make", [lambda: gg.rmat(11, 16, seed=210), lambda: gg.grid(24, "0.05", seed=211),
                                  lambda: gg.star(30)])
def test_unit_weights_give_the_unweighted_bits(gb, make):
    g = make()
    S = gg.sample_sources(g.n, min(200, g.n), seed=212)
    _, fixed, _, _ = run_w(gb, g, np.ones(g.nnz, np.int32), S)
    with gb.BC.from_graph(g) as bc:
        bc.compute(S)
        assert np.array_equal(bc.read_fixed(), fixed)


def test_weighted_edge_cases(gb):
    # isolated vertices, duplicated sources, a source repeated within a batch
    g = gg.from_edges(8, [(0, 1), (1, 2), (2, 3), (5, 6)])
    u = np.repeat(np.arange(8), np.diff(g.row_ptr))
    w = np.array([1 + (int(a) + int(b)) % 3 for a, b in zip(u, g.col)], np.int32)
    S = [0, 0, 4, 5, 3, 7, 2, 2]
    check_w(gb, g, w, S, keep=(0, 1, 2))
    # more than one batch, ragged tail, on a multi-level graph
    h = gg.grid(20, "0.1", seed=213)
    wh = gg.edge_weights(h, 5, seed=214)
    check_w(gb, h, wh, gg.sample_sources(h.n, 199, seed=215), keep=(64, 198))


def test_weighted_counts_past_2_64_run_wide(gb):
    # 2^70 shortest paths at unit weights (diamond chain), C(2k, k) on grids:
    # the batch is rerun in the wide format; sigma mod 2^64 and the flags
    # stay exact, BC within tolerance
    g = gg.diamond_chain(70)
    S = np.arange(g.n, dtype=np.int32)
    _, _, stats = check_w(gb, g, np.ones(g.nnz, np.int32), S, keep=(0, g.n - 1))
    assert stats["wide_batches"] > 0
    h = gg.grid(48, "0.05", seed=220)
    wh = gg.edge_weights(h, 2, seed=221)
    check_w(gb, h, wh, gg.sample_sources(h.n, 150, seed=222), keep=(0, 149))


def test_weighted_invalid_weights(gb):
    h = gg.path(5)
    for bad in (np.zeros(h.nnz, np.int32), np.full(h.nnz, gb.MAX_WEIGHT + 1, np.int32)):
        with pytest.raises(gb.GbbcError) as e:
            gb.BC.from_weighted(h.n, h.row_ptr, h.col, bad)
        assert e.value.status == gb.GBBC_ERR_INVALID
    asym = np.arange(1, h.nnz + 1, dtype=np.int32)
    with pytest.raises(gb.GbbcError) as e:
        gb.BC.from_weighted(h.n, h.row_ptr, h.col, asym, validate=True)
    assert e.value.status == gb.GBBC_ERR_INVALID
    with gb.BC.from_weighted(h.n, h.row_ptr, h.col, np.ones(h.nnz, np.int32), batch_width=1) as bc:
        with pytest.raises(gb.GbbcError) as e:
            bc.compute([0])
        assert e.value.status == gb.GBBC_ERR_INVALID


def test_weighted_full_size_sampled(gb):
    g, S = gg.workload("rmat18")
    w = gg.edge_weights(g, 16, seed=216)
    check_w(gb, g, w, S[:64], keep=(0, 63))


# ---- the same kernel for unweighted graphs (GBBC_SCHEDULE_PAIR) ----------------

PAIR_CASES = [
    ("grid64_wide", lambda: gg.grid(64, "0.05", seed=230), 200),
    ("tri48", lambda: gg.tri(48, seed=231), 160),
    ("rgg3000", lambda: gg.rgg(3000, 10.0, seed=232), 300),
    ("mesh12", lambda: gg.mesh27(12), 200),
    ("rmat12", lambda: gg.rmat(12, 16, seed=233), 400),
    ("diamond70", lambda: gg.diamond_chain(70), 211),
]


@pytest.mark.parametrize("name,make,k", PAIR_CASES, ids=[c[0] for c in PAIR_CASES])
def test_pair_schedule_parity(gb, name, make, k):
    import oracle as orc
    g = make()
    S = gg.sample_sources(g.n, min(k, g.n), seed=234)
    keep = (0, len(S) - 1)
    want, ost = orc.bc_graph(g, S, dump=keep)
    with gb.BC.from_graph(g, schedule="pair", flags=gb.GBBC_KEEP_STATE) as bc:
        bc.compute(S)
        got = bc.read()
        assert bc.stats()["schedule"] == 3
        for i in keep:
            d, s, o = bc.source_state(i)
            assert np.array_equal(d, ost[i].dist)
            assert np.array_equal(s, ost[i].sigma)
            assert np.array_equal(o, ost[i].ovf)
    assert_bc_close(got, want)
    with gb.BC.from_graph(g, schedule="pair") as bc:
        bc.compute(S)
        pair_fixed = bc.read_fixed()
        wide = bc.stats()["wide_batches"]
    if wide == 0:  # counts below 2^64: the same integer sums as the bitset path
        with gb.BC.from_graph(g, schedule="grid") as bc:
            bc.compute(S)
            assert np.array_equal(bc.read_fixed(), pair_fixed)


def test_auto_schedule_routes_high_diameter_graphs_of_a_multi_handle_to_pairs(gb):
    # a large grid (above 65,536 vertices, eccentricity >= 64) goes to the pair
    # schedule, the R-MAT graphs and the small grid to the bitset schedules;
    # every graph's BC matches the oracle
    import oracle as orc
    graphs = [gg.rmat(10, 16, seed=240), gg.grid(300, "0.03", seed=241), gg.grid(40, "0.03", seed=242),
              gg.rmat(11, 16, seed=243)]
    per = [gg.sample_sources(g.n, min(100, g.n), seed=244 + i) for i, g in enumerate(graphs)]
    gids = np.concatenate([np.full(len(S), i, np.int32) for i, S in enumerate(per)])
    locs = np.concatenate(per).astype(np.int32)
    with gb.BC.from_graphs(graphs) as bc:
        bc.compute_multi(gids, locs)
        st = bc.stats()
        got = [bc.read(graph_id=i) for i in range(len(graphs))]
    assert st["schedule"] == 0  # pair and bitset schedules in one call
    for i, g in enumerate(graphs):
        want, _ = orc.bc_graph(g, per[i])
        assert_bc_close(got[i], want)
