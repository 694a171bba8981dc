"""Learned source grouping: the device features against a numpy restatement,
the scores against the FP16 inference reference, the grouping only reorders
work (identical BC bits, kept state still in list order), and the shipped
network's gain on a held-out R-MAT graph."""
import numpy as np
import pytest

from oracle import mlp


# ---- CPU: host logic of the training module --------------------------------------


def test_rank_correlation_matches_scipy():
    from scipy.stats import spearmanr
    from paper_2008_05718_gb300.grouping import rank_correlation
    r = np.random.default_rng(3)
    for _ in range(5):
        a = r.integers(0, 20, 300).astype(float)  # many ties
        b = a + r.normal(0, 4, 300)
        assert np.isclose(rank_correlation(a, b), spearmanr(a, b).statistic, rtol=1e-12)
    assert rank_correlation(np.arange(10), np.arange(10)[::-1]) == pytest.approx(-1.0)


def test_mean_distance_over_reached_vertices():
    from paper_2008_05718_gb300.grouping import mean_distance
    assert mean_distance(np.array([0, 1, 2, 3, -1])) == pytest.approx(2.0)
    assert mean_distance(np.array([0, -1, -1])) == 0.0


def test_init_params_layout():
    from paper_2008_05718_gb300.grouping import init_params
    assert len(init_params()) == mlp.param_count(1)


# ---- GPU ----------------------------------------------------------------------


def _features_numpy(graphs, sources_per_graph):
    out = []
    for g, S in zip(graphs, sources_per_graph):
        deg = np.diff(g.row_ptr).astype(np.float64)
        n, nnz, dmax = float(g.n), float(g.nnz), float(deg.max(initial=0))
        for s in S:
            nb = g.col[g.row_ptr[s]:g.row_ptr[s + 1]]
            out.append([np.log2(1 + deg[s]) / 24, np.log2(1 + deg[nb].sum()) / 32,
                        np.log2(1 + deg[nb].max(initial=0)) / 24, np.log2(1 + n) / 32,
                        np.log2(1 + nnz / n) / 16, np.log2(1 + dmax) / 24])
    return np.array(out)


@pytest.mark.gpu
def test_source_features_match_numpy(gb):
    from paper_2008_05718_gb300 import graphgen as gg
    graphs = [gg.rmat(11, 16, seed=41), gg.grid(20, "0.1", seed=42), gg.star(50), gg.path(7)]
    S = [gg.sample_sources(g.n, min(70, g.n), seed=43) for g in graphs]
    off = np.cumsum([0] + [g.n for g in graphs])
    glob = np.concatenate([s + off[i] for i, s in enumerate(S)]).astype(np.int32)
    with gb.BC.from_graphs(graphs) as bc:
        x = bc.source_features(glob)
        assert x.shape == (len(glob), 6)
        assert np.allclose(x, _features_numpy(graphs, S), rtol=2e-6, atol=1e-7)
        assert bc.source_features(np.zeros(0, np.int32)).shape == (0, 6)
        with pytest.raises(gb.GbbcError) as e:
            bc.source_features([int(off[-1])])
        assert e.value.status == gb.GBBC_ERR_INVALID


@pytest.mark.gpu
def test_grouping_scores_match_fp16_reference(gb):
    from paper_2008_05718_gb300 import graphgen as gg
    g = gg.rmat(12, 16, seed=44)
    S = gg.sample_sources(g.n, 500, seed=45)
    p = mlp.init(1, seed=46).astype(np.float32)
    with gb.BC.from_graph(g) as bc:
        with pytest.raises(gb.GbbcError) as e:
            bc.grouping_scores(S)
        assert e.value.status == gb.GBBC_ERR_STATE
        bc.load_grouping(p)
        sc = bc.grouping_scores(S)
        ref = mlp.forward_fp16_weights(p, bc.source_features(S), 1)[:, 0]
        assert np.allclose(sc, ref, atol=1e-3, rtol=1e-3)
        with pytest.raises(gb.GbbcError) as e:
            bc.load_grouping(p[:-1])
        assert e.value.status == gb.GBBC_ERR_INVALID
        bc.load_grouping(None)
        with pytest.raises(gb.GbbcError):
            bc.grouping_scores(S)


@pytest.mark.gpu
@pytest.mark.parametrize("schedule", ["grid", "block"])
def test_grouping_only_reorders(gb, schedule):
    # a random network gives an arbitrary order; the BC bits are those of list
    # order, and both agree with the oracle
    import oracle
    from paper_2008_05718_gb300 import graphgen as gg
    g = gg.rmat(12, 16, seed=47)
    S = gg.sample_sources(g.n, 300, seed=48)  # 4 full words and a ragged one
    with gb.BC.from_graph(g, schedule=schedule) as bc:
        bc.compute(S)
        ref = bc.read_fixed()
        base = bc.read()
    for seed in range(2):
        with gb.BC.from_graph(g, schedule=schedule) as bc:
            bc.load_grouping(mlp.init(1, seed=200 + seed).astype(np.float32))
            bc.compute(S)
            assert np.array_equal(bc.read_fixed(), ref)
    expect, _ = oracle.bc_graph(g, S)
    assert np.allclose(base, expect, rtol=1e-12, atol=1e-15)


@pytest.mark.gpu
def test_grouping_multi_graph_handle(gb):
    from paper_2008_05718_gb300 import graphgen as gg
    from paper_2008_05718_gb300 import grouping
    graphs = [gg.rmat(10, 16, seed=50 + i) for i in range(3)] + [gg.grid(24, "0.05", seed=60)]
    gid = np.repeat(np.arange(4, dtype=np.int32), 90)
    loc = np.concatenate([gg.sample_sources(g.n, 90, seed=61) for g in graphs]).astype(np.int32)
    w = grouping.shipped_weights()
    if w is None:
        w = grouping.init_params(1)
    outs = []
    for load in (False, True):
        with gb.BC.from_graphs(graphs) as bc:
            if load:
                bc.load_grouping(w)
            bc.compute_multi(gid, loc)
            outs.append([bc.read_fixed(i) for i in range(4)])
    assert all(np.array_equal(a, b) for a, b in zip(*outs))


@pytest.mark.gpu
def test_kept_state_follows_list_order_with_grouping_loaded(gb):
    import oracle
    from paper_2008_05718_gb300 import graphgen as gg
    g = gg.rmat(10, 16, seed=62)
    S = gg.sample_sources(g.n, 100, seed=63)
    _, ost = oracle.bc_graph(g, S, dump=(0, 37, 99))
    with gb.BC.from_graph(g, flags=gb.GBBC_KEEP_STATE) as bc:
        bc.load_grouping(mlp.init(1, seed=64).astype(np.float32))
        bc.compute(S)
        for i in (0, 37, 99):
            d, sig, _ = bc.source_state(i)
            assert np.array_equal(d, ost[i].dist)
            assert np.array_equal(sig, ost[i].sigma)


@pytest.mark.gpu
def test_shipped_grouping_gains_on_held_out_rmat(gb):
    # seeds not used in training; the predicted order must rank sources like
    # the true mean BFS distance and make the whole computation faster
    from paper_2008_05718_gb300 import graphgen as gg
    from paper_2008_05718_gb300 import grouping, policy
    p = grouping.shipped_weights()
    assert p is not None and len(p) == gb.bc_mlp_param_count(1)
    x, t, names = grouping.collect([("rmat15", gg.rmat(15, 16, seed=4245))], sources=256, seed=4246)
    rho = grouping.rank_correlation(grouping.predict(p, x), t)
    g = gg.rmat(16, 16, seed=4247)
    S = gg.sample_sources(g.n, 1024, seed=4248)
    r = grouping.time_orders(g, S, p, policy.shipped_weights(), reps=3)
    print("held-out rho", rho, "times", r)
    assert rho > 0.9
    assert r["identical_bits"]
    assert r["grouped"] < 0.85 * r["list"]
