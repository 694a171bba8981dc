"""Pins of the weighted (Dijkstra) oracle to facts fixed by the definition of
BC with weighted path lengths (Eq. 1 measured by weight) and by mathematics:
a hand-worked example, brute-force enumeration of minimum-weight paths with
exact rationals, the reduction to the unweighted oracle (itself pinned by
closed forms) at unit weights, and subdivision: an edge of weight c behaves,
for distances and path counts between original vertices, like a path of c
unit edges.  The mutation test at the end plants plausible slips in a copy of
the oracle and checks that a pin catches each."""
import os
import random
import subprocess

import numpy as np
import pytest

import oracle
from oracle.brute import brute_bc_weighted
from paper_2008_05718_gb300 import graphgen as gg

REL = 1e-12


def weighted_graph(n, wedges):
    g = gg.from_edges(n, [(u, v) for u, v, _ in wedges])
    w = {}
    for u, v, c in wedges:
        w[(u, v)] = w[(v, u)] = c
    u = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    return g, np.array([w[(int(a), int(b))] for a, b in zip(u, g.col)], np.int32)


def test_hand_example_weights_decide_the_paths():
    # square 0-1-3-2-0 with weights 01:1, 13:1, 02:1, 23:2.  Shortest paths:
    # 0->3 only via 1 (2 < 3); 1->2 only via 0 (2 < 3); 2->3 direct (2 < 3).
    # Ordered pairs: BC = [2, 2, 0, 0].  With unit weights every pair of
    # opposite corners has two paths: BC = [1, 1, 1, 1].
    g, w = weighted_graph(4, [(0, 1, 1), (1, 3, 1), (0, 2, 1), (2, 3, 2)])
    bc, st = oracle.bc_graph_weighted(g, w, np.arange(4), dump=(0,))
    assert np.array_equal(bc, [2.0, 2.0, 0.0, 0.0])
    assert np.array_equal(st[0].dist, [0, 1, 1, 2]) and np.array_equal(st[0].sigma, [1, 1, 1, 1])
    bc1, _ = oracle.bc_graph_weighted(g, np.ones_like(w), np.arange(4))
    assert np.array_equal(bc1, [1.0, 1.0, 1.0, 1.0])


@pytest.mark.parametrize("n", [2, 5, 9])
def test_weighted_path_closed_form(n):
    # a path has one path per pair whatever the weights: BC(i) = 2 i (n-1-i)
    g, w = weighted_graph(n, [(i, i + 1, 1 + (7 * i) % 5) for i in range(n - 1)])
    bc, _ = oracle.bc_graph_weighted(g, w, np.arange(n))
    assert np.array_equal(bc, [2.0 * i * (n - 1 - i) for i in range(n)])


def test_brute_force_random_weighted_graphs():
    rnd = random.Random(20)
    for trial in range(150):
        n = rnd.randint(2, 8)
        pairs = [(u, v) for u in range(n) for v in range(u + 1, n) if rnd.random() < 0.45]
        if not pairs:
            continue
        wedges = [(u, v, rnd.randint(1, 3)) for u, v in pairs]
        g, w = weighted_graph(n, wedges)
        want, dist, sigma = brute_bc_weighted(n, wedges)
        got, st = oracle.bc_graph_weighted(g, w, np.arange(n), dump=range(n))
        for v in range(n):
            assert abs(got[v] - float(want[v])) <= REL * max(1.0, abs(float(want[v]))), (trial, v)
        for s in range(n):
            assert list(st[s].dist) == dist[s]
            assert [int(x) for x in st[s].sigma] == sigma[s]


@pytest.mark.parametrize("make", [lambda: gg.rmat(9, 8, seed=31), lambda: gg.grid(20, "0.1", seed=32),
                                  lambda: gg.diamond_chain(70)])
def test_unit_weights_reduce_to_the_unweighted_oracle(make):
    g = make()
    S = gg.sample_sources(g.n, min(40, g.n), seed=33)
    keep = (0, len(S) - 1)
    a, sa = oracle.bc_graph(g, S, dump=keep)
    b, sb = oracle.bc_graph_weighted(g, np.ones(g.nnz, np.int32), S, dump=keep)
    assert np.allclose(b, a, rtol=REL, atol=1e-15)
    for i in keep:
        assert np.array_equal(sa[i].dist, sb[i].dist)
        assert np.array_equal(sa[i].sigma, sb[i].sigma)
        assert np.array_equal(sa[i].ovf, sb[i].ovf)


@pytest.mark.parametrize("maxw", [2, 4])
def test_subdivision_gives_the_same_distances_and_path_counts(maxw):
    g = gg.rmat(8, 6, seed=40 + maxw)
    w = gg.edge_weights(g, maxw, seed=41)
    h = gg.subdivide(g, w)
    S = gg.sample_sources(g.n, 12, seed=42)
    keep = tuple(range(len(S)))
    _, sw = oracle.bc_graph_weighted(g, w, S, dump=keep)
    _, su = oracle.bc_graph(h, S, dump=keep)
    for i in keep:
        assert np.array_equal(sw[i].dist, su[i].dist[: g.n])
        assert np.array_equal(sw[i].sigma, su[i].sigma[: g.n])


def test_scaling_all_weights_changes_nothing():
    g = gg.grid(15, "0.1", seed=50)
    w = gg.edge_weights(g, 3, seed=51)
    S = gg.sample_sources(g.n, 30, seed=52)
    a, _ = oracle.bc_graph_weighted(g, w, S)
    b, _ = oracle.bc_graph_weighted(g, 5 * w, S)
    assert np.array_equal(a, b)


def test_unreachable_and_rejections():
    g, w = weighted_graph(5, [(0, 1, 2), (1, 2, 3)])  # 3, 4 isolated
    bc, st = oracle.bc_graph_weighted(g, w, [0, 3], dump=(0, 1))
    assert list(st[0].dist) == [0, 2, 5, -1, -1] and list(st[1].dist) == [-1, -1, -1, 0, -1]
    assert bc[1] == 1.0 and bc[0] == 0.0 and bc[3] == 0.0
    with pytest.raises(ValueError):
        oracle.bc_graph_weighted(g, np.zeros_like(w), [0])
    with pytest.raises(ValueError):
        oracle.bc_graph_weighted(g, w, [5])
    big, wb = weighted_graph(3, [(0, 1, 2**30), (1, 2, 2**30)])
    with pytest.raises(ValueError):
        oracle.bc_graph_weighted(big, wb, [0])


# ---- mutation check ----------------------------------------------------------

MUTANTS = {
    "relax_ignores_weight": ("int64_t nd = dist[u] + (int64_t)weight[p];", "int64_t nd = dist[u] + 1;"),
    "drop_one_plus_weighted": ("* (1.0 + delta[w]);", "* (delta[w]);"),
    "heap_max_first": ("if (l < *len && h[l].d < h[m].d) m = l;", "if (l < *len && h[l].d > h[m].d) m = l;"),
    "sigma_skips_first_settled": ("for (int64_t q = 1; q < nset; ++q) {\n            int32_t w = order[q];\n"
                                  "            int32_t maxlen = 1;",
                                  "for (int64_t q = 2; q < nset; ++q) {\n            int32_t w = order[q];\n"
                                  "            int32_t maxlen = 1;"),
    "backward_in_settle_order": ("for (int64_t q = nset - 1; q > 0; --q) {", "for (int64_t q = 1; q < nset; ++q) {"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_weighted_pins_catch_planted_mistake(name, tmp_path):
    import ctypes
    src = open(os.path.join(os.path.dirname(oracle.__file__), "brandes.c")).read()
    a, b = MUTANTS[name]
    assert src.count(a) == 1, name
    p = tmp_path / "m.c"
    p.write_text(src.replace(a, b))
    so = tmp_path / "m.so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-o", str(so), str(p), "-lm"])
    lib = ctypes.CDLL(str(so))
    ref = oracle._load()
    for f in ("oracle_bc", "oracle_bc_weighted", "oracle_big_to_scaled"):
        getattr(lib, f).argtypes = getattr(ref, f).argtypes
        getattr(lib, f).restype = getattr(ref, f).restype
    saved = oracle._lib
    try:
        oracle._lib = lib
        failed = False
        for check in (test_hand_example_weights_decide_the_paths, lambda: test_weighted_path_closed_form(9),
                      test_brute_force_random_weighted_graphs,
                      lambda: test_subdivision_gives_the_same_distances_and_path_counts(4)):
            try:
                check()
            except AssertionError:
                failed = True
                break
        assert failed, f"mutant {name} survived every pin"
    finally:
        oracle._lib = saved
