"""Input generators: CSR validity, shapes of the workload classes, and
byte-for-byte determinism across machines (goldens written by
tests/golden/make_graph_hashes.py)."""
import json
import os

import numpy as np
import pytest

from paper_2008_05718_gb300 import graphgen as gg

GOLD = os.path.join(os.path.dirname(__file__), "golden", "graph_hashes.json")


def assert_valid_csr(g):
    rp, col = g.row_ptr, g.col
    assert rp.dtype == np.int32 and col.dtype == np.int32
    assert rp[0] == 0 and len(rp) == g.n + 1 and rp[-1] == len(col)
    assert np.all(np.diff(rp) >= 0)
    if len(col):
        assert col.min() >= 0 and col.max() < g.n
    u = np.repeat(np.arange(g.n), np.diff(rp))
    assert not np.any(u == col), "self-loop"
    key = u.astype(np.int64) * g.n + col
    assert np.all(np.diff(key) > 0), "rows not strictly sorted (duplicate or unsorted)"
    rev = col.astype(np.int64) * g.n + u
    assert np.array_equal(np.sort(rev), key), "not symmetric"


@pytest.mark.parametrize("make", [
    lambda: gg.er(500, "0.01", seed=3),
    lambda: gg.rmat(10, 16, seed=4),
    lambda: gg.rmat(11, 8, seed=4, permute=False),
    lambda: gg.grid(50, "0.05", seed=5),
    lambda: gg.grid(30, "0", seed=5, lcc=False),
    lambda: gg.diamond_chain(5),
    lambda: gg.full_grid(7, 9),
    lambda: gg.from_edges(6, [(0, 0), (1, 2), (2, 1), (1, 2), (5, 3)]),
])
def test_csr_valid(make):
    assert_valid_csr(make())


def test_goldens_match():
    import importlib.util
    spec = importlib.util.spec_from_file_location("mk", os.path.join(os.path.dirname(GOLD), "make_graph_hashes.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    assert mk.compute() == json.load(open(GOLD))


def test_er_shape():
    g, S = gg.workload("er4096")
    assert g.n == 4096 and len(S) == 4096
    assert abs(g.nnz / g.n - 8) < 0.3  # average degree 8


def test_rmat_shape_and_permutation():
    g = gg.rmat(12, 16, seed=1)
    assert g.n == 4096 and 0.5 * 2 * 16 * 4096 < g.nnz <= 2 * 16 * 4096
    d = g.degrees()
    # permuted: the hub is not vertex 0 and max degree is heavy-tailed
    assert d.max() > 20 * d.mean()
    h = gg.rmat(12, 16, seed=1, permute=False)
    assert h.degrees()[0] == h.degrees().max()


def test_grid_lcc_connected_and_degree():
    g = gg.grid(80, "0.05", seed=2)
    assert g.degrees().max() <= 4
    lcc, old = gg.largest_cc(g)
    assert lcc.n == g.n and np.array_equal(old, np.arange(g.n))
    full = gg.grid(80, "0", seed=2)
    assert full.n == 6400 and full.nnz == 4 * 80 * 79


def test_sources_distinct_and_deterministic():
    a = gg.sample_sources(1000, 500, seed=9)
    assert len(set(a.tolist())) == 500 and a.min() >= 0 and a.max() < 1000
    assert np.array_equal(a, gg.sample_sources(1000, 500, seed=9))
    assert not np.array_equal(a, gg.sample_sources(1000, 500, seed=10))


def test_union_offsets():
    gs = [gg.path(3), gg.star(4), gg.cycle(5)]
    u, off = gg.union(gs)
    assert list(off) == [0, 3, 7, 12]
    assert_valid_csr(u)
    assert u.nnz == sum(g.nnz for g in gs)


def test_bad_edge_rejected():
    with pytest.raises(ValueError):
        gg.from_edges(3, [(0, 3)])
