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
    lambda: gg.tri(40, seed=6),
    lambda: gg.rgg(3000, 10.0, seed=7),
    lambda: gg.rgg(3000, 3.0, seed=7, lcc=False),
    lambda: gg.mesh27(7, 5, 4),
])
def test_csr_valid(make):
    assert_valid_csr(make())


def test_tri_is_a_lattice_triangulation():
    side = 37
    g = gg.tri(side, seed=11)
    assert g.n == side * side
    cells = (side - 1) ** 2
    assert g.nnz == 2 * (2 * side * (side - 1) + cells)  # grid edges + one diagonal per cell
    assert g.nnz // 2 <= 3 * g.n - 6  # planar (Euler)
    E = {(int(a), int(b)) for a, b in g.edges()}
    for i in range(side - 1):
        for j in range(side - 1):
            a = i * side + j
            d1 = (a, a + side + 1) in E
            d2 = (a + 1, a + side) in E
            assert d1 != d2  # exactly one diagonal per cell
    deg = g.degrees()
    assert deg.min() >= 2 and deg.max() <= 8
    assert 5.7 < deg.mean() < 6.0  # 6 inside, less on the boundary


def test_rgg_edges_are_exactly_the_close_pairs():
    # brute force over all pairs with the generator's own coordinates (the
    # SplitMix64 stream of the seed), mapped through the spatial numbering
    import math
    n, seed = 700, 21
    g = gg.rgg(n, 10.0, seed=seed, lcc=False)
    r2 = gg.rgg_threshold(n, 10.0)
    xs = np.array([gg.rng(seed, 7, 2 * i) >> 32 for i in range(n)], dtype=np.int64)
    ys = np.array([gg.rng(seed, 7, 2 * i + 1) >> 32 for i in range(n)], dtype=np.int64)
    cs = math.isqrt(r2)
    cs += cs * cs < r2
    C = -(-(1 << 32) // cs)
    cmax = max(1, math.isqrt(n))
    if C > cmax:
        C = cmax
        cs = -(-(1 << 32) // C)
    cell = (ys // cs) * C + xs // cs
    order = np.lexsort((np.arange(n), cell))  # cell order, generation order within a cell
    new_id = np.empty(n, np.int64)
    new_id[order] = np.arange(n)
    want = set()
    for i in range(n):
        for j in range(i + 1, n):
            dx, dy = int(xs[i] - xs[j]), int(ys[i] - ys[j])
            if dx * dx + dy * dy < r2:
                a, b = sorted((int(new_id[i]), int(new_id[j])))
                want.add((a, b))
    got = {(int(a), int(b)) for a, b in g.edges()}
    assert got == want
    assert 7.0 < 2 * len(want) / n < 11.0  # expected degree 10 less the boundary loss


def test_mesh27_degrees_closed_form():
    nx, ny, nz = 6, 5, 4
    g = gg.mesh27(nx, ny, nz)
    deg = g.degrees()
    for x in range(nx):
        for y in range(ny):
            for z in range(nz):
                per = [1 + (c > 0) + (c < m - 1) for c, m in ((x, nx), (y, ny), (z, nz))]
                assert deg[(x * ny + y) * nz + z] == per[0] * per[1] * per[2] - 1
    assert g.nnz == deg.sum()
    # the chebyshev distance is the BFS distance: diameter = max side - 1
    assert gg.mesh27(9, 3, 2).n == 54


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
