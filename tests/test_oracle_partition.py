"""Pins of the oracle's border nodes and border matrices (Sec. IV-B, and the
sigma matrix of Sec. V-A) against closed forms: paths, cycles and grids cut
into parts, where shortest paths inside a part are known exactly."""
from math import comb

import numpy as np

from oracle import partition as op
from paper_2008_05718_gb300 import graphgen as gg


def test_path_cut_in_two():
    g = gg.path(10)
    part = np.array([0] * 4 + [1] * 6)
    res = op.border_matrices(g.n, g.row_ptr, g.col, part)
    assert [list(b) for b, _, _ in res] == [[3], [4]]
    for _, bm, sm in res:
        assert bm.tolist() == [[0]] and sm == [[1]]


def test_cycle_cut_into_arcs():
    n, a = 15, 6
    g = gg.cycle(n)
    part = np.array([0] * a + [1] * (n - a))
    (b0, bm0, sm0), (b1, bm1, sm1) = op.border_matrices(g.n, g.row_ptr, g.col, part)
    assert list(b0) == [0, a - 1] and list(b1) == [a, n - 1]
    # the only path inside an arc runs along it
    assert bm0.tolist() == [[0, a - 1], [a - 1, 0]] and sm0 == [[1, 1], [1, 1]]
    assert bm1.tolist() == [[0, n - 1 - a], [n - 1 - a, 0]] and sm1 == [[1, 1], [1, 1]]


def test_grid_cut_into_two_halves_by_columns():
    rows, cols, c = 7, 9, 4
    g = gg.full_grid(rows, cols)
    part = np.array([0 if (v % cols) < c else 1 for v in range(g.n)])
    (b0, bm0, sm0), (b1, bm1, sm1) = op.border_matrices(g.n, g.row_ptr, g.col, part)
    assert list(b0) == [i * cols + c - 1 for i in range(rows)]
    assert list(b1) == [i * cols + c for i in range(rows)]
    # along one column: distance |i - j|, and a single shortest path (any
    # step away from the column costs two more)
    for bm, sm in ((bm0, sm0), (bm1, sm1)):
        for i in range(rows):
            for j in range(rows):
                assert bm[i, j] == abs(i - j) and sm[i][j] == 1


def test_grid_cut_into_four_quadrants():
    # in the top-left quadrant the border nodes are its last column and its
    # last row; between two of them every monotone lattice path stays inside
    # the quadrant, so BM is the Manhattan distance and sigmaM the binomial
    R = C = 10
    r, c = 5, 6
    g = gg.full_grid(R, C)
    part = np.array([(0 if (v // C) < r else 2) + (0 if (v % C) < c else 1) for v in range(g.n)])
    res = op.border_matrices(g.n, g.row_ptr, g.col, part)
    b, bm, sm = res[0]
    want = sorted({i * C + c - 1 for i in range(r)} | {(r - 1) * C + j for j in range(c)})
    assert list(b) == want
    for x, u in enumerate(b):
        for y, w in enumerate(b):
            di, dj = abs(u // C - w // C), abs(u % C - w % C)
            assert bm[x, y] == di + dj
            assert sm[x][y] == comb(di + dj, di)
    # every part: symmetric, zero diagonal, one path to itself
    for b, bm, sm in res:
        assert np.array_equal(bm, bm.T) and np.all(np.diag(bm) == 0)
        assert all(sm[i][i] == 1 for i in range(len(b)))


def test_no_cut_no_border_nodes_and_inside_distances_bound_the_graph():
    g = gg.rmat(8, 8, seed=3)
    assert all(len(b) == 0 for b in op.border_nodes(g.n, g.row_ptr, g.col, np.zeros(g.n, np.int64)))
    import oracle
    part = (np.arange(g.n) * 3) // g.n
    for b, bm, _ in op.border_matrices(g.n, g.row_ptr, g.col, part):
        for i, bi in enumerate(b[:5]):
            _, st = oracle.bc_graph(g, [int(bi)], dump=(0,))
            d = st[0].dist[b]
            # a path inside the part is a path of the graph: never shorter
            assert np.all((bm[i] < 0) | (bm[i] >= d))
