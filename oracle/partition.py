"""ORACLE - test infrastructure, not part of the product.

Border nodes and border matrices of a partitioned graph, by their plain
definitions (Sec. IV: notations and Sec. IV-B; the sigma matrix of Sec. V-A):

  - a border edge (edge cut) joins two vertices of different parts; its end
    points are border nodes;
  - for part p with border nodes b_0 < b_1 < ... (vertex order),
    BM_p[i][j] is the length of a shortest path from b_i to b_j that uses
    only vertices and edges of part p (-1 when there is none), and
    sigmaM_p[i][j] the number of such shortest paths (0 when none).

Everything is plain Python over the CSR: a queue BFS inside the part from
each border node, with exact (unbounded) integer path counts.  For the small
graphs of the tests only.
"""
from __future__ import annotations

from collections import deque

import numpy as np


def border_nodes(n, row_ptr, col, part):
    """Sorted vertex ids of the border nodes of each part: [array per part]."""
    part = np.asarray(part)
    P = int(part.max()) + 1 if n else 0
    out = [[] for _ in range(P)]
    for v in range(n):
        for p in range(row_ptr[v], row_ptr[v + 1]):
            if part[col[p]] != part[v]:
                out[part[v]].append(v)
                break
    return [np.array(b, np.int32) for b in out]


def bfs_in_part(n, row_ptr, col, part, s):
    """(dist, sigma) from s over the vertices and edges of part[s] only:
    dist -1 and sigma 0 outside it or where unreachable; sigma exact ints."""
    dist = [-1] * n
    sigma = [0] * n
    dist[s] = 0
    sigma[s] = 1
    q = deque([s])
    ps = part[s]
    while q:
        v = q.popleft()
        for p in range(row_ptr[v], row_ptr[v + 1]):
            w = int(col[p])
            if part[w] != ps:
                continue
            if dist[w] < 0:
                dist[w] = dist[v] + 1
                q.append(w)
            if dist[w] == dist[v] + 1:
                sigma[w] += sigma[v]
    return dist, sigma


def border_matrices(n, row_ptr, col, part):
    """[(border ids, BM int64 [b, b], sigmaM as a list of lists of exact ints)] per part."""
    part = np.asarray(part)
    res = []
    for b in border_nodes(n, row_ptr, col, part):
        k = len(b)
        bm = np.full((k, k), -1, np.int64)
        sm = [[0] * k for _ in range(k)]
        for i, bi in enumerate(b):
            d, s = bfs_in_part(n, row_ptr, col, part, int(bi))
            for j, bj in enumerate(b):
                bm[i, j] = d[bj]
                sm[i][j] = s[bj]
        res.append((b, bm, sm))
    return res
