"""ORACLE - test infrastructure, not part of the product.

Betweenness centrality straight from its definition (Eq. 1):
BC[v] = sum over ordered pairs (s, t), s != v != t, of sigma_st(v) / sigma_st,
where sigma_st counts shortest s-t paths and sigma_st(v) those passing v.

Every simple path from every source is enumerated by depth-first search; for
each target the shortest length found is d(s, t), the number of paths of that
length is sigma_st, and each interior vertex of such a path gets one count.
Sums are exact (fractions.Fraction).  Exponential time: graphs with n <= 10.
Works from an adjacency list built here from the edge list, independent of
any CSR builder.  The weighted form measures a path by the sum of its edge
weights (positive integers) instead of its edge count.
"""
from __future__ import annotations

from fractions import Fraction


def _adjacency(n, edges):
    adj = [set() for _ in range(n)]
    for u, v in edges:
        u, v = int(u), int(v)
        if u != v:
            adj[u].add(v)
            adj[v].add(u)
    return [sorted(a) for a in adj]


def shortest_paths(n, edges, s):
    """dict t -> (length, [paths]) of all shortest simple paths s -> t."""
    adj = _adjacency(n, edges)
    best = {}

    def dfs(path, on):
        x = path[-1]
        L = len(path) - 1
        if x != s:
            cur = best.get(x)
            if cur is None or L < cur[0]:
                best[x] = (L, [tuple(path)])
            elif L == cur[0]:
                cur[1].append(tuple(path))
        for y in adj[x]:
            if y not in on:
                on.add(y)
                path.append(y)
                dfs(path, on)
                path.pop()
                on.discard(y)

    dfs([s], {s})
    return best


def brute_bc(n, edges, sources=None):
    """(bc as list of Fraction, dist[s][t], sigma[s][t]) over the given sources
    (default: all vertices).  dist -1 and sigma 0 when t is unreachable;
    dist 0 and sigma 1 at t = s."""
    srcs = range(n) if sources is None else [int(s) for s in sources]
    bc = [Fraction(0)] * n
    dist, sigma = {}, {}
    for s in srcs:
        sp = shortest_paths(n, edges, s)
        d = [-1] * n
        c = [0] * n
        d[s], c[s] = 0, 1
        for t, (L, paths) in sp.items():
            d[t], c[t] = L, len(paths)
            through = [0] * n
            for p in paths:
                for v in p[1:-1]:
                    through[v] += 1
            for v in range(n):
                if through[v]:
                    bc[v] += Fraction(through[v], len(paths))
        dist[s], sigma[s] = d, c
    return bc, dist, sigma


def shortest_paths_weighted(n, wedges, s):
    """dict t -> (weight, [paths]) of all minimum-weight simple paths s -> t;
    wedges lists (u, v, weight) with positive integer weights."""
    adj = [dict() for _ in range(n)]
    for u, v, w in wedges:
        u, v, w = int(u), int(v), int(w)
        if u != v:
            adj[u][v] = w
            adj[v][u] = w
    best = {}

    def dfs(path, on, length):
        x = path[-1]
        if x != s:
            cur = best.get(x)
            if cur is None or length < cur[0]:
                best[x] = (length, [tuple(path)])
            elif length == cur[0]:
                cur[1].append(tuple(path))
        for y in sorted(adj[x]):
            if y not in on:
                on.add(y)
                path.append(y)
                dfs(path, on, length + adj[x][y])
                path.pop()
                on.discard(y)

    dfs([s], {s}, 0)
    return best


def brute_bc_weighted(n, wedges, sources=None):
    """Eq. 1 with path lengths measured by weight: (bc as Fractions,
    dist[s][t], sigma[s][t]) like brute_bc."""
    srcs = range(n) if sources is None else [int(x) for x in sources]
    bc = [Fraction(0)] * n
    dist, sigma = {}, {}
    for s in srcs:
        sp = shortest_paths_weighted(n, wedges, s)
        d = [-1] * n
        c = [0] * n
        d[s], c[s] = 0, 1
        for t, (L, paths) in sp.items():
            d[t], c[t] = L, len(paths)
            through = [0] * n
            for p in paths:
                for v in p[1:-1]:
                    through[v] += 1
            for v in range(n):
                if through[v]:
                    bc[v] += Fraction(through[v], len(paths))
        dist[s], sigma[s] = d, c
    return bc, dist, sigma
