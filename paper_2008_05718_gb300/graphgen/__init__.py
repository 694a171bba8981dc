"""Seeded synthetic inputs: undirected graphs in CSR form and source lists.

This module is the one piece shared by the CUDA library's tests and the CPU
oracle: it writes inputs and holds none of the betweenness-centrality
arithmetic.  The generators live in ``graphgen.c`` (plain C, integer-only
SplitMix64 randomness, so the same seed gives the same bytes on x86-64 and
AArch64); this wrapper compiles it on first use and returns numpy arrays.

Graph families (shapes of the paper's workload classes, Table I of Sec. VI):
Erdos-Renyi G(n, p), R-MAT scale-free graphs (social/web class), 4-neighbour
grids with edges removed (road-network class: high diameter, degree <= 4),
and small closed-form graphs (path, star, cycle, complete, complete
bipartite, diamond chain, full grid) used to pin the oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgbgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into libgbgen.so (gcc, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _CSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.POINTER(ctypes.c_int32)), ("col", ctypes.POINTER(ctypes.c_int32))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            i32p = P(ctypes.c_int32)
            lib.gg_from_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, P(_CSR)]
            lib.gg_er.argtypes = [ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64, P(_CSR)]
            lib.gg_rmat.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, P(_CSR)]
            lib.gg_grid.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, P(_CSR)]
            lib.gg_lcc.argtypes = [P(_CSR), P(_CSR), i32p]
            lib.gg_components.argtypes = [P(_CSR), i32p]
            lib.gg_components.restype = ctypes.c_int32
            lib.gg_tri.argtypes = [ctypes.c_int32, ctypes.c_uint64, P(_CSR)]
            lib.gg_weights.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int32, ctypes.c_uint64, i32p]
            lib.gg_rgg.argtypes = [ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int32, P(_CSR)]
            lib.gg_mesh27.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P(_CSR)]
            lib.gg_sample_sources.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, i32p]
            lib.gg_permutation.argtypes = [ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64, i32p]
            lib.gg_rng.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
            lib.gg_rng.restype = ctypes.c_uint64
            lib.gg_free_csr.argtypes = [P(_CSR)]
            for f in ("gg_from_edges", "gg_er", "gg_rmat", "gg_grid", "gg_lcc", "gg_sample_sources",
                      "gg_permutation"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclass
class Graph:
    """Undirected graph in CSR form (symmetric, sorted rows, no loops/duplicates)."""
    n: int
    row_ptr: np.ndarray  # int32[n + 1]
    col: np.ndarray      # int32[nnz]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))

    def edges(self):
        """Undirected edge list (u < v) as an int32 [m, 2] array."""
        u = np.repeat(np.arange(self.n, dtype=np.int32), self.degrees())
        keep = u < self.col
        return np.stack([u[keep], self.col[keep]], axis=1)


def _take(c: _CSR, name: str, meta=None) -> Graph:
    lib = _load()
    n = c.n
    rp = np.ctypeslib.as_array(c.row_ptr, shape=(n + 1,)).copy() if c.row_ptr else np.zeros(1, np.int32)
    nnz = int(rp[-1])
    col = np.ctypeslib.as_array(c.col, shape=(max(nnz, 1),))[:nnz].copy() if c.col else np.zeros(0, np.int32)
    lib.gg_free_csr(ctypes.byref(c))
    return Graph(n, rp, col, name, dict(meta or {}))


def _i32p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def from_edges(n: int, edges, name: str = "edges") -> Graph:
    """Symmetrise, drop self-loops, deduplicate and sort an edge list into CSR."""
    e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
    u = np.ascontiguousarray(e[:, 0])
    v = np.ascontiguousarray(e[:, 1])
    c = _CSR()
    if _load().gg_from_edges(int(n), int(len(u)), _i32p(u), _i32p(v), ctypes.byref(c)) != 0:
        raise ValueError("gg_from_edges: bad vertex id or graph too large")
    return _take(c, name)


def rng(seed: int, stream: int, i: int) -> int:
    """Value i of the SplitMix64 stream (seed, stream)."""
    return int(_load().gg_rng(seed, stream, i))


def er(n: int, p, seed: int) -> Graph:
    """Erdos-Renyi G(n, p) with p given exactly (Fraction or str)."""
    p = Fraction(p)
    thr = min((p * (1 << 64)).__floor__(), (1 << 64) - 1)
    c = _CSR()
    if _load().gg_er(int(n), thr, int(seed), ctypes.byref(c)) != 0:
        raise MemoryError("gg_er failed")
    return _take(c, f"er_n{n}", {"p": str(p), "seed": seed})


RMAT_ABCD = ("0.57", "0.19", "0.19", "0.05")


def rmat(scale: int, edge_factor: int = 16, abcd=RMAT_ABCD, seed: int = 0, permute: bool = True) -> Graph:
    """R-MAT graph: 2^scale vertices, edge_factor * 2^scale generated edges,
    quadrant probabilities (a, b, c, d), symmetrised and deduplicated."""
    a, b, c_, d = (Fraction(x) for x in abcd)
    if a + b + c_ + d != 1:
        raise ValueError("R-MAT probabilities must sum to 1")
    t = [min(int(x * (1 << 32)), (1 << 32) - 1) for x in (a, a + b, a + b + c_)]
    c = _CSR()
    if _load().gg_rmat(int(scale), int(edge_factor), t[0], t[1], t[2], int(seed), int(bool(permute)),
                       ctypes.byref(c)) != 0:
        raise MemoryError("gg_rmat failed")
    return _take(c, f"rmat_s{scale}_ef{edge_factor}", {"seed": seed, "abcd": tuple(abcd)})


def grid(side: int, remove_frac="0", seed: int = 0, lcc: bool = True) -> Graph:
    """side x side 4-neighbour grid with floor(remove_frac * |E|) edges removed
    uniformly at random; the largest component is kept (row-major relabel)."""
    E = 2 * side * (side - 1)
    rm = (Fraction(remove_frac) * E).__floor__()
    c = _CSR()
    if _load().gg_grid(int(side), int(rm), int(seed), int(bool(lcc)), ctypes.byref(c)) != 0:
        raise MemoryError("gg_grid failed")
    return _take(c, f"grid_{side}", {"removed": rm, "seed": seed})


def tri(side: int, seed: int = 0) -> Graph:
    """Planar triangulation of a side x side lattice (grid edges plus one
    random diagonal per cell): a Delaunay-like planar graph, average degree
    about 6, diameter about 2 * side."""
    c = _CSR()
    if _load().gg_tri(int(side), int(seed), ctypes.byref(c)) != 0:
        raise ValueError("gg_tri failed")
    return _take(c, f"tri{side}", {"side": side, "seed": seed})


def rgg_threshold(n: int, avg_deg: float) -> int:
    """Squared radius, in units of the 2^32-sided square, that gives expected
    degree avg_deg (boundary effects aside): r^2 = avg_deg / (pi * n)."""
    import math
    r2 = int(avg_deg / (math.pi * n) * float(1 << 64))
    return max(1, min(r2, (1 << 64) - 1))


def rgg(n: int, avg_deg: float = 10.0, seed: int = 0, lcc: bool = True) -> Graph:
    """Random geometric graph on n uniform points of the unit square, an edge
    where the distance is below r with pi r^2 n = avg_deg; vertices numbered in
    spatial cell order; the largest component kept by default."""
    c = _CSR()
    r2 = rgg_threshold(n, avg_deg)
    if _load().gg_rgg(int(n), r2, int(seed), 1 if lcc else 0, ctypes.byref(c)) != 0:
        raise ValueError("gg_rgg failed")
    return _take(c, f"rgg_n{n}", {"n": n, "avg_deg": avg_deg, "seed": seed, "r2": r2})


def mesh27(nx: int, ny: int = None, nz: int = None) -> Graph:
    """3-D mesh with the 27-point stencil (26 neighbours inside): the banded
    sparsity of the KKT matrices of 3-D PDE-constrained optimisation."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    c = _CSR()
    if _load().gg_mesh27(int(nx), int(ny), int(nz), ctypes.byref(c)) != 0:
        raise ValueError("gg_mesh27 failed")
    return _take(c, f"mesh27_{nx}x{ny}x{nz}", {"dims": (nx, ny, nz)})


def edge_weights(g: Graph, max_weight: int, seed: int) -> np.ndarray:
    """Positive integer weights in [1, max_weight] aligned with g.col, one per
    undirected edge (both CSR entries of an edge carry the same weight)."""
    out = np.zeros(max(g.nnz, 1), np.int32)
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(g.col if g.nnz else np.zeros(1, np.int32), dtype=np.int32)
    if _load().gg_weights(int(g.n), _i32p(rp), _i32p(cl), int(max_weight), int(seed), _i32p(out)) != 0:
        raise ValueError("gg_weights: bad arguments")
    return out[: g.nnz]


def subdivide(g: Graph, weight: np.ndarray) -> Graph:
    """Replace every edge {u, v} of weight c by a path of c unit edges through
    c - 1 new vertices (numbered from g.n on); original vertices keep their ids."""
    edges = []
    nxt = g.n
    for u in range(g.n):
        for p in range(g.row_ptr[u], g.row_ptr[u + 1]):
            v = int(g.col[p])
            if u >= v:
                continue
            c = int(weight[p])
            prev = u
            for _ in range(c - 1):
                edges.append((prev, nxt))
                prev = nxt
                nxt += 1
            edges.append((prev, v))
    return from_edges(nxt, edges, name=g.name + "_subdivided")


def largest_cc(g: Graph) -> tuple[Graph, np.ndarray]:
    """Largest connected component and the old id of each kept vertex."""
    src = _CSR(g.n, g.nnz, _i32p(g.row_ptr), _i32p(g.col))
    old = np.zeros(max(g.n, 1), np.int32)
    c = _CSR()
    if _load().gg_lcc(ctypes.byref(src), ctypes.byref(c), _i32p(old)) != 0:
        raise MemoryError("gg_lcc failed")
    out = _take(c, g.name + "_lcc")
    return out, old[: out.n].copy()


def component_labels(g: Graph) -> np.ndarray:
    """Connected-component label of every vertex (labels numbered from the
    smallest vertex id)."""
    src = _CSR(g.n, g.nnz, _i32p(g.row_ptr), _i32p(g.col))
    comp = np.zeros(max(g.n, 1), np.int32)
    if _load().gg_components(ctypes.byref(src), _i32p(comp)) < 0:
        raise MemoryError("gg_components failed")
    return comp[: g.n].copy()


def component_entries(g: Graph) -> np.ndarray:
    """For every vertex, the CSR entries (directed edges) of its connected
    component: the edges a BFS from that vertex traverses."""
    comp = component_labels(g)
    per = np.bincount(comp, weights=np.diff(g.row_ptr).astype(np.float64), minlength=int(comp.max(initial=-1)) + 1)
    return per[comp].astype(np.int64)


def sample_sources(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct vertices drawn uniformly from [0, n) (seeded Fisher-Yates)."""
    out = np.zeros(max(k, 1), np.int32)
    if _load().gg_sample_sources(int(n), int(k), int(seed), _i32p(out)) != 0:
        raise ValueError("k > n")
    return out[:k].copy()


def permutation(n: int, seed: int, stream: int = 7) -> np.ndarray:
    out = np.zeros(max(n, 1), np.int32)
    _load().gg_permutation(int(n), int(seed), int(stream), _i32p(out))
    return out[:n].copy()


def relabel(g: Graph, perm: np.ndarray) -> Graph:
    """Graph with vertex v renamed perm[v]."""
    e = g.edges()
    return from_edges(g.n, perm[e], g.name + "_perm")


# ---- closed-form graphs (inputs for the oracle's pins) ----------------------

def path(n: int) -> Graph:
    return from_edges(n, [(i, i + 1) for i in range(n - 1)], f"path{n}")


def star(n: int) -> Graph:
    """Centre 0 joined to leaves 1..n-1."""
    return from_edges(n, [(0, i) for i in range(1, n)], f"star{n}")


def cycle(n: int) -> Graph:
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], f"cycle{n}")


def complete(n: int) -> Graph:
    return from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)], f"K{n}")


def complete_bipartite(a: int, b: int) -> Graph:
    """Side A = 0..a-1, side B = a..a+b-1."""
    return from_edges(a + b, [(i, a + j) for i in range(a) for j in range(b)], f"K{a},{b}")


def diamond_chain(k: int) -> Graph:
    """k diamonds in a row: c_0 - {a_1, b_1} - c_1 - ... - c_k.
    Ids: c_i = 3i, a_i = 3i - 2, b_i = 3i - 1 (i >= 1); n = 3k + 1."""
    e = []
    for i in range(1, k + 1):
        c0, a, b, c1 = 3 * (i - 1), 3 * i - 2, 3 * i - 1, 3 * i
        e += [(c0, a), (c0, b), (a, c1), (b, c1)]
    return from_edges(3 * k + 1, e, f"diamond{k}")


def full_grid(rows: int, cols: int) -> Graph:
    """rows x cols 4-neighbour grid, vertex (i, j) = i * cols + j."""
    e = []
    for i in range(rows):
        for j in range(cols):
            v = i * cols + j
            if j + 1 < cols:
                e.append((v, v + 1))
            if i + 1 < rows:
                e.append((v, v + cols))
    return from_edges(rows * cols, e, f"fullgrid{rows}x{cols}")


def union(graphs) -> tuple[Graph, np.ndarray]:
    """Disjoint union; returns the union graph and vertex offsets[len+1]."""
    offs = np.zeros(len(graphs) + 1, np.int64)
    for i, g in enumerate(graphs):
        offs[i + 1] = offs[i] + g.n
    rps, cols = [np.zeros(1, np.int64)], []
    base = 0
    for i, g in enumerate(graphs):
        rps.append(g.row_ptr[1:].astype(np.int64) + base)
        cols.append(g.col.astype(np.int64) + offs[i])
        base += g.nnz
    rp = np.concatenate(rps)
    if rp[-1] >= 2**31 or offs[-1] >= 2**31:
        raise ValueError("union too large for int32 CSR")
    col = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    return Graph(int(offs[-1]), rp.astype(np.int32), col.astype(np.int32), "union"), offs


# ---- the five benchmark workloads ------------------------------------------

def workload(name: str):
    """Return (graph, sources) for the named workload.

    er4096   : ER n=4096, p=8/4095, seed 1, all vertices as sources.
    rmat18   : R-MAT scale 18, ef 16, seed 2, 4096 uniform sources.
    grid1024 : 1024^2 grid, 5% edges removed, LCC, seed 3, 1024 uniform sources.
    rmat22   : R-MAT scale 22, ef 16, seed 5, 16384 uniform sources.
    tri1024  : planar triangulation of a 1024^2 lattice (Delaunay-like), seed 6,
               1024 uniform sources.
    rgg20    : random geometric graph, 2^20 points, expected degree 10, LCC,
               seed 7, 1024 uniform sources.
    mesh100  : 100^3 mesh, 27-point stencil (KKT-like), 4096 uniform sources
               (seed 8).
    Small variants for tests: rmat<s> (any scale), grid<side>, tri<side>,
    rgg<log2 n>, mesh<side>.
    """
    if name == "er4096":
        g = er(4096, Fraction(8, 4095), seed=1)
        return g, np.arange(g.n, dtype=np.int32)
    if name == "grid1024":
        g = grid(1024, Fraction(5, 100), seed=3)
        return g, sample_sources(g.n, 1024, seed=3)
    if name.startswith("rmat"):
        s = int(name[4:])
        seed = {18: 2, 22: 5}.get(s, 1000 + s)
        k = {18: 4096, 22: 16384}.get(s, 256)
        g = rmat(s, 16, seed=seed)
        return g, sample_sources(g.n, min(k, g.n), seed=seed)
    if name.startswith("grid"):
        side = int(name[4:])
        g = grid(side, Fraction(5, 100), seed=3000 + side)
        return g, sample_sources(g.n, min(256, g.n), seed=3000 + side)
    if name.startswith("tri"):
        side = int(name[3:])
        seed = 6 if side == 1024 else 6000 + side
        g = tri(side, seed=seed)
        return g, sample_sources(g.n, min(1024 if side == 1024 else 256, g.n), seed=seed)
    if name.startswith("rgg"):
        s = int(name[3:])
        seed = 7 if s == 20 else 7000 + s
        g = rgg(1 << s, 10.0, seed=seed)
        return g, sample_sources(g.n, min(1024 if s == 20 else 256, g.n), seed=seed)
    if name.startswith("mesh"):
        side = int(name[4:])
        g = mesh27(side)
        seed = 8 if side == 100 else 8000 + side
        return g, sample_sources(g.n, min(4096 if side == 100 else 256, g.n), seed=seed)
    raise KeyError(name)


@dataclass
class MultiWorkload:
    graphs: list
    sources: list  # per-graph local source arrays
    kinds: list


def multi_workload(seed: int = 4, count: int = 256, scale_range=(10, 16), side_range=(64, 512),
                   remove_frac="0.03", full_scale=12, full_side=128, sampled=1024) -> MultiWorkload:
    """256 independent graphs: the first half R-MAT (scale uniform in
    scale_range, ef 16), the second half grids (side uniform in side_range,
    remove_frac removed, LCC).  All vertices are sources on graphs with
    scale <= full_scale or side <= full_side, else `sampled` uniform sources."""
    graphs, sources, kinds = [], [], []
    half = count // 2
    for i in range(count):
        sub = rng(seed, 11, i)
        if i < half:
            s = scale_range[0] + rng(seed, 12, i) % (scale_range[1] - scale_range[0] + 1)
            g = rmat(int(s), 16, seed=sub)
            full = s <= full_scale
            kinds.append(("rmat", int(s)))
        else:
            side = side_range[0] + rng(seed, 13, i) % (side_range[1] - side_range[0] + 1)
            g = grid(int(side), remove_frac, seed=sub)
            full = side <= full_side
            kinds.append(("grid", int(side)))
        graphs.append(g)
        src = np.arange(g.n, dtype=np.int32) if full else sample_sources(g.n, min(sampled, g.n), seed=sub)
        sources.append(src)
    return MultiWorkload(graphs, sources, kinds)
