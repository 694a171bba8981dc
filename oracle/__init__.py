"""ORACLE - test infrastructure, not part of the product.

Plain CPU reference for exact Brandes betweenness centrality (Sec. II of the
paper: Eq. 1, Eq. 2 and Algorithm 1).  Only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import this
package.  It shares no code with the CUDA library: the C source here is
compiled on its own with gcc, and nothing here imports the product package
except, in tests, through the separate input generators.

  brandes.c  single-threaded Brandes per Algorithm 1, exact (multi-limb)
             sigma, FP64 delta and BC                              -> bc()
             and its weighted (Dijkstra) form                      -> bc_weighted()
  brute.py   Eq. 1 evaluated by enumerating every shortest path, exact
             rationals, for graphs with n <= 10 (edge counts or
             weights as path lengths)                              -> brute
  mlp.py     FP64 numpy reference of the policy network (forward, analytic
             gradients, Adam step)                                 -> mlp
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "brandes.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile brandes.c with gcc (no -ffast-math: IEEE double semantics)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            lib.oracle_bc.argtypes = [ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_int32), ctypes.c_int64,
                                      P(ctypes.c_int32), P(ctypes.c_double), ctypes.c_int64, P(ctypes.c_int64),
                                      P(ctypes.c_int32), P(ctypes.c_uint64), P(ctypes.c_uint8),
                                      P(ctypes.c_double)]
            lib.oracle_bc.restype = ctypes.c_int
            lib.oracle_bc_weighted.argtypes = [ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_int32),
                                               P(ctypes.c_int32), ctypes.c_int64, P(ctypes.c_int32),
                                               P(ctypes.c_double), ctypes.c_int64, P(ctypes.c_int64),
                                               P(ctypes.c_int32), P(ctypes.c_uint64), P(ctypes.c_uint8),
                                               P(ctypes.c_double)]
            lib.oracle_bc_weighted.restype = ctypes.c_int
            lib.oracle_big_to_scaled.argtypes = [P(ctypes.c_uint64), ctypes.c_int32, P(ctypes.c_double),
                                                 P(ctypes.c_int64)]
            lib.oracle_big_to_scaled.restype = None
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t)) if a is not None else None


class SourceState:
    """Per-source dumps: dist int32, sigma mod 2^64 uint64, overflow uint8, delta f64."""

    def __init__(self, dist, sigma, ovf, delta):
        self.dist, self.sigma, self.ovf, self.delta = dist, sigma, ovf, delta


def bc(n: int, row_ptr, col, sources, dump=(), bc_init=None):
    """Brandes BC summed over `sources` (list order, multiplicity counted).

    Returns (bc float64[n], {source_position: SourceState}) where the dict
    holds the dumps for the source positions listed in `dump`.
    """
    lib = _load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    src = np.ascontiguousarray(sources, dtype=np.int32).reshape(-1)
    out = np.zeros(n, np.float64) if bc_init is None else np.array(bc_init, np.float64, copy=True)
    di = np.ascontiguousarray(sorted(set(int(x) for x in dump)), dtype=np.int64)
    nd = len(di)
    dist = np.zeros((nd, n), np.int32)
    sig = np.zeros((nd, n), np.uint64)
    ovf = np.zeros((nd, n), np.uint8)
    dlt = np.zeros((nd, n), np.float64)
    if len(cl) == 0:
        cl = np.zeros(1, np.int32)
    rc = lib.oracle_bc(int(n), _p(rp, ctypes.c_int32), _p(cl, ctypes.c_int32), len(src), _p(src, ctypes.c_int32),
                       _p(out, ctypes.c_double), nd, _p(di, ctypes.c_int64), _p(dist, ctypes.c_int32),
                       _p(sig, ctypes.c_uint64), _p(ovf, ctypes.c_uint8), _p(dlt, ctypes.c_double))
    if rc == -1:
        raise ValueError("oracle_bc: invalid input (source out of range)")
    if rc != 0:
        raise MemoryError("oracle_bc: allocation failed")
    states = {int(d): SourceState(dist[i], sig[i], ovf[i], dlt[i]) for i, d in enumerate(di)}
    return out, states


def bc_weighted(n: int, row_ptr, col, weight, sources, dump=(), bc_init=None):
    """Weighted Brandes BC (Dijkstra distances, positive integer weights
    aligned with col) summed over `sources`; returns like bc()."""
    lib = _load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    wt = np.ascontiguousarray(weight, dtype=np.int32)
    if len(wt) != len(cl):
        raise ValueError("weight must align with col")
    src = np.ascontiguousarray(sources, dtype=np.int32).reshape(-1)
    out = np.zeros(n, np.float64) if bc_init is None else np.array(bc_init, np.float64, copy=True)
    di = np.ascontiguousarray(sorted(set(int(x) for x in dump)), dtype=np.int64)
    nd = len(di)
    dist = np.zeros((nd, n), np.int32)
    sig = np.zeros((nd, n), np.uint64)
    ovf = np.zeros((nd, n), np.uint8)
    dlt = np.zeros((nd, n), np.float64)
    if len(cl) == 0:
        cl = np.zeros(1, np.int32)
        wt = np.ones(1, np.int32)
    rc = lib.oracle_bc_weighted(int(n), _p(rp, ctypes.c_int32), _p(cl, ctypes.c_int32), _p(wt, ctypes.c_int32),
                                len(src), _p(src, ctypes.c_int32), _p(out, ctypes.c_double), nd,
                                _p(di, ctypes.c_int64), _p(dist, ctypes.c_int32), _p(sig, ctypes.c_uint64),
                                _p(ovf, ctypes.c_uint8), _p(dlt, ctypes.c_double))
    if rc == -1:
        raise ValueError("oracle_bc_weighted: invalid input (source out of range or weight < 1)")
    if rc == -3:
        raise ValueError("oracle_bc_weighted: a distance exceeds 2^31 - 1")
    if rc != 0:
        raise MemoryError("oracle_bc_weighted: allocation failed")
    states = {int(d): SourceState(dist[i], sig[i], ovf[i], dlt[i]) for i, d in enumerate(di)}
    return out, states


def bc_graph_weighted(g, weight, sources, dump=()):
    """bc_weighted() for a graph object and its weight array."""
    return bc_weighted(g.n, g.row_ptr, g.col, weight, sources, dump)


def bc_graph(g, sources, dump=()):
    """bc() for an object with .n, .row_ptr, .col (e.g. graphgen.Graph)."""
    return bc(g.n, g.row_ptr, g.col, sources, dump)


def big_to_scaled(x: int):
    """(mantissa in [1, 2), exponent) of the correctly rounded 53-bit value of
    the non-negative integer x, from the oracle's C helper."""
    limbs = []
    while x:
        limbs.append(x & ((1 << 64) - 1))
        x >>= 64
    arr = np.array(limbs or [0], dtype=np.uint64)
    m = ctypes.c_double()
    e = ctypes.c_int64()
    _load().oracle_big_to_scaled(_p(arr, ctypes.c_uint64), len(arr), ctypes.byref(m), ctypes.byref(e))
    return m.value, e.value
