"""ORACLE - test infrastructure, not part of the product.

Source-parallel harness around the unmodified single-threaded oracle
(brandes.c).  Sources are independent (the sum after Eq. 2 runs over
sources), so P worker processes each run the oracle over a share of the
list, and the shares' BC vectors are added in share order.  Only the order
of the FP64 additions across shares differs from one process running the
whole list.

Workers are started with `spawn` (a process forked after CUDA work would
hang), and receive the graph as memory-mapped .npy files in a temporary
directory rather than as pickled arrays, so a 128M-entry CSR is not copied
once per worker.
"""
from __future__ import annotations

import os
import shutil
import tempfile
import time

import numpy as np

_G = None


def _init(path, weighted):
    global _G
    import oracle
    oracle.build()
    n = int(np.load(os.path.join(path, "n.npy")))
    rp = np.load(os.path.join(path, "row_ptr.npy"), mmap_mode="r")
    col = np.load(os.path.join(path, "col.npy"), mmap_mode="r")
    w = np.load(os.path.join(path, "weight.npy"), mmap_mode="r") if weighted else None
    _G = (n, rp, col, w)


def _run(sources):
    import oracle
    n, rp, col, w = _G
    if w is None:
        return oracle.bc(n, rp, col, sources)[0]
    return oracle.bc_weighted(n, rp, col, w, sources)[0]


def _run_state(source):
    """dist, sigma mod 2^64 and overflow flags of one source."""
    import oracle
    n, rp, col, w = _G
    src = np.array([source], np.int32)
    if w is None:
        _, st = oracle.bc(n, rp, col, src, dump=(0,))
    else:
        _, st = oracle.bc_weighted(n, rp, col, w, src, dump=(0,))
    return st[0].dist, st[0].sigma, st[0].ovf


def _run_graph(task):
    import oracle
    n, rp, col, sources = task
    return oracle.bc(n, rp, col, sources)[0]


def _noop(_):
    import oracle
    oracle.build()
    return 0


def map_graphs(tasks, procs=None):
    """oracle.bc over independent (n, row_ptr, col, sources) tasks, one task
    per worker at a time (for many small graphs); returns their BC vectors
    in task order."""
    import multiprocessing as mp
    procs = max(1, min(int(procs or host_cores()), len(tasks) or 1))
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map(_noop, range(procs))
        return pool.map(_run_graph, tasks, chunksize=1)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """P processes running the oracle over shares of a source list."""

    def __init__(self, g, weight=None, procs=None):
        import multiprocessing as mp
        self.n = int(g.n)
        self.procs = max(1, int(procs or host_cores()))
        self.dir = tempfile.mkdtemp(prefix="oracle_pool_")
        np.save(os.path.join(self.dir, "n.npy"), np.int64(g.n))
        np.save(os.path.join(self.dir, "row_ptr.npy"), np.ascontiguousarray(g.row_ptr, np.int32))
        np.save(os.path.join(self.dir, "col.npy"), np.ascontiguousarray(g.col, np.int32))
        if weight is not None:
            np.save(os.path.join(self.dir, "weight.npy"), np.ascontiguousarray(weight, np.int32))
        self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_init,
                                                 initargs=(self.dir, weight is not None))
        # every worker up, the oracle loaded and the graph mapped
        self.pool.map(_run, [np.zeros(0, np.int32)] * self.procs, chunksize=1)

    def bc(self, sources, shares_per_proc=1):
        """BC over `sources` (list order within a share, shares summed in
        order); returns (bc float64[n], seconds)."""
        src = np.ascontiguousarray(sources, np.int32).reshape(-1)
        parts = [p for p in np.array_split(src, self.procs * max(1, shares_per_proc)) if len(p)]
        t = time.perf_counter()
        total = np.zeros(self.n, np.float64)
        for part in self.pool.imap(_run, parts, chunksize=1):
            total += part
        return total, time.perf_counter() - t

    def states(self, sources):
        """[(dist, sigma, overflow)] of each source, one per worker task."""
        return self.pool.map(_run_state, [int(x) for x in sources], chunksize=1)

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None
        shutil.rmtree(self.dir, ignore_errors=True)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
