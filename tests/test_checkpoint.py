"""Checkpoint and resume (paper_2008_05718_gb300/checkpoint.py) on the CPU.

The library needs a GPU, so the handle is a stand-in whose exact
fixed-point BC grows by the oracle's dependency vector of each source,
converted to fixed point by the oracle's reference helper (oracle/fixed.py):
the sums are exact integers, as the library's are, so any split of the
source list gives the same bits.  A run interrupted after some chunks and
resumed by a new handle from the file must reach the uninterrupted run's
bits."""
import numpy as np
import pytest

import oracle
from oracle import fixed as fx
from paper_2008_05718_gb300 import checkpoint as ckpt
from paper_2008_05718_gb300 import graphgen as gg


class Crash(RuntimeError):
    pass


class StandIn:
    def __init__(self, g, delta, crash_after=None):
        self.g, self.n, self.delta = g, g.n, delta
        self.vals = [0] * g.n
        self.calls, self.crash_after = 0, crash_after

    def compute(self, sources, stream=None):
        if self.crash_after is not None and self.calls == self.crash_after:
            raise Crash("process lost")
        self.calls += 1
        for s in np.asarray(sources):
            self.vals = [a + b for a, b in zip(self.vals, self.delta[int(s)])]

    def read_fixed(self, stream=None):
        return fx.from_int(self.vals)

    def add_fixed(self, partial, stream=None):
        self.vals = [a + b for a, b in zip(self.vals, fx.to_int(partial))]


@pytest.fixture(scope="module")
def setup():
    g = gg.rmat(8, 8, seed=71)
    S = gg.sample_sources(g.n, 40, seed=72)
    delta = {}
    for s in set(int(x) for x in S):
        bc1, _ = oracle.bc_graph(g, np.array([s], np.int32))  # the dependencies of one source
        delta[s] = fx.to_int(fx.from_double(bc1))
    return g, S, delta


def test_resumed_run_has_the_uninterrupted_bits(setup, tmp_path):
    g, S, delta = setup
    whole = StandIn(g, delta)
    assert ckpt.compute_resumable(whole, S, str(tmp_path / "a.npz"), chunk=7) == len(S)
    path = str(tmp_path / "b.npz")
    first = StandIn(g, delta, crash_after=3)
    with pytest.raises(Crash):
        ckpt.compute_resumable(first, S, path, chunk=7)
    assert ckpt.load(path)["done"] == 21
    second = StandIn(g, delta)
    assert ckpt.compute_resumable(second, S, path, chunk=7) == len(S) - 21
    assert second.vals == whole.vals
    assert ckpt.load(path)["done"] == len(S)
    # a finished checkpoint resumes to the same bits with no work
    third = StandIn(g, delta)
    assert ckpt.compute_resumable(third, S, path, chunk=5) == 0 and third.vals == whole.vals
    # the uninterrupted bits equal the oracle's BC over all sources, rounded once
    ref, _ = oracle.bc_graph(g, S)
    assert np.allclose(fx.to_double(whole.vals), ref, rtol=1e-12, atol=1e-15)


def test_checkpoint_of_another_list_or_graph_is_refused(setup, tmp_path):
    g, S, delta = setup
    path = str(tmp_path / "c.npz")
    ckpt.compute_resumable(StandIn(g, delta), S[:10], path, chunk=4)
    with pytest.raises(ValueError):
        ckpt.compute_resumable(StandIn(g, delta), S, path, chunk=4)
    h = gg.rmat(7, 8, seed=73)
    with pytest.raises(ValueError):
        ckpt.compute_resumable(StandIn(h, {}), S[:10], path, chunk=4)
    with pytest.raises(ValueError):
        ckpt.save(path, np.zeros((3, 2), np.uint64), 1, 4, "x")
