"""Autotuning of the grid schedule's launch configuration: batch width,
heavy-row threshold and level loop, picked by timed trials on a handle's
first large call and kept for the handle.  Whatever it picks, BC must be
bit-identical to a fixed configuration (exact integer sums)."""
import numpy as np
import pytest

from paper_2008_05718_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def test_autotuner_picks_a_candidate_and_keeps_the_bits(gb):
    g = gg.rmat(17, 16, seed=501)  # 131,072 vertices, average degree above 6: grid schedule
    S = gg.sample_sources(g.n, 3000, seed=501)
    with gb.BC.from_graph(g) as bc:
        bc.compute(S)
        tuned = bc.read_fixed()
        st = bc.stats()
        assert st["batch_width"] in (32, 64)
        assert st["tuned_heavy_degree"] in (512, 1024, 2048)
        assert st["tuned_device_loop"] in (0, 1)
        assert st["sources"] == len(S)
        # the choice is kept: a second call runs no trials and adds the same bits again
        bc.compute(S)
        twice = bc.read_fixed()
    with gb.BC.from_graph(g, batch_width=64, heavy_degree=1024) as bc:
        bc.compute(S)
        fixed = bc.read_fixed()
        st2 = bc.stats()
    assert st2["tuned_heavy_degree"] == 0  # explicit options: no trials
    assert np.array_equal(tuned, fixed)
    lo = twice[:, 0].astype(object) + (twice[:, 1].astype(object) << 64)
    one = fixed[:, 0].astype(object) + (fixed[:, 1].astype(object) << 64)
    assert all(a == 2 * b for a, b in zip(lo, one))


def test_small_calls_are_not_tuned(gb):
    g = gg.rmat(17, 16, seed=502)
    S = gg.sample_sources(g.n, 500, seed=502)
    with gb.BC.from_graph(g) as bc:
        bc.compute(S)
        assert bc.stats()["tuned_heavy_degree"] == 0
