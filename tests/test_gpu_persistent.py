"""The persistent grid schedule: one cooperative launch per call, several
batches in flight, the level loop on the device between bounded grid
barriers.

It runs with GBBC_DEVICE_LOOP; its BC must be bit-identical to the default
host-driven level loop (per-step kernels, a read-back per level) and agree
with the oracle; a grid
barrier that waits longer than timeout_spins must end the launch with
GBBC_ERR_TIMEOUT and leave the handle usable after bc_reset.
"""
import numpy as np
import pytest

import oracle
from paper_2008_05718_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

REL, ABS = 1e-12, 1e-15


def assert_bc_close(got, want):
    excess = np.abs(np.asarray(got) - want) - (REL * np.abs(want) + ABS)
    i = int(np.argmax(excess))
    assert excess[i] <= 0, f"vertex {i}: gpu {got[i]!r} oracle {want[i]!r}"


def fixed_bits(gb, g, S, device=True, **opts):
    if device:
        opts["flags"] = opts.get("flags", 0) | gb.GBBC_DEVICE_LOOP
    with gb.BC.from_graph(g, schedule="grid", **opts) as bc:
        bc.compute(S)
        return bc.read_fixed(), bc.read(), bc.stats()


CASES = [
    ("er4096", lambda: gg.workload("er4096")[0], 700, {}),
    ("rmat13_heavy32", lambda: gg.rmat(13, 16, seed=301), 300, {"heavy_degree": 32}),
    ("rmat13_pull", lambda: gg.rmat(13, 16, seed=302), 300, {"policy": "pull"}),
    ("rmat13_push", lambda: gg.rmat(13, 16, seed=303), 300, {"policy": "push"}),
    ("rmat16", lambda: gg.rmat(16, 16, seed=304), 520, {}),
    ("grid96_sparse", lambda: gg.grid(96, "0.05", seed=305), 200, {}),
    ("mesh24", lambda: gg.mesh27(24), 150, {"streams": 3}),
]


@pytest.mark.parametrize("name,make,k,opts", CASES, ids=[c[0] for c in CASES])
def test_persistent_bits_equal_host_loop_and_oracle(gb, name, make, k, opts):
    g = make()
    S = gg.sample_sources(g.n, min(k, g.n), seed=17)
    fx_p, bc_p, st_p = fixed_bits(gb, g, S, **opts)
    fx_h, _, st_h = fixed_bits(gb, g, S, device=False, **opts)
    assert np.array_equal(fx_p, fx_h)
    assert st_p["batches"] == st_h["batches"] == (len(S) + 63) // 64
    assert st_p["levels_fwd"] == st_h["levels_fwd"]
    assert st_p["kernel_launches"] < st_h["kernel_launches"]
    want, _ = oracle.bc_graph(g, S)
    assert_bc_close(bc_p, want)


def test_persistent_reruns_wide_batches_on_the_host(gb):
    # corner-to-corner path counts of a 70 x 70 grid pass 2^64: the narrow
    # persistent pass hands those batches back and the host reruns them wide
    g = gg.full_grid(70, 70)
    S = np.array([0, 69, 4899, 2450, 100, 1000, 3000], np.int32)
    fx_p, bc_p, st = fixed_bits(gb, g, S)
    fx_h, _, _ = fixed_bits(gb, g, S, device=False)
    assert st["wide_batches"] >= 1 and st["batches"] == 1 and st["sources"] == len(S)
    assert np.array_equal(fx_p, fx_h)
    want, _ = oracle.bc_graph(g, S)
    assert_bc_close(bc_p, want)


def test_persistent_multi_graph_handle(gb):
    graphs = [gg.rmat(s, 16, seed=310 + s) for s in (9, 11, 12)] + [gg.grid(40, "0.05", seed=313)]
    gid, loc = [], []
    for i, h in enumerate(graphs):
        s = gg.sample_sources(h.n, min(130, h.n), seed=320 + i)
        gid += [i] * len(s)
        loc += list(s)
    gid, loc = np.array(gid, np.int32), np.array(loc, np.int32)
    outs = []
    for flags in (gb.GBBC_DEVICE_LOOP, 0):
        with gb.BC.from_graphs(graphs, schedule="grid", flags=flags) as bc:
            bc.compute_multi(gid, loc)
            outs.append(bc.read_fixed())
            if flags:
                per = [bc.read(graph_id=i) for i in range(len(graphs))]
    assert np.array_equal(outs[0], outs[1])
    for i, h in enumerate(graphs):
        want, _ = oracle.bc_graph(h, loc[gid == i])
        assert_bc_close(per[i], want)


def test_timeout_spins_ends_the_launch_with_an_error(gb):
    # one poll per barrier wait: every block that reaches a barrier before
    # the last one gives up at its first poll, so the launch must end with
    # GBBC_ERR_TIMEOUT (a host-side status; the context stays usable)
    g = gg.rmat(14, 16, seed=331)
    S = gg.sample_sources(g.n, 256, seed=331)
    with gb.BC.from_graph(g, schedule="grid", timeout_spins=1, flags=gb.GBBC_DEVICE_LOOP) as bc:
        with pytest.raises(gb.GbbcError) as e:
            bc.compute(S)
        assert e.value.status == gb.GBBC_ERR_TIMEOUT
        bc.reset()
        bc.compute(S[:0])  # the handle still takes calls
        assert np.all(bc.read() == 0)
    # the device is fine: a handle with the default bound gives the host
    # loop's bits
    want_fx, _, _ = fixed_bits(gb, g, S, device=False)
    got_fx, _, _ = fixed_bits(gb, g, S)
    assert np.array_equal(got_fx, want_fx)


def test_persistent_launch_count(gb):
    g = gg.rmat(15, 16, seed=341)
    S = gg.sample_sources(g.n, 1024, seed=341)
    with gb.BC.from_graph(g, schedule="grid", flags=gb.GBBC_DEVICE_LOOP) as bc:
        before = bc.stats()["kernel_launches"]
        bc.compute(S)
        launches = bc.stats()["kernel_launches"] - before
    assert launches <= 4  # one cooperative launch for 16 batches
