"""The partitioned method (Sec. IV, Sec. V-A) on one GPU: P logical parts.

Border matrices against the oracle's plain definition (a BFS inside the part
from each border node, exact counts); then, per source, Step 1, the
refinement of Steps 2-5, the border sigma, the Step 6 relaxation and the
backward phase must reach exactly what the unpartitioned bc_compute reaches:
dist and sigma (mod 2^64, with the overflow flag) bit for bit against the
oracle, BC bit for bit against bc_compute while counts stay below 2^64, and
within 1e-12 of the oracle everywhere.
"""
import numpy as np
import pytest

import oracle
from oracle import partition as op
from oracle.pool import OraclePool
from paper_2008_05718_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

REL, ABS = 1e-12, 1e-15
M64 = (1 << 64) - 1


def assert_bc_close(got, want):
    excess = np.abs(np.asarray(got) - want) - (REL * np.abs(want) + ABS)
    i = int(np.argmax(excess))
    assert excess[i] <= 0, f"vertex {i}: gpu {got[i]!r} oracle {want[i]!r}"


def contiguous(n, P):
    return (np.arange(n, dtype=np.int64) * P // max(n, 1)).astype(np.int32)


def scrambled(n, P, seed=7):
    return ((np.arange(n, dtype=np.uint64) * np.uint64(2654435761) + np.uint64(seed)) % np.uint64(P)).astype(np.int32)


def quadrants(rows, cols):
    v = np.arange(rows * cols)
    return (((v // cols) >= rows // 2) * 2 + ((v % cols) >= cols // 2)).astype(np.int32)


MATRIX_CASES = [
    ("path", lambda: gg.path(12), lambda g: contiguous(g.n, 2)),
    ("cycle", lambda: gg.cycle(21), lambda g: contiguous(g.n, 3)),
    ("grid_quadrants", lambda: gg.full_grid(12, 10), lambda g: quadrants(12, 10)),
    ("grid_wide_counts", lambda: gg.full_grid(80, 80), lambda g: quadrants(80, 80)),
    ("rmat10_scrambled", lambda: gg.rmat(10, 8, seed=5), lambda g: scrambled(g.n, 3)),
]


@pytest.mark.parametrize("name,make,partf", MATRIX_CASES, ids=[c[0] for c in MATRIX_CASES])
def test_border_matrices_match_the_definition(gb, name, make, partf):
    g = make()
    part = partf(g)
    P = int(part.max()) + 1
    want = op.border_matrices(g.n, g.row_ptr, g.col, part)
    with gb.BC.from_graph(g) as bc:
        bc.partition(part, P)
        info = bc.partition_info()
        assert info["parts"] == P and info["border_nodes"] == sum(len(b) for b, _, _ in want)
        assert info["border_edges"] + info["intra_entries"] == g.nnz
        for p, (wb, wbm, wsm) in enumerate(want):
            b, bm, sm, ov = bc.border_matrix(p)
            assert np.array_equal(b, wb)
            assert np.array_equal(bm, wbm.astype(np.int32))
            exact = np.array([[x & M64 for x in row] for row in wsm], np.uint64).reshape(bm.shape)
            big = np.array([[x > M64 for x in row] for row in wsm], np.uint8).reshape(bm.shape)
            assert np.array_equal(sm, exact) and np.array_equal(ov, big)


def _partitioned(gb, g, S, part, P, keep=(), flags=0, **opts):
    flags |= gb.GBBC_KEEP_STATE if keep else 0
    with gb.BC.from_graph(g, flags=flags, **opts) as bc:
        bc.partition(part, P)
        bc.compute_partitioned(S)
        return bc.read_fixed(), bc.read(), {i: bc.source_state(i) for i in keep}, bc.partition_info()


CASES = [
    ("er4096_p2", lambda: gg.workload("er4096")[0], 200, 2, "contiguous"),
    ("er4096_p4", lambda: gg.workload("er4096")[0], 200, 4, "contiguous"),
    ("rmat12_p2", lambda: gg.rmat(12, 16, seed=401), 150, 2, "contiguous"),
    ("rmat12_p4_scrambled", lambda: gg.rmat(12, 16, seed=402), 150, 4, "scrambled"),
    ("grid64_p4", lambda: gg.grid(64, "0.05", seed=403), 100, 4, "contiguous"),
    ("p1_no_border", lambda: gg.rmat(11, 16, seed=404), 70, 1, "contiguous"),
]


@pytest.mark.parametrize("name,make,k,P,kind", CASES, ids=[c[0] for c in CASES])
def test_partitioned_equals_bc_compute_and_the_oracle(gb, name, make, k, P, kind):
    g = make()
    S = gg.sample_sources(g.n, min(k, g.n), seed=41)
    part = contiguous(g.n, P) if kind == "contiguous" else scrambled(g.n, P)
    keep = (0, len(S) - 1)
    fx, got, st, info = _partitioned(gb, g, S, part, P, keep=keep)
    with gb.BC.from_graph(g) as bc:
        bc.compute(S)
        whole_fx = bc.read_fixed()
        whole_wide = bc.stats()["wide_batches"]
    want, ost = oracle.bc_graph(g, S, dump=keep)
    assert_bc_close(got, want)
    if whole_wide == 0:
        assert np.array_equal(fx, whole_fx)
    for i in keep:
        d, s, o = st[i]
        assert np.array_equal(d, ost[i].dist), f"dist of source #{i}"
        assert np.array_equal(s, ost[i].sigma), f"sigma of source #{i}"
        assert np.array_equal(o, ost[i].ovf), f"overflow flags of source #{i}"
    if P > 1:
        assert info["border_nodes"] > 0 and info["refinement_sweeps"] >= (k + 63) // 64


@pytest.mark.parametrize("P", [2, 4])
def test_partitioned_grid1024_full_size(gb, P):
    # the high-diameter workload: strips of the 1024^2 grid (contiguous
    # row-major ranges); path counts far beyond 2^64 run in the wide format
    g, S = gg.workload("grid1024")
    S = S[:64]
    keep = (0, 63)
    fx, got, st, info = _partitioned(gb, g, S, None, P, keep=keep)
    assert info["parts"] == P and info["border_nodes"] > 1000
    with OraclePool(g) as pool:
        want, _ = pool.bc(S)
        ost = pool.states(S[list(keep)])
    assert_bc_close(got, want)
    for i, (od, os_, oo) in zip(keep, ost):
        d, s, o = st[i]
        assert np.array_equal(d, od) and np.array_equal(s, os_) and np.array_equal(o, oo)


def test_partition_errors(gb):
    g = gg.rmat(9, 8, seed=9)
    with gb.BC.from_graph(g) as bc:
        with pytest.raises(gb.GbbcError) as e:
            bc.compute_partitioned([0, 1])
        assert e.value.status == gb.GBBC_ERR_STATE
        with pytest.raises(gb.GbbcError) as e:
            bc.partition(np.full(g.n, 5, np.int32), 3)
        assert e.value.status == gb.GBBC_ERR_INVALID
        with pytest.raises(gb.GbbcError) as e:
            bc.partition(None, 0)
        assert e.value.status == gb.GBBC_ERR_INVALID
    w = gg.edge_weights(g, 4, seed=1)
    with gb.BC.from_weighted(g.n, g.row_ptr, g.col, w) as bc:
        with pytest.raises(gb.GbbcError) as e:
            bc.partition(None, 2)
        assert e.value.status == gb.GBBC_ERR_INVALID


@pytest.mark.parametrize("name,make,k,P", [("er4096_p4", lambda: gg.workload("er4096")[0], 130, 4),
                                           ("grid64_p3", lambda: gg.grid(64, "0.05", seed=405), 100, 3),
                                           ("rmat12_p2", lambda: gg.rmat(12, 16, seed=406), 100, 2)])
def test_asynchronous_backward_equals_level_synchronous(gb, name, make, k, P):
    # each part walks its own levels and waits only where a border node's
    # successor lies in another part one level deeper: the same integer sums
    g = make()
    S = gg.sample_sources(g.n, min(k, g.n), seed=43)
    fx_a, _, _, info_a = _partitioned(gb, g, S, None, P)
    fx_s, _, _, info_s = _partitioned(gb, g, S, None, P, flags=gb.GBBC_SYNC_BACKWARD)
    assert np.array_equal(fx_a, fx_s)
    assert info_a["backward_waits"] > 0 and info_s["backward_waits"] == 0


def test_asynchronous_backward_wait_bound(gb):
    g = gg.grid(64, "0.05", seed=407)
    S = gg.sample_sources(g.n, 64, seed=44)
    with gb.BC.from_graph(g, timeout_spins=1) as bc:
        bc.partition(None, 4)
        with pytest.raises(gb.GbbcError) as e:
            bc.compute_partitioned(S)
        assert e.value.status == gb.GBBC_ERR_TIMEOUT
        bc.reset()
    # the device is fine afterwards (grid counts pass 2^64: compare with the oracle)
    _, got, _, _ = _partitioned(gb, g, S, None, 4)
    want, _ = oracle.bc_graph(g, S)
    assert_bc_close(got, want)
