"""bc_compute_noalloc through the C ABI against bc_compute and the oracle.

The no-allocation entry point serves callers that may not allocate memory
(a pool allocator owning the device, a plug-in host, a real-time loop): it
keeps its working state in a static device array of the library.  This file
is collected last so that, if it fails, a run stopping at the first failure
has already run every other test; it must pass alone and after the others.
"""
import numpy as np
import pytest

import oracle
from paper_2008_05718_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu
REL, ABS = 1e-12, 1e-15


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_05718_gb300 import _build, gbbc
    _build.build()
    gbbc.load()
    return torch, gbbc


def _close(got, want):
    excess = np.abs(got - want) - (REL * np.abs(want) + ABS)
    assert excess.max() <= 0, f"max excess {excess.max()} at vertex {int(np.argmax(excess))}"


def _noalloc_twice(torch, gb, g, S):
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    stream = torch.cuda.current_stream(dev)
    outs = []
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        out = torch.zeros(g.n, dtype=torch.float64, device=dev)
        gb.bc_compute_noalloc(g.n, g.nnz, rp, col, S, out, stream=stream)
        outs.append(out.cpu().numpy())
    return outs


@pytest.mark.parametrize("scale,k", [(13, 150), (14, 130)])
def test_noalloc_matches_bc_compute_and_the_oracle_twice(env, scale, k):
    # scale 14 is the largest graph the static array holds (16,384 vertices)
    torch, gb = env
    g = gg.rmat(scale, 16, seed=41 + scale)  # heavy rows present
    assert g.n <= gb.NOALLOC_MAX_VERTICES
    S = gg.sample_sources(g.n, k, seed=41 + scale)
    with gb.BC.from_graph(g, batch_width=64) as bc:
        bc.compute(S)
        want = bc.read()
    ref, _ = oracle.bc_graph(g, S)
    for got in _noalloc_twice(torch, gb, g, S):
        _close(got, want)
        _close(got, ref)


def test_noalloc_rejects_too_large_graph(env):
    torch, gb = env
    dev = torch.device("cuda:0")
    n = gb.NOALLOC_MAX_VERTICES + 1
    rp = torch.zeros(n + 1, dtype=torch.int32, device=dev)
    col = torch.zeros(1, dtype=torch.int32, device=dev)
    out = torch.zeros(n, dtype=torch.float64, device=dev)
    with pytest.raises(gb.GbbcError) as e:
        gb.bc_compute_noalloc(n, 0, rp, col, np.array([0], np.int32), out)
    assert e.value.status == gb.GBBC_ERR_CAPACITY


def test_noalloc_path_count_past_2_64_leaves_output_unchanged(env):
    # corner to corner of a 128 x 128 grid there are C(254, 127) ~ 2^250
    # shortest paths: the 64-bit format cannot hold them
    torch, gb = env
    dev = torch.device("cuda:0")
    g = gg.full_grid(128, 128)
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    before = torch.arange(g.n, dtype=torch.float64, device=dev) * 0.25 + 1.0
    out = before.clone()
    with pytest.raises(gb.GbbcError) as e:
        gb.bc_compute_noalloc(g.n, g.nnz, rp, col, np.array([0, 5, g.n - 1], np.int32), out)
    assert e.value.status == gb.GBBC_ERR_CAPACITY
    assert torch.equal(out, before)
    # the next call on the same scratch still gives the right answer
    S = np.array([3, 700], np.int32)
    h = gg.rmat(10, 8, seed=5)
    got = _noalloc_twice(torch, gb, h, S)
    ref, _ = oracle.bc_graph(h, S)
    _close(got[0], ref)


def test_noalloc_rejects_an_invalid_csr(env):
    torch, gb = env
    dev = torch.device("cuda:0")
    out = torch.zeros(4, dtype=torch.float64, device=dev)
    cases = {
        "asymmetric": (np.array([0, 1, 2, 3, 3], np.int32), np.array([1, 2, 3], np.int32)),
        "col out of range": (np.array([0, 1, 2, 3, 4], np.int32), np.array([1, 0, 9, 2], np.int32)),
        "self-loop": (np.array([0, 1, 2, 2, 2], np.int32), np.array([0, 0], np.int32)),
        "row_ptr[n] != nnz": (np.array([0, 1, 2, 2, 3], np.int32), np.array([1, 0], np.int32)),
    }
    for name, (rp, col) in cases.items():
        with pytest.raises(gb.GbbcError) as e:
            gb.bc_compute_noalloc(4, len(col), torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev),
                                  np.array([0], np.int32), out)
        assert e.value.status == gb.GBBC_ERR_INVALID, name
    assert torch.count_nonzero(out) == 0
