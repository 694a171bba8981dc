"""bc_compute_noalloc through the C ABI against bc_compute.

The no-allocation entry point serves callers that may not allocate memory
(a pool allocator owning the device, a plug-in host, a real-time loop): it
keeps its working state in a static device array of the library.  This file
is collected last so that, if it fails, a run stopping at the first failure
has already run every other test; it must pass alone and after the others.
"""
import numpy as np
import pytest

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


def test_noalloc_matches_bc_compute_twice(env):
    torch, gb = env
    dev = torch.device("cuda:0")
    g = gg.rmat(13, 16, seed=41)  # 8192 vertices, heavy rows present
    assert g.n <= gb.NOALLOC_MAX_VERTICES
    S = gg.sample_sources(g.n, 150, seed=41)
    with gb.BC.from_graph(g, batch_width=64) as bc:
        bc.compute(S)
        want = bc.read()
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        out = torch.zeros(g.n, dtype=torch.float64, device=dev)
        gb.bc_compute_noalloc(g.n, g.nnz, rp, col, S, out, stream=stream)
        got = out.cpu().numpy()
        excess = np.abs(got - want) - (REL * np.abs(want) + ABS)
        assert excess.max() <= 0, f"max excess {excess.max()}"


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
