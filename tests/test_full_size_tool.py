"""Host logic of tests/full_size_check.py (no GPU): the slices of the source
list, the sum of the slices' BC vectors and the comparison at the parity bar
of the GPU tests (1e-12 relative, 1e-15 absolute floor)."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOOL = os.path.join(ROOT, "tests", "full_size_check.py")


def _run(*args):
    p = subprocess.run([sys.executable, TOOL, *args], capture_output=True, text=True, cwd=ROOT)
    return p.returncode, json.loads(p.stdout.strip().splitlines()[-1])


def test_slices_cover_the_list_once_in_order():
    # the oracle step splits the list with np.array_split: contiguous slices,
    # every source exactly once, whatever the list length and slice count
    for k in (1, 15, 16, 17, 16384):
        S = np.arange(k, dtype=np.int32)
        for n in (1, 3, 16):
            parts = np.array_split(S, n)
            assert len(parts) == n
            assert np.array_equal(np.concatenate(parts), S)


def test_sum_and_compare(tmp_path):
    rng = np.random.default_rng(7)
    want = rng.random(1000) * 1e6
    want[:10] = 0.0  # vertices no path passes: exact zeros
    a, b = want * 0.25, want * 0.75  # two slices' partial BC (exact in binary)
    pa, pb = str(tmp_path / "a.npy"), str(tmp_path / "b.npy")
    np.save(pa, a)
    np.save(pb, b)
    tot = str(tmp_path / "tot.npy")
    rc, out = _run("sum", "--out", tot, pa, pb)
    assert rc == 0 and out["parts"] == 2
    assert np.array_equal(np.load(tot), want)
    # within the bar: one ulp-scale difference; outside: 1e-11 relative
    close = want * (1 + 4e-13)
    pc = str(tmp_path / "close.npy")
    np.save(pc, close)
    rc, out = _run("compare", tot, pc)
    assert rc == 0 and out["pass"] and out["vertices"] == 1000
    far = want.copy()
    far[500] *= 1 + 1e-11
    pf = str(tmp_path / "far.npy")
    np.save(pf, far)
    rc, out = _run("compare", tot, pf)
    assert rc == 1 and not out["pass"] and out["worst_vertex"] == 500
    # a zero that the GPU reports as 1e-14 fails the 1e-15 absolute floor
    z = want.copy()
    z[3] = 1e-14
    pz = str(tmp_path / "z.npy")
    np.save(pz, z)
    rc, out = _run("compare", tot, pz)
    assert rc == 1 and out["worst_vertex"] == 3
