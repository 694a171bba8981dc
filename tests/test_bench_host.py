"""Host logic of bench.py (no GPU): DRAM traffic is reported only from an ncu
summary of the current kernel sources, the pair kernel's bytes model, the weighted
workloads, and the reference arm's JSON line."""
import hashlib
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_traffic_is_reported_only_from_a_summary_of_the_current_kernels(tmp_path, monkeypatch):
    # bench.py reports ncu DRAM traffic only from a committed summary taken on
    # the current kernel sources with the bench's source grouping; any kernel
    # edit without a new capture gives null
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = tmp_path / "paper_2008_05718_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in bench.KERNEL_SOURCES:
        (csrc / name).write_text("kernel " + name)
    (tmp_path / "profiles").mkdir()
    sha = bench.kernel_source_hash()
    (tmp_path / "profiles" / "persistent_rmat18.txt").write_text(
        f"kernel_source_sha256_16: {sha}\nsource_grouping: learned\ndram_bytes_per_launch: 123.0\n")
    assert bench.traffic_from_profiles("persistent", "rmat18", "learned") == 123.0
    assert bench.traffic_from_profiles("persistent", "rmat18", "list order") is None
    assert bench.traffic_from_profiles("persistent", "rmat22", "learned") is None
    (csrc / bench.KERNEL_SOURCES[0]).write_text("edited")
    assert bench.traffic_from_profiles("persistent", "rmat18", "learned") is None


def test_pair_bytes_model():
    n, nnz, k, nb = 1000, 6000, 300, 10
    unweighted = bench.pair_bytes_per_step(n, nnz, k, nb, False)
    weighted = bench.pair_bytes_per_step(n, nnz, k, nb, True)
    assert unweighted == nb * (2 * (4 * nnz + 4 * (n + 1)) + 16 * n) + 4 * k * n * 12
    assert weighted - unweighted == nb * 2 * 4 * nnz


def test_weighted_workloads_carry_symmetric_weights():
    g, S, w = bench.load_workload("wrmat18", 0)
    assert w is not None and len(w) == g.nnz and w.min() >= 1 and w.max() <= 16
    u = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    fwd = dict(zip(zip(u.tolist(), g.col.tolist()), w.tolist()))
    for (a, b), c in list(fwd.items())[:5000]:
        assert fwd[(b, a)] == c
    g2, S2, w2 = bench.load_workload("rmat18", 0)
    assert w2 is None and np.array_equal(S2, S)
    _, S3, _ = bench.load_workload("rmat18", 1)  # another rank: another sample of the same size
    assert len(S3) == len(S) and not np.array_equal(S3, S)


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "er4096", "--steps", "1", "--warmup", "0", "--cpu-sample", "4"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
