"""Host logic of bench.py (no GPU): the committed DRAM-traffic summary is tied
to the current kernel source, the pair kernel's bytes model, the weighted
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


def test_traffic_summary_matches_the_kernel_source():
    # bench.py only reports the committed ncu traffic when it was taken on the
    # current kernels with the bench's grouping: a kernel edit without a new
    # capture shows up here
    src = os.path.join(ROOT, "paper_2008_05718_gb300", "csrc", "bc_kernels.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    vals = {}
    for line in open(os.path.join(ROOT, "profiles", "backward_rmat18.txt")):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    assert vals["kernel_source_sha256_16"] == sha
    assert vals["source_grouping"] == "learned"
    t = bench.traffic_from_profiles("backward", "rmat18", "learned")
    assert t is not None and t > float(vals["algorithmic_bytes_per_launch_in_bench"])
    assert bench.traffic_from_profiles("backward", "rmat18", "list order") is None
    assert bench.traffic_from_profiles("gather", "rmat18", "learned") is None


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
