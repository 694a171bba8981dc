"""Full-size parity check of a benchmark workload over ALL of its sources.

Too slow for the test suite (R-MAT 22 with 16,384 sources takes the oracle
about half an hour on 8 cores), so it runs offline in three steps:

    python tests/full_size_check.py oracle  --workload rmat22 --out oracle_bc.npy [--procs P]
    python tests/full_size_check.py gpu     --workload rmat22 --out gpu_bc.npy
    python tests/full_size_check.py compare oracle_bc.npy gpu_bc.npy

The oracle step can be split: `oracle --part K/N` covers the K-th of N
contiguous slices of the source list (K = 0 .. N-1), so that the slices can
run on different machines or at different times, and
`sum --out oracle_bc.npy part0.npy part1.npy ...` adds the slices' BC
vectors in the order given.

`oracle` runs the plain CPU oracle over every source of the workload, in
worker processes (oracle/pool.py); `gpu` runs the CUDA library through the
C ABI in the benchmark's launch configuration (shipped direction and
grouping networks, automatic schedule, concurrent batches); `compare`
applies the parity bar of the GPU tests: BC within 1e-12 relative with a
1e-15 absolute floor, vertex by vertex.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

REL, ABS = 1e-12, 1e-15


def _workload(name):
    from paper_2008_05718_gb300 import graphgen as gg
    return gg.workload(name)


def run_oracle(args):
    from oracle.pool import OraclePool
    g, S = _workload(args.workload)
    part = "0/1"
    if args.part:
        k, n = (int(x) for x in args.part.split("/"))
        assert 0 <= k < n, args.part
        S = np.array_split(S, n)[k]
        part = args.part
    with OraclePool(g, procs=args.procs) as pool:
        bc, dt = pool.bc(S, shares_per_proc=4)
    np.save(args.out, bc)
    print(json.dumps({"workload": args.workload, "part": part, "sources": len(S), "n": g.n, "nnz": g.nnz,
                      "procs": pool.procs, "seconds": round(dt, 1), "out": args.out}))


def run_sum(args):
    total = None
    for path in args.parts:
        x = np.load(path)
        total = x.copy() if total is None else total + x
    np.save(args.out, total)
    print(json.dumps({"parts": len(args.parts), "out": args.out}))


def run_gpu(args):
    import torch
    from paper_2008_05718_gb300 import _build, gbbc, grouping, policy
    _build.build()
    gbbc.load()
    g, S = _workload(args.workload)
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    with gbbc.BC.from_csr(g.n, rp, col) as bc:
        bc.load_policy(policy.shipped_weights())
        bc.load_grouping(grouping.shipped_weights())
        torch.cuda.synchronize()
        t = time.perf_counter()
        bc.compute(torch.from_numpy(S).to(dev))
        out = bc.read()
        dt = time.perf_counter() - t
        st = bc.stats()
    np.save(args.out, out)
    print(json.dumps({"workload": args.workload, "sources": len(S), "seconds": round(dt, 3),
                      "schedule": st["schedule"], "batches": st["batches"], "out": args.out,
                      "sha256_16": hashlib.sha256(out.tobytes()).hexdigest()[:16]}))


def run_compare(args):
    want = np.load(args.oracle)
    got = np.load(args.gpu)
    assert want.shape == got.shape, (want.shape, got.shape)
    excess = np.abs(got - want) - (REL * np.abs(want) + ABS)
    i = int(np.argmax(excess))
    with np.errstate(divide="ignore", invalid="ignore"):
        rel = np.where(want != 0, np.abs(got - want) / np.abs(want), np.abs(got - want))
    res = {"vertices": int(len(want)), "max_excess": float(excess[i]), "worst_vertex": i,
           "gpu": float(got[i]), "oracle": float(want[i]), "max_rel": float(np.nanmax(rel)),
           "bit_identical": int(np.sum(got == want)), "sum_oracle": float(want.sum()),
           "sum_gpu": float(got.sum()), "pass": bool(excess[i] <= 0)}
    print(json.dumps(res))
    return 0 if res["pass"] else 1


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    a = sub.add_parser("oracle")
    a.add_argument("--workload", default="rmat22")
    a.add_argument("--out", required=True)
    a.add_argument("--procs", type=int, default=None)
    a.add_argument("--part", default=None, help="K/N: the K-th of N contiguous slices of the source list")
    d = sub.add_parser("sum")
    d.add_argument("--out", required=True)
    d.add_argument("parts", nargs="+")
    b = sub.add_parser("gpu")
    b.add_argument("--workload", default="rmat22")
    b.add_argument("--out", required=True)
    c = sub.add_parser("compare")
    c.add_argument("oracle")
    c.add_argument("gpu")
    args = ap.parse_args()
    if args.cmd == "oracle":
        return run_oracle(args)
    if args.cmd == "gpu":
        return run_gpu(args)
    if args.cmd == "sum":
        return run_sum(args)
    return run_compare(args)


if __name__ == "__main__":
    sys.exit(main() or 0)
