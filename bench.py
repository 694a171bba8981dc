"""Benchmark: exact Brandes BC throughput in GTEPS (sources x directed edges / s).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload rmat22]
                    [--policy auto] [--width 64] [--impl ours|reference]

Default workload: R-MAT scale 22 (4,194,304 vertices, 128,304,280 directed
CSR entries) with 16,384 sources, the configuration on which the learned-
batched vs plain comparison is stated.  One step = one bc_compute over the
workload's whole source list (forward, backward and BC accumulation for
every source) followed by bc_read of the BC vector into device memory; the
graph and sources are resident in HBM.  An L2 flush (a 512 MiB device
write) separates timed steps and is not timed.  Steps are timed with CUDA
events on the compute stream.

Beside the headline the line carries:
  plain      the plain one-source-at-a-time GPU Brandes (batch width 1,
             the same handle options) on a seeded sample of the list, timed
             the same way; beside it the same sample with one source per
             thread block, many blocks at once (plain.concurrent), and the
             batched form on the sample; vs_plain = value / plain.value
  traversed  GTEPS counting only the edges each source's BFS reaches (the
             CSR entries of its connected component)
  e2e        the same metric through the C ABI with host buffers:
             bc_graph_create from pinned host CSR, bc_compute from pinned
             host sources, bc_read into pinned host memory, destroy
  roofline   the dominant step kind's algorithmic bytes over its CUDA-event
             time (a traced run), against the measured HBM copy peak
  cpu_baseline  the CPU oracle (oracle/) on a bounded sample, one process
             per host core, and on one core
`--impl reference` times the CPU oracle alone on a bounded sample per step.

With torchrun (N > 1) every rank runs the same number of sources, its own
seeded share of the job's source list (weak scaling), over its own replica
of the graph; each timed step ends with the one exchange the method has:
the ranks' exact fixed-point partial BC vectors are all-gathered (NCCL) and
added into every rank's handle by the library (multirank.reduce_bc), so
every rank holds the BC of the whole list.  Rank 0 prints the line with the
time of the slowest rank, and checks outside the timed region that the
reduced BC of a small sub-list equals one GPU's run over it bit for bit.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact-BC GTEPS (sources×edges/s), learned-batched vs plain GPU; % HBM roofline"
UNIT = "GTEPS"
WORKLOADS = {
    "rmat18": "R-MAT scale 18 (262,144 vertices, edge factor 16, a=0.57 b=0.19 c=0.19 d=0.05), symmetrised, "
              "deduplicated, int32 CSR, seed 2; 4096 uniform sources in bitset batches of 64",
    "er4096": "Erdos-Renyi n=4096, p=8/4095, seed 1, all 4096 vertices as sources",
    "grid1024": "1024x1024 4-neighbour grid, 5% edges removed, LCC, seed 3, 1024 uniform sources",
    "rmat22": "R-MAT scale 22, edge factor 16, seed 5, 16,384 uniform sources",
    "tri1024": "planar triangulation of a 1024x1024 lattice (grid edges plus one random diagonal per cell, "
               "Delaunay-like, average degree 6), seed 6, 1024 uniform sources",
    "rgg20": "random geometric graph, 2^20 uniform points, expected degree 10, LCC, seed 7, 1024 uniform sources",
    "mesh100": "100x100x100 mesh, 27-point stencil (KKT-like banded pattern, average degree 25.5), "
               "4096 uniform sources (seed 8)",
    "grid256": "256x256 4-neighbour grid, 5% edges removed, LCC, seed 3256, 256 uniform sources "
               "(a small case for profiling)",
    "wrmat18": "the rmat18 graph and sources with integer edge weights uniform in [1, 16] (seed 216); "
               "weighted shortest paths",
    "wgrid1024": "the grid1024 graph and sources with integer edge weights uniform in [1, 16] (seed 217); "
                 "weighted shortest paths",
}
WEIGHTED = {"wrmat18": ("rmat18", 16, 216), "wgrid1024": ("grid1024", 16, 217)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="rmat22", choices=sorted(WORKLOADS))
    ap.add_argument("--policy", default="auto")
    ap.add_argument("--width", type=int, default=64)
    ap.add_argument("--schedule", default="auto", choices=["auto", "grid", "block", "pair"])
    ap.add_argument("--streams", type=int, default=0,
                    help="batches the grid schedule runs at once (0: the library's default)")
    ap.add_argument("--grouping", default="learned", choices=["learned", "none"],
                    help="order sources by the shipped grouping network before packing them into words")
    ap.add_argument("--device-loop", action="store_true",
                    help="grid schedule: run the level loop in the persistent kernel instead of from the host")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="sources of the single-core oracle sample (0: sized from the graph, about 10-30 s)")
    ap.add_argument("--plain-sources", type=int, default=256,
                    help="sources of the plain one-source-at-a-time arm's seeded sample (0: no plain arm)")
    ap.add_argument("--sources", type=int, default=0,
                    help="use the first K sources of the workload's list (0: all of them)")
    ap.add_argument("--partitions", type=int, default=0,
                    help="run the partitioned method (border matrices, refinement, relaxation, asynchronous "
                         "backward) with this many contiguous parts instead of bc_compute (0: off); no plain arm "
                         "and no traced roofline then")
    ap.add_argument("--plain-concurrent-sources", type=int, default=1216,
                    help="sources of the one-source-per-thread-block plain arm's sample (two waves of the "
                         "resident blocks on a 152-SM GPU)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_sources(g, S, rank):
    """Rank `rank`'s share of the job's source list: rank 0 takes the
    workload's list, rank r > 0 another seeded sample of the same size
    (weak scaling: the job's list is the concatenation of the shares)."""
    from paper_2008_05718_gb300 import graphgen as gg
    if rank == 0:
        return S
    return gg.sample_sources(g.n, len(S), seed=10_000 + 97 * rank + len(S))


def load_workload(name, rank):
    """(graph, sources of this rank, edge weights or None)."""
    from paper_2008_05718_gb300 import graphgen as gg
    base, maxw, wseed = WEIGHTED.get(name, (name, 0, 0))
    g, S = gg.workload(base)
    w = gg.edge_weights(g, maxw, seed=wseed) if maxw else None
    return g, rank_sources(g, S, rank), w


def pair_bytes_per_step(n, nnz, k, nb, weighted):
    """Compulsory bytes of one call of the pair-granular kernel (k sources in
    nb batches): per batch the CSR (and weights) read in the forward and the
    backward and BC read and written; per (vertex, source) pair dist (4 B)
    and sigma/psi (8 B) written and read in each phase."""
    csr = (8 if weighted else 4) * nnz + 4 * (n + 1)
    return nb * (2 * csr + 16 * n) + 2 * 2 * k * n * (4 + 8)


# ---- clocks -----------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    rows.append((float(p[1]), float(p[2]), p[5:9]))
                except ValueError:
                    continue
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---- reference arm: the CPU oracle -------------------------------------------
# The oracle (oracle/brandes.c, unmodified) runs single-threaded per process;
# oracle/pool.py runs one process per host core (spawn) over shares of a
# source sample and sums their BC.  Sample sizes follow the graph's size so
# that each timed piece stays within seconds: the oracle's cost per source
# grows with the CSR entries (about 10 s per source on R-MAT 22 and 0.1 s on
# R-MAT 18 for one core).

def oracle_sources_per_core(nnz, budget_entries):
    """Sources per core so that one core reads about budget_entries CSR entries."""
    return int(max(1, min(48, budget_entries // max(nnz, 1))))


def cpu_oracle_gteps(g, S, sample, w=None):
    import oracle
    oracle.build()
    src = np.asarray(S[:sample], np.int32)
    t = time.perf_counter()
    if w is None:
        oracle.bc_graph(g, src)
    else:
        oracle.bc_graph_weighted(g, w, src)
    dt = time.perf_counter() - t
    return len(src) * g.nnz / dt / 1e9, dt, len(src)


def run_reference(args):
    from oracle.pool import OraclePool, host_cores
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    g, S, w = load_workload(args.workload, 0)
    cores = host_cores()
    per = oracle_sources_per_core(g.nnz, 10**8)
    sample = max(1, min(per * cores, len(S)))
    times = []
    with OraclePool(g, w, cores) as pool:
        for i in range(args.warmup + args.steps):
            lo = i * sample % len(S)
            src = np.concatenate([S[lo:], S[:lo]])[:sample]
            _, dt = pool.bc(src)
            if i >= args.warmup:
                times.append(dt)
    value = args.steps * sample * g.nnz / sum(times) / 1e9
    desc = (f"{sample} sources per step ({per} per process) of the {len(S)}-source list over {cores} "
            f"processes, full graph (n={g.n}, nnz={g.nnz})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload], "name": args.workload,
                                            "sources": len(S), "n": g.n, "nnz": g.nnz},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---- our arm -------------------------------------------------------------------

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = ("bc_kernels.cu", "bc_persist.cu", "bc_rows.cuh", "bc_fixed.cuh", "bc_internal.cuh")


def kernel_source_hash():
    """SHA-256 (16 hex digits) of the kernel sources an ncu summary covers."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2008_05718_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def traffic_from_profiles(kernel_kind, workload, grouping):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources with the same source grouping (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel_kind}_{workload}.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != kernel_source_hash() or \
            vals.get("source_grouping", "list order") != grouping:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def run_ours(args):
    import torch
    from paper_2008_05718_gb300 import _build, gbbc

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _build.build()
    gbbc.load()
    g, S, wts = load_workload(args.workload, rank)
    if args.sources > 0:
        S = S[:args.sources]
    k = len(S)
    stream = torch.cuda.current_stream(dev)
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    wt = torch.from_numpy(wts).to(dev) if wts is not None else None
    src = torch.from_numpy(S).to(dev)
    out = torch.zeros(g.n, dtype=torch.float64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    opts = dict(batch_width=args.width, policy=args.policy, streams=args.streams, schedule=args.schedule,
                flags=gbbc.GBBC_DEVICE_LOOP if args.device_loop else 0)

    weights = None
    if args.policy in ("auto", "learned") and args.width != 1:
        from paper_2008_05718_gb300 import policy as pol
        weights = pol.shipped_weights()
    gweights = None
    if args.grouping == "learned" and args.width != 1:
        from paper_2008_05718_gb300 import grouping as grp
        gweights = grp.shipped_weights()

    def prepare(h):
        if weights is not None:
            h.load_policy(weights)
        if gweights is not None:
            h.load_grouping(gweights)
        return h

    def make(rp_, col_, wt_, **kw):
        if wt_ is None:
            return gbbc.BC.from_csr(g.n, rp_, col_, stream=stream, **kw)
        return gbbc.BC.from_weighted(g.n, rp_, col_, wt_, stream=stream, **kw)

    P = args.partitions

    def compute(h, sources):
        if P > 0:
            h.compute_partitioned(sources, stream=stream)
        else:
            h.compute(sources, stream=stream)

    bc = prepare(make(rp, col, wt, **opts))
    t_part = None
    if P > 0:  # once per graph, outside the timed region (border matrices)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bc.partition(None, P, stream=stream)
        torch.cuda.synchronize()
        t_part = time.perf_counter() - t0
    if world > 1:
        from paper_2008_05718_gb300 import multirank as mr

    def step():
        bc.reset()
        compute(bc, src)
        if world > 1:  # the exchange step: every rank ends with the whole BC
            mr.reduce_bc(bc, stream=stream, device=dev)
        bc.read(out, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stats0 = bc.stats()
    launches0 = stats0["kernel_launches"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = clk.summary()
    stats1 = bc.stats()
    launches = stats1["kernel_launches"] - launches0
    p_launches = stats1["persist_launches"] - stats0["persist_launches"]
    p_ms = stats1["persist_ms"] - stats0["persist_ms"]
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    if world > 1:
        t = torch.tensor([total_s], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    value = world * args.steps * k * g.nnz / total_s / 1e9
    # edges the sources' searches actually reach: each source's component
    from paper_2008_05718_gb300 import graphgen as gg
    reach = int(gg.component_entries(g)[S].sum())
    traversed = {"value": world * args.steps * reach / total_s / 1e9, "unit": UNIT,
                 "reachable_fraction": reach / (k * g.nnz)}

    def timed(h, sources, steps, warm):
        """CUDA-event milliseconds per step of reset + compute + read on h
        (an L2 flush before each timed step, not timed)."""
        def once():
            h.reset()
            h.compute(sources, stream=stream)
            h.read(out, stream=stream)
        for _ in range(warm):
            once()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.fill_((i + 7) & 0xFF)
            evs[i][0].record(stream)
            once()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / steps

    # ---- the plain one-source-at-a-time GPU path on a seeded sample ----
    plain = None
    if args.plain_sources > 0 and wts is None and args.width != 1 and P == 0:
        kp = min(args.plain_sources, k)
        sp = torch.from_numpy(gg.sample_sources(k, kp, seed=4242)).to(dev)
        sp = src[sp.long()].contiguous()  # a seeded sample of the list itself
        p_steps = max(1, min(args.steps, 3))
        with make(rp, col, None, **dict(opts, batch_width=1)) as hp:
            ms_plain = timed(hp, sp, p_steps, 1)
        # one source per thread block needs many more sources than resident
        # blocks before it fills the GPU: its own, larger sample
        kc = min(max(args.plain_concurrent_sources, kp), k)
        sc = torch.from_numpy(gg.sample_sources(k, kc, seed=4243)).to(dev)
        sc = src[sc.long()].contiguous()
        with make(rp, col, None, **dict(opts, batch_width=1, schedule="block")) as hp:
            ms_conc = timed(hp, sc, 1, 1)
        ms_batched = timed(bc, sp, p_steps, 1)
        plain = {"value": kp * g.nnz / (ms_plain / 1e3) / 1e9, "unit": UNIT, "sources": kp, "steps": p_steps,
                 "ms_per_step": ms_plain, "sample": "seeded uniform sample (seed 4242) of the source list",
                 "concurrent": {"value": kc * g.nnz / (ms_conc / 1e3) / 1e9, "ms_per_step": ms_conc,
                                "sources": kc, "steps": 1,
                                "sample": "seeded uniform sample (seed 4243) of the source list",
                                "design": "one source per thread block, many blocks at once "
                                          "(batch width 1, block schedule)"},
                 "batched_on_sample": {"value": kp * g.nnz / (ms_batched / 1e3) / 1e9, "ms_per_step": ms_batched}}

    # ---- end to end through the C ABI with host buffers ----
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    src_h = torch.from_numpy(S).pin_memory()
    out_h = torch.zeros(g.n, dtype=torch.float64).pin_memory()
    wt_h = torch.from_numpy(wts).pin_memory() if wts is not None else None
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        with make(rp_h, col_h, wt_h, **opts) as h:
            prepare(h)
            if P > 0:
                h.partition(None, P, stream=stream)
            compute(h, src_h)
            h.read(out_h, stream=stream)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_val = k * g.nnz / e2e_s / 1e9 * world
    h2d = (g.n + 1) * 4 + g.nnz * 4 + k * 4 + (g.nnz * 4 if wts is not None else 0)
    d2h = g.n * 8

    # ---- roofline of the dominant step kind (one traced step) ----
    st_all = bc.stats()
    if P > 0:
        prof = None
    elif wts is None and st_all["schedule"] != 3:
        with make(rp, col, None, **dict(opts, flags=opts["flags"] | gbbc.GBBC_TRACE)) as tb:
            prepare(tb)
            tb.compute(src, stream=stream)
            tb.sync()
            prof = tb.profile()
    else:  # one launch of the pair-granular kernel per step: the timed steps themselves
        ms = 1e3 * total_s / args.steps
        nb = st_all["batches"] // max(1, args.warmup + args.steps)
        prof = {"pair": {"ms": ms, "launches": 1,
                         "bytes": pair_bytes_per_step(g.n, g.nnz, k, nb, wts is not None)}}
    peak, peak_src = measured_peaks()
    grouping_name = "learned" if gweights is not None else "list order"
    if prof is None:
        prof = {}
    total_ms = sum(v["ms"] for v in prof.values())
    step_bytes = sum(v["bytes"] for v in prof.values())
    steps_ctx = {x: {"ms": round(v["ms"], 3), "GBps": (v["bytes"] / v["ms"] / 1e6) if v["ms"] else 0.0,
                     "bytes": v["bytes"]} for x, v in prof.items()}
    if P > 0:
        roof = None  # the per-step trace covers bc_compute's step kinds only
    elif p_launches > 0:
        # the persistent grid-schedule kernel runs every level step of every
        # batch: its algorithmic bytes per launch are the whole step's (every
        # step kind's compulsory bytes, from a traced run of the same
        # batches and directions) over its CUDA-event duration in the timed
        # region
        per_launch_bytes = step_bytes * args.steps / p_launches
        ms_launch = p_ms / p_launches
        achieved = per_launch_bytes / (ms_launch / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic_from_profiles("persistent", args.workload, grouping_name),
                "kernel": "k_persist", "launches_per_step": p_launches / args.steps,
                "bytes_per_launch": per_launch_bytes, "ms_per_launch": ms_launch,
                "share_of_step": p_ms / (1e3 * total_s), "peak_source": f"{peak_src} hbm_gbs (copy)",
                "slots": stats1["persist_slots"], "blocks": stats1["persist_blocks"],
                "steps": steps_ctx}
    else:
        kind = max(prof, key=lambda x: prof[x]["ms"])
        p = prof[kind]
        achieved = p["bytes"] / (p["ms"] / 1e3) / 1e9 if p["ms"] > 0 else 0.0
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic_from_profiles(kind, args.workload, grouping_name), "kernel": kind,
                "launches_per_step": p["launches"], "bytes_per_launch": p["bytes"] / max(p["launches"], 1),
                "ms_per_launch": p["ms"] / max(p["launches"], 1),
                "share_of_step": p["ms"] / total_ms if total_ms else None,
                "peak_source": f"{peak_src} hbm_gbs (copy)", "steps": steps_ctx}
    # the whole step in the timed region: every step kind's algorithmic bytes
    # over the timed step time
    if roof is not None:
        roof["timed_step"] = {"algorithmic_bytes": step_bytes, "ms": 1e3 * total_s / args.steps,
                              "GBps": step_bytes / total_s * args.steps / 1e9,
                              "frac": step_bytes / total_s * args.steps / 1e9 / peak}

    # ---- N > 1: the reduced BC of a sub-list against one GPU, bit for bit ----
    mcheck = None
    if world > 1:
        sub = 64
        with prepare(make(rp, col, wt, **opts)) as hs:
            hs.compute(src[:sub], stream=stream)
            mr.reduce_bc(hs, stream=stream, device=dev)
            red = hs.read_fixed()
        if rank == 0:
            allsub = np.concatenate([rank_sources(g, S, r)[:sub] for r in range(world)])
            with prepare(make(rp, col, wt, **opts)) as h1:
                h1.compute(allsub, stream=stream)
                one = h1.read_fixed()
            mcheck = {"sources": int(len(allsub)), "bit_identical": bool(np.array_equal(red, one))}

    # ---- CPU baseline: the oracle on a bounded sample ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle.pool import OraclePool, host_cores
        one = args.cpu_sample or oracle_sources_per_core(g.nnz, 4 * 10**8)
        val1, dt1, ks1 = cpu_oracle_gteps(g, S, min(one, k), wts)
        cores = host_cores()
        per = oracle_sources_per_core(g.nnz, 4 * 10**8)
        ks = min(per * cores, k)
        with OraclePool(g, wts, cores) as pool:
            _, dt = pool.bc(S[:ks])
        cpu = {"value": ks * g.nnz / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {ks} of the {k} sources over {cores} processes ({per} each), full graph; "
                         f"{dt:.1f} s",
               "single_core": {"value": val1, "sources": ks1, "seconds": round(dt1, 2)}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64+f64", "data": "synthetic",
                "config": {"workload": WORKLOADS[args.workload], "name": args.workload, "sources": k,
                           "n": g.n, "nnz": g.nnz, "batch_width": args.width,
                           "policy": args.policy + (" (learned, shipped weights)" if weights is not None else ""),
                           "source_grouping": "learned (shipped weights)" if gweights is not None else "list order",
                           "schedule": ["auto", "grid", "block", "pair"][st_all["schedule"]],
                           "tuned": {"batch_width": st_all["batch_width"],
                                     "heavy_degree": st_all["tuned_heavy_degree"],
                                     "device_loop": st_all["tuned_device_loop"]}
                           if st_all["tuned_heavy_degree"] else None,
                           "source_sample": (f"the first {k} sources of the workload's list" if args.sources > 0
                                             else None),
                           "l2": "flushed between timed steps (512 MiB device write)",
                           "partitions": ({"parts": P, "kind": "contiguous vertex ranges",
                                           "border_matrices_s": round(t_part, 3),
                                           **bc.partition_info()} if P > 0 else None)},
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "plain": plain, "vs_plain": (value / world / plain["value"]) if plain else None,
                "traversed": traversed, "multi_gpu_check": mcheck, "gpu_launches": launches, "clocks": clocks, "roofline": roof, "cpu_baseline": cpu,
                "step_ms": [round(x, 3) for x in step_ms]}
        print(json.dumps(line))
    bc.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
