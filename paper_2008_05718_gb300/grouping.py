"""Training the learned source-grouping network (which sources share a word).

A 64-lane batch runs as many levels as its deepest source needs, and every
level pays for the union of the lanes' frontiers.  Sources whose BFS level
profiles line up therefore make cheaper words than a random mix: a source
whose mean BFS distance is small (a hub, or a vertex of a tiny component)
finishes in a few levels, a peripheral one needs many more.  The network
(6 -> 32 -> 32 -> 1, the same shape as the direction network, one output)
predicts log2(1 + mean BFS distance) of each source from six features the
library computes on the device (bc_source_features); bc_compute then orders
each graph's sources by that score before packing them into words.  The BC
bits do not depend on the order: only the time does.

Targets come from the method itself: kept per-source BFS distances
(GBBC_KEEP_STATE) of the library's own forward pass.  Training runs on the
library's CUDA kernels (bc_mlp_train, squared error, Adam).

    python -m paper_2008_05718_gb300.grouping train   # writes grouping_weights.f32
    python -m paper_2008_05718_gb300.grouping eval    # held-out rank correlation and timing
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "grouping_weights.f32")


def shipped_weights():
    """FP32 parameters of the shipped grouping network, or None."""
    if not os.path.exists(WEIGHTS):
        return None
    return np.fromfile(WEIGHTS, dtype=np.float32)


def training_graphs(seed=0):
    """R-MAT scales 14-17 (skewed degrees, many isolated vertices), two
    Erdos-Renyi graphs and two perturbed grids."""
    from . import graphgen as gg
    out = [(f"rmat{s}", gg.rmat(s, 16, seed=seed + 100 + s)) for s in (14, 15, 16, 17)]
    out += [(f"er{n}", gg.er(n, f"8/{n}", seed=seed + 300 + n)) for n in (4096, 16384)]
    out += [(f"grid{side}", gg.grid(side, "0.05", seed=seed + 200 + side)) for side in (96, 256)]
    return out


def mean_distance(dist):
    """Mean BFS distance over the vertices a source reaches (0 when it reaches none)."""
    r = dist[dist > 0]
    return float(r.mean()) if len(r) else 0.0


def collect(graphs, sources=512, seed=1):
    """Features (device kernel) and targets log2(1 + mean distance) of sampled sources."""
    from . import gbbc
    from . import graphgen as gg
    xs, ts, names = [], [], []
    for name, g in graphs:
        S = gg.sample_sources(g.n, min(sources, g.n), seed=seed)
        with gbbc.BC.from_graph(g, flags=gbbc.GBBC_KEEP_STATE) as bc:
            xs.append(bc.source_features(S))
            bc.compute(S)
            md = np.array([mean_distance(bc.source_state(i)[0]) for i in range(len(S))])
        ts.append(np.log2(1.0 + md).astype(np.float32))
        names += [name] * len(S)
    return np.concatenate(xs), np.concatenate(ts), np.array(names)


def init_params(seed=0):
    """He-style initialisation of the 6-32-32-1 network (FP32)."""
    r = np.random.default_rng(seed)
    H, IN = 32, 6
    parts = [r.normal(0, np.sqrt(2 / IN), H * IN), np.zeros(H), r.normal(0, np.sqrt(2 / H), H * H), np.zeros(H),
             r.normal(0, np.sqrt(1 / H), H), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def train(x, t, epochs=3000, lr=3e-3, seed=0):
    from . import gbbc
    p, hist = gbbc.bc_mlp_train(init_params(seed), x, t, None, k_out=1, loss_kind=1, epochs=epochs, lr=lr)
    return p.cpu().numpy().astype(np.float32), hist


def rank_correlation(a, b):
    """Spearman's rho (average ranks for ties)."""
    def ranks(v):
        v = np.asarray(v, dtype=np.float64)
        order = np.argsort(v, kind="stable")
        r = np.empty(len(v))
        r[order] = np.arange(len(v), dtype=np.float64)
        _, inv, cnt = np.unique(v, return_inverse=True, return_counts=True)
        sums = np.bincount(inv, weights=r)
        return (sums / cnt)[inv]
    ra, rb = ranks(a), ranks(b)
    ra -= ra.mean()
    rb -= rb.mean()
    den = np.sqrt((ra * ra).sum() * (rb * rb).sum())
    return float((ra * rb).sum() / den) if den > 0 else 0.0


def predict(params, x):
    from . import gbbc
    return gbbc.bc_mlp_forward(params, x, k_out=1).cpu().numpy()[:, 0]


def per_graph_correlation(params, x, t, names):
    p = predict(params, x)
    return {nm: round(rank_correlation(p[names == nm], t[names == nm]), 4) for nm in dict.fromkeys(names)}


def time_orders(g, S, params, policy_weights=None, reps=2):
    """Seconds for list order and for the grouped order (best of reps) and whether the bits agree."""
    import torch
    from . import gbbc
    res = {}
    outs = []
    for label, w in (("list", None), ("grouped", params)):
        with gbbc.BC.from_graph(g) as bc:
            if policy_weights is not None:
                bc.load_policy(policy_weights)
            if w is not None:
                bc.load_grouping(w)
            bc.compute(S[:64])
            bc.sync()
            best = None
            for _ in range(reps):
                bc.reset()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                bc.compute(S)
                bc.sync()
                dt = time.perf_counter() - t0
                best = dt if best is None else min(best, dt)
            outs.append(bc.read_fixed())
        res[label] = best
    res["identical_bits"] = bool(np.array_equal(outs[0], outs[1]))
    return res


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "eval"])
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--sources", type=int, default=512)
    a = ap.parse_args(argv)
    import torch
    torch.cuda.init()
    from . import graphgen as gg
    from . import policy
    if a.cmd == "train":
        x, t, names = collect(training_graphs(), sources=a.sources)
        p, hist = train(x, t, epochs=a.epochs)
        p.tofile(a.out)
        report = {"samples": int(len(t)), "loss_first": float(hist[0]), "loss_last": float(hist[-1]),
                  "train_rho": per_graph_correlation(p, x, t, names)}
    else:
        p = np.fromfile(a.out, dtype=np.float32)
        report = {}
    hx, ht, hn = collect(training_graphs(seed=7), sources=a.sources, seed=9)
    report["held_out_rho"] = per_graph_correlation(p, hx, ht, hn)
    g = gg.rmat(17, 16, seed=901)
    S = gg.sample_sources(g.n, 2048, seed=5)
    report["held_out_time_rmat17"] = time_orders(g, S, p, policy.shipped_weights())
    report["out"] = a.out
    print(json.dumps(report))
    return 0


if __name__ == "__main__":
    sys.exit(main())
