"""Training the learned direction policy from traces of the method itself.

Every forward step of a batch can run top-down (push) or bottom-up (pull);
both compute the same level, so a trace that times both directions at every
level (GBBC_TRACE | GBBC_TRACE_BOTH) gives the exact cost of either choice.
The network learns, from the six level features of the trace, which
direction is cheaper: softmax cross-entropy with the faster direction as the
class and |t_push - t_pull| as the sample weight, trained by the library's
own CUDA kernels (bc_mlp_train: forward, backward and Adam on the device).

    python -m paper_2008_05718_gb300.policy train   # writes policy_weights.f32
    python -m paper_2008_05718_gb300.policy eval    # learned vs threshold rule

The shipped weights (policy_weights.f32, FP32, bc_mlp_param_count(2) values)
are loaded with BC.load_policy (bench.py does so by default); a handle with
them loaded and GBBC_POLICY_AUTO uses the network, else the threshold rule.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "policy_weights.f32")


def shipped_weights():
    """FP32 parameters of the shipped direction network, or None."""
    if not os.path.exists(WEIGHTS):
        return None
    return np.fromfile(WEIGHTS, dtype=np.float32)


def training_graphs(seed=0):
    """R-MAT scales 14-17 (the social/web class) and grids (the road class)."""
    from . import graphgen as gg
    out = []
    for s in (14, 15, 16, 17):
        out.append((f"rmat{s}", gg.rmat(s, 16, seed=seed + 100 + s)))
    for side in (96, 160, 256, 512, 1024):
        out.append((f"grid{side}", gg.grid(side, "0.05", seed=seed + 200 + side)))
    return out


def collect(graphs, sources=256, width=64, policy="beamer", seed=1):
    """Per-level records with both directions timed: dict of arrays."""
    from . import gbbc
    from . import graphgen as gg
    recs = []
    for name, g in graphs:
        # large high-diameter graphs: one batch is thousands of levels
        S = gg.sample_sources(g.n, min(sources if g.n < 200000 else 64, g.n), seed=seed)
        flags = gbbc.GBBC_TRACE | gbbc.GBBC_TRACE_BOTH
        with gbbc.BC.from_graph(g, batch_width=width, policy=policy, flags=flags) as bc:
            bc.compute(S[:min(64, len(S), 8 if g.n >= 200000 else 64)])  # warm-up (not kept)
            bc.clear_trace()
            bc.compute(S)
            tr = bc.trace()
        ok = (tr["ms_push"] > 0) & (tr["ms_pull"] > 0)
        recs.append({"graph": np.array([name] * int(ok.sum())), "features": tr["features"][ok],
                     "ms_push": tr["ms_push"][ok], "ms_pull": tr["ms_pull"][ok],
                     "direction": tr["direction"][ok], "level": tr["level"][ok]})
    return {k: np.concatenate([r[k] for r in recs]) for k in recs[0]}


def dataset(tr):
    x = tr["features"].astype(np.float32)
    t = (tr["ms_pull"] < tr["ms_push"]).astype(np.float32)
    w = np.abs(tr["ms_push"] - tr["ms_pull"]).astype(np.float32)
    return x, t, w / max(float(w.mean()), 1e-9)


def init_params(seed=0):
    """He-style initialisation of the 6-32-32-2 network (FP32)."""
    r = np.random.default_rng(seed)
    H, IN = 32, 6
    parts = [r.normal(0, np.sqrt(2 / IN), H * IN), np.zeros(H), r.normal(0, np.sqrt(2 / H), H * H), np.zeros(H),
             r.normal(0, np.sqrt(1 / H), 2 * H), np.zeros(2)]
    return np.concatenate(parts).astype(np.float32)


def train(tr, epochs=1500, lr=3e-3, seed=0):
    from . import gbbc
    x, t, w = dataset(tr)
    p, hist = gbbc.bc_mlp_train(init_params(seed), x, t, w, k_out=2, loss_kind=0, epochs=epochs, lr=lr)
    return p.cpu().numpy().astype(np.float32), hist


def costs(params, tr):
    """Total step time (ms) under each schedule on traced levels."""
    from . import gbbc
    _, choice = gbbc.bc_policy_eval(params, tr["features"])
    t = np.stack([tr["ms_push"], tr["ms_pull"]], axis=1)
    idx = np.arange(len(t))
    return {"learned": float(t[idx, choice].sum()), "threshold": float(t[idx, tr["direction"]].sum()),
            "best": float(t.min(axis=1).sum()), "push": float(t[:, 0].sum()), "pull": float(t[:, 1].sum()),
            "levels": int(len(t))}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "eval"])
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--epochs", type=int, default=1500)
    ap.add_argument("--sources", type=int, default=256)
    a = ap.parse_args(argv)
    import torch
    torch.cuda.init()
    if a.cmd == "train":
        tr = collect(training_graphs(), sources=a.sources)
        p, hist = train(tr, epochs=a.epochs)
        p.tofile(a.out)
        held = collect(training_graphs(seed=7), sources=a.sources, seed=9)
        print(json.dumps({"levels": int(len(tr["level"])), "loss_first": float(hist[0]), "loss_last": float(hist[-1]),
                          "train": costs(p, tr), "held_out": costs(p, held), "out": a.out}))
    else:
        p = np.fromfile(a.out, dtype=np.float32)
        held = collect(training_graphs(seed=7), sources=a.sources, seed=9)
        print(json.dumps({"held_out": costs(p, held)}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
