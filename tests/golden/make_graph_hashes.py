"""Write graph_hashes.json: SHA-256 of the CSR bytes of seeded generator
outputs.  Calls only the input generators; re-run after an intended change
to a generator and commit the result with the reason."""
import hashlib
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from paper_2008_05718_gb300 import graphgen as gg  # noqa: E402

CASES = {
    "er4096": lambda: gg.workload("er4096")[0],
    "rmat12": lambda: gg.rmat(12, 16, seed=1012),
    "rmat14_nopermute": lambda: gg.rmat(14, 16, seed=7, permute=False),
    "grid64": lambda: gg.grid(64, "0.03", seed=64),
    "grid200": lambda: gg.grid(200, "0.05", seed=3),
    "tri64": lambda: gg.tri(64, seed=6064),
    "rgg12": lambda: gg.rgg(1 << 12, 10.0, seed=7012),
    "mesh12": lambda: gg.mesh27(12),
}


def digest(g):
    h = hashlib.sha256()
    h.update(g.row_ptr.astype("<i4").tobytes())
    h.update(g.col.astype("<i4").tobytes())
    return h.hexdigest()


def compute():
    out = {}
    for name, make in CASES.items():
        g = make()
        out[name] = {"n": int(g.n), "nnz": int(g.nnz), "sha256": digest(g)}
    out["sources_rmat18"] = hashlib.sha256(gg.sample_sources(262144, 4096, seed=2).astype("<i4").tobytes()).hexdigest()
    return out


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "graph_hashes.json")
    with open(path, "w") as f:
        json.dump(compute(), f, indent=1, sort_keys=True)
    print("wrote", path)
