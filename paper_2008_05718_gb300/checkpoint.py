"""Checkpoint and resume of a long BC computation over a source list.

BC is a sum over sources (Eq. 2), and the library keeps a handle's BC as an
exact 128-bit fixed-point vector (bc_read_fixed; units 2^-64).  A computation
over a long source list can therefore be cut into chunks: after each chunk
the handle's exact BC and the number of sources done are written to a file,
and a later process (a new handle over the same graph) adds the saved vector
back with bc_add_fixed and goes on after the last finished chunk.  Integer
sums do not depend on how the sources were split, so a resumed run gives the
bits of an uninterrupted one.

File: a NumPy .npz with the format number, the graph's vertex count, the
number of sources done, a SHA-256 digest of the int32 source list, and the
fixed-point vector (uint64, 2n words: low, high per vertex).  It is written
to a temporary name and renamed over the old file, so a crash while writing
leaves the previous checkpoint intact.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np

FORMAT = 1


def sources_digest(sources) -> str:
    """SHA-256 (32 hex digits) of the source list as int32."""
    s = np.ascontiguousarray(sources, dtype=np.int32)
    return hashlib.sha256(s.tobytes()).hexdigest()[:32]


def save(path: str, bc_fixed, done: int, n: int, digest: str) -> None:
    """Write a checkpoint: the exact BC of the first `done` sources."""
    words = np.ascontiguousarray(bc_fixed).view(np.uint64).reshape(-1)
    if words.size != 2 * n:
        raise ValueError(f"fixed-point vector of {words.size} words for {n} vertices")
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        np.savez(f, format=np.int64(FORMAT), n=np.int64(n), done=np.int64(done), sources=np.array(digest),
                 bc_fixed=words)
    os.replace(tmp, path)


def load(path: str) -> dict:
    """The checkpoint's fields: format, n, done, sources (digest), bc_fixed."""
    with np.load(path) as z:
        ck = {"format": int(z["format"]), "n": int(z["n"]), "done": int(z["done"]),
              "sources": str(z["sources"]), "bc_fixed": z["bc_fixed"].copy()}
    if ck["format"] != FORMAT:
        raise ValueError(f"checkpoint format {ck['format']}, expected {FORMAT}")
    return ck


def compute_resumable(bc, sources, path: str, chunk: int = 4096, stream=None) -> int:
    """Add the dependencies of `sources` into `bc` in chunks of `chunk`
    sources, writing a checkpoint to `path` after each chunk.  If `path`
    holds a checkpoint of the same vertex count and source list, its BC is
    added into `bc` first and the computation goes on after its last chunk.
    `bc` (a gbbc.BC handle, or anything with n, compute, read_fixed and
    add_fixed) must hold no other sources' BC.  Returns the number of sources
    this call computed."""
    if chunk < 1:
        raise ValueError("chunk must be at least 1")
    S = np.ascontiguousarray(sources, dtype=np.int32)
    digest = sources_digest(S)
    done = 0
    if os.path.exists(path):
        ck = load(path)
        if ck["n"] != bc.n or ck["sources"] != digest:
            raise ValueError(f"{path} belongs to another graph or source list")
        if not 0 <= ck["done"] <= len(S):
            raise ValueError(f"{path}: {ck['done']} sources done of {len(S)}")
        bc.add_fixed(ck["bc_fixed"], stream=stream)
        done = ck["done"]
    start = done
    while done < len(S):
        hi = min(len(S), done + chunk)
        bc.compute(S[done:hi], stream=stream)
        done = hi
        save(path, bc.read_fixed(stream=stream), done, bc.n, digest)
    return done - start
