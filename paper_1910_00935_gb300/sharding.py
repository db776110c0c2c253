"""Splitting independent scenes across ranks (one process per GPU).

Scenes of a batch never exchange data, so a multi-GPU run needs no collective on the data
path: every rank simulates its own scenes.  `shard_scenes` assigns scenes to ranks
greedily by particle count (largest first, to the least-loaded rank, ties to the lower
rank), which is deterministic and balances uneven batches; `subset` extracts those
scenes from a scene dict of `paper_1910_00935_gb300.scenes`.
"""
from __future__ import annotations

import numpy as np


def shard_scenes(n_particles, world_size: int, rank: int):
    """Indices (ascending) of the scenes that `rank` simulates."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("bad world_size / rank")
    order = sorted(range(len(n_particles)), key=lambda i: (-int(n_particles[i]), i))
    load = [0] * world_size
    owner = [0] * len(n_particles)
    for i in order:
        r = min(range(world_size), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += int(n_particles[i])
    return [i for i in range(len(n_particles)) if owner[i] == rank]


def subset(scene, idx):
    """The batch made of scenes `idx` of `scene` (arrays sliced, description updated)."""
    idx = list(idx)
    desc = dict(scene["desc"])
    a = scene["arrays"]
    off = np.concatenate([[0], np.cumsum(desc["n_particles"])])
    sl = [slice(int(off[i]), int(off[i + 1])) for i in idx]
    cols = lambda k: np.ascontiguousarray(np.concatenate([a[k][..., s] for s in sl], axis=-1))
    arr = {k: cols(k) for k in ("x0", "v0", "C0", "F0", "E", "nu", "group") + (
        ("material",) if "material" in a else ())}
    arr["w"] = np.ascontiguousarray(a["w"][idx])
    arr["target"] = np.ascontiguousarray(a["target"][idx])
    desc["n_particles"] = [int(desc["n_particles"][i]) for i in idx]
    desc["n_scenes"] = len(idx)
    return {"desc": desc, "arrays": arr}
