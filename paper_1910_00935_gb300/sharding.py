"""Splitting independent scenes across ranks (one process per GPU).

Scenes of a batch never exchange data, so a multi-GPU run needs no collective on the data
path: every rank simulates its own scenes.  `shard_scenes` assigns scenes to ranks
greedily by particle count (largest first, to the least-loaded rank, ties to the lower
rank), which is deterministic and balances uneven batches; `subset` extracts those
scenes from a scene dict of `paper_1910_00935_gb300.scenes`.
"""
from __future__ import annotations

import pickle
from datetime import timedelta

import numpy as np


class RankFailure(RuntimeError):
    """Ranks that did not report their shard before the deadline."""

    def __init__(self, missing):
        super().__init__(f"ranks {sorted(missing)} did not report their shards")
        self.missing = sorted(missing)


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


def collect_shards(store, rank: int, world_size: int, payload, timeout_s: float = 60.0,
                   tag: str = "shard"):
    """Every rank publishes its shard's result in the rendezvous store; rank 0 waits for all
    of them for at most timeout_s and returns {rank: payload}, or raises RankFailure naming
    the ranks that never reported (a rank that crashed, hung or left).  Other ranks return
    None.  No collective runs, so a missing rank cannot hang the others."""
    store.set(f"{tag}/{rank}", pickle.dumps(payload))
    if rank != 0:
        return None
    keys = [f"{tag}/{r}" for r in range(world_size)]
    try:
        store.wait(keys, timedelta(seconds=timeout_s))
    except Exception:
        missing = [r for r, k in enumerate(keys) if not store.check([k])]
        if missing:
            raise RankFailure(missing) from None
        raise
    return {r: pickle.loads(store.get(k)) for r, k in enumerate(keys)}
