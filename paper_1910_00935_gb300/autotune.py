"""Autotuner for the launch knobs of libmpm (measurement-based, cached).

The knobs are the library's runtime options: the capacity of the shared gather box
(MPM_OPT_GATHER_CAPACITY), the scatter path (MPM_OPT_SMEM_TILE: shared node box vs. float4
reductions straight to the grid; MPM_OPT_BUCKET_SCATTER: one reduction per stencil base and
node, summed by a warp, vs. one per particle and node), the shared box capacity (MPM_OPT_TILE_CAPACITY), the
CTA count of the end-of-sequence grid clear (MPM_OPT_GRID_BLOCKS), the launch form
(MPM_OPT_PERSISTENT: one launch per pass, or persistent launches over the pass plan), and two
memory-vs-recompute choices of the backward: a re-simulated segment's grids kept or recomputed
per step (MPM_OPT_GRID_RECOMPUTE) and the re-simulation overlapped with the adjoint passes on a
second stream or run before them (MPM_OPT_OVERLAP_RESIM).  `tune` times a short forward+backward
of the caller's own simulator for each candidate, one knob at a time (coordinate descent
from the defaults), keeps the fastest, and caches the result in a JSON file keyed by the
workload's shape class and the device name.  Results never change numerics beyond FP32
atomic-order rounding (the GPU tests check every knob setting against the oracle).
"""
from __future__ import annotations

import json
import math
import os

SPACE = {
    "gather_capacity": [512, 0, 1024, 2048],
    "smem_tile": [0, 1],
    "bucket_scatter": [0, 1],
    "pair_scatter": [0, 1, 3],
    "sort_order": [0, 1, 2],
    "tile_capacity": [1024, 2048],
    "grid_blocks": [0, 32, 64, 128],
    "persistent": [0, 1],
    "grid_recompute": [0, 1],
    "overlap_resim": [1, 0],
}
DEFAULTS = {"gather_capacity": 512, "smem_tile": 0, "bucket_scatter": 0, "pair_scatter": 0, "sort_order": 0,
            "tile_capacity": 1024,
            "grid_blocks": 0,
            "persistent": 0, "grid_recompute": 0, "overlap_resim": 1}

_OPTION_IDS = {"gather_capacity": 5, "smem_tile": 2, "bucket_scatter": 14, "pair_scatter": 15, "sort_order": 16,
               "tile_capacity": 3,
               "grid_blocks": 6,
               "persistent": 8, "grid_recompute": 12, "overlap_resim": 13}


def default_cache_path() -> str:
    return os.environ.get("MPM_TUNE_CACHE",
                          os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build",
                                       "autotune.json"))


def shape_key(desc: dict, device_name: str = "") -> str:
    """Workloads of the same dimension, material, grid, scene count and particle count
    (to within a factor of 2) share tuned knobs."""
    N = int(sum(desc["n_particles"]))
    return "|".join(str(v) for v in (
        device_name, desc["dim"], desc["material"], desc["n_grid"], len(desc["n_particles"]),
        int(math.log2(max(N, 1))), 1 if desc.get("n_groups", 0) else 0))


def load_cache(path: str | None = None) -> dict:
    path = path or default_cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str | None = None) -> None:
    path = path or default_cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def coordinate_descent(measure, space=SPACE, start=DEFAULTS, rounds: int = 1):
    """Minimise measure(config) -> seconds one knob at a time.  Returns (best config,
    best time, list of (config, time) evaluated)."""
    best = dict(start)
    best_t = measure(best)
    log = [(dict(best), best_t)]
    for _ in range(rounds):
        improved = False
        for knob, values in space.items():
            for v in values:
                if v == best[knob]:
                    continue
                cand = dict(best, **{knob: v})
                t = measure(cand)
                log.append((dict(cand), t))
                if t < best_t:
                    best, best_t, improved = cand, t, True
        if not improved:
            break
    return best, best_t, log


def apply(sim, config: dict) -> None:
    """Set the knobs of `config` on a Simulator (the particle order takes effect through a
    new set-up from the simulator's inputs)."""
    for knob, value in config.items():
        sim.set_option(_OPTION_IDS[knob], int(value))
    if "sort_order" in config and getattr(sim, "_inputs", None) is not None:
        sim.reload()


def tune(sim, T: int = 32, repeats: int = 2, cache_path: str | None = None, force: bool = False):
    """Tune the knobs for `sim` (a Simulator with its initial state set) and apply them.
    Returns the chosen configuration."""
    import torch

    from .mpm import MPMError

    key = shape_key(sim.desc, torch.cuda.get_device_name(sim.device))
    cache = load_cache(cache_path)
    if not force and key in cache:
        apply(sim, cache[key]["config"])
        return cache[key]["config"]
    T = min(T, sim.max_steps)
    target = torch.zeros(sim.n_scenes, sim.dim, device=sim.device)

    failed = []

    def measure(config):
        # a candidate the library refuses (an error status from any call) is infeasible:
        # it is recorded and never chosen, and the next candidate starts from a new set-up
        try:
            apply(sim, config)
            best = float("inf")
            for _ in range(repeats + 1):  # the first run captures the graphs
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                sim.forward(T)
                _, gT, _ = sim.loss(0, target)
                sim.backward(dL_dx=gT)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1e3)
            sim.check()
            return best
        except MPMError as e:
            failed.append([dict(config), str(e)])
            return float("inf")

    config, t, log = coordinate_descent(measure)
    sim.autotune_failed = failed
    apply(sim, config)
    if "sort_order" not in config and getattr(sim, "_inputs", None) is not None:
        sim.reload()
    cache[key] = {"config": config, "seconds_per_probe": t, "T_probe": T,
                  "evaluated": [[c, s] for c, s in log], "failed": failed}
    save_cache(cache, cache_path)
    return config
