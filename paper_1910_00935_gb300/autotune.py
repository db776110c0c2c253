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

`tune_build` does the same for the build-time shapes: particles (= threads) per CTA,
`MPM_TILE`, with the CTAs per SM of each pass that follow from it.  Each candidate is a
library build of its own (`build.build(tag=...)`), timed in a child process (one process
loads one library) on the caller's scene and checked against the default build's final
positions; the fastest valid build's path is returned for `MPM_LIB`.
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


# build-time block shapes: variant tag -> extra nvcc flags (the default build is "tile128")
BUILD_SPACE = {"tile128": [], "tile64": ["-DMPM_TILE=64"], "tile256": ["-DMPM_TILE=256"]}

_CHILD = r"""
import json, sys, time
import numpy as np
sys.path.insert(0, {root!r})
import torch
from paper_1910_00935_gb300 import mpm
desc = json.load(open({desc!r}))
arrays = dict(np.load({npz!r}))
scene = {{"desc": desc, "arrays": arrays}}
T = {T}
sim = mpm.from_scene(scene, max_steps=T)
S = len(desc["n_particles"])
tgt = torch.as_tensor(arrays["target"]).cuda() if "target" in arrays else torch.zeros(S, desc["dim"], device="cuda")
def run():
    sim.forward(T)
    _, gT, _ = sim.loss(desc.get("loss_kind", 0), tgt)
    sim.backward(dL_dx=gT)
run()
torch.cuda.synchronize()
best = float("inf")
for _ in range({repeats}):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    run()
    e1.record()
    torch.cuda.synchronize()
    best = min(best, e0.elapsed_time(e1) / 1e3)
sim.check()
sim.forward(T)
np.save({xout!r}, sim.state()[0].cpu().numpy())
sim.check()
print(json.dumps({{"seconds": best}}))
"""


def _jsonable(v):
    import numpy as np
    if isinstance(v, np.ndarray):
        return v.tolist()
    if isinstance(v, np.generic):
        return v.item()
    raise TypeError(type(v))


def tune_build(scene: dict, T: int = 32, repeats: int = 2, space: dict = BUILD_SPACE,
               cache_path: str | None = None, force: bool = False, device_name: str | None = None,
               timeout: float = 900.0) -> dict:
    """Pick the build-time block shape for `scene` (a scenes.make dict) by measurement.
    Returns {"tag", "lib", "seconds": {tag: s}, "refused": {tag: reason}}; the library path
    is the one to load through MPM_LIB."""
    import subprocess
    import sys
    import tempfile

    import numpy as np

    from . import build as _build

    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name(0)
    key = "build|" + shape_key(scene["desc"], device_name)
    cache = load_cache(cache_path)
    if not force and key in cache and os.path.exists(cache[key]["lib"]):
        return cache[key]
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    seconds, refused, xs, libs = {}, {}, {}, {}
    with tempfile.TemporaryDirectory() as tmp:
        desc_path, npz = os.path.join(tmp, "desc.json"), os.path.join(tmp, "arrays.npz")
        with open(desc_path, "w") as f:
            json.dump(scene["desc"], f, default=_jsonable)
        np.savez(npz, **scene["arrays"])
        for tag, flags in space.items():
            try:
                libs[tag] = _build.build(extra_flags=flags, tag=tag if flags else "")
            except RuntimeError as e:
                refused[tag] = f"build failed: {str(e)[:200]}"
                continue
            xout = os.path.join(tmp, f"x_{tag}.npy")
            script = _CHILD.format(root=root, desc=desc_path, npz=npz, T=int(T), repeats=int(repeats),
                                   xout=xout)
            r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True,
                               env=dict(os.environ, MPM_LIB=libs[tag]), timeout=timeout)
            if r.returncode != 0:
                refused[tag] = "run failed: " + (r.stderr.strip().splitlines() or [""])[-1][:200]
                continue
            seconds[tag] = json.loads(r.stdout.strip().splitlines()[-1])["seconds"]
            xs[tag] = np.load(xout)
        ref = next(iter(space))  # the first entry is the default build: the others must agree
        if ref in xs:
            for tag in list(seconds):
                d = float(np.linalg.norm(xs[tag] - xs[ref]) / max(np.linalg.norm(xs[ref]), 1e-30))
                if not d <= 1e-5:
                    refused[tag] = f"final positions differ from {ref} by {d:.2e}"
                    del seconds[tag]
    if not seconds:
        raise RuntimeError(f"no build-time variant ran: {refused}")
    best = min(seconds, key=seconds.get)
    res = {"tag": best, "lib": libs[best], "flags": list(space[best]), "seconds": seconds,
           "refused": refused, "T_probe": int(T)}
    cache[key] = res
    save_cache(cache, cache_path)
    return res
