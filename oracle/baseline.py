"""Timing of the FP64 oracle on the host cores -- TEST INFRASTRUCTURE (the CPU baseline).

    python -m oracle.baseline --workload cube3d --steps 64 --threads 16

Runs the oracle as it stands (``loss_and_grad``: forward with every state kept, the loss,
the reverse replay of Appendix D.1 in FP64) on a bounded sample of a workload and prints
one JSON line with particle-steps per second.  ``--threads 1`` uses the serial build,
``--threads N`` (N > 1) the OpenMP build of the same source on N threads.  It is run as a
child process of the benchmark so that its OpenMP runtime never shares a process with the
GPU path's libraries.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# the scene sample each workload is timed on: (generator kwargs, description)
SAMPLES = {
    "robots3d": (dict(n_scenes=1), "one of the 16 independent robots (65,536 particles)"),
    "robots_nn": (dict(n_scenes=1), "one of the 4 independent robots (27,648 particles)"),
}


def run(workload: str, steps: int, threads: int) -> dict:
    if threads > 1:
        os.environ["ORACLE_OPENMP"] = "1"
        os.environ["OMP_NUM_THREADS"] = str(threads)
    import oracle
    from paper_1910_00935_gb300 import scenes
    kw, what = SAMPLES.get(workload, ({}, "the whole workload"))
    scene = scenes.make(workload, **kw)
    N = int(sum(scene["desc"]["n_particles"]))
    view = scenes.oracle_view(scene)
    used = oracle.threads(threads if threads > 1 else 0)
    t0 = time.perf_counter()
    oracle.loss_and_grad(view, steps)
    dt = time.perf_counter() - t0
    return {"value": N * steps / dt, "unit": "particle-steps/s", "cores": used,
            "kind": "oracle", "build": "OpenMP" if threads > 1 else "serial",
            "sample": f"{what} of {workload}: {N} particles x {steps} steps forward + loss + "
                      f"backward (FP64)",
            "seconds": round(dt, 3), "units": N * steps}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cube3d")
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--threads", type=int, default=1)
    a = ap.parse_args()
    print(json.dumps(run(a.workload, a.steps, a.threads)), flush=True)


if __name__ == "__main__":
    main()
