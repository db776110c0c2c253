"""Benchmark of the differentiable MLS-MPM hot path (forward + reverse tape) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload cube3d|robots3d|...]
    python bench.py --impl reference ...     # the FP64 CPU oracle, timed on host cores

One bench step = one pass of the whole hot path on one batch: set the initial state,
forward T MLS-MPM steps with checkpoints, centre-of-mass loss, backward through the
tape (segment re-simulation, per-step grid recompute, adjoint kernels), gradients out.
The metric is particle-steps per second of forward+backward (N particles x T steps per
bench step).  `value` is measured with the inputs already on the device; `e2e` times
the same step through the public API from pinned host buffers, the host<->device copies
inside the timed region.  Prints one JSON line (rank 0).

Multi-GPU (torchrun): the scenes of a batch are independent, so no collective runs on the
data path.  By default every rank owns one seeded batch of the workload (the job's batch is
the union, partitioned by rank: weak scaling); with --shard the one batch's scenes are split
across the ranks by shard_scenes, balanced by particle count (strong scaling).  The ranks'
losses are gathered after the timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# the workload's headline metric; `value` is the forward+backward figure, the forward one is in
# the line's `forward` object and the HBM fraction in `roofline`
METRIC = ("particle-steps/s fwd and fwd+bwd (3D, FP32, grad err<=1e-3 vs FP64 oracle); "
          "% HBM roofline")
UNIT = "particle-steps/s"

# algorithmic bytes per particle of each pass category (3D, FP32 state rows):
# x, v: 12 B each; C, F: 36 B each; mu, la: 8 B; full state 96 B.
def alg_bytes(d):
    """Algorithmic bytes per particle of each pass category (FP32 state rows; the minimum
    each pass must move).  S: full state x, v, C, F; XF: x and F rows; M: mu, la;
    MB: mu-bar, la-bar (FP64 sums over the steps) read and written."""
    S, XF, X, C = 4 * (2 * d + 2 * d * d), 4 * (d + d * d), 4 * d, 4 * d * d
    M, MB = 8, 32
    return {
        "p2g": S + M,                       # read x, v, C, F, mu, la
        "g2p_p2g": XF + M + XF,             # read x, F, mu, la; write x, F
        "g2p_p2g_full": XF + M + S,         # read x, F, mu, la; write x, v, C, F
        "g2p": XF + S,                      # read x, F; write the full state
        "adj_g2p": S + XF + (X + C) + XF,   # read adj, x F of state s, x C of state s+1; write adj x F
        "adj_fused": S + XF + 2 * XF + M + MB + S,  # state s+1, x F of state s, adj x F (rw),
                                                    # mu la, mubar labar (rw), state s-1 (P2G)
        "adj_p2g": S + XF + M + MB + S,     # state 0, adj x F, mu la, mubar labar; write full adj
    }




def pass_bytes(N, T, K, dim=3, kept=True):
    """Algorithmic bytes of one bench step per kernel category, for both launch forms (the
    per-pass categories and the persistent launches that run the same passes), following
    the library's schedule: the forward writes the full state at checkpoints and over its
    last segment (left resident); the backward computes the grid of step T-1 with one P2G
    pass, re-simulates every other segment, and each fused adjoint pass also recomputes
    the grid of the step before unless the segment's grids were kept (kept=True) -- the
    resident segment always recomputes."""
    a = alg_bytes(dim)
    state_s_minus_1 = 4 * (2 * dim + 2 * dim * dim)
    by = {k: 0 for k in ("p2g", "g2p_p2g", "g2p_p2g_full", "g2p", "adj_g2p", "adj_fused",
                         "adj_p2g")}
    sL = ((T - 1) // K) * K
    by["p2g"] += a["p2g"]
    for t in range(1, T):
        by["g2p_p2g_full" if (t % K == 0 or t > sL) else "g2p_p2g"] += 1
    by["g2p_p2g"] *= a["g2p_p2g"]
    by["g2p_p2g_full"] *= a["g2p_p2g_full"]
    by["g2p"] += a["g2p"]
    fwd = sum(by.values())
    back = {k: 0 for k in by}
    back["p2g"] += a["p2g"]  # grid of step T-1 (resident last segment)
    for s0 in range(0, sL, K):
        n = min(K, T - s0)
        back["p2g"] += a["p2g"]
        back["g2p_p2g_full"] += (n - 1) * a["g2p_p2g_full"]
        back["g2p"] += a["g2p"]
    back["adj_g2p"] += a["adj_g2p"]
    for s in range(T - 2, -1, -1):
        s0 = (s // K) * K
        recompute = s - 1 >= s0 and (s0 == sL or not kept)
        back["adj_fused"] += a["adj_fused"] - (0 if recompute else state_s_minus_1)
    back["adj_p2g"] += a["adj_p2g"]
    out = {k: by[k] + back[k] for k in by}
    out["persistent_step"] = fwd + back["p2g"] + back["g2p_p2g_full"] + back["g2p"]
    out["persistent_adj"] = back["adj_g2p"] + back["adj_fused"] + back["adj_p2g"]
    return {k: v * N for k, v in out.items()}


def pass_bytes_ctrl(N, T, K, dim=3, kept=True):
    """pass_bytes for a closed-loop controller scene (ctrl_hidden > 0), following its split
    schedule: the forward runs G2P (full state written), the controller and P2G (from the
    full state) for every step; the backward runs, per step, the P2G adjoint of step s+1
    (full adjoint written), the controller's reverse and the G2P adjoint of step s (from the
    full adjoint), recomputing a grid with its own P2G pass where it is neither kept nor
    re-simulated.  The controller's sensing reads x, v and the group id; its reverse adds to
    the x and v rows of the adjoint."""
    a = alg_bytes(dim)
    S = 4 * (2 * dim + 2 * dim * dim)
    XF, M, MB = 4 * (dim + dim * dim), 8, 32
    sense, sense_adj = 4 * 2 * dim + 4, 4 + 2 * 4 * 2 * dim
    by = {k: 0 for k in ("p2g", "g2p_p2g", "g2p_p2g_full", "g2p", "adj_g2p", "adj_fused",
                         "adj_p2g", "controller")}
    by["p2g"] += T * a["p2g"]
    by["g2p"] += T * a["g2p"]
    by["controller"] += T * sense
    sL = ((T - 1) // K) * K
    by["p2g"] += a["p2g"]  # grid of step T-1 (resident last segment)
    for s0 in range(0, sL, K):
        n = min(K, T - s0)
        by["p2g"] += a["p2g"]
        by["g2p_p2g_full"] += (n - 1) * a["g2p_p2g_full"]
        by["g2p"] += a["g2p"]
        if not kept:
            by["p2g"] += (n - 1) * a["p2g"]
    by["p2g"] += (T - 1 - sL) * a["p2g"]  # the resident segment's grids
    adj_p2g = S + XF + M + MB + S
    by["adj_p2g"] += T * adj_p2g
    by["controller"] += T * sense_adj
    by["adj_g2p"] += T * a["adj_g2p"]
    return {k: v * N for k, v in by.items()}


def source_digest():
    """Digest of the particle-pass kernels' sources (mpm_kernels.cuh, mpm_common.cuh,
    kernels_launch.cuh, kernels_*.cu): a DRAM-traffic figure read from a profile summary
    counts only if the summary was taken on these exact kernels."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1910_00935_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f in ("mpm_kernels.cuh", "mpm_common.cuh", "kernels_launch.cuh") or \
                (f.startswith("kernels_") and f.endswith(".cu")):
            h.update(f.encode())
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(workload, category):
    """DRAM bytes per launch (read + write) from profiles/ncu_<category>_<workload>.md when
    that summary carries this source digest; else None."""
    path = os.path.join(ROOT, "profiles", f"ncu_{category}_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    if f"source digest: {source_digest()}" not in text:
        return None
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    total = 0.0
    for metric in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
        row = [ln for ln in text.splitlines() if ln.startswith(f"| `{metric}` |")]
        if not row:
            return None
        cells = [c.strip() for c in row[0].strip("|").split("|")]
        vals = [float(c) for c in cells[1:-1]]
        total += statistics.mean(vals) * scale.get(cells[-1], float("nan"))
    return total


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def precision_label(desc):
    """What the workload's passes compute in: FP32 arithmetic, with the polar factor of
    fixed-corotated particles resolved to FP64 accuracy by compensated FP32 arithmetic."""
    mat = desc.get("material", 0)
    fcr = ("FP32 state, grid and stress; polar factor resolved to FP64 accuracy in compensated "
           "FP32, FP32 polar adjoint")
    nh = "FP32 throughout (neo-Hookean: J - 1 and ln J in FP32; no polar factor)"
    liq = "FP32 throughout (Tait liquid: J - 1, log1p/expm1 in FP32; no polar factor)"
    return {0: fcr, 1: nh, 3: liq,
            4: "per-particle materials: " + fcr + " for the solid, FP32 for the liquid"}.get(mat, fcr)


def make_workload(name, seed=0):
    from paper_1910_00935_gb300 import scenes
    scene = scenes.make(name, seed=seed)
    d = scene["desc"]
    N = sum(d["n_particles"])
    descr = {
        "cube3d": "3D elastic cube: 262,144 particles (64^3 lattice, 2/cell/axis), 128^3 grid, "
                  "neo-Hookean E=5e3 nu=0.3, dt=1e-4, T=1024, checkpoint every 64, COM loss",
        "robots3d": "16 batched 3D actuated robots x 65,536 particles, 64^3 grids, "
                    "fixed-corotated, 8 groups x 4 sine terms, T=2048, ckpt 64",
        "rects2d": "64 batched 2D rectangles (1k-16k particles), 128^2 grids, T=512",
        "square2d_grad": "2D square 4,096 particles, 128^2 grid, T=512, ckpt 32",
        "robots_nn": "4 batched 3D robots x 27,648 particles, 64^3 grids, fixed-corotated, "
                     "8 groups driven by a closed-loop MLP controller (52 inputs, 32 tanh "
                     "units), T=512, ckpt 64",
        "liquid2d": "2D dam break: 6,144 weakly compressible liquid particles (Tait, E=500 "
                    "nu=0.3), 128^2 grid, dt=1e-4, T=256, ckpt 32, COM loss",
        "liquid3d": "3D dam break: 49,152 weakly compressible liquid particles (Tait, E=500 "
                    "nu=0.3), 64^3 grid, dt=1e-4, T=256, ckpt 32, COM loss",
        "robot_in_liquid": "3D actuated fixed-corotated robot (8,192 particles, 8 groups x 4 "
                           "sine terms) in a liquid pool (55,296 particles), per-particle "
                           "materials in one 64^3 grid, T=256, ckpt 32, x-displacement loss",
    }.get(name, name)
    return scene, N, d["steps"], descr


# bounded oracle samples: steps of the all-cores run and of the single-thread run
CPU_WINDOWS = {"cube3d": (64, 2), "robots3d": (64, 4), "rects2d": (16, 4),
               "square2d_grad": (64, 32), "robots_nn": (16, 4)}


def host_cores():
    """Cores available to this process, and the host CPU's model name (lscpu)."""
    cores = len(os.sched_getaffinity(0))
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return cores, model


def oracle_timing(name, steps, threads):
    """One timing of the FP64 oracle (oracle/baseline.py) in a child process: its OpenMP
    runtime never shares a process with the GPU path's libraries."""
    cmd = [sys.executable, "-m", "oracle.baseline", "--workload", name, "--steps", str(steps),
           "--threads", str(threads)]
    r = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(f"oracle baseline failed: {r.stderr[-2000:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(name, single_thread=True):
    """The FP64 oracle, as it stands, on a bounded sample of the workload, on all cores
    available to the process (the OpenMP build of the same source) and on one thread."""
    cores, model = host_cores()
    w_all, w_one = CPU_WINDOWS.get(name, (8, 2))
    one = oracle_timing(name, w_one, 1) if single_thread or cores == 1 else None
    res = oracle_timing(name, w_all, cores) if cores > 1 else dict(one)
    res["cpu_model"] = model
    res["cores_available"] = cores
    if one is not None:
        res["single_thread"] = {k: one[k] for k in ("value", "sample", "seconds", "units")}
    return res


def run_reference(args, rank, world):
    if rank != 0:
        return
    if args.workload == "springs":
        w = springs_workload()
        T = args.T or w["T"]
        times, cb = [], None
        for i in range(args.warmup + args.steps):
            r = springs_cpu_baseline(w, T, k=1024)
            if i >= args.warmup:
                times.append(r["seconds"])
                cb = r
        ms_ = 1e3 * sum(times) / len(times)
        value = cb["units"] / (ms_ / 1e3)
        print(json.dumps({"impl": "reference", "metric": SPRINGS_METRIC, "value": value,
                          "unit": SPRINGS_UNIT, "n_gpus": world, "steps": args.steps,
                          "warmup": args.warmup, "ms_per_step": ms_, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "the mass-spring triangle batch (a sample of "
                                                 "1,024 systems per step)", "T": T},
                          "cpu_baseline": {**cb, "value": value},
                          "e2e": {"value": value, "unit": SPRINGS_UNIT, "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return
    import oracle  # noqa: F401
    name = args.workload
    _, N, T, descr = make_workload(name)
    times = []
    cb = None
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(name, single_thread=False)
        if i >= args.warmup:
            times.append(r["seconds"])
            cb = r
    ms = 1e3 * sum(times) / len(times)
    value = cb["units"] / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": descr, "particles": N, "T": T},
            "cpu_baseline": {**cb, "value": value},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


SPRINGS_METRIC = "mass-point-steps/s fwd+bwd (batched mass-spring, Section 2 example)"
SPRINGS_UNIT = "mass-point-steps/s"


def springs_workload(seed=0, S=1 << 20, T=256):
    """1,048,576 copies of the paper's 2D triangle (3 masses, 3 springs; masses at (0,0),
    (0,0.1), (0.1,0) jittered by U(+-0.005), rest lengths U(0.09, 0.15)), k = 100,
    alpha = 10, dt = 2e-3, 256 states, loss (area - 0.2)^2 per system."""
    from paper_1910_00935_gb300.scenes import uniform
    import numpy as np
    tri = np.array([[0.0, 0.0], [0.0, 0.1], [0.1, 0.0]])
    x0 = (tri.reshape(-1)[:, None] + (uniform(seed, 600, 6 * S).reshape(6, S) - 0.5) * 0.01)
    rest = 0.09 + 0.06 * uniform(seed, 601, 3 * S).reshape(3, S)
    return dict(S=S, T=T, x0=x0.astype(np.float32), rest=rest.astype(np.float32),
                springs=[(0, 1), (0, 2), (1, 2)], k=100.0, alpha=10.0, dt=2e-3, m=1.0)


def springs_digest():
    """Digest of the mass-spring kernels' source (csrc/mass_spring.cu)."""
    import hashlib
    path = os.path.join(ROOT, "paper_1910_00935_gb300", "csrc", "mass_spring.cu")
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def springs_traffic(kernel, T):
    """DRAM bytes per launch of `kernel` from profiles/ncu_springs.md when it was captured on
    these kernels, scaled from the captured run's states to T (the tape traffic grows with
    the states; the capture runs a shorter tape of the same systems); else None."""
    path = os.path.join(ROOT, "profiles", "ncu_springs.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    if f"source digest: {springs_digest()}" not in text:
        return None
    import re
    m = re.search(r"captured states: (\d+)", text)
    sec = text.split(f"## {kernel}")
    if not m or len(sec) < 2:
        return None
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    total = 0.0
    for metric in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
        row = [ln for ln in sec[1].splitlines() if ln.startswith(f"| `{metric}` |")]
        if not row:
            return None
        cells = [c.strip() for c in row[0].strip("|").split("|")]
        total += statistics.mean(float(c) for c in cells[1:-1]) * scale.get(cells[-1], float("nan"))
    return total * (T - 1) / (int(m.group(1)) - 1)


def springs_cpu_baseline(w, T, k=4096):
    """The FP64 oracle, as it stands, on the first k systems: forward, area loss, backward
    (1 host thread)."""
    import numpy as np
    import oracle
    n = 3
    t0 = time.perf_counter()
    x0h = w["x0"][:, :k].astype(np.float64)
    for sidx in range(k):
        X, _ = oracle.ms_forward(x0h[:, sidx].reshape(3, 2), np.zeros((3, 2)), w["springs"],
                                 w["rest"][:, sidx], w["k"], w["alpha"], w["dt"], w["m"], T)
        _, xb = oracle.ms_area_loss(X[-1], 0.2)
        oracle.ms_backward(X, w["springs"], w["rest"][:, sidx], w["k"], w["alpha"], w["dt"],
                           w["m"], xb, np.zeros((3, 2)))
    dt_cpu = time.perf_counter() - t0
    return {"value": k * n * (T - 1) / dt_cpu, "unit": SPRINGS_UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{k} of the systems x {T} states forward+backward", "seconds": round(dt_cpu, 3),
            "units": k * n * (T - 1)}


def run_springs(args, rank, world):
    """The mass-spring line: forward (records 256 states of 1,048,576 systems), the area
    loss and its gradient in torch, backward through the tape; inputs resident."""
    import numpy as np
    import torch
    from paper_1910_00935_gb300 import build as mbuild
    mbuild.build()
    from paper_1910_00935_gb300 import mass_spring as ms
    torch.cuda.set_device(0 if world == 1 else _env_int("LOCAL_RANK", 0))
    dev = torch.device("cuda", torch.cuda.current_device())
    w = springs_workload(seed=rank)
    S, T, n = w["S"], args.T or w["T"], 3
    sim = ms.MassSprings(2, n, w["springs"], S, w["k"], w["alpha"], w["dt"], w["m"], steps=T,
                         device=dev)
    host = {"x0": torch.as_tensor(w["x0"]).pin_memory(),
            "v0": torch.zeros(6, S).pin_memory(),
            "rest": torch.as_tensor(w["rest"]).pin_memory()}
    devin = {k: v.to(dev) for k, v in host.items()}
    out = {}

    def device_step():
        sim.forward(devin["x0"], devin["v0"], devin["rest"], T)
        xT, _ = sim.state()
        xT.requires_grad_(True)
        L = ms.triangle_area(xT)
        (gT,) = torch.autograd.grad(L.sum(), xT)
        gx, gv, gl = sim.backward(gT, None)
        out.update(loss=L.detach(), grest=gl, gx0=gx)

    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        device_step()
    sim.sync()
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    torch.cuda.synchronize()
    for e0, e1 in evs:
        flush.fill_(1)
        e0.record(stream)
        device_step()
        e1.record(stream)
    torch.cuda.synchronize()
    ms_step = sum(e0.elapsed_time(e1) for e0, e1 in evs) / args.steps
    clk = clocks.stop() if clocks else None
    units = S * n * (T - 1)
    value = world * units / (ms_step / 1e3)
    # each pass alone (one kernel each): forward writes every state, backward reads the positions
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    flush.fill_(1)
    ev[0].record(stream)
    sim.forward(devin["x0"], devin["v0"], devin["rest"], T)
    ev[1].record(stream)
    gT = torch.ones(6, S, device=dev)
    flush.fill_(1)
    torch.cuda.synchronize()
    ev[1].record(stream)
    sim.backward(gT, None)
    ev[2].record(stream)
    torch.cuda.synchronize()
    f_ms, b_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    rows = n * 2
    fwd_bytes = S * 4 * (2 * rows * T + 2 * rows + 3)      # states written, x0 v0 rest read
    bwd_bytes = S * 4 * (rows * (T - 1) + 2 * rows + 3)    # positions read, seeds, outputs
    hbm, peak_src = measured_peaks()
    dom, dom_ms, dom_bytes = ("ms_backward", b_ms, bwd_bytes) if b_ms >= f_ms else ("ms_forward", f_ms, fwd_bytes)
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": springs_traffic(dom, T), "kernel": dom,
            "alg_bytes_per_launch": dom_bytes, "avg_launch_ms": dom_ms,
            "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
            else "fallback 6.8 TB/s",
            "forward_ms": f_ms, "backward_ms": b_ms}
    # e2e: host arrays in, loss and dL/drest out
    e2e = None
    if not args.no_e2e:
        out_host = {"loss": torch.empty(S).pin_memory(), "grest": torch.empty(3, S).pin_memory()}

        def e2e_step():
            for k, v in host.items():
                devin[k].copy_(v, non_blocking=True)
            device_step()
            out_host["loss"].copy_(out["loss"], non_blocking=True)
            out_host["grest"].copy_(out["grest"], non_blocking=True)
            torch.cuda.synchronize()

        e2e_step()
        times = []
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step()
            times.append(time.perf_counter() - t0)
        e_ms = 1e3 * sum(times) / len(times)
        e2e = {"value": world * units / (e_ms / 1e3), "unit": SPRINGS_UNIT, "ms_per_step": e_ms,
               "h2d_bytes_per_step": int(sum(v.numel() * 4 for v in host.values())),
               "d2h_bytes_per_step": int(sum(v.numel() * 4 for v in out_host.values()))}
    cb = springs_cpu_baseline(w, T) if rank == 0 and not args.no_cpu_baseline else None
    sim.sync()
    if rank == 0:
        line = {"metric": SPRINGS_METRIC, "value": value, "unit": SPRINGS_UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": f"1,048,576 copies of the paper's 2D mass-spring triangle "
                                       f"(3 masses, 3 springs), k=100, alpha=10, dt=2e-3, {T} states, "
                                       "area loss", "systems": S, "T": T,
                           "l2": "flushed between timed iterations (512 MiB write)",
                           "parallelism": "1 GPU" if world == 1 else f"{world} replicas"},
                "e2e": e2e, "gpu_launches": 2 * args.steps, "roofline": roof, "cpu_baseline": cb,
                "clocks": clk}
        print(json.dumps(line), flush=True)
    sim.close()


def flop_per_particle(workload, category, precision="FP64"):
    """FP64 (or FP32) FLOP per particle of one launch of `category` (2 per fused multiply-add,
    1 per add or multiply), from profiles/fp64_<category>_<workload>.md when that summary was
    taken on these kernels (same source digest); else None."""
    path = os.path.join(ROOT, "profiles", f"fp64_{category}_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    if f"source digest: {source_digest()}" not in text:
        return None
    import re
    m = re.search(precision + r" FLOP per particle: ([0-9.eE+-]+)", text)
    return float(m.group(1)) if m else None


def fp64_roofline(mpm, workload, category, n_launch, cat_ms, particles_per_launch):
    """Achieved FP64 FLOP/s of a kernel category against the GPU's FP64 FMA peak measured
    live with the library's own kernel (mpm_measure_peak), and the same for FP32 (the
    fixed-corotated passes' polar factor and adjoint left the FP64 pipe; their FP32
    arithmetic is the ALU share that remains)."""
    per = flop_per_particle(workload, category, "FP64")
    peak = mpm.mpm_measure_peak(mpm.MPM_PEAK_FP64_FMA)
    out = {"bound": "fp64", "peak": peak / 1e12, "unit": "TFLOP/s", "kernel": category,
           "peak_source": "measured live: mpm_measure_peak (FP64 FMA chains, CUDA events)"}
    if per is None or not n_launch:
        out.update(achieved=None, frac=None,
                   note="no FP64 FLOP count captured on these kernels (profiles/fp64_*.md)")
        return out
    avg_ms = cat_ms / n_launch
    achieved = per * particles_per_launch / (avg_ms / 1e3) / 1e12
    out.update(achieved=achieved, frac=achieved / out["peak"], flop_per_particle=per,
               avg_launch_ms=avg_ms)
    per32 = flop_per_particle(workload, category, "FP32")
    if per32 is not None:
        peak32 = mpm.mpm_measure_peak(mpm.MPM_PEAK_FP32_FMA) / 1e12
        a32 = per32 * particles_per_launch / (avg_ms / 1e3) / 1e12
        out["fp32"] = {"achieved": a32, "peak": peak32, "unit": "TFLOP/s", "frac": a32 / peak32,
                       "flop_per_particle": per32}
    return out


def scatter_roofline(mpm, prof, N, dim):
    """Grid reductions per second of the scattering passes against this GPU's float4
    reduction rate measured live (mpm_measure_peak): one float4 reduction per particle and
    stencil node (3^dim), the work that bounds these L2-resident passes rather than bytes.
    The recomputed P2G of a resident segment's adjoint passes is not counted."""
    red = mpm.mpm_measure_peak(mpm.MPM_PEAK_RED_F32X4)
    spread = mpm.mpm_measure_peak(mpm.MPM_PEAK_RED_F32X4_SPREAD)
    out = {"bound": "l2_reductions", "unit": "float4 reductions/s", "peak": red,
           "peak_spread": spread,
           "peak_source": "measured live: mpm_measure_peak (float4 reductions, 32 lanes on 32 "
                          "consecutive nodes; peak_spread: on 32 cache lines)",
           "reductions_per_particle": 3 ** dim, "kernels": {}}
    for cat in ("g2p_p2g", "g2p_p2g_full", "adj_fused"):
        if cat in prof and prof[cat][0]:
            n, ms = prof[cat]
            avg = ms / n
            ach = 3 ** dim * N / (avg / 1e3)
            out["kernels"][cat] = {"achieved": ach, "frac": ach / red, "frac_spread": ach / spread,
                                   "avg_launch_ms": avg}
    return out


def batched_line(name, dev, flush, steps=2, warmup=1, autotune_probe=True):
    """One batched configuration measured compactly for the headline's JSON line: forward and
    forward+backward particle-steps/s with inputs resident (L2 flushed between timed steps),
    the dominant kernel's roofline (HBM, and FP64 for the fixed-corotated passes), the same
    batch as one scene per launch sequence, the persistent launch form, and the autotuned
    knobs."""
    import torch
    from paper_1910_00935_gb300 import autotune, mpm
    from paper_1910_00935_gb300.sharding import subset
    scene, N, T, descr = make_workload(name)
    desc, a = scene["desc"], scene["arrays"]
    G = desc.get("n_groups", 0)
    S = len(desc["n_particles"])
    t = lambda k: torch.as_tensor(a[k]).to(dev)
    target = t("target")

    def run(sim):
        sim.forward(T)
        _, gT, _ = sim.loss(desc["loss_kind"], target)
        sim.backward(dL_dx=gT)

    def timed(fn, n):
        ms = []
        for _ in range(n):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return sum(ms) / len(ms)

    sim = mpm.from_scene(scene, max_steps=T, device=dev)
    for _ in range(warmup):
        run(sim)
    torch.cuda.synchronize()
    sim.check()
    ms = timed(lambda: run(sim), steps)
    fwd_ms = timed(lambda: sim.forward(T), 1)
    # per-kernel timing pass (CUDA events around every launch on its stream)
    sim.set_option(mpm.MPM_OPT_PROFILE, 1)
    flush.fill_(1)
    run(sim)
    torch.cuda.synchronize()
    prof = sim.profile()
    sim.set_option(mpm.MPM_OPT_PROFILE, 0)
    dom = max(prof, key=lambda k: prof[k][1])
    n_launch, dom_ms = prof[dom]
    step_bytes = pass_bytes(N, T, desc["ckpt_every"], desc["dim"],
                            kept=bool(sim.info(mpm.MPM_INFO_KEEPS_SEGMENT_GRIDS)))
    hbm, peak_src = measured_peaks()
    roof = None
    if dom in step_bytes and n_launch:
        avg = dom_ms / n_launch
        ach = step_bytes[dom] / n_launch / (avg / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": profiled_traffic(name, dom), "kernel": dom,
                "alg_bytes_per_launch": step_bytes[dom] / n_launch, "avg_launch_ms": avg,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)"}
    roof64 = None
    if desc["material"] in (mpm.MPM_FIXED_COROTATED, mpm.MPM_MIXED) and desc["dim"] == 3:
        roof64 = fp64_roofline(mpm, name, dom, n_launch, dom_ms, N)
    line = {"workload": descr, "particles": N, "scenes": S, "T": T,
            "value": N * T / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "forward": {"value": N * T / (fwd_ms / 1e3), "ms": fwd_ms},
            "roofline": roof, "roofline_fp64": roof64,
            "roofline_scatter": scatter_roofline(mpm, prof, N, desc["dim"]),
            "kernel_times_ms": {k: round(v[1], 3) for k, v in prof.items() if v[0]},
            "precision": precision_label(desc)}
    # the same batch through persistent launches (each run of same-kind passes one launch)
    sim.set_option(mpm.MPM_OPT_PERSISTENT, 1)
    run(sim)
    torch.cuda.synchronize()
    pms = timed(lambda: run(sim), steps)
    sim.set_option(mpm.MPM_OPT_PERSISTENT, 0)
    line["persistent"] = {"value": N * T / (pms / 1e3), "ms_per_step": pms}
    # autotuned knobs (coordinate descent over the library's options, short probes)
    if autotune_probe:
        cfg = autotune.tune(sim, T=min(T, 64), repeats=1, force=True)
        run(sim)
        torch.cuda.synchronize()
        ams = timed(lambda: run(sim), steps)
        line["autotuned"] = {"value": N * T / (ams / 1e3), "ms_per_step": ams, "config": cfg,
                             "refused": getattr(sim, "autotune_failed", [])}
    sim.check()
    sim.close()
    # one scene per launch sequence, scenes back to back
    sims = []
    for i in range(S):
        sub = subset(scene, [i])
        si = mpm.from_scene(sub, max_steps=T, device=dev)
        si._tgt = torch.as_tensor(sub["arrays"]["target"]).to(dev)
        sims.append(si)

    def per_scene():
        for si in sims:
            si.forward(T)
            _, gT, _ = si.loss(desc["loss_kind"], si._tgt)
            si.backward(dL_dx=gT)

    per_scene()
    torch.cuda.synchronize()
    sms = timed(per_scene, 1)
    for si in sims:
        si.check()
        si.close()
    line["one_scene_per_launch"] = {"value": N * T / (sms / 1e3), "ms_per_step": sms,
                                    "form": "one scene per launch sequence, back to back"}
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cube3d")
    ap.add_argument("--T", type=int, default=0, help="override the workload's step count")
    ap.add_argument("--ckpt-every", type=int, default=0, help="override the checkpoint interval")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--compare-per-scene", action="store_true",
                    help="also time the same batch one scene per launch sequence")
    ap.add_argument("--persistent", type=int, default=0,
                    help="1: run each run of same-kind passes as one persistent launch")
    ap.add_argument("--opt", action="append", default=[], metavar="MPM_OPT_NAME=VALUE",
                    help="set a library option (include/mpm.h) for the run; repeatable")
    ap.add_argument("--deterministic", action="store_true",
                    help="bitwise-reproducible fixed-point grid sums (deterministic_p2g = 1)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched configurations (rects2d, robots3d) that the default "
                         "cube3d line carries under 'batched'")
    ap.add_argument("--shard", action="store_true",
                    help="under torchrun: split the one batch's scenes across the ranks, "
                         "balanced by particle count (strong scaling; default: every rank "
                         "owns its own seeded batch, weak scaling)")
    args = ap.parse_args()

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local_rank = _env_int("LOCAL_RANK", 0)

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "springs":
        run_springs(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_1910_00935_gb300 import build as mbuild
    if rank == 0 or world == 1:
        mbuild.build()
    if world > 1:
        dist.init_process_group("nccl", rank=rank, world_size=world)
        torch.cuda.set_device(local_rank)
        dist.barrier()
        mbuild.build()
    else:
        torch.cuda.set_device(0)
    from paper_1910_00935_gb300 import mpm

    dev = torch.device("cuda", torch.cuda.current_device())
    shard = bool(args.shard and world > 1)
    if shard:
        # one batch, its scenes partitioned across the ranks by particle count; no data
        # crosses between ranks (the scenes are independent)
        from paper_1910_00935_gb300.sharding import shard_scenes, subset
        full, N_total, T, descr = make_workload(args.workload, seed=0)
        mine = shard_scenes(full["desc"]["n_particles"], world, rank)
        if not mine:
            raise RuntimeError(f"rank {rank} of {world} got no scene of {args.workload}")
        scene = subset(full, mine)
        N = int(sum(scene["desc"]["n_particles"]))
    else:
        # every rank simulates its own seeded batch: the job's batch is the union of the
        # ranks' batches, partitioned by rank (weak scaling)
        scene, N, T, descr = make_workload(args.workload, seed=rank)
        N_total = world * N
    if args.T:
        T = args.T
    if args.ckpt_every:
        scene["desc"]["ckpt_every"] = args.ckpt_every
    if args.deterministic:
        scene["desc"]["deterministic_p2g"] = 1
    desc = scene["desc"]
    a = scene["arrays"]
    G = desc.get("n_groups", 0)
    sim = mpm.Simulator(desc, T, device=dev)
    sim.set_option(mpm.MPM_OPT_PERSISTENT, args.persistent)
    options = {}
    for o in args.opt:
        k, v = o.split("=")
        sim.set_option(getattr(mpm, k), int(v))
        options[k] = int(v)
    names = ["x0", "v0", "C0", "F0", "E", "nu"]
    host = {k: torch.as_tensor(a[k]).pin_memory() for k in names + ["target"]}
    if G:
        host["group"] = torch.as_tensor(a["group"]).pin_memory()
        host["w"] = torch.as_tensor(a["w"]).pin_memory()
    devin = {k: v.to(dev) for k, v in host.items()}
    stream = torch.cuda.current_stream()

    if desc.get("material") == mpm.MPM_MIXED:
        devin["material"] = torch.as_tensor(a["material"]).to(dev)

    def device_step():
        mpm.mpm_set_initial(sim.h, devin["x0"], devin["v0"], devin["C0"], devin["F0"], devin["E"],
                            devin["nu"], devin.get("group"), devin.get("w"))
        if "material" in devin:
            mpm.mpm_set_particle_materials(sim.h, devin["material"])
        mpm.mpm_forward(sim.h, T)
        mpm.mpm_loss(sim.h, desc["loss_kind"], devin["target"], bufs["loss"], bufs["gT"], bufs["g0"])
        mpm.mpm_backward(sim.h, bufs["gT"], None, None, None, bufs["gx0"], bufs["gv0"], None, None,
                         bufs["gE"], bufs["gnu"], bufs["gw"] if G else None)

    d = desc["dim"]
    S = len(desc["n_particles"])
    bufs = {k: torch.empty(*shape, device=dev) for k, shape in
            (("loss", (S,)), ("gT", (d, N)), ("g0", (d, N)), ("gx0", (d, N)), ("gv0", (d, N)),
             ("gE", (N,)), ("gnu", (N,)), ("gw", (S, max(G, 1), max(desc.get("n_basis", 0), 1))))}

    # L2 flush buffer (larger than the 129 MB L2), written between timed iterations
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)

    for _ in range(args.warmup):
        device_step()
    torch.cuda.synchronize()
    rc = mpm.mpm_sync_status(sim.h)
    if rc != mpm.MPM_OK:
        raise RuntimeError(f"device error during warm-up: {mpm.mpm_last_error(sim.h)}")

    # ---- timed region: device-resident inputs ----
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
    launches0 = sim.info(mpm.MPM_INFO_KERNEL_LAUNCHES)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for e0, e1 in evs:
        flush.fill_(1)
        e0.record(stream)
        device_step()
        e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = sim.info(mpm.MPM_INFO_KERNEL_LAUNCHES) - launches0
    ms = sum(e0.elapsed_time(e1) for e0, e1 in evs) / args.steps
    clk = clocks.stop() if clocks else None
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = N_total * T / (ms / 1e3)

    # ---- forward-only throughput (same inputs, same stream) ----
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.fill_(1)
    mpm.mpm_set_initial(sim.h, devin["x0"], devin["v0"], devin["C0"], devin["F0"], devin["E"],
                        devin["nu"], devin.get("group"), devin.get("w"))
    if "material" in devin:
        mpm.mpm_set_particle_materials(sim.h, devin["material"])
    f0.record(stream)
    mpm.mpm_forward(sim.h, T)
    f1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = f0.elapsed_time(f1)

    # ---- e2e: host buffers through the public API, copies inside the timed region ----
    e2e = None
    if not args.no_e2e:
        out_host = {k: torch.empty_like(bufs[k], device="cpu").pin_memory()
                    for k in ("loss", "gv0", "gx0", "gE", "gnu", "gw")}
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        d2h = sum(v.numel() * v.element_size() for k, v in out_host.items() if G or k != "gw")

        def e2e_step():
            for k, v in host.items():
                devin[k].copy_(v, non_blocking=True)
            device_step()
            for k, v in out_host.items():
                if G or k != "gw":
                    v.copy_(bufs[k], non_blocking=True)
            torch.cuda.synchronize()

        e2e_step()
        times = []
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step()
            times.append(time.perf_counter() - t0)
        e_ms = 1e3 * sum(times) / len(times)
        if world > 1:
            t = torch.tensor([e_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e_ms = float(t.item())
        e2e = {"value": N_total * T / (e_ms / 1e3), "unit": UNIT, "ms_per_step": e_ms,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # ---- live per-kernel timing: CUDA events around every launch on its stream ----
    sim.set_option(mpm.MPM_OPT_PROFILE, 1)
    flush.fill_(1)
    device_step()
    torch.cuda.synchronize()
    prof = sim.profile()
    sim.set_option(mpm.MPM_OPT_PROFILE, 0)
    rc = mpm.mpm_sync_status(sim.h)
    if rc != mpm.MPM_OK:
        raise RuntimeError(f"device error: {mpm.mpm_last_error(sim.h)}")
    total_prof = sum(ms_ for _, ms_ in prof.values()) or 1.0
    dom = max(prof, key=lambda k: prof[k][1])
    n_launch, dom_ms = prof[dom]
    hbm, peak_src = measured_peaks()
    step_bytes = (pass_bytes_ctrl if desc.get("ctrl_hidden", 0) else pass_bytes)(
        N, T, desc["ckpt_every"], desc["dim"],
        kept=bool(sim.info(mpm.MPM_INFO_KEEPS_SEGMENT_GRIDS)))
    roof = None
    if dom in step_bytes and n_launch:
        avg_ms = dom_ms / n_launch
        alg_per_launch = step_bytes[dom] / n_launch
        achieved = alg_per_launch / (avg_ms / 1e3) / 1e9
        traffic = profiled_traffic(args.workload, dom)
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic, "kernel": dom,
                "alg_bytes_per_launch": alg_per_launch, "avg_launch_ms": avg_ms,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                else "fallback 6.8 TB/s",
                "share_of_step": dom_ms / total_prof}

    per_scene = None
    if args.compare_per_scene and len(desc["n_particles"]) > 1:
        from paper_1910_00935_gb300.sharding import subset
        sims = []
        for i in range(len(desc["n_particles"])):
            sub = subset(scene, [i])
            si = mpm.from_scene(sub, max_steps=T, device=dev)
            si._tgt = torch.as_tensor(sub["arrays"]["target"]).to(dev)
            sims.append(si)

        def per_scene_step():
            for si in sims:
                si.forward(T)
                L_, gT_, g0_ = si.loss(desc["loss_kind"], si._tgt)
                si.backward(dL_dx=gT_)

        per_scene_step()
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1)
        p0.record(stream)
        per_scene_step()
        p1.record(stream)
        torch.cuda.synchronize()
        pms = p0.elapsed_time(p1)
        per_scene = {"value": N * T / (pms / 1e3), "unit": UNIT, "ms_per_step": pms,
                     "form": "one scene per launch sequence, scenes run back to back"}
        for si in sims:
            si.close()

    # the job's loss: every rank's per-scene losses, gathered after the timed region (a
    # report, not part of the simulated path)
    losses = bufs["loss"].cpu().tolist()
    if world > 1:
        every = [None] * world
        dist.all_gather_object(every, losses)
        losses = [v for r in every for v in r]
    # the batched configurations of the same workload family (one GPU, default line only)
    batched = None
    if world == 1 and args.workload == "cube3d" and not args.no_batched and not args.T:
        sim.close()
        batched = {w: batched_line(w, dev, flush) for w in ("rects2d", "robots3d")}
    if rank != 0:
        return
    cb = None
    if world == 1 and not args.no_cpu_baseline:
        try:
            cb = cpu_baseline(args.workload)
        except Exception as e:  # the oracle needs gcc; report, never fake
            cb = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": str(e)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if shard else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": descr, "particles": N_total, "scenes": S if not shard else
                   len(full["desc"]["n_particles"]), "T": T,
                   "ckpt_every": desc["ckpt_every"], "grid": f"{desc['n_grid']}^{desc['dim']}",
                   "l2": "flushed between timed iterations (512 MiB write)",
                   "precision": precision_label(desc),
                   "parallelism": ("1 GPU" if world == 1 else
                                   f"dp{world}: the batch's scenes sharded by particle count"
                                   if shard else f"dp{world}: one seeded batch per rank"),
                   "launch_form": "persistent" if args.persistent else "one launch per pass",
                   "grid_sums": ("64-bit fixed point (deterministic)" if desc.get("deterministic_p2g")
                                 else "FP32 atomics"),
                   "options": options or "library defaults"},
        "forward": {"value": N * T / (fwd_ms / 1e3), "unit": UNIT, "ms": fwd_ms,
                    "scope": "rank 0's scenes"},
        "loss": {"sum": float(sum(losses)), "scenes": len(losses)},
        "one_scene_per_launch": per_scene,
        "batched": batched,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "roofline": roof,
        "roofline_scatter": scatter_roofline(mpm, prof, N, desc["dim"]),
        "kernel_times_ms": {k: round(v[1], 3) for k, v in prof.items() if v[0]},
        "cpu_baseline": cb,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
