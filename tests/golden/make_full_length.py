"""Write the FP64 expected values of the full-length parity tests (oracle only).

For each workload at its full size and step count this script runs the FP64 oracle
(`oracle/`) with the tape of Section 3.2 / Appendix D.2: the forward keeps the state every
k steps, the backward re-simulates each segment from its checkpoint and replays the step
adjoints of Appendix D.1 (`advance_grad`) in reverse.  Appendix D.2's segment invariance
holds bitwise in the oracle (pinned in tests/test_oracle_adjoint.py), so the gradients equal
those of one uncheckpointed reverse replay.  Two seeds are propagated on the same
re-simulation:

* the workload's own loss (the centre-of-mass loss of Section 3.2's compute_loss pattern:
  |COM_T - target|^2, or -(COM_x(T) - COM_x(0)) for the robots), whose dL/dx0 includes the
  loss's direct x0 term;
* a fixed random linear functional <a, state_T> (scenes.linear_functional), which exercises
  every adjoint term (the centre-of-mass loss alone leaves dL/dE at zero when no wall is
  touched, since internal forces conserve momentum).

Stored per workload (tests/golden/full_<name>.npz, FP32 unless noted): the final positions
x_T of every particle; v_T, C_T, F_T and every gradient block on a seeded sample of
particles (scenes.sample_indices); dL/dw in full; the losses and the full-array L2 norms
(FP64).  Only oracle/ and the input generator are called; nothing here comes from the CUDA
path.

    python tests/golden/make_full_length.py cube3d rects2d robots3d   # ~1 h on 8 cores
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1910_00935_gb300 import scenes  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

# workload -> (generator kwargs, scenes whose particles are compared, particles sampled
# per compared scene)
WORKLOADS = {
    "cube3d": (dict(), [0], 32768),
    "rects2d": (dict(), list(range(64)), 768),
    "robots3d": (dict(), [0, 9], 16384),
}
FUNCTIONAL_SEED = 0


def _scene(name):
    kw = WORKLOADS[name][0]
    return scenes.make(name, **kw)


def _one_scene(args):
    """Forward T steps with checkpoints every k, then the reverse replay of both seeds.
    Returns the per-scene results (FP64)."""
    name, si = args
    sc = scenes.oracle_view(_scene(name))
    desc, a = sc["desc"], sc["arrays"]
    d, T, k = desc["dim"], int(desc["steps"]), int(desc["ckpt_every"])
    off = np.concatenate([[0], np.cumsum(desc["n_particles"])]).astype(np.int64)
    sl = slice(int(off[si]), int(off[si + 1]))
    n = sl.stop - sl.start
    p = oracle.scene_params(sc, sl)
    mu, la = oracle.lame(a["E"][sl], a["nu"][sl])
    grp = a["group"][sl] if desc["n_groups"] else None
    w = a["w"][si] if desc["n_groups"] else None
    x0 = a["x0"][:, sl]

    t0 = time.time()
    state = [np.ascontiguousarray(a[key][:, sl]) for key in ("x0", "v0", "C0", "F0")]
    ckpt = {0: oracle.pack_state(*state)}
    for t in range(T):
        state = oracle.step(p, t, *state, mu, la, grp, w)
        if (t + 1) % k == 0 and t + 1 < T:
            ckpt[t + 1] = oracle.pack_state(*state)
    xT, vT, CT, FT = state
    tgt = a["target"][si] if "target" in a else None
    loss, xTb, x0b = oracle.com_loss(d, desc["loss_kind"], xT, x0, tgt)

    seeds_all = scenes.linear_functional(d, int(sum(desc["n_particles"])), FUNCTIONAL_SEED)
    adj = {
        "loss": oracle.pack_state(xTb, np.zeros((d, n)), np.zeros((d * d, n)),
                                  np.zeros((d * d, n))),
        "lin": oracle.pack_state(*[seeds_all[key][:, sl].astype(np.float64)
                                   for key in ("dL_dx", "dL_dv", "dL_dC", "dL_dF")]),
    }
    nw = oracle.n_act_params(p)
    acc = {s: dict(mub=np.zeros(n), lab=np.zeros(n), wb=np.zeros(nw)) for s in adj}
    t_fwd = time.time() - t0

    starts = sorted(ckpt)
    for s0 in reversed(starts):
        s1 = min(s0 + k, T)
        seg = [ckpt[s0]]
        st = oracle.unpack_state(ckpt[s0], d, n)
        st = [np.ascontiguousarray(q) for q in st]
        for t in range(s0, s1 - 1):
            st = oracle.step(p, t, *st, mu, la, grp, w)
            seg.append(oracle.pack_state(*st))
        for t in range(s1 - 1, s0 - 1, -1):
            for s in adj:
                adj[s], mub, lab, wb = oracle.step_adjoint(p, t, seg[t - s0], mu, la, adj[s],
                                                           grp, w)
                acc[s]["mub"] += mub
                acc[s]["lab"] += lab
                if nw:
                    acc[s]["wb"] += np.asarray(wb).reshape(-1)
        del seg
    out = dict(si=si, n=n, L=loss, xT=xT, vT=vT, CT=CT, FT=FT, t_fwd=t_fwd,
               t_all=time.time() - t0)
    for s in adj:
        gx, gv, gC, gF = oracle.unpack_state(adj[s], d, n)
        if s == "loss":
            gx = gx + x0b
        gE, gnu = oracle.lame_adjoint(a["E"][sl], a["nu"][sl], acc[s]["mub"], acc[s]["lab"])
        out[s] = dict(gx0=gx, gv0=gv, gC0=gC, gF0=gF, gE=gE, gnu=gnu,
                      gw=acc[s]["wb"].reshape(np.shape(w)) if nw else np.zeros(0))
    return out


def make(name, procs):
    kw, compared, m = WORKLOADS[name]
    sc = _scene(name)
    desc = sc["desc"]
    off = np.concatenate([[0], np.cumsum(desc["n_particles"])]).astype(np.int64)
    jobs = [(name, si) for si in compared]
    if procs > 1 and len(jobs) > 1:
        with mp.get_context("spawn").Pool(min(procs, len(jobs))) as pool:
            res = pool.map(_one_scene, jobs, chunksize=1)
    else:
        res = [_one_scene(j) for j in jobs]
    rec = dict(workload=np.array(name), T=np.int64(desc["steps"]),
               ckpt_every=np.int64(desc["ckpt_every"]),
               n_particles=np.asarray(desc["n_particles"], np.int64),
               compared_scenes=np.asarray(compared, np.int64),
               functional_seed=np.int64(FUNCTIONAL_SEED))
    losses, idx_all, xT_all = [], [], []
    blocks = {}
    norms = {}
    for r in res:
        si, n = r["si"], r["n"]
        idx = scenes.sample_indices(n, m, seed=si)
        idx_all.append(idx + off[si])
        losses.append(r["L"])
        xT_all.append(r["xT"])
        for key in ("vT", "CT", "FT"):
            blocks.setdefault(key, []).append(r[key][:, idx])
            norms.setdefault(key, []).append(np.linalg.norm(r[key]))
        for s in ("loss", "lin"):
            for g, v in r[s].items():
                if g == "gw":
                    blocks.setdefault(f"{s}_gw", []).append(v)
                    continue
                v2 = v if v.ndim == 2 else v[None, :]
                blocks.setdefault(f"{s}_{g}", []).append(v2[:, idx])
                norms.setdefault(f"{s}_{g}", []).append(np.linalg.norm(v))
        print(f"{name} scene {si}: n={n} forward {r['t_fwd']:.0f} s, all {r['t_all']:.0f} s",
              flush=True)
    rec["sample_index"] = np.concatenate(idx_all)
    rec["loss"] = np.asarray(losses, np.float64)
    rec["xT"] = np.concatenate(xT_all, axis=1).astype(np.float32)
    for key, v in blocks.items():
        if key.endswith("_gw"):
            rec[key] = np.stack(v).astype(np.float32)
        else:
            rec[key] = np.concatenate(v, axis=1).astype(np.float32)
    for key, v in norms.items():
        rec[f"norm_{key}"] = np.asarray(v, np.float64)
    path = os.path.join(HERE, f"full_{name}.npz")
    np.savez_compressed(path, **rec)
    print("wrote", path, os.path.getsize(path), "bytes", flush=True)


if __name__ == "__main__":
    names = sys.argv[1:] or list(WORKLOADS)
    oracle.build()
    procs = int(os.environ.get("GOLDEN_PROCS", str(os.cpu_count() or 1)))
    for nm in names:
        make(nm, procs)
