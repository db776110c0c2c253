"""Shared helpers of the GPU parity tests (no simulation arithmetic here)."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def to_np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def scene_slice(scene, i):
    off = np.concatenate([[0], np.cumsum(scene["desc"]["n_particles"])])
    return slice(int(off[i]), int(off[i + 1]))


def subset_scenes(scene, idx):
    """A batch made of some scenes of another batch (arrays sliced, desc updated)."""
    desc = dict(scene["desc"])
    a = scene["arrays"]
    sl = [scene_slice(scene, i) for i in idx]
    cat = lambda k, ax=1: np.ascontiguousarray(np.concatenate([a[k][..., s] for s in sl], axis=ax))
    arr = {k: cat(k) for k in ("x0", "v0", "C0", "F0")}
    arr["E"] = np.ascontiguousarray(np.concatenate([a["E"][s] for s in sl]))
    arr["nu"] = np.ascontiguousarray(np.concatenate([a["nu"][s] for s in sl]))
    arr["group"] = np.ascontiguousarray(np.concatenate([a["group"][s] for s in sl]))
    arr["w"] = np.ascontiguousarray(a["w"][list(idx)])
    arr["target"] = np.ascontiguousarray(a["target"][list(idx)])
    desc["n_particles"] = [int(scene["desc"]["n_particles"][i]) for i in idx]
    desc["n_scenes"] = len(idx)
    return {"desc": desc, "arrays": arr}
