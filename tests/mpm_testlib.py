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
    from paper_1910_00935_gb300.sharding import subset
    return subset(scene, idx)
