"""Seeded synthetic scenes for the differentiable MLS-MPM path.

This module only builds INPUTS (particle lattices, seeded noise, material parameters,
actuator groups, controller weights, loss targets).  It holds none of the method's
arithmetic (no weights, no stress, no Lame conversion) so that both the CUDA path and
the FP64 oracle can consume the exact same FP32 arrays.

Random numbers come from splitmix64 (Steele, Lea & Flood 2014): output i of a stream
is mix(state0 + (i + 1) * 0x9E3779B97F4A7C15) and a uniform double is the top 53 bits
times 2^-53.  Every stream is keyed by (seed, stream id).

The five workloads mirror the paper's soft-body experiments (Section 4.1, Fig. 7):
a 2D elastic square, its differentiable run, a 3D elastic cube, a batch of uneven 2D
scenes and a batch of 3D actuated robots.  All arrays are component-major
([component][particle]) and scenes of a batch are concatenated in particle order.
"""
from __future__ import annotations

import math

import numpy as np

FIXED_COROTATED, NEO_HOOKEAN, LIQUID, MIXED = 0, 1, 3, 4
LOSS_COM_TARGET, LOSS_COM_X_DISP = 0, 1

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from the splitmix64 stream keyed by (seed, stream)."""
    with np.errstate(over="ignore"):
        s0 = _mix(np.uint64((seed * 1000003 + stream) & 0xFFFFFFFFFFFFFFFF))
        states = s0 + _GOLDEN * np.arange(1, n + 1, dtype=np.uint64)
    z = _mix(states)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def lattice(dim, counts, corner, spacing):
    """Particle positions corner + (idx + 0.5) * spacing, row-major over idx."""
    axes = [np.arange(c, dtype=np.float64) for c in counts]
    grids = np.meshgrid(*axes, indexing="ij")
    pos = [corner[a] + (grids[a].reshape(-1) + 0.5) * spacing for a in range(dim)]
    return np.stack(pos), [g.reshape(-1).astype(np.int64) for g in grids]


def _identity(dim, n):
    F = np.zeros((dim * dim, n))
    for i in range(dim):
        F[i * dim + i] = 1.0
    return F


def _base_desc(**kw):
    desc = dict(dim=2, n_grid=128, dt=2e-4, gravity=(0.0, -9.8, 0.0), wall_cells=3,
                material=FIXED_COROTATED, rho=1.0, ckpt_every=32, n_groups=0, n_basis=0,
                act_period=50.0, act_phase=0.0, loss_kind=LOSS_COM_TARGET, steps=128)
    desc.update(kw)
    return desc


def _assemble(desc, parts):
    """parts: list of dicts with x0, v0, E, nu (+ group, w, target) per scene."""
    d = desc["dim"]
    n = [p["x0"].shape[1] for p in parts]
    desc = dict(desc, n_particles=[int(k) for k in n], n_scenes=len(parts))
    arr = {
        "x0": _f32(np.concatenate([p["x0"] for p in parts], axis=1)),
        "v0": _f32(np.concatenate([p["v0"] for p in parts], axis=1)),
        "C0": _f32(np.zeros((d * d, sum(n)))),
        "F0": _f32(_identity(d, sum(n))),
        "E": _f32(np.concatenate([p["E"] for p in parts])),
        "nu": _f32(np.concatenate([p["nu"] for p in parts])),
        "group": np.ascontiguousarray(np.concatenate(
            [p.get("group", np.zeros(k, np.int32)) for p, k in zip(parts, n)]).astype(np.int32)),
        "target": _f32(np.stack([p.get("target", np.zeros(d)) for p in parts])),
    }
    G, K = desc["n_groups"], desc["n_basis"]
    arr["w"] = _f32(np.stack([p.get("w", np.zeros((G, K))) for p in parts])
                    if G * K else np.zeros((len(parts), 0, 0)))
    return {"desc": desc, "arrays": arr}


def _noise(seed, stream, shape, half_width=0.05):
    n = int(np.prod(shape))
    return (uniform(seed, stream, n).reshape(shape) * 2.0 - 1.0) * half_width


def linear_functional(dim: int, n: int, seed: int = 0, c_scale: float = 1e-3):
    """Seeds of a fixed random linear functional L = <a, state_T> of the final state:
    U(-1, 1) weights on x, v and F and c_scale * U(-1, 1) on C (C is O(1/dt) larger).
    Returned as FP32 component-major arrays dL_dx[d, n], dL_dv, dL_dC[d^2, n], dL_dF."""
    f = lambda stream, rows, s=1.0: _f32((uniform(seed, stream, rows * n).reshape(rows, n)
                                          * 2.0 - 1.0) * s)
    return dict(dL_dx=f(900, dim), dL_dv=f(901, dim), dL_dC=f(902, dim * dim, c_scale),
                dL_dF=f(903, dim * dim))


def sample_indices(n: int, m: int, seed: int = 0) -> np.ndarray:
    """m distinct particle indices of [0, n), sorted, drawn with the splitmix64 stream
    (seed, 950): the particles a full-length comparison samples."""
    if m >= n:
        return np.arange(n, dtype=np.int64)
    return np.sort(np.argsort(uniform(seed, 950, n), kind="stable")[:m]).astype(np.int64)


def elastic_square_2d(seed=0, steps=128, n_side=64, ckpt_every=32):
    """2D square of n_side^2 particles (2 per cell per axis), side n_side/256,
    centred at (0.3, 0.5); fixed-corotated E=1e3, nu=0.2; v0 = (1, 0) + U(+-0.05)."""
    n_grid = 128
    h = 0.5 / n_grid
    side = n_side * h
    x0, _ = lattice(2, (n_side, n_side), (0.3 - side / 2, 0.5 - side / 2), h)
    n = x0.shape[1]
    v0 = np.array([[1.0], [0.0]]) + _noise(seed, 1, (2, n))
    desc = _base_desc(dim=2, n_grid=n_grid, dt=2e-4, steps=steps, ckpt_every=ckpt_every)
    return _assemble(desc, [dict(x0=x0, v0=v0, E=np.full(n, 1e3), nu=np.full(n, 0.2),
                                 target=np.array([0.7, 0.5]))])


def elastic_cube_3d(seed=0, steps=1024, n_side=64, n_grid=128, ckpt_every=64):
    """3D cube of n_side^3 particles (2 per cell per axis), side n_side/(2 n_grid),
    centred at (0.3, 0.5, 0.5); neo-Hookean E=5e3, nu=0.3; v0 = (1,0,0) + U(+-0.05);
    loss |COM_T - (0.7, 0.5, 0.5)|^2."""
    h = 0.5 / n_grid
    side = n_side * h
    x0, _ = lattice(3, (n_side,) * 3, (0.3 - side / 2, 0.5 - side / 2, 0.5 - side / 2), h)
    n = x0.shape[1]
    v0 = np.array([[1.0], [0.0], [0.0]]) + _noise(seed, 1, (3, n))
    desc = _base_desc(dim=3, n_grid=n_grid, dt=1e-4, material=NEO_HOOKEAN, steps=steps,
                      ckpt_every=ckpt_every)
    return _assemble(desc, [dict(x0=x0, v0=v0, E=np.full(n, 5e3), nu=np.full(n, 0.3),
                                 target=np.array([0.7, 0.5, 0.5]))])


def batched_rects_2d(seed=0, n_scenes=64, steps=512, n_min=1024, n_max=16384, ckpt_every=32):
    """n_scenes independent 2D rectangles: N log-uniform in [n_min, n_max] (2 particles
    per cell per axis), aspect U[0.5, 2], placed uniformly inside [0.15, 0.85]^2,
    E log-uniform in [5e2, 5e3] per scene, nu = 0.2, v0 = (1, 0) + U(+-0.05)."""
    n_grid = 128
    h = 0.5 / n_grid
    u = uniform(seed, 7, 5 * n_scenes).reshape(n_scenes, 5)
    parts = []
    for s in range(n_scenes):
        n_target = math.exp(math.log(n_min) + u[s, 0] * (math.log(n_max) - math.log(n_min)))
        aspect = 0.5 + 1.5 * u[s, 1]
        nx = max(1, int(round(math.sqrt(n_target * aspect))))
        ny = max(1, int(round(n_target / nx)))
        wx, wy = nx * h, ny * h
        cx = 0.15 + u[s, 2] * (0.7 - wx)
        cy = 0.15 + u[s, 3] * (0.7 - wy)
        x0, _ = lattice(2, (nx, ny), (cx, cy), h)
        n = x0.shape[1]
        v0 = np.array([[1.0], [0.0]]) + _noise(seed, 100 + s, (2, n))
        E = math.exp(math.log(5e2) + u[s, 4] * (math.log(5e3) - math.log(5e2)))
        parts.append(dict(x0=x0, v0=v0, E=np.full(n, E), nu=np.full(n, 0.2),
                          target=np.array([0.7, 0.5])))
    desc = _base_desc(dim=2, n_grid=n_grid, dt=1e-4, steps=steps, ckpt_every=ckpt_every)
    return _assemble(desc, parts)


def actuated_robots_3d(seed=0, n_scenes=16, steps=2048, dims=(64, 32, 32), n_grid=64,
                       ckpt_every=64, n_basis=4, bottom_dx=4.0):
    """n_scenes 3D box robots of dims[0]*dims[1]*dims[2] particles at spacing dx/2,
    bottom at y = bottom_dx * dx (4 dx), x from 0.1, centred in z; 8 actuator groups (octants: bit0
    x-half, bit1 y-half, bit2 z-half; fibre axis g mod 3); w ~ U(-50, 50) per scene;
    fixed-corotated E=5e3, nu=0.3; v0 = U(+-0.05); loss -(COM_x(T) - COM_x(0))."""
    dx = 1.0 / n_grid
    h = 0.5 * dx
    corner = (0.1, bottom_dx * dx, 0.5 - dims[2] * h / 2)
    parts = []
    for s in range(n_scenes):
        x0, idx = lattice(3, dims, corner, h)
        n = x0.shape[1]
        grp = ((idx[0] >= dims[0] // 2).astype(np.int32)
               | ((idx[1] >= dims[1] // 2).astype(np.int32) << 1)
               | ((idx[2] >= dims[2] // 2).astype(np.int32) << 2))
        v0 = _noise(seed, 200 + s, (3, n))
        w = (uniform(seed, 300 + s, 8 * n_basis).reshape(8, n_basis) * 2.0 - 1.0) * 50.0
        parts.append(dict(x0=x0, v0=v0, E=np.full(n, 5e3), nu=np.full(n, 0.3), group=grp, w=w))
    desc = _base_desc(dim=3, n_grid=n_grid, dt=1e-4, steps=steps, ckpt_every=ckpt_every,
                      n_groups=8, n_basis=n_basis, act_period=50.0, act_phase=0.0,
                      loss_kind=LOSS_COM_X_DISP)
    return _assemble(desc, parts)


def controller_params(seed, stream, dim, n_groups, n_basis, hidden, sensor_gain=10.0):
    """Seeded controller parameters theta = [W1 | b1 | W2 | b2] (the layout of
    mpm_scene_desc.ctrl_hidden): uniform with variance 1/fan_in per layer, the columns of W1
    that read the sensors (centre offsets, mean velocities) scaled by sensor_gain, biases
    zero."""
    n_in = n_basis + 2 * dim * n_groups
    u = uniform(seed, stream, hidden * n_in + n_groups * hidden) * 2.0 - 1.0
    W1 = u[:hidden * n_in].reshape(hidden, n_in) * np.sqrt(3.0 / n_in)
    W1[:, n_basis:] *= sensor_gain
    W2 = u[hidden * n_in:].reshape(n_groups, hidden) * np.sqrt(3.0 / hidden)
    return np.concatenate([W1.reshape(-1), np.zeros(hidden), W2.reshape(-1), np.zeros(n_groups)])


def controlled_robots_3d(seed=0, n_scenes=4, steps=512, dims=(48, 24, 24), n_grid=64,
                         ckpt_every=64, n_basis=4, hidden=32, scale=50.0, sensor_gain=10.0,
                         material=FIXED_COROTATED, bottom_dx=4.0):
    """Closed-loop robots (the neural-network controllers of Section 4.1): n_scenes 3D box
    robots of dims particles (48 x 24 x 24 = 27,648, about the paper's 30K-particle 3D
    robot) at spacing dx/2 on the floor, 8 octant actuator groups (fibre axis g mod 3), each
    driven at every step by its own controller: inputs sin(2 pi k t / 50), k = 1..n_basis,
    and per group the centre-of-mass offset and mean velocity; hidden tanh layer of `hidden`
    units; outputs scale * tanh(.).  E = 5e3, nu = 0.3; v0 = U(+-0.05); loss
    -(COM_x(T) - COM_x(0)).  The bottom sits at y = bottom_dx * dx (at 3 dx its lowest
    particles reach the sticky floor from the first step)."""
    dx = 1.0 / n_grid
    h = 0.5 * dx
    corner = (0.1, bottom_dx * dx, 0.5 - dims[2] * h / 2)
    parts = []
    for s in range(n_scenes):
        x0, idx = lattice(3, dims, corner, h)
        n = x0.shape[1]
        grp = ((idx[0] >= dims[0] // 2).astype(np.int32)
               | ((idx[1] >= dims[1] // 2).astype(np.int32) << 1)
               | ((idx[2] >= dims[2] // 2).astype(np.int32) << 2))
        v0 = _noise(seed, 400 + s, (3, n))
        th = controller_params(seed, 500 + s, 3, 8, n_basis, hidden, sensor_gain)
        parts.append(dict(x0=x0, v0=v0, E=np.full(n, 5e3), nu=np.full(n, 0.3), group=grp, w=th))
    desc = _base_desc(dim=3, n_grid=n_grid, dt=1e-4, steps=steps, ckpt_every=ckpt_every,
                      material=material, n_groups=8, n_basis=n_basis, act_period=50.0,
                      act_phase=0.0, loss_kind=LOSS_COM_X_DISP, ctrl_hidden=hidden,
                      ctrl_scale=scale)
    return _assemble(desc, parts)


def liquid_column(seed=0, dim=3, steps=256, n_grid=64, cols=(32, 48, 32), E=500.0, nu=0.3,
                  ckpt_every=32):
    """Dam break: a column of weakly compressible liquid (cols particles per axis, 2 per
    cell per axis) standing in the low-x corner on the sticky floor, released at t = 0;
    v0 = U(+-0.05); bulk modulus from E, nu (E = 500, nu = 0.3: kappa = 417 in 3D, sound
    speed sqrt(7 kappa / rho) = 54 within the dt = 1e-4, dx = 1/64 stability limit);
    loss |COM_T - target|^2 with the target downstream on the floor."""
    h = 0.5 / n_grid
    cols = tuple(cols[:dim])
    lo = [0.1, 4.0 / n_grid] + ([0.5 - cols[2] * h / 2] if dim == 3 else [])
    x0, _ = lattice(dim, cols, tuple(lo), h)
    n = x0.shape[1]
    v0 = _noise(seed, 1, (dim, n))
    desc = _base_desc(dim=dim, n_grid=n_grid, dt=1e-4, material=LIQUID, steps=steps,
                      ckpt_every=ckpt_every)
    target = np.array([0.4, 0.1, 0.5][:dim])
    return _assemble(desc, [dict(x0=x0, v0=v0, E=np.full(n, E), nu=np.full(n, nu), target=target)])


def robot_in_liquid(seed=0, steps=256, n_grid=64, robot=(32, 16, 16), pool=(96, 12, 48),
                    ckpt_every=32, w_scale=50.0):
    """Two-way coupling in one grid (the paper's robot-in-liquid experiment): an actuated
    fixed-corotated robot (robot particles per axis, 8 octant groups, 4 sine terms, w ~
    U(+-w_scale)) standing in a shallow pool of weakly compressible liquid (pool particles
    per axis, 2 per cell per axis, on the sticky floor).  Robot E = 5e3, nu = 0.3; liquid
    E = 500, nu = 0.3.  Per-particle materials (MIXED); loss -(COM_x(T) - COM_x(0)) of the
    whole scene.  The robot stands on the floor beside the pool's far end."""
    h = 0.5 / n_grid
    floor = 4.0 / n_grid
    px0 = 0.1
    xl, _ = lattice(3, pool, (px0, floor, 0.5 - pool[2] * h / 2), h)
    rx0 = px0 + 2 * h
    xr, _ = lattice(3, robot, (rx0, floor + pool[1] * h * 0.5, 0.5 - robot[2] * h / 2), h)
    nr, nl = xr.shape[1], xl.shape[1]
    x0 = np.concatenate([xr, xl], axis=1)
    n = nr + nl
    v0 = _noise(seed, 1, (3, n))
    rel = (xr - xr.min(1, keepdims=True)) / (xr.max(1, keepdims=True) - xr.min(1, keepdims=True))
    bits = (rel > 0.5).astype(np.int32)
    group = np.concatenate([bits[0] + 2 * bits[1] + 4 * bits[2], np.full(nl, -1, np.int32)])
    G, K = 8, 4
    w = (uniform(seed, 2, G * K).reshape(G, K) * 2.0 - 1.0) * w_scale
    E = np.concatenate([np.full(nr, 5e3), np.full(nl, 500.0)])
    desc = _base_desc(dim=3, n_grid=n_grid, dt=1e-4, material=MIXED, steps=steps,
                      ckpt_every=ckpt_every, n_groups=G, n_basis=K, loss_kind=LOSS_COM_X_DISP)
    scene = _assemble(desc, [dict(x0=x0, v0=v0, E=E, nu=np.full(n, 0.3), group=group, w=w)])
    scene["arrays"]["material"] = np.ascontiguousarray(
        np.concatenate([np.full(nr, FIXED_COROTATED), np.full(nl, LIQUID)]).astype(np.int32))
    return scene


def make(name: str, seed: int = 0, **kw):
    """Named workloads: 'square2d', 'square2d_grad', 'cube3d', 'rects2d', 'robots3d',
    'liquid2d', 'liquid3d', 'robot_in_liquid', 'robots_nn'."""
    if name == "robots_nn":
        return controlled_robots_3d(seed, **kw)
    if name == "liquid2d":
        return liquid_column(seed, **{"dim": 2, "n_grid": 128, "cols": (64, 96), **kw})
    if name == "liquid3d":
        return liquid_column(seed, **{"dim": 3, **kw})
    if name == "robot_in_liquid":
        return robot_in_liquid(seed, **kw)
    if name == "square2d":
        return elastic_square_2d(seed, **{"steps": 128, **kw})
    if name == "square2d_grad":
        return elastic_square_2d(seed, **{"steps": 512, "ckpt_every": 32, **kw})
    if name == "cube3d":
        return elastic_cube_3d(seed, **kw)
    if name == "rects2d":
        return batched_rects_2d(seed, **kw)
    if name == "robots3d":
        return actuated_robots_3d(seed, **kw)
    raise KeyError(name)


def oracle_view(scene):
    """The same scene with every float array promoted to float64 (exactly)."""
    arr = {k: (v.astype(np.float64) if v.dtype == np.float32 else v)
           for k, v in scene["arrays"].items()}
    return {"desc": scene["desc"], "arrays": arr}
