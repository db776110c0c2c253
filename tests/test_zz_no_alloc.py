"""mpm_step_noalloc: one forward step with no workspace, for callers that cannot allocate
device memory (code inside a host application that owns the device memory budget and
forbids allocation after start-up, or a small C caller without an allocator).  Its grid
scratch is a fixed array inside the library, shared by every call on a device.

The GPU test calls it through the C ABI several times in a row, on problems of different
sizes, and checks each result against the workspace path (mpm_create, mpm_set_initial,
mpm_forward with T = 1, mpm_get_state) at the one-step tolerance of the parity tests.
A stale grid left by the previous call would show up as a mismatch."""
import numpy as np
import pytest

from mpm_testlib import rel_l2, to_np
from paper_1910_00935_gb300 import scenes

torch = pytest.importorskip("torch")

# one-step bars of the parity tests: x and F at 1e-5; v (a difference of positions) at 10x
# and C (a velocity gradient) at 100x, as in tests/test_gpu_parity.py
STEP_TOL = 1e-5
FIELD_TOL = {"x": STEP_TOL, "F": STEP_TOL, "v": 10 * STEP_TOL, "C": 100 * STEP_TOL}


@pytest.fixture(scope="module")
def mpm():
    from paper_1910_00935_gb300 import build, mpm as m
    build.build()
    return m


def _state_block(scene):
    a = scene["arrays"]
    return np.ascontiguousarray(np.concatenate([a["x0"], a["v0"], a["C0"], a["F0"]], axis=0))


def _workspace_step(mpm, scene):
    sim = mpm.from_scene(scene, max_steps=1)
    sim.forward(1)
    x, v, C, F = sim.state()
    assert mpm.mpm_sync_status(sim.h) == mpm.MPM_OK
    sim.close()
    return np.concatenate([to_np(t) for t in (x, v, C, F)], axis=0)


def _noalloc_step(mpm, scene, device_err):
    desc = mpm.make_desc(scene["desc"])
    state_in = torch.as_tensor(_state_block(scene)).cuda()
    state_out = torch.full_like(state_in, float("nan"))
    E = torch.as_tensor(scene["arrays"]["E"]).cuda()
    nu = torch.as_tensor(scene["arrays"]["nu"]).cuda()
    rc = mpm.mpm_step_noalloc(desc, state_in, E, nu, state_out, device_err)
    torch.cuda.synchronize()
    return rc, to_np(state_out)


def _compare(out, ref, dim):
    rows = {"x": (0, dim), "v": (dim, 2 * dim), "C": (2 * dim, 2 * dim + dim * dim),
            "F": (2 * dim + dim * dim, 2 * dim + 2 * dim * dim)}
    for name, (a, b) in rows.items():
        r = rel_l2(out[a:b], ref[a:b])
        assert r <= FIELD_TOL[name], (name, r)


@pytest.mark.gpu
def test_noalloc_step_matches_workspace_path_calls_in_a_row(mpm):
    # the documented start-up call: no particles, only the set-up (nothing read or written)
    warm = dict(scenes.make("cube3d", n_side=24, n_grid=64)["desc"], n_particles=[0])
    assert mpm.mpm_step_noalloc(mpm.make_desc(warm), 256, 256, 256, 512, None) == mpm.MPM_OK
    device_err = torch.zeros(1, dtype=torch.int32, device="cuda")
    cube = scenes.make("cube3d", n_side=24, n_grid=64)   # 13,824 particles, 64^3 nodes (the limit)
    square = scenes.make("square2d")                     # 4,096 particles, 128^2 nodes
    first = None
    for scene in (cube, square, cube):
        ref = _workspace_step(mpm, scene)
        rc, out = _noalloc_step(mpm, scene, device_err)
        assert rc == mpm.MPM_OK
        _compare(out, ref, scene["desc"]["dim"])
        if scene is cube:
            if first is None:
                first = out
            else:  # the repeat sees the array as the 2D call left it
                _compare(out, first, scene["desc"]["dim"])
    assert int(device_err.item()) == 0


def test_noalloc_rejects_problems_beyond_its_scratch(mpm):
    """Size checks run on the host before any CUDA call (no GPU needed); each rejection
    leaves its reason where mpm_last_error(NULL) reads it."""
    big_grid = dict(scenes.make("cube3d", n_side=8, n_grid=128)["desc"])  # 128^3 > 2^18 nodes
    assert mpm.mpm_step_noalloc(mpm.make_desc(big_grid), 256, 256, 256, 512, None, 0) == \
        mpm.MPM_ERR_TOO_LARGE
    assert "MPM_NOALLOC_MAX_NODES" in mpm.mpm_last_error(None)
    many = dict(big_grid, n_grid=64, n_particles=[mpm.MPM_NOALLOC_MAX_PARTICLES + 1])
    assert mpm.mpm_step_noalloc(mpm.make_desc(many), 256, 256, 256, 512, None, 0) == \
        mpm.MPM_ERR_TOO_LARGE
    two = dict(big_grid, n_grid=64, n_particles=[100, 100])
    assert mpm.mpm_step_noalloc(mpm.make_desc(two), 256, 256, 256, 512, None, 0) == mpm.MPM_ERR_ARG
    assert "one scene" in mpm.mpm_last_error(None)
    act = dict(big_grid, n_grid=64, n_groups=2, n_basis=1)
    assert mpm.mpm_step_noalloc(mpm.make_desc(act), 256, 256, 256, 512, None, 0) == mpm.MPM_ERR_ARG
    det = dict(big_grid, n_grid=64, deterministic_p2g=1)
    assert mpm.mpm_step_noalloc(mpm.make_desc(det), 256, 256, 256, 512, None, 0) == mpm.MPM_ERR_ARG


@pytest.mark.gpu
def test_noalloc_liquid_and_error_word(mpm):
    """The liquid material through the entry point, a call whose error bits go to the fixed
    array (device_err NULL), and a particle placed where its stencil leaves the grid: the
    kernels' own bounds check skips it and sets bit 1 of the caller's error word."""
    liquid = scenes.make("liquid3d", cols=(16, 20, 16), n_grid=64)
    ref = _workspace_step(mpm, liquid)
    rc, out = _noalloc_step(mpm, liquid, None)
    assert rc == mpm.MPM_OK
    _compare(out, ref, 3)

    square = scenes.make("square2d")
    bad = {"desc": square["desc"], "arrays": dict(square["arrays"])}
    x0 = bad["arrays"]["x0"].copy()
    x0[0, 5] = 0.2 / square["desc"]["n_grid"]  # x/dx = 0.2: stencil base -1, off the grid
    bad["arrays"]["x0"] = x0
    device_err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc, out = _noalloc_step(mpm, bad, device_err)
    assert rc == mpm.MPM_OK
    assert int(device_err.item()) & 1
    assert np.isfinite(out).all()
