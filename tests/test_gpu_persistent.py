"""The persistent form (MPM_OPT_PERSISTENT): each run of same-kind passes is one
cooperative launch that steps through the recorded pass plan with a bounded grid-wide
barrier between passes.  It must give the oracle's results (same bars as the
one-launch-per-pass form), agree with that form to FP32 atomic-order rounding, replace
thousands of launches by a handful, and report a barrier wait that runs out as
MPM_ERR_TIMEOUT without faulting or hanging (the wait is made to run out on purpose by
the test hook that adds arrivals no CTA will ever make).
"""
import time

import numpy as np
import pytest

from mpm_testlib import rel_l2
from paper_1910_00935_gb300 import scenes
from test_gpu_parity import (GRAD_TOL, POS_TOL, _compare_grads, _compare_states, _oracle_grad_linear,
                             _oracle_states, _random_seeds, _run_gpu)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpm():
    from paper_1910_00935_gb300 import build, mpm as m
    build.build()
    return m


CASES = [
    # uneven 2D batch (5 scenes, ragged tiles), segments 7 + ... + ragged last one
    ("rects2d", dict(n_scenes=5, n_min=300, n_max=2000), 24, 7),
    ("cube3d", dict(n_side=16, n_grid=64), 12, 5),
    # fixed-corotated 3D with actuation: polar cache and w-bar reduction inside the plan
    ("robots3d", dict(n_scenes=2, dims=(16, 8, 8)), 12, 5),
]


@pytest.mark.parametrize("name,kw,T,k", CASES)
@pytest.mark.parametrize("graphs", [1, 0])
def test_persistent_matches_oracle_and_per_pass_form(mpm, name, kw, T, k, graphs):
    scene = scenes.make(name, **kw)
    scene["desc"]["ckpt_every"] = k
    seeds = _random_seeds(scene, np.random.default_rng(11))
    per_pass = _run_gpu(mpm, scene, T, seeds=seeds, loss=False,
                        options={mpm.MPM_OPT_USE_GRAPHS: graphs})
    pers = _run_gpu(mpm, scene, T, seeds=seeds, loss=False,
                    options={mpm.MPM_OPT_USE_GRAPHS: graphs, mpm.MPM_OPT_PERSISTENT: 1})
    _compare_states(pers["state"], _oracle_states(scene, T), scene, POS_TOL)
    o = _oracle_grad_linear(scene, T, {kk: v.astype(np.float64) for kk, v in seeds.items()})
    keys = ["gx0", "gv0", "gC0", "gF0", "gE", "gnu"] + (["gw"] if scene["desc"]["n_groups"] else [])
    _compare_grads(pers["grad"], o, keys)
    # x and F to FP32 atomic-order rounding; v and C (differences of nearby grid values) with
    # the same 10x / 100x relaxation as their oracle bars
    for i, tol in enumerate((1e-5, 1e-4, 1e-3, 1e-5)):
        assert rel_l2(pers["state"][i], per_pass["state"][i]) <= tol, (i, rel_l2(pers["state"][i], per_pass["state"][i]))
    for key in keys:
        assert rel_l2(pers["grad"][key], per_pass["grad"][key]) <= 1e-4, key


def test_persistent_launch_counts(mpm):
    """Each run of passes of one kind and one pass mode is one persistent launch.  Forward:
    three (the first P2G, the G2P+P2G steps, the last G2P) plus the end-of-sequence clears
    and box reset; backward: at most six per segment (re-simulation and adjoint, each with
    its first, middle and last pass modes) plus the same clean-up and the gradient I/O
    kernels."""
    scene = scenes.make("cube3d", n_side=16, n_grid=64)
    T, k = 12, 5
    scene["desc"]["ckpt_every"] = k
    counts = {}
    for persistent in (0, 1):
        sim = mpm.from_scene(scene, max_steps=T)
        sim.set_option(mpm.MPM_OPT_USE_GRAPHS, 0)
        sim.set_option(mpm.MPM_OPT_PERSISTENT, persistent)
        n0 = sim.info(mpm.MPM_INFO_KERNEL_LAUNCHES)
        sim.forward(T)
        n1 = sim.info(mpm.MPM_INFO_KERNEL_LAUNCHES)
        sim.backward(dL_dx=torch.ones(3, sim.N, device="cuda"))
        n2 = sim.info(mpm.MPM_INFO_KERNEL_LAUNCHES)
        assert mpm.mpm_sync_status(sim.h) == mpm.MPM_OK
        counts[persistent] = (n1 - n0, n2 - n1)
        sim.close()
    n_seg = -(-T // k)
    s_last = ((T - 1) // k) * k  # the forward leaves the last segment resident
    fwd_pp, bwd_pp = counts[0]
    fwd_p, bwd_p = counts[1]
    # per-pass backward: re-simulation of the other segments, one P2G for the grid of
    # step T-1, T + 1 adjoint passes; the rest is clean-up and gradient I/O
    passes = (s_last + n_seg - 1) + 1 + (T + 1)
    assert fwd_pp >= T + 1 and bwd_pp >= passes, counts
    assert fwd_p <= 3 + 5, counts
    assert bwd_p <= 6 * n_seg + (bwd_pp - passes) + 1, counts


def test_persistent_repeated_runs_reuse_the_plan(mpm):
    """Same T twice, then a different T, then the first again: the plan regions are
    refreshed only when the plan changes, and every run matches the oracle."""
    scene = scenes.make("square2d", n_side=40)
    sim = mpm.from_scene(scene, max_steps=40)
    sim.set_option(mpm.MPM_OPT_PERSISTENT, 1)
    for T in (16, 16, 40, 16):
        sim.forward(T)
        got = [a.cpu().numpy() for a in sim.state()]
        assert mpm.mpm_sync_status(sim.h) == mpm.MPM_OK
        _compare_states(got, _oracle_states(scene, T), scene, POS_TOL)
    sim.close()


def test_barrier_timeout_is_reported_and_the_handle_recovers(mpm):
    scene = scenes.make("square2d", n_side=32)  # 1,024 particles: 4 tiles, 4 CTAs
    T = 6
    sim = mpm.from_scene(scene, max_steps=T)
    sim.set_option(mpm.MPM_OPT_PERSISTENT, 1)
    sim.set_option(mpm.MPM_OPT_BARRIER_TIMEOUT_US, 20000)
    sim.set_option(mpm.MPM_OPT_BARRIER_TEST_EXTRA, 1)  # an arrival that never comes
    t0 = time.perf_counter()
    sim.forward(T)
    rc = mpm.mpm_sync_status(sim.h)
    elapsed = time.perf_counter() - t0
    assert rc == mpm.MPM_ERR_TIMEOUT, (rc, mpm.mpm_last_error(sim.h))
    assert elapsed < 10.0
    # the context is still usable; the handle wants a fresh initial state first
    with pytest.raises(mpm.MPMError) as ei:
        sim.forward(T)
    assert ei.value.code == mpm.MPM_ERR_STATE
    sim.set_option(mpm.MPM_OPT_BARRIER_TEST_EXTRA, 0)
    a = scene["arrays"]
    t = lambda key: torch.as_tensor(a[key])
    sim.set_initial(t("x0"), t("v0"), t("C0"), t("F0"), t("E"), t("nu"))
    sim.forward(T)
    got = [x.cpu().numpy() for x in sim.state()]
    assert mpm.mpm_sync_status(sim.h) == mpm.MPM_OK
    _compare_states(got, _oracle_states(scene, T), scene, POS_TOL)
    x = torch.ones(4, device="cuda")
    assert float((x * 2).sum()) == 8.0  # the CUDA context survived
    sim.close()
