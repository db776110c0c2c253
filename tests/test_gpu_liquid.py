"""The weakly compressible liquid (MPM_LIQUID, the material of the paper's liquid
simulator) through the same passes as the solids: one step, a dam break of many steps,
gradients of random linear functionals through the tape, and the deterministic mode —
all against the FP64 oracle at the bars of the solid workloads."""
import numpy as np
import pytest

from mpm_testlib import rel_l2
from paper_1910_00935_gb300 import scenes
from test_gpu_parity import (GRAD_TOL, POS_TOL, STEP_TOL, _compare_grads, _compare_states,
                             _oracle_grad_linear, _oracle_states, _random_seeds, _run_gpu)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpm():
    from paper_1910_00935_gb300 import build, mpm as m
    build.build()
    return m


@pytest.mark.parametrize("name,kw", [("liquid2d", dict(cols=(48, 64))),
                                     ("liquid3d", dict(cols=(20, 28, 20)))])
def test_liquid_one_step(mpm, name, kw):
    scene = scenes.make(name, **kw)
    g = _run_gpu(mpm, scene, 1, loss=False)
    _compare_states(g["state"], _oracle_states(scene, 1), scene, STEP_TOL)


@pytest.mark.parametrize("name,kw,T", [("liquid2d", dict(cols=(48, 64)), 200),
                                       ("liquid3d", dict(cols=(16, 24, 16)), 80)])
def test_liquid_dam_break_forward(mpm, name, kw, T):
    scene = scenes.make(name, **kw)
    g = _run_gpu(mpm, scene, T, loss=False)
    _compare_states(g["state"], _oracle_states(scene, T), scene, POS_TOL)


@pytest.mark.parametrize("name,kw,T,k", [("liquid2d", dict(cols=(32, 40)), 40, 12),
                                         ("liquid3d", dict(cols=(12, 16, 12)), 24, 8)])
def test_liquid_gradients(mpm, name, kw, T, k):
    scene = scenes.make(name, **kw)
    scene["desc"]["ckpt_every"] = k
    seeds = _random_seeds(scene, np.random.default_rng(31))
    g = _run_gpu(mpm, scene, T, seeds=seeds, loss=False)
    o = _oracle_grad_linear(scene, T, {kk: v.astype(np.float64) for kk, v in seeds.items()})
    _compare_grads(g["grad"], o, ["gx0", "gv0", "gC0", "gF0", "gE", "gnu"])


def test_liquid_loss_gradient_and_deterministic_mode(mpm):
    """COM-loss gradients (the dam-break optimisation target), and the deterministic mode
    bitwise equal across two runs and within the gradient bar of the oracle."""
    import oracle
    scene = scenes.make("liquid3d", cols=(12, 16, 12))
    T = 32
    g = _run_gpu(mpm, scene, T)
    o = oracle.loss_and_grad(scenes.oracle_view(scene), T)
    assert rel_l2(g["loss"], o["losses"]) <= 1e-3
    _compare_grads(g["grad"], o, ["gx0", "gv0"])
    scene["desc"]["deterministic_p2g"] = 1
    seeds = _random_seeds(scene, np.random.default_rng(32))
    a = _run_gpu(mpm, scene, T, seeds=seeds, loss=False)
    b = _run_gpu(mpm, scene, T, seeds=seeds, loss=False)
    for key in ("gx0", "gv0", "gF0", "gE"):
        assert np.array_equal(a["grad"][key], b["grad"][key]), key
    od = _oracle_grad_linear(scene, T, {kk: v.astype(np.float64) for kk, v in seeds.items()})
    _compare_grads(a["grad"], od, ["gx0", "gv0", "gF0", "gE"], GRAD_TOL)


# ---------------------------------------------------------------------------
# two-way coupling: an actuated fixed-corotated robot in a liquid pool, one grid
# (MPM_MIXED, per-particle materials)
# ---------------------------------------------------------------------------

COUPLED = dict(robot=(16, 8, 8), pool=(48, 8, 24))


def test_robot_in_liquid_one_step_and_forward(mpm):
    scene = scenes.make("robot_in_liquid", **COUPLED)
    g = _run_gpu(mpm, scene, 1, loss=False)
    _compare_states(g["state"], _oracle_states(scene, 1), scene, STEP_TOL)
    T = 60
    g = _run_gpu(mpm, scene, T, loss=False)
    _compare_states(g["state"], _oracle_states(scene, T), scene, POS_TOL)


def test_robot_in_liquid_gradients(mpm):
    """Random linear functionals of the final state: every adjoint term of both materials,
    the actuation weights (only the robot is actuated) and the polar cache of the robot's
    particles."""
    scene = scenes.make("robot_in_liquid", **COUPLED)
    T, k = 24, 10
    scene["desc"]["ckpt_every"] = k
    seeds = _random_seeds(scene, np.random.default_rng(33))
    g = _run_gpu(mpm, scene, T, seeds=seeds, loss=False)
    o = _oracle_grad_linear(scene, T, {kk: v.astype(np.float64) for kk, v in seeds.items()})
    _compare_grads(g["grad"], o, ["gx0", "gv0", "gC0", "gF0", "gE", "gnu", "gw"])


def test_mixed_scene_needs_its_materials(mpm):
    scene = scenes.make("robot_in_liquid", robot=(8, 8, 8), pool=(16, 4, 16))
    sim = mpm.Simulator(scene["desc"], 4)
    a = scene["arrays"]
    t = lambda key: torch.as_tensor(a[key])
    mpm.mpm_set_initial(sim.h, *[t(k).cuda().contiguous() for k in ("x0", "v0", "C0", "F0", "E", "nu")],
                        t("group").cuda().contiguous(), t("w").cuda().contiguous())
    with pytest.raises(mpm.MPMError) as ei:
        sim.forward(4)
    assert ei.value.code == mpm.MPM_ERR_STATE
    mpm.mpm_set_particle_materials(sim.h, t("material").cuda().contiguous())
    sim.forward(4)
    assert mpm.mpm_sync_status(sim.h) == mpm.MPM_OK
    sim.close()
