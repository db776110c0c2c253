"""Closed-loop controller (mpm_scene_desc.ctrl_hidden > 0; the neural-network controllers
of Section 4.1): at every step the sensors of the current state drive a small MLP whose
outputs actuate the groups.  The CUDA path (split passes around the controller's sensing,
MLP and reverse kernels) against the FP64 oracle: states, then gradients of random linear
functionals of the final state -- the initial state (which reaches the loss through the
sensors as well as the dynamics), E, nu and the controller's parameters theta."""
import numpy as np
import pytest

from mpm_testlib import rel_l2
from paper_1910_00935_gb300 import scenes
from test_gpu_parity import (GRAD_TOL, POS_TOL, STEP_TOL, _compare_grads, _compare_states,
                             _oracle_grad_linear, _oracle_states, _random_seeds, _run_gpu)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SMALL = dict(n_scenes=2, dims=(16, 8, 8), hidden=16)
KEYS = ["gx0", "gv0", "gC0", "gF0", "gE", "gnu", "gw"]


@pytest.fixture(scope="module")
def mpm():
    from paper_1910_00935_gb300 import build, mpm as m
    build.build()
    return m


def _square2d_controlled(hidden=8, n_basis=2, G=4):
    """The 2D square with four quadrant groups driven by a controller."""
    s = scenes.make("square2d", n_side=32)
    a, d = s["arrays"], s["desc"]
    x = a["x0"]
    c = x.mean(axis=1, keepdims=True)
    a["group"] = np.ascontiguousarray(((x[0] > c[0]).astype(np.int32)
                                       + 2 * (x[1] > c[1]).astype(np.int32)))
    th = scenes.controller_params(0, 77, 2, G, n_basis, hidden)
    a["w"] = np.ascontiguousarray(th[None].astype(np.float32))
    d.update(n_groups=G, n_basis=n_basis, ctrl_hidden=hidden, ctrl_scale=60.0, act_period=40.0)
    return s


def test_controller_one_step_and_forward(mpm):
    scene = scenes.make("robots_nn", **SMALL)
    g = _run_gpu(mpm, scene, 1, loss=False)
    _compare_states(g["state"], _oracle_states(scene, 1), scene, STEP_TOL)
    T = 80
    g = _run_gpu(mpm, scene, T, loss=False)
    _compare_states(g["state"], _oracle_states(scene, T), scene, POS_TOL)


def test_controller_actuates(mpm):
    """The controller's output reaches the particles: zeroing theta changes the run."""
    scene = scenes.make("robots_nn", **SMALL)
    a = _run_gpu(mpm, scene, 40, loss=False)["state"][0]
    scene["arrays"]["w"] = np.zeros_like(scene["arrays"]["w"])
    b = _run_gpu(mpm, scene, 40, loss=False)["state"][0]
    assert rel_l2(a, b) > 1e-6


@pytest.mark.parametrize("T,k,options", [
    (24, 10, {}),      # two re-simulated segments with kept grids, resident last segment
    (24, 10, "recompute"),  # every grid recomputed by its own P2G pass
    (12, 64, {}),      # one resident segment: no re-simulation
    (24, 7, "nographs"),
])
def test_controller_gradients(mpm, T, k, options):
    scene = scenes.make("robots_nn", **SMALL)
    scene["desc"]["ckpt_every"] = k
    opts = {}
    if options == "recompute":
        opts = {mpm.MPM_OPT_GRID_RECOMPUTE: 1}
    elif options == "nographs":
        opts = {mpm.MPM_OPT_USE_GRAPHS: 0}
    seeds = _random_seeds(scene, np.random.default_rng(41))
    g = _run_gpu(mpm, scene, T, seeds=seeds, loss=False, options=opts)
    o = _oracle_grad_linear(scene, T, {kk: v.astype(np.float64) for kk, v in seeds.items()})
    _compare_grads(g["grad"], o, KEYS)


def test_controller_2d(mpm):
    scene = _square2d_controlled()
    T, k = 30, 8
    scene["desc"]["ckpt_every"] = k
    g = _run_gpu(mpm, scene, T, loss=False)
    _compare_states(g["state"], _oracle_states(scene, T), scene, POS_TOL)
    seeds = _random_seeds(scene, np.random.default_rng(42))
    g = _run_gpu(mpm, scene, T, seeds=seeds, loss=False)
    o = _oracle_grad_linear(scene, T, {kk: v.astype(np.float64) for kk, v in seeds.items()})
    _compare_grads(g["grad"], o, KEYS)


def test_controller_deterministic_and_persistent_option(mpm):
    """The deterministic mode stays bitwise reproducible with the controller (its sums run
    in a fixed order) and within the oracle bars; the persistent option is ignored."""
    scene = scenes.make("robots_nn", **SMALL)
    scene["desc"]["ckpt_every"] = 8
    scene["desc"]["deterministic_p2g"] = 1
    T = 20
    seeds = _random_seeds(scene, np.random.default_rng(43))
    a = _run_gpu(mpm, scene, T, seeds=seeds, loss=False)
    b = _run_gpu(mpm, scene, T, seeds=seeds, loss=False, options={mpm.MPM_OPT_PERSISTENT: 1})
    for i in range(4):
        assert np.array_equal(a["state"][i], b["state"][i]), i
    for key in KEYS:
        assert np.array_equal(a["grad"][key], b["grad"][key]), key
    o = _oracle_grad_linear(scene, T, {kk: v.astype(np.float64) for kk, v in seeds.items()})
    _compare_grads(a["grad"], o, KEYS)


def test_controller_loss_gradient_and_backward_twice(mpm):
    """A centre-of-mass loss end to end (mpm_loss seeds the backward), with the robots on
    the sticky floor so that the actuation moves the centre of mass, and a second backward
    of the same forward giving the same gradients."""
    import oracle
    scene = scenes.make("robots_nn", bottom_dx=3.0, **SMALL)  # on the sticky floor
    scene["desc"]["ckpt_every"] = 16
    scene["desc"]["loss_kind"] = oracle.LOSS_COM_TARGET
    scene["arrays"]["target"] = np.tile(np.float32([0.7, 0.5, 0.5]), (2, 1))
    T = 40
    sim = mpm.from_scene(scene, max_steps=T)
    sim.forward(T)
    L, gT, g0 = sim.loss(scene["desc"]["loss_kind"], torch.as_tensor(scene["arrays"]["target"]))
    g1 = {k: v.cpu().numpy().copy() for k, v in sim.backward(dL_dx=gT).items()}
    g2 = {k: v.cpu().numpy().copy() for k, v in sim.backward(dL_dx=gT).items()}
    assert mpm.mpm_sync_status(sim.h) == mpm.MPM_OK
    sim.close()
    o = oracle.loss_and_grad(scenes.oracle_view(scene), T)
    assert rel_l2(L.cpu().numpy(), np.asarray(o["losses"])) <= 1e-3
    for key in ("gw", "gx0", "gv0"):
        assert rel_l2(g1[key], o[key]) <= GRAD_TOL, key
        assert rel_l2(g2[key], g1[key]) <= 1e-5, key
