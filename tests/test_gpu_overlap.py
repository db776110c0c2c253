"""Checkpoint schedules and the launch form of the re-simulation: the backward's
re-simulation of segment j-1 on a second stream, overlapped with the adjoint passes of
segment j (MPM_OPT_OVERLAP_RESIM, on by default); the automatic O(sqrt T) interval; two
levels of checkpoints (ckpt_coarse).  None of them changes what is computed: in the
deterministic mode the gradients are bitwise those of the single-stream, one-level backward
(kept and recomputed grids, resident or re-simulated last segment, fixed-corotated polar
caches), and the default mode meets the oracle bars."""
import numpy as np
import pytest

from paper_1910_00935_gb300 import scenes
from test_gpu_parity import (_compare_grads, _oracle_grad_linear, _random_seeds, _run_gpu)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ["gx0", "gv0", "gC0", "gF0", "gE", "gnu"]


@pytest.fixture(scope="module")
def mpm():
    from paper_1910_00935_gb300 import build, mpm as m
    build.build()
    return m


CASES = [
    ("cube3d", dict(n_side=16, n_grid=64), 40, 8, 0),
    ("cube3d", dict(n_side=16, n_grid=64), 40, 8, 1),    # every grid recomputed
    ("cube3d", dict(n_side=16, n_grid=64), 37, 9, 0),    # ragged last segment
    ("robots3d", dict(n_scenes=2, dims=(16, 8, 8)), 30, 7, 0),
    ("rects2d", dict(n_scenes=4, n_min=300, n_max=1500), 33, 5, 0),
]


@pytest.mark.parametrize("name,kw,T,k,recompute", CASES)
def test_overlap_is_bitwise_the_single_stream_backward(mpm, name, kw, T, k, recompute):
    scene = scenes.make(name, **kw)
    scene["desc"]["ckpt_every"] = k
    scene["desc"]["deterministic_p2g"] = 1
    seeds = _random_seeds(scene, np.random.default_rng(51))
    base = {mpm.MPM_OPT_GRID_RECOMPUTE: recompute}
    runs = [_run_gpu(mpm, scene, T, seeds=seeds, loss=False,
                     options={**base, mpm.MPM_OPT_OVERLAP_RESIM: ov, mpm.MPM_OPT_USE_GRAPHS: gr})
            for ov, gr in ((1, 1), (0, 1), (1, 0))]
    ref = runs[1]
    for r in (runs[0], runs[2]):
        for key, v in ref["grad"].items():
            if v is not None:
                assert np.array_equal(r["grad"][key], v), key


def test_overlap_backward_twice_and_oracle(mpm):
    """Default (FP32) mode with the overlap: the oracle bars, and a second backward of the
    same forward within rounding of the first."""
    from mpm_testlib import rel_l2
    scene = scenes.make("cube3d", n_side=16, n_grid=64)
    scene["desc"]["ckpt_every"] = 6
    T = 26
    seeds = _random_seeds(scene, np.random.default_rng(52))
    sim = mpm.from_scene(scene, max_steps=T)
    sim.forward(T)
    tseeds = {kk: torch.as_tensor(v) for kk, v in seeds.items()}
    g1 = {kk: v.cpu().numpy().copy() for kk, v in sim.backward(**tseeds).items()}
    g2 = {kk: v.cpu().numpy().copy() for kk, v in sim.backward(**tseeds).items()}
    assert mpm.mpm_sync_status(sim.h) == mpm.MPM_OK
    sim.close()
    o = _oracle_grad_linear(scene, T, {kk: v.astype(np.float64) for kk, v in seeds.items()})
    _compare_grads(g1, o, KEYS)
    # the second backward re-simulates the last segment as well (the first found it
    # resident): FP32 atomics in a different order, so agreement to rounding, not bitwise
    for key in KEYS:
        assert rel_l2(g2[key], g1[key]) <= 1e-4, key


def test_automatic_checkpoint_interval(mpm):
    """ckpt_every = 0 takes k = ceil(sqrt(max_steps)) (T/k checkpoints + k segment states,
    Appendix D's O(sqrt(T)) memory); the gradients still meet the oracle bars."""
    scene = scenes.make("robots3d", n_scenes=2, dims=(12, 8, 8))
    scene["desc"]["ckpt_every"] = 0
    T = 40
    sim = mpm.from_scene(scene, max_steps=T)
    assert sim.info(mpm.MPM_INFO_CKPT_EVERY) == 7
    sim.close()
    seeds = _random_seeds(scene, np.random.default_rng(53))
    g = _run_gpu(mpm, scene, T, seeds=seeds, loss=False)
    o = _oracle_grad_linear(scene, T, {kk: v.astype(np.float64) for kk, v in seeds.items()})
    _compare_grads(g["grad"], o, KEYS + ["gw"])


@pytest.mark.parametrize("name,kw,T,k,M", [
    ("cube3d", dict(n_side=16, n_grid=64), 40, 4, 3),    # coarse segments of 12, ragged end
    ("robots3d", dict(n_scenes=2, dims=(12, 8, 8)), 29, 3, 4),  # polar caches, actuation
    ("robots_nn", dict(n_scenes=2, dims=(12, 8, 8), hidden=8), 21, 4, 2),  # controller
])
def test_two_level_checkpoints_bitwise_equal_one_level(mpm, name, kw, T, k, M):
    """ckpt_coarse = M: the forward keeps the state every k*M steps and the backward rebuilds
    each coarse segment's checkpoints before its segments' re-simulation; in the
    deterministic mode the gradients are bitwise those of one level at interval k (the
    rebuilt checkpoints equal the forward's), for the first and a second backward."""
    scene = scenes.make(name, **kw)
    scene["desc"]["ckpt_every"] = k
    scene["desc"]["deterministic_p2g"] = 1
    seeds = _random_seeds(scene, np.random.default_rng(54))
    keys = KEYS + (["gw"] if scene["desc"].get("n_groups", 0) else [])
    one = _run_gpu(mpm, scene, T, seeds=seeds, loss=False)
    scene["desc"]["ckpt_coarse"] = M
    sim = mpm.from_scene(scene, max_steps=T)
    sim.forward(T)
    tseeds = {kk: torch.as_tensor(v) for kk, v in seeds.items()}
    for _ in range(2):
        g = {kk: v.cpu().numpy() for kk, v in sim.backward(**tseeds).items()}
        for key in keys:
            assert np.array_equal(g[key], one["grad"][key]), key
    assert mpm.mpm_sync_status(sim.h) == mpm.MPM_OK
    sim.close()


def test_two_level_checkpoints_store_fewer_states(mpm):
    scene = scenes.make("cube3d", n_side=16, n_grid=64)
    d1 = dict(scene["desc"], ckpt_every=4)
    d2 = dict(d1, ckpt_coarse=8)
    b1 = mpm.mpm_workspace_bytes(mpm.make_desc(d1), 1024)
    b2 = mpm.mpm_workspace_bytes(mpm.make_desc(d2), 1024)
    state = 24 * 4 * sum(scene["desc"]["n_particles"])
    # 256 checkpoints -> 32 coarse ones + 8 rebuilt ones
    assert b1 - b2 >= (256 - 32 - 8) * state


def test_budget_chosen_schedule_bitwise_equal_one_level(mpm):
    """A two-level schedule chosen by mpm_plan_checkpoints for a budget just below the
    smallest one-level workspace gives, in the deterministic mode, bitwise the gradients of
    the one-level schedule at the same interval (Appendix D.2's segment invariance, carried
    to two levels), through the Simulator's workspace_budget argument."""
    scene = scenes.make("cube3d", n_side=24, n_grid=32)
    scene["desc"]["deterministic_p2g"] = 1
    T = 512
    desc = scene["desc"]
    one_min = min(mpm.mpm_workspace_bytes(mpm.make_desc(dict(desc, ckpt_every=k)), T)
                  for k in range(1, T + 1))
    sim = mpm.Simulator(desc, T, workspace_budget=one_min - 1)
    k, M = sim.desc["ckpt_every"], sim.desc["ckpt_coarse"]
    assert M >= 2 and sim.ws_bytes < one_min, (k, M, sim.ws_bytes, one_min)
    seeds = _random_seeds(scene, np.random.default_rng(61))
    a = scene["arrays"]
    t = lambda key: torch.as_tensor(a[key])
    sim.set_initial(t("x0"), t("v0"), t("C0"), t("F0"), t("E"), t("nu"))
    sim.forward(T)
    g = {kk: v.cpu().numpy() for kk, v in sim.backward(**{kk: torch.as_tensor(v)
                                                         for kk, v in seeds.items()}).items()}
    assert mpm.mpm_sync_status(sim.h) == mpm.MPM_OK
    sim.close()
    scene["desc"]["ckpt_every"], scene["desc"]["ckpt_coarse"] = k, 0
    one = _run_gpu(mpm, scene, T, seeds=seeds, loss=False)
    for key in KEYS:
        assert np.array_equal(g[key], one["grad"][key]), key
