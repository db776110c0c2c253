"""CUDA path (through the C ABI) against the FP64 oracle, element by element on the
same seeded FP32 inputs.

Bars: positions (and the rest of the state) within 1e-4 relative L2 after the
workload's steps; gradients within 1e-3 relative L2 per block; one-step results
within 1e-5 (FP32 rounding of one step).  Sizes span many 256-particle tiles with a
ragged last tile; the full-size workloads are checked on reduced step counts and, for
the 16-scene robot batch, on sampled scenes the oracle computes one by one.
"""
import numpy as np
import pytest

import oracle
from mpm_testlib import rel_l2, scene_slice, subset_scenes, to_np
from paper_1910_00935_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

POS_TOL, GRAD_TOL, STEP_TOL = 1e-4, 1e-3, 1e-5


@pytest.fixture(scope="module")
def mpm():
    from paper_1910_00935_gb300 import build, mpm as m
    build.build()
    return m


def _run_gpu(mpm, scene, T, seeds=None, loss=True, options=None, max_steps=None):
    sim = mpm.from_scene(scene, max_steps=max_steps or T)
    for k, v in (options or {}).items():
        sim.set_option(k, v)
    sim.forward(T)
    out = {"state": [to_np(t) for t in sim.state()]}
    if loss:
        L, gT, g0 = sim.loss(scene["desc"]["loss_kind"], torch.as_tensor(scene["arrays"]["target"]))
        out["loss"], out["seedT"], out["seed0"] = to_np(L), gT, g0
        if seeds is None:
            seeds = dict(dL_dx=gT)
    if seeds is not None:
        g = sim.backward(**{k: (torch.as_tensor(v) if isinstance(v, np.ndarray) else v)
                            for k, v in seeds.items()})
        out["grad"] = {k: to_np(v) for k, v in g.items()}
        if loss and "seed0" in out and seeds.get("dL_dx") is out.get("seedT"):
            out["grad"]["gx0"] = out["grad"]["gx0"] + to_np(out["seed0"])
    rc = mpm.mpm_sync_status(sim.h)
    assert rc == mpm.MPM_OK, mpm.mpm_last_error(sim.h)
    out["launches"] = sim.info(mpm.MPM_INFO_KERNEL_LAUNCHES)
    sim.close()
    return out


def _oracle_states(scene, T):
    return oracle.simulate(scenes.oracle_view(scene), T)


def _compare_states(gpu_state, orc_blocks, scene, tol):
    d = scene["desc"]["dim"]
    for si, blk in enumerate(orc_blocks):
        sl = scene_slice(scene, si)
        n = sl.stop - sl.start
        ox, ov, oC, oF = oracle.unpack_state(blk, d, n)
        gx, gv, gC, gF = [a[:, sl] for a in gpu_state]
        assert rel_l2(gx, ox) <= tol, ("x", si, rel_l2(gx, ox))
        assert rel_l2(gF, oF) <= tol, ("F", si, rel_l2(gF, oF))
        # velocities/affine fields are differences of positions: looser by dt-scaling,
        # still checked at 10x the position bar
        assert rel_l2(gv, ov) <= 10 * tol, ("v", si, rel_l2(gv, ov))
        assert rel_l2(gC, oC) <= 100 * tol, ("C", si, rel_l2(gC, oC))


def _random_seeds(scene, rng, scale=1.0):
    d = scene["desc"]["dim"]
    N = sum(scene["desc"]["n_particles"])
    f = lambda r: (scale * rng.standard_normal((r, N))).astype(np.float32)
    return dict(dL_dx=f(d), dL_dv=f(d), dL_dC=f(d * d) * 1e-3, dL_dF=f(d * d))


def _oracle_grad_linear(scene, T, seeds):
    """Oracle gradient of L = <seeds, state_T> (per scene)."""
    desc = scene["desc"]
    d = desc["dim"]
    a = scene["arrays"]
    res = {k: [] for k in ("gx0", "gv0", "gC0", "gF0", "gE", "gnu", "gw")}
    for si in range(len(desc["n_particles"])):
        sl = scene_slice(scene, si)
        p = oracle.scene_params(scene, sl)  # with the slice's per-particle materials if any
        mu, la = oracle.lame(a["E"][sl], a["nu"][sl])
        grp = a["group"][sl] if desc["n_groups"] else None
        w = a["w"][si] if desc["n_groups"] else None
        states = oracle.run(p, T, a["x0"][:, sl], a["v0"][:, sl], a["C0"][:, sl], a["F0"][:, sl],
                            mu, la, grp, w)
        adjT = oracle.pack_state(*[seeds[k][:, sl] for k in ("dL_dx", "dL_dv", "dL_dC", "dL_dF")])
        adj0, mub, lab, wb = oracle.grad(p, T, states, adjT, mu, la, grp, w)
        gx, gv, gC, gF = oracle.unpack_state(adj0, d, sl.stop - sl.start)
        eb, nb = oracle.lame_adjoint(a["E"][sl], a["nu"][sl], mub, lab)
        for k, v in (("gx0", gx), ("gv0", gv), ("gC0", gC), ("gF0", gF), ("gE", eb), ("gnu", nb),
                     ("gw", wb)):
            res[k].append(v)
    cat = {k: np.concatenate(v, axis=-1) for k, v in res.items() if k != "gw"}
    cat["gw"] = np.stack(res["gw"]) if desc["n_groups"] else None
    return cat


def _compare_grads(gpu, orc, keys, tol=GRAD_TOL):
    for k in keys:
        r = rel_l2(gpu[k], orc[k])
        assert r <= tol, (k, r)


# ---------------------------------------------------------------------------
# one step: grid-level and state-level parity
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,kw", [("square2d", {}), ("cube3d", dict(n_side=24, n_grid=64)),
                                     ("robots3d", dict(n_scenes=2, dims=(20, 10, 12)))])
def test_one_step_matches_oracle(mpm, name, kw):
    scene = scenes.make(name, **kw)
    g = _run_gpu(mpm, scene, 1, loss=False)
    _compare_states(g["state"], _oracle_states(scene, 1), scene, STEP_TOL)


@pytest.mark.parametrize("name,kw", [("cube3d", dict(n_side=24, n_grid=64)),
                                     ("rects2d", dict(n_scenes=3, n_min=300, n_max=900)),
                                     ("robots3d", dict(n_scenes=2, dims=(12, 8, 8)))])
def test_p2g_grid_matches_oracle(mpm, name, kw):
    """Sub-stage: the (m, p) grid one P2G pass scatters from the initial state (stress,
    actuation and the APIC affine term included) against the oracle's P2G, per scene."""
    scene = scenes.make(name, **kw)
    sim = mpm.from_scene(scene, max_steps=2)
    d, n, S = scene["desc"]["dim"], scene["desc"]["n_grid"], len(scene["desc"]["n_particles"])
    grid = torch.empty(S, n ** d, 4, device="cuda")
    mpm.mpm_initial_p2g_grid(sim.h, grid)
    assert mpm.mpm_sync_status(sim.h) == mpm.MPM_OK
    sim.close()
    g = grid.cpu().numpy().astype(np.float64)
    a = scene["arrays"]
    for si in range(S):
        sl = scene_slice(scene, si)
        mu, la = oracle.lame(a["E"][sl], a["nu"][sl])
        grp = a["group"][sl] if scene["desc"]["n_groups"] else None
        w = a["w"][si] if scene["desc"]["n_groups"] else None
        gm, gp = oracle.p2g(oracle.scene_params(scene, sl), 0, a["x0"][:, sl], a["v0"][:, sl],
                            a["C0"][:, sl], a["F0"][:, sl], mu, la, grp, w)
        assert rel_l2(g[si, :, 0], gm) <= 1e-6, (si, "m")
        assert rel_l2(g[si, :, 1:1 + d], gp) <= 1e-6, (si, "p")


def test_one_step_adjoint_matches_oracle(mpm):
    """Sub-stage: the adjoint of a single step (the G2P-adjoint pass from the seeds and the
    last P2G-adjoint pass) against the oracle's step adjoint, given the same seeds."""
    scene = scenes.make("robots3d", n_scenes=2, dims=(12, 8, 8))
    seeds = _random_seeds(scene, np.random.default_rng(11))
    g = _run_gpu(mpm, scene, 1, seeds=seeds, loss=False)
    o = _oracle_grad_linear(scene, 1, {kk: v.astype(np.float64) for kk, v in seeds.items()})
    for key in ("gx0", "gv0", "gC0", "gF0", "gE", "gnu", "gw"):
        assert rel_l2(g["grad"][key], o[key]) <= 1e-5, key


# ---------------------------------------------------------------------------
# the workloads' forward passes
# ---------------------------------------------------------------------------

def test_square2d_forward_128_steps(mpm):
    scene = scenes.make("square2d")  # 4096 particles, 16 tiles, fixed-corotated, T = 128
    g = _run_gpu(mpm, scene, 128)
    orc = _oracle_states(scene, 128)
    _compare_states(g["state"], orc, scene, POS_TOL)
    assert g["launches"] > 0


def test_ragged_tiles_and_uneven_batch(mpm):
    # 3 scenes of log-uniform sizes (none a multiple of the 256-particle tile)
    base = scenes.make("rects2d", n_scenes=6)
    scene = subset_scenes(base, [0, 3, 5])
    T = 24
    g = _run_gpu(mpm, scene, T)
    _compare_states(g["state"], _oracle_states(scene, T), scene, POS_TOL)


@pytest.mark.parametrize("n_min,n_max", [(1, 3), (1, 300)])
def test_degenerate_and_tiny_scenes(mpm, n_min, n_max):
    """Scenes of one to three particles (a lone particle keeps C = 0 and F = I, so its
    material gradients vanish) and a batch spanning 4 to 210 particles (partial tiles,
    scenes smaller than a warp) in one batch: states and the gradients of a random
    functional against the oracle."""
    scene = scenes.make("rects2d", n_scenes=8, n_min=n_min, n_max=n_max)
    T = 16
    seeds = _random_seeds(scene, np.random.default_rng(5))
    g = _run_gpu(mpm, scene, T, seeds=seeds, loss=False)
    d, dx = 2, 1.0 / scene["desc"]["n_grid"]
    # C of a lone particle is 0 in exact arithmetic (its 9 weighted node terms cancel); in
    # FP32 each term is about (4/dx) |v|, so C is compared on that absolute scale
    c_bar = 16 * np.finfo(np.float32).eps * (4 / dx) * np.abs(scene["arrays"]["v0"]).max()
    for si, blk in enumerate(_oracle_states(scene, T)):
        sl = scene_slice(scene, si)
        ox, ov, oC, oF = oracle.unpack_state(blk, d, sl.stop - sl.start)
        gx, gv, gC, gF = [a[:, sl] for a in g["state"]]
        assert rel_l2(gx, ox) <= POS_TOL and rel_l2(gF, oF) <= POS_TOL, si
        assert rel_l2(gv, ov) <= 10 * POS_TOL, si
        assert np.abs(gC - oC).max() <= c_bar, (si, np.abs(gC - oC).max(), c_bar)
    o = _oracle_grad_linear(scene, T, {k: v.astype(np.float64) for k, v in seeds.items()})
    _compare_grads(g["grad"], o, ("gx0", "gv0", "gC0", "gF0", "gE", "gnu"))


def test_rects2d_batch_forward(mpm):
    scene = scenes.make("rects2d")  # 64 scenes, log-uniform sizes
    T = 32
    g = _run_gpu(mpm, scene, T)
    _compare_states(g["state"], _oracle_states(scene, T), scene, POS_TOL)


def test_cube3d_full_size_short_run(mpm):
    scene = scenes.make("cube3d")  # 262,144 particles, 128^3 grid, neo-Hookean
    T = 6
    g = _run_gpu(mpm, scene, T)
    _compare_states(g["state"], _oracle_states(scene, T), scene, POS_TOL)


def test_robots3d_full_batch_sampled_scenes(mpm):
    scene = scenes.make("robots3d")  # 16 x 65,536 particles, actuation, fixed-corotated
    T = 8
    g = _run_gpu(mpm, scene, T)
    sampled = [0, 11]
    sub = subset_scenes(scene, sampled)
    orc = _oracle_states(sub, T)
    state_sub = [np.concatenate([a[:, scene_slice(scene, i)] for i in sampled], axis=1)
                 for a in g["state"]]
    _compare_states(state_sub, orc, sub, POS_TOL)


# ---------------------------------------------------------------------------
# gradients
# ---------------------------------------------------------------------------

def test_square2d_grad_full_run(mpm):
    """The differentiable run: T = 512, checkpoint every 32, COM loss."""
    scene = scenes.make("square2d_grad")
    T = 512
    g = _run_gpu(mpm, scene, T, max_steps=T)
    o = oracle.loss_and_grad(scenes.oracle_view(scene), T)
    assert abs(g["loss"][0] - o["loss"]) <= 1e-4 * abs(o["loss"])
    _compare_grads(g["grad"], o, ["gv0", "gx0"])
    # gradient w.r.t. the 2-vector initial-velocity bias = sum over particles of dL/dv0
    bias_g, bias_o = g["grad"]["gv0"].sum(1), o["gv0"].sum(1)
    assert rel_l2(bias_g, bias_o) <= GRAD_TOL
    # internal forces conserve momentum and the body never meets a wall, so dL/dE
    # vanishes identically: both sides must be ~0 on the scale of the loss
    E = scene["arrays"]["E"].astype(np.float64)
    assert np.sum(np.abs(o["gE"]) * E) <= 1e-9 * o["loss"]
    assert np.sum(np.abs(g["grad"]["gE"]) * E) <= 1e-3 * o["loss"]


@pytest.mark.parametrize("name,kw,T,k", [
    ("square2d", dict(n_side=40), 64, 8),
    ("cube3d", dict(n_side=20, n_grid=64), 24, 8),
    ("robots3d", dict(n_scenes=2, dims=(16, 8, 8)), 40, 16),
])
def test_gradients_of_random_functional(mpm, name, kw, T, k):
    """dL/d(x0, v0, C0, F0, E, nu, w) of L = <c, state_T> for random c: exercises every
    adjoint term (the COM loss alone leaves most of them untouched)."""
    scene = scenes.make(name, **kw)
    scene["desc"]["ckpt_every"] = k
    seeds = _random_seeds(scene, np.random.default_rng(5))
    g = _run_gpu(mpm, scene, T, seeds=seeds, loss=False)
    o = _oracle_grad_linear(scene, T, {kk: v.astype(np.float64) for kk, v in seeds.items()})
    keys = ["gx0", "gv0", "gC0", "gF0", "gE", "gnu"] + (["gw"] if scene["desc"]["n_groups"] else [])
    _compare_grads(g["grad"], o, keys)


def test_cube3d_full_size_gradient(mpm):
    scene = scenes.make("cube3d")
    T = 4
    scene["desc"]["ckpt_every"] = 2
    seeds = _random_seeds(scene, np.random.default_rng(9))
    g = _run_gpu(mpm, scene, T, seeds=seeds, loss=False)
    o = _oracle_grad_linear(scene, T, {kk: v.astype(np.float64) for kk, v in seeds.items()})
    _compare_grads(g["grad"], o, ["gx0", "gv0", "gC0", "gF0", "gE", "gnu"])


def test_robots3d_displacement_loss_gradient(mpm):
    """Robots standing on the sticky floor (lowest stencils reach the wall nodes), so
    the actuation moves the centre of mass and dL/dw is not identically zero."""
    scene = scenes.make("robots3d", n_scenes=2, dims=(16, 8, 8), bottom_dx=3.0)
    T = 64
    g = _run_gpu(mpm, scene, T)
    o = oracle.loss_and_grad(scenes.oracle_view(scene), T)
    assert rel_l2(g["loss"], o["losses"]) <= 1e-3
    _compare_grads(g["grad"], o, ["gw", "gx0", "gv0"])


# ---------------------------------------------------------------------------
# tape and launch-form invariances
# ---------------------------------------------------------------------------

def test_checkpoint_interval_invariance(mpm):
    """Appendix D.2: segment-wise recomputation gives the same gradient for every
    segment length (here against the oracle, which stores every state, and against
    each other; the GPU re-simulation differs from the forward only by FP32
    atomic-order rounding)."""
    scene = scenes.make("square2d", n_side=32)
    T = 48
    seeds = _random_seeds(scene, np.random.default_rng(1))
    o = _oracle_grad_linear(scene, T, {k: v.astype(np.float64) for k, v in seeds.items()})
    grads = []
    for k in (1, 7, 16, 48):
        scene["desc"]["ckpt_every"] = k
        grads.append(_run_gpu(mpm, scene, T, seeds=seeds, loss=False)["grad"])
    for g in grads:
        _compare_grads(g, o, ["gx0", "gv0", "gF0", "gE"])
    for g in grads[1:]:
        for key in ("gx0", "gv0", "gF0", "gE"):
            assert rel_l2(g[key], grads[0][key]) <= GRAD_TOL, key


def test_graphs_and_tiles_do_not_change_results(mpm):
    scene = scenes.make("cube3d", n_side=16, n_grid=64)
    T = 12
    seeds = _random_seeds(scene, np.random.default_rng(2))
    ref = _run_gpu(mpm, scene, T, seeds=seeds, loss=False)
    for opts in ({mpm.MPM_OPT_USE_GRAPHS: 0}, {mpm.MPM_OPT_SMEM_TILE: 1},
                 {mpm.MPM_OPT_SMEM_TILE: 1, mpm.MPM_OPT_TILE_CAPACITY: 64}):
        g = _run_gpu(mpm, scene, T, seeds=seeds, loss=False, options=opts)
        assert rel_l2(g["state"][0], ref["state"][0]) <= 1e-6
        for key in ("gx0", "gv0", "gF0"):
            assert rel_l2(g["grad"][key], ref["grad"][key]) <= 1e-4, (opts, key)


def test_backward_twice_and_single_segment(mpm):
    """The forward leaves its last segment in the segment buffer, so the backward starts
    without re-simulating it (nothing is re-simulated when ckpt_every >= T).  A second
    backward of the same forward must still be right (the earlier segments' re-simulation
    reused that buffer), and the single-segment run needs no re-simulation passes."""
    scene = scenes.make("robots3d", n_scenes=2, dims=(16, 8, 8))
    T = 20
    seeds = _random_seeds(scene, np.random.default_rng(6))
    o = _oracle_grad_linear(scene, T, {k: v.astype(np.float64) for k, v in seeds.items()})
    keys = ["gx0", "gv0", "gC0", "gF0", "gE", "gnu", "gw"]
    for k in (6, 20):
        scene["desc"]["ckpt_every"] = k
        sim = mpm.from_scene(scene, max_steps=T)
        sim.set_option(mpm.MPM_OPT_USE_GRAPHS, 0)
        sim.forward(T)
        grads, launches = [], []
        for _ in range(2):
            n0 = sim.info(mpm.MPM_INFO_KERNEL_LAUNCHES)
            g = sim.backward(**{kk: torch.as_tensor(v) for kk, v in seeds.items()})
            launches.append(sim.info(mpm.MPM_INFO_KERNEL_LAUNCHES) - n0)
            grads.append({kk: v.cpu().numpy() for kk, v in g.items()})
        assert mpm.mpm_sync_status(sim.h) == mpm.MPM_OK
        sim.close()
        for g in grads:
            _compare_grads(g, o, keys)
        if k == T:
            # one P2G pass for the grid of step T-1, T + 1 adjoint passes, clean-up and I/O
            assert launches[0] == launches[1] and launches[0] < T + 1 + 20, launches
        else:
            assert launches[1] > launches[0], launches  # the second one re-simulates it


def test_kept_segment_grids_equal_recomputed_grids(mpm):
    """A re-simulated segment's grids kept for its adjoint passes give the gradients of the
    per-step recompute of Appendix D.1 (both against the oracle, and against each other
    to FP32 atomic-order rounding)."""
    scene = scenes.make("robots3d", n_scenes=2, dims=(16, 8, 8))
    T = 20
    scene["desc"]["ckpt_every"] = 6  # segments 0-5, 6-11, 12-17 re-simulated; 18-19 resident
    seeds = _random_seeds(scene, np.random.default_rng(8))
    kept = _run_gpu(mpm, scene, T, seeds=seeds, loss=False)
    rec = _run_gpu(mpm, scene, T, seeds=seeds, loss=False, options={mpm.MPM_OPT_GRID_RECOMPUTE: 1})
    o = _oracle_grad_linear(scene, T, {k: v.astype(np.float64) for k, v in seeds.items()})
    keys = ["gx0", "gv0", "gC0", "gF0", "gE", "gnu", "gw"]
    _compare_grads(kept["grad"], o, keys)
    _compare_grads(rec["grad"], o, keys)
    for key in keys:
        assert rel_l2(kept["grad"][key], rec["grad"][key]) <= 1e-4, key


def test_polar_cache_does_not_change_results(mpm):
    """3D fixed-corotated: backward passes that read the polar factors cached by the
    re-simulation give the gradients of the passes that recompute them (both against the
    oracle, and against each other to FP32 atomic-order rounding)."""
    scene = scenes.make("robots3d", n_scenes=2, dims=(16, 8, 8))
    T = 20
    scene["desc"]["ckpt_every"] = 6  # ragged last segment: 0, 6, 12, 18
    seeds = _random_seeds(scene, np.random.default_rng(4))
    on = _run_gpu(mpm, scene, T, seeds=seeds, loss=False)
    off = _run_gpu(mpm, scene, T, seeds=seeds, loss=False, options={mpm.MPM_OPT_POLAR_CACHE: 0})
    o = _oracle_grad_linear(scene, T, {k: v.astype(np.float64) for k, v in seeds.items()})
    keys = ["gx0", "gv0", "gC0", "gF0", "gE", "gnu", "gw"]
    _compare_grads(on["grad"], o, keys)
    _compare_grads(off["grad"], o, keys)
    for key in keys:
        assert rel_l2(on["grad"][key], off["grad"][key]) <= 1e-4, key


def test_batched_equals_unbatched(mpm):
    base = scenes.make("rects2d", n_scenes=5)
    T = 20
    seeds = _random_seeds(base, np.random.default_rng(3))
    batched = _run_gpu(mpm, base, T, seeds=seeds, loss=False)
    for i in (1, 4):
        single = subset_scenes(base, [i])
        sl = scene_slice(base, i)
        s_seeds = {k: np.ascontiguousarray(v[:, sl]) for k, v in seeds.items()}
        g = _run_gpu(mpm, single, T, seeds=s_seeds, loss=False)
        assert rel_l2(batched["state"][0][:, sl], g["state"][0]) <= 1e-6
        assert rel_l2(batched["grad"]["gv0"][:, sl], g["grad"]["gv0"]) <= 1e-4


def test_autograd_function_matches_backward(mpm):
    scene = scenes.make("square2d", n_side=24)
    T = 16
    sim = mpm.from_scene(scene, max_steps=T)
    a = {k: torch.as_tensor(v).cuda() for k, v in scene["arrays"].items()}
    v0 = a["v0"].clone().requires_grad_(True)
    E = a["E"].clone().requires_grad_(True)
    xT, vT, CT, FT = mpm.simulate(sim, T, a["x0"], v0, a["C0"], a["F0"], E, a["nu"])
    loss = ((xT.mean(1) - torch.tensor([0.7, 0.5], device="cuda")) ** 2).sum() + (vT ** 2).sum()
    gv, gE = torch.autograd.grad(loss, [v0, E])
    seeds = dict(dL_dx=to_np(2 * (xT.mean(1, keepdim=True) - torch.tensor([[0.7], [0.5]], device="cuda"))
                             / xT.shape[1] * torch.ones_like(xT)).astype(np.float32),
                 dL_dv=to_np(2 * vT).astype(np.float32),
                 dL_dC=np.zeros((4, xT.shape[1]), np.float32),
                 dL_dF=np.zeros((4, xT.shape[1]), np.float32))
    orc = _oracle_grad_linear(scene, T, {k: v.astype(np.float64) for k, v in seeds.items()})
    assert rel_l2(to_np(gv), orc["gv0"]) <= GRAD_TOL
    assert rel_l2(to_np(gE), orc["gE"]) <= GRAD_TOL
    sim.close()


# ---------------------------------------------------------------------------
# error behaviour (host-made failures only; nothing here can fault the GPU)
# ---------------------------------------------------------------------------

def test_out_of_grid_particle_reports_oob(mpm):
    scene = scenes.make("square2d", n_side=16)
    scene["arrays"]["x0"][0, 5] = 0.001  # x/dx = 0.128 < 0.5: stencil base -1
    sim = mpm.from_scene(scene, max_steps=4)
    sim.forward(2)
    assert mpm.mpm_sync_status(sim.h) == mpm.MPM_ERR_OOB
    assert "grid" in mpm.mpm_last_error(sim.h)
    assert mpm.mpm_sync_status(sim.h) == mpm.MPM_OK  # the error word was cleared
    sim.close()


def test_state_errors(mpm):
    scene = scenes.make("square2d", n_side=8)
    sim = mpm.Simulator(scene["desc"], 8)
    with pytest.raises(mpm.MPMError) as e:
        sim.forward(4)  # before set_initial
    assert e.value.code == mpm.MPM_ERR_STATE
    grid = torch.empty(128 * 128, 4, device="cuda")
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_initial_p2g_grid(sim.h, grid)
    assert e.value.code == mpm.MPM_ERR_STATE
    sim.close()
    det = scenes.make("square2d", n_side=8)
    det["desc"]["deterministic_p2g"] = 1
    sim = mpm.from_scene(det, max_steps=8)
    with pytest.raises(mpm.MPMError) as e:  # its grids are fixed point
        mpm.mpm_initial_p2g_grid(sim.h, grid)
    assert e.value.code == mpm.MPM_ERR_ARG
    sim.close()
    sim = mpm.from_scene(scene, max_steps=8)
    with pytest.raises(mpm.MPMError) as e:
        sim.backward()
    assert e.value.code == mpm.MPM_ERR_STATE
    with pytest.raises(mpm.MPMError) as e:
        sim.forward(9)
    assert e.value.code == mpm.MPM_ERR_STATE
    sim.close()


# ---------------------------------------------------------------------------
# scatter forms: the per-base bucket table and its fall-backs
# ---------------------------------------------------------------------------

def _dense_cube(spacing_div=4):
    """A 3D cube packed at dx/spacing_div (64 particles per stencil base at 4): every base's
    group overflows the bucket table's 8 slots, so most particles scatter on their own."""
    scene = scenes.make("cube3d", n_side=16, n_grid=64)
    x0 = scene["arrays"]["x0"].astype(np.float64)
    c = x0.mean(axis=1, keepdims=True)
    scene["arrays"]["x0"] = np.ascontiguousarray((c + (x0 - c) * (2.0 / spacing_div)).astype(np.float32))
    return scene


def _random_cloud():
    """Particles scattered uniformly over [0.2, 0.8]^3: a 128-particle tile's base box spans
    most of the grid, beyond the bucket table's keys, so the tiles take the per-particle path."""
    scene = scenes.make("cube3d", n_side=12, n_grid=64)
    n = scene["arrays"]["x0"].shape[1]
    u = scenes.uniform(3, 77, 3 * n).reshape(3, n)
    scene["arrays"]["x0"] = np.ascontiguousarray((0.2 + 0.6 * u).astype(np.float32))
    return scene


SCATTER_FORMS = {"pairs": {}, "pairs_forward_only": {"MPM_OPT_PAIR_SCATTER": 1},
                 "per_particle": {"MPM_OPT_PAIR_SCATTER": 0},
                 "bucket": {"MPM_OPT_PAIR_SCATTER": 0, "MPM_OPT_BUCKET_SCATTER": 1}}


@pytest.mark.parametrize("case", ["dense", "cloud", "rects2d", "robots3d"])
@pytest.mark.parametrize("form", list(SCATTER_FORMS))
def test_scatter_forms_match_oracle(mpm, case, form):
    """States and random-functional gradients for each scatter form (pair-merged reductions,
    the default; one reduction per particle and node; the per-base bucket table) on scenes
    that exercise pairs whose bases differ and the bucket table's overflow (dense cube), its
    fall-back (random cloud), 2D (three bucket groups per warp step) and actuated robots."""
    scene = {"dense": _dense_cube, "cloud": _random_cloud,
             "rects2d": lambda: scenes.make("rects2d", n_scenes=4, n_min=500, n_max=3000),
             "robots3d": lambda: scenes.make("robots3d", n_scenes=2, dims=(12, 8, 8))}[case]()
    T = 6
    scene["desc"]["ckpt_every"] = 3
    seeds = _random_seeds(scene, np.random.default_rng(21))
    g = _run_gpu(mpm, scene, T, seeds=seeds, loss=False,
                 options={getattr(mpm, k): v for k, v in SCATTER_FORMS[form].items()})
    _compare_states(g["state"], _oracle_states(scene, T), scene, POS_TOL)
    o = _oracle_grad_linear(scene, T, {kk: v.astype(np.float64) for kk, v in seeds.items()})
    keys = ["gx0", "gv0", "gC0", "gF0", "gE", "gnu"] + (["gw"] if scene["desc"]["n_groups"] else [])
    _compare_grads(g["grad"], o, keys)


@pytest.mark.parametrize("name,kw", [("square2d", dict(n_side=40)),
                                     ("cube3d", dict(n_side=16, n_grid=64))])
@pytest.mark.parametrize("gather", [1536, 2048, 4096])
def test_gather_capacities_near_the_static_limit(mpm, name, kw, gather):
    """Gather boxes whose dynamic shared memory lands just under or over 48 KB (where the
    kernel's static shared memory decides whether the limit must be raised) run and give
    the default's results; graphs on, re-simulation overlapped."""
    scene = scenes.make(name, **kw)
    T = 12
    scene["desc"]["ckpt_every"] = 5
    seeds = _random_seeds(scene, np.random.default_rng(3))
    ref = _run_gpu(mpm, scene, T, seeds=seeds, loss=False)
    g = _run_gpu(mpm, scene, T, seeds=seeds, loss=False,
                 options={mpm.MPM_OPT_GATHER_CAPACITY: gather})
    assert rel_l2(g["state"][0], ref["state"][0]) <= 1e-6
    for key in ("gx0", "gv0", "gF0"):
        assert rel_l2(g["grad"][key], ref["grad"][key]) <= 1e-4, key


def test_capacity_beyond_shared_memory_is_refused(mpm):
    """A gather box that cannot fit one CTA's shared memory is refused by the option call
    (MPM_ERR_ARG, option unchanged), and the handle keeps working."""
    scene = scenes.make("cube3d", n_side=12, n_grid=32)
    sim = mpm.from_scene(scene, max_steps=4)
    with pytest.raises(mpm.MPMError) as ei:
        sim.set_option(mpm.MPM_OPT_GATHER_CAPACITY, 12288)
    assert ei.value.code == mpm.MPM_ERR_ARG and "shared memory" in str(ei.value)
    sim.forward(4)
    sim.check()
    sim.close()


def test_gather_box_counters(mpm):
    """MPM_INFO_GATHER_BOXES / _OVERFLOWS count the forward's gathers and those whose stencil
    box did not fit the shared gather box; a set-up resets them."""
    scene = scenes.make("cube3d", n_side=16, n_grid=64)  # 4,096 particles: 32 tiles of 128
    sim = mpm.from_scene(scene, max_steps=8)
    assert sim.info(mpm.MPM_INFO_GATHER_BOXES) == 0
    sim.forward(8)
    boxes = sim.info(mpm.MPM_INFO_GATHER_BOXES)
    # the first step is a P2G from the initial state; then 7 fused G2P+P2G passes and the last
    # G2P each gather once per tile
    assert boxes == 8 * 32, boxes
    assert sim.info(mpm.MPM_INFO_GATHER_BOX_OVERFLOWS) == 0  # a compact tile's box fits 512
    sim.set_option(mpm.MPM_OPT_GATHER_CAPACITY, 27)  # smaller than any 3D stencil box of a tile
    sim.reload()
    assert sim.info(mpm.MPM_INFO_GATHER_BOXES) == 0
    sim.forward(8)
    assert sim.info(mpm.MPM_INFO_GATHER_BOX_OVERFLOWS) == sim.info(mpm.MPM_INFO_GATHER_BOXES) == boxes
    sim.check()
    sim.close()
