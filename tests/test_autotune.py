"""Autotuner logic on the host (no GPU): coordinate descent finds the minimum of a known
cost over the knob space, the cache round-trips, and shape keys group workloads."""
import pytest

from paper_1910_00935_gb300 import autotune

torch = pytest.importorskip("torch")


def test_coordinate_descent_finds_separable_minimum():
    target = {"gather_capacity": 1024, "smem_tile": 1, "bucket_scatter": 1, "pair_scatter": 3, "sort_order": 1,
              "tile_capacity": 2048,
              "grid_blocks": 64, "persistent": 1, "grid_recompute": 1, "overlap_resim": 0}
    cost = lambda c: sum((0 if c[k] == target[k] else 1.0 + i) for i, k in enumerate(c))
    best, t, log = autotune.coordinate_descent(cost, rounds=3)
    assert best == target and t == 0
    assert all(set(c) == set(autotune.SPACE) for c, _ in log)


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "t.json")
    assert autotune.load_cache(path) == {}
    autotune.save_cache({"k": {"config": autotune.DEFAULTS}}, path)
    assert autotune.load_cache(path)["k"]["config"] == autotune.DEFAULTS


def test_shape_key_groups_by_size_class():
    d = dict(dim=3, material=1, n_grid=128, n_particles=[262144])
    assert autotune.shape_key(d, "gpu") == autotune.shape_key(dict(d, n_particles=[300000]), "gpu")
    assert autotune.shape_key(d, "gpu") != autotune.shape_key(dict(d, n_particles=[600000]), "gpu")
    assert autotune.shape_key(d, "gpu") != autotune.shape_key(dict(d, dim=2), "gpu")


@pytest.mark.gpu
def test_tune_on_gpu_keeps_results(tmp_path):
    import numpy as np
    from paper_1910_00935_gb300 import build, mpm, scenes
    build.build()
    sc = scenes.make("cube3d", n_side=16, n_grid=64)
    T = 8
    ref = mpm.from_scene(sc, max_steps=T)
    ref.forward(T)
    x_ref = ref.state()[0].cpu().numpy()
    ref.close()
    sim = mpm.from_scene(sc, max_steps=T)
    cfg = autotune.tune(sim, T=T, repeats=1, cache_path=str(tmp_path / "c.json"))
    assert set(cfg) == set(autotune.SPACE)
    sim.forward(T)
    x = sim.state()[0].cpu().numpy()
    sim.check()
    assert np.linalg.norm(x - x_ref) <= 1e-6 * np.linalg.norm(x_ref)
    # second call hits the cache
    assert autotune.tune(sim, T=T, cache_path=str(tmp_path / "c.json")) == cfg
    sim.close()


def test_tune_build_selection_validation_and_cache(tmp_path, monkeypatch):
    """tune_build with the builds and the child runs replaced by fakes: the fastest variant
    whose final positions agree with the default build's is chosen, a variant that
    disagrees or fails is listed as refused, and the result is cached by shape."""
    import json
    import os
    import re
    import subprocess

    import numpy as np

    from paper_1910_00935_gb300 import build, scenes

    space = {"tile128": [], "tile64": ["-DMPM_TILE=64"], "tile256": ["-DMPM_TILE=256"],
             "bad": ["-DBAD"], "broken": ["-DBROKEN"]}
    built = []

    def fake_build(extra_flags=(), tag="", **kw):
        built.append((tuple(extra_flags), tag))
        return f"/fake/{tag or 'default'}/libmpm.so"

    seconds = {"default": 2.0, "tile64": 1.0, "tile256": 3.0, "bad": 0.5, "broken": 0.1}

    def fake_run(cmd, capture_output=True, text=True, env=None, timeout=None, **kw):
        tag = env["MPM_LIB"].split("/")[2]
        xout = re.search(r"np\.save\('([^']+)'", cmd[-1]).group(1)
        x = np.ones((3, 8))
        if tag == "bad":
            x = x * 1.01  # a build that computes something else
        if tag == "broken":
            return subprocess.CompletedProcess(cmd, 1, "", "Traceback\nRuntimeError: launch failed")
        np.save(xout, x)
        return subprocess.CompletedProcess(cmd, 0, json.dumps({"seconds": seconds[tag]}) + "\n", "")

    monkeypatch.setattr(build, "build", fake_build)
    monkeypatch.setattr(subprocess, "run", fake_run)
    scene = scenes.make("square2d", n_side=8)
    cache = str(tmp_path / "tune.json")
    res = autotune.tune_build(scene, T=4, space=space, cache_path=cache, device_name="fake-gpu")
    assert res["tag"] == "tile64" and res["lib"] == "/fake/tile64/libmpm.so"
    assert set(res["seconds"]) == {"tile128", "tile64", "tile256"}
    assert set(res["refused"]) == {"bad", "broken"}
    assert "differ" in res["refused"]["bad"] and "launch failed" in res["refused"]["broken"]
    assert ((), "") in built  # the default build has no flags and no tag
    # cached: a second call builds nothing new when the chosen library exists
    monkeypatch.setattr(os.path, "exists", lambda p: True)
    n = len(built)
    assert autotune.tune_build(scene, T=4, space=space, cache_path=cache, device_name="fake-gpu")["tag"] == "tile64"
    assert len(built) == n
