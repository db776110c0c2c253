"""The two precisions of the fixed-corotated polar factor, against the oracle and each other.

The default library refines Newton's FP32 polar factor with error-free FP32 transforms (R to
~1e-14) and runs the polar adjoint in FP32; the build variant MPM_POLAR_FP64=1 does both in
FP64.  Each library runs in a child process of its own (one process loads one library) on
the same seeded scenes: 2D squares and two actuated 3D robots, a random linear functional
of the final state as the loss.  Both must meet the oracle bars (state 1e-4, every gradient
block 1e-3), and per gradient block the FP32 forms must be about as close to the oracle as
the FP64 forms (FP32 atomic-order noise differs from run to run, so the builds are compared
through the oracle, not with each other).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from mpm_testlib import rel_l2
from paper_1910_00935_gb300 import scenes
from test_gpu_parity import (GRAD_TOL, POS_TOL, _compare_grads, _compare_states, _oracle_grad_linear,
                             _oracle_states, _random_seeds)

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASES = {
    "square2d": (dict(n_side=40), 48, 16),
    "robots3d": (dict(n_scenes=2, dims=(16, 8, 8)), 40, 16),
}

CHILD = r"""
import json, sys
import numpy as np
sys.path[:0] = [{root!r}, {tests!r}]
from paper_1910_00935_gb300 import mpm, scenes
from test_gpu_parity import _random_seeds, _run_gpu
out = {{}}
for name, (kw, T, k) in json.loads({cases!r}).items():
    scene = scenes.make(name, **kw)
    scene["desc"]["ckpt_every"] = k
    seeds = _random_seeds(scene, np.random.default_rng(11))
    g = _run_gpu(mpm, scene, T, seeds=seeds, loss=False)
    for i, a in enumerate(g["state"]):
        out[f"{{name}}/state{{i}}"] = a
    for key, a in g["grad"].items():
        if a is not None:
            out[f"{{name}}/{{key}}"] = np.asarray(a)
sim = mpm.from_scene(scenes.make("square2d", n_side=8), max_steps=1)
out["polar_fp64"] = np.array(sim.info(mpm.MPM_INFO_POLAR_FP64))
sim.close()
np.savez({path!r}, **out)
"""


def _child(lib, path):
    script = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"),
                          cases=json.dumps({k: list(v) for k, v in CASES.items()}), path=str(path))
    env = dict(os.environ, MPM_LIB=lib)
    subprocess.run([sys.executable, "-c", script], check=True, env=env, cwd=ROOT, timeout=900)
    return dict(np.load(path))


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    from paper_1910_00935_gb300 import build
    tmp = tmp_path_factory.mktemp("polar")
    libs = {"fp32": build.build(), "fp64": build.build(polar_fp64=True)}
    return {k: _child(lib, tmp / f"{k}.npz") for k, lib in libs.items()}


def test_variants_are_the_builds_they_claim(results):
    assert int(results["fp32"]["polar_fp64"]) == 0
    assert int(results["fp64"]["polar_fp64"]) == 1


_ORACLE = {}


def _oracle(name):
    if name not in _ORACLE:
        kw, T, k = CASES[name]
        scene = scenes.make(name, **kw)
        scene["desc"]["ckpt_every"] = k
        seeds = _random_seeds(scene, np.random.default_rng(11))
        _ORACLE[name] = (scene, _oracle_states(scene, T),
                         _oracle_grad_linear(scene, T, {kk: v.astype(np.float64) for kk, v in seeds.items()}))
    return _ORACLE[name]


def _keys(scene):
    return ["gx0", "gv0", "gC0", "gF0", "gE", "gnu"] + (["gw"] if scene["desc"]["n_groups"] else [])


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("variant", ["fp32", "fp64"])
def test_each_precision_matches_the_oracle(results, name, variant):
    scene, states, o = _oracle(name)
    r = results[variant]
    _compare_states([r[f"{name}/state{i}"] for i in range(4)], states, scene, POS_TOL)
    keys = _keys(scene)
    _compare_grads({kk: r[f"{name}/{kk}"] for kk in keys}, o, keys, GRAD_TOL)


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_forms_are_as_close_to_the_oracle(results, name):
    """Per gradient block, the FP32 forms' distance to the oracle is at most twice the FP64
    forms' (or 1% of the bar): run-to-run FP32 atomic-order noise is in both, so the two
    builds are compared through the oracle rather than bitwise."""
    scene, _, o = _oracle(name)
    for kk in _keys(scene):
        e32 = rel_l2(results["fp32"][f"{name}/{kk}"], o[kk])
        e64 = rel_l2(results["fp64"][f"{name}/{kk}"], o[kk])
        assert e32 <= max(2.0 * e64, 0.01 * GRAD_TOL), (kk, e32, e64)
