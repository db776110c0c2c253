"""The build-time shape autotuner (`autotune.tune_build`): particles per CTA chosen among
library builds by measurement, each build checked against the default build's result."""
import json
import os

import numpy as np
import pytest

from paper_1910_00935_gb300 import autotune, scenes

pytestmark = pytest.mark.gpu


def test_tune_build_picks_a_measured_valid_variant(tmp_path):
    scene = scenes.make("cube3d", n_side=16, n_grid=64)  # 4,096 particles
    space = {"tile128": [], "tile64": ["-DMPM_TILE=64"]}
    cache = str(tmp_path / "tune.json")
    res = autotune.tune_build(scene, T=12, repeats=2, space=space, cache_path=cache, force=True)
    assert res["tag"] in space
    assert set(res["seconds"]) == set(space), res  # both ran and agreed with the default build
    assert all(np.isfinite(v) and v > 0 for v in res["seconds"].values())
    assert res["seconds"][res["tag"]] == min(res["seconds"].values())
    assert os.path.exists(res["lib"])
    assert not res["refused"], res["refused"]
    stored = json.load(open(cache))
    assert any(k.startswith("build|") and v["tag"] == res["tag"] for k, v in stored.items())
    # a second call is answered from the cache
    assert autotune.tune_build(scene, T=12, space=space, cache_path=cache)["tag"] == res["tag"]
