"""The C-ABI library builds for sm_103a, loads without a GPU, exports every entry point
that include/mpm.h and include/mass_spring.h declare, and validates arguments on the host
(no compute calls)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpm.h")
MS_HEADER = os.path.join(ROOT, "include", "mass_spring.h")


def declared(header=HEADER, prefix="mpm"):
    text = open(header).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(" + prefix + r"_\w+)\(",
                                 text, re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1910_00935_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared()
    for n in ("mpm_create", "mpm_forward", "mpm_backward", "mpm_workspace_bytes",
              "mpm_set_initial", "mpm_get_state", "mpm_loss", "mpm_sync_status",
              "mpm_last_error", "mpm_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT ((?:mpm|ms)_\w+)$", out, re.M))
    missing = [n for n in declared() + declared(MS_HEADER, "ms") if n not in exported]
    assert not missing, missing


def test_binding_names_match_header(libpath):
    from paper_1910_00935_gb300 import mpm
    assert sorted(mpm.EXPORTED) == declared()
    for n in declared():
        assert callable(getattr(mpm, n))


def test_host_side_validation_without_gpu(libpath):
    from paper_1910_00935_gb300 import mpm
    good = dict(dim=3, n_grid=64, n_particles=[1000, 2000], dt=1e-4, ckpt_every=16,
                material=mpm.MPM_NEO_HOOKEAN)
    d = mpm.make_desc(good)
    b1 = mpm.mpm_workspace_bytes(d, 64)
    b2 = mpm.mpm_workspace_bytes(d, 256)
    assert b2 > b1 > 0
    for bad in (dict(dim=4), dict(n_grid=4), dict(dt=0.0), dict(ckpt_every=-1),
                dict(n_particles=[0]), dict(wall_cells=40), dict(material=7),
                dict(n_groups=9), dict(n_groups=2, n_basis=0), dict(deterministic_p2g=2)):
        with pytest.raises(mpm.MPMError) as e:
            mpm.mpm_workspace_bytes(mpm.make_desc({**good, **bad}), 64)
        assert e.value.code == mpm.MPM_ERR_ARG
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_workspace_bytes(d, 0)
    assert e.value.code == mpm.MPM_ERR_ARG
    # the deterministic mode keeps 64-bit fixed-point grids: twice the grid memory
    bd = mpm.mpm_workspace_bytes(mpm.make_desc({**good, "deterministic_p2g": 1}), 64)
    grids = 10 * 2 * 64 ** 3 * 16  # ten (m, p) and ubar buffers, two scenes, float4 nodes
    assert bd - b1 >= grids
    # ckpt_every = 0: the interval that minimises the stored states, ceil(sqrt(max_steps))
    # (T/k checkpoints + k segment states); its workspace matches an explicit k of that size
    for T_max in (64, 1000, 1024):
        k = int(np.ceil(np.sqrt(T_max)))
        assert (mpm.mpm_workspace_bytes(mpm.make_desc({**good, "ckpt_every": 0}), T_max)
                == mpm.mpm_workspace_bytes(mpm.make_desc({**good, "ckpt_every": k}), T_max))
    # the closed-loop controller: limits, and its per-step tables in the workspace
    ctrl = dict(good, n_groups=8, n_basis=4, ctrl_hidden=32, ctrl_scale=50.0)
    for bad in (dict(ctrl_hidden=65), dict(ctrl_hidden=-1), dict(n_groups=0),
                dict(ctrl_scale=float("inf")), dict(act_period=0.0)):
        with pytest.raises(mpm.MPMError) as e:
            mpm.mpm_workspace_bytes(mpm.make_desc({**ctrl, **bad}), 64)
        assert e.value.code == mpm.MPM_ERR_ARG, bad
    # no time inputs: n_basis 0 is allowed with the controller (not without it)
    assert mpm.mpm_workspace_bytes(mpm.make_desc({**ctrl, "n_basis": 0}), 64) > 0
    bc = mpm.mpm_workspace_bytes(mpm.make_desc(ctrl), 64)
    n_in = 4 + 2 * 3 * 8
    per_step = 2 * (n_in + 32 + 8) * 8 + 2 * 8 * 4  # u, h, y (FP64) and the actuation row
    assert bc - b1 >= 65 * per_step
    # NULL or misaligned workspace is rejected before any CUDA call
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_create(d, 0, b1, 64)
    assert e.value.code == mpm.MPM_ERR_WORKSPACE
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_create(d, 4096 + 8, b1, 64)
    assert e.value.code == mpm.MPM_ERR_WORKSPACE
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_create(d, 4096, b1 - 1, 64)
    assert e.value.code == mpm.MPM_ERR_WORKSPACE
    assert "workspace" in mpm.mpm_last_error(None)
    # NULL handle
    assert mpm.lib().mpm_forward(None, 1, None) == mpm.MPM_ERR_ARG
    assert mpm.lib().mpm_sync_status(None) == mpm.MPM_ERR_ARG
    assert mpm.lib().mpm_initial_p2g_grid(None, None, None) == mpm.MPM_ERR_ARG
    assert mpm.lib().mpm_measure_peak(7, None, None) == mpm.MPM_ERR_ARG


def test_mass_spring_binding_and_host_validation(libpath):
    from paper_1910_00935_gb300 import mass_spring as ms, mpm
    assert sorted(ms.EXPORTED) == declared(MS_HEADER, "ms")
    tri = [(0, 1), (0, 2), (1, 2)]
    d = ms.make_desc(2, 3, tri, 1000, 100.0, 10.0, 1e-3)
    b = ms.ms_workspace_bytes(d, 100)
    assert b >= 2 * 100 * 6 * 1000 * 4  # positions and velocities of every state
    for args in ((4, 3, tri), (2, 9, tri), (2, 3, [(0, 0)]), (2, 3, [(0, 3)]),
                 (2, 3, [(0, 1)] * 33)):
        with pytest.raises(mpm.MPMError) as e:
            ms.ms_workspace_bytes(ms.make_desc(*args, 1000, 100.0, 10.0, 1e-3), 100)
        assert e.value.code == mpm.MPM_ERR_ARG, args
    for bad in (dict(dt=0.0), dict(mass=-1.0), dict(n_systems=0)):
        kw = dict(dim=2, n_masses=3, springs=tri, n_systems=10, stiffness=1.0, damping=0.0,
                  dt=1e-3, mass=1.0)
        kw.update(bad)
        with pytest.raises(mpm.MPMError):
            ms.ms_workspace_bytes(ms.make_desc(**kw), 10)
    with pytest.raises(mpm.MPMError):
        ms.ms_workspace_bytes(d, 0)
    assert ms.lib().ms_forward(None, None, None, None, 1, None) == mpm.MPM_ERR_ARG


@pytest.mark.gpu
def test_measured_peaks_are_sane(libpath):
    """The FMA peaks the ALU rooflines divide by: positive, FP32 well above FP64 (this
    part's FP64 rate is a small fraction of FP32), both below the chip's nominal ceilings
    (FP32: 152 SMs x 128 lanes x 2 FLOP x ~2.1 GHz = 82 TFLOP/s)."""
    from paper_1910_00935_gb300 import mpm
    f64 = mpm.mpm_measure_peak(mpm.MPM_PEAK_FP64_FMA)
    f32 = mpm.mpm_measure_peak(mpm.MPM_PEAK_FP32_FMA)
    assert 1e11 < f64 < 2e13, f64
    assert 1e13 < f32 < 1e14, f32
    assert f32 > 4 * f64
    # float4 reductions per second: the scatter roofline's denominators; lanes on 32
    # consecutive nodes touch 4 cache lines, on 32 spread nodes 32, so the spread rate is
    # the lower one
    red = mpm.mpm_measure_peak(mpm.MPM_PEAK_RED_F32X4)
    spread = mpm.mpm_measure_peak(mpm.MPM_PEAK_RED_F32X4_SPREAD)
    assert 1e10 < spread <= 1.1 * red < 1e13, (spread, red)


def test_planned_schedule_fits_budget_and_prefers_fewer_passes(libpath):
    """mpm_plan_checkpoints (host only): within a budget it returns the schedule with the
    fewest re-simulated steps; a huge budget keeps every state (nothing re-simulated), the
    smallest one-level workspace keeps one level, one byte less needs two levels, and a
    budget below any schedule is refused."""
    from paper_1910_00935_gb300 import mpm, scenes
    desc = dict(scenes.make("cube3d", n_side=24, n_grid=32)["desc"], ckpt_every=16)
    T = 512
    ws = lambda k, M=0: mpm.mpm_workspace_bytes(mpm.make_desc(dict(desc, ckpt_every=k,
                                                                   ckpt_coarse=M)), T)
    k, M, b = mpm.mpm_plan_checkpoints(mpm.make_desc(desc), T, 1 << 50)
    assert (k, M) == (T, 0) and b == ws(T)
    one_min = min(ws(k) for k in range(1, T + 1))
    k, M, b = mpm.mpm_plan_checkpoints(mpm.make_desc(desc), T, one_min)
    assert M == 0 and b == one_min == ws(k)
    k, M, b = mpm.mpm_plan_checkpoints(mpm.make_desc(desc), T, one_min - 1)
    assert M >= 2 and b < one_min and b == ws(k, M)
    with pytest.raises(mpm.MPMError) as e:
        mpm.mpm_plan_checkpoints(mpm.make_desc(desc), T, one_min // 2)
    assert e.value.code == mpm.MPM_ERR_WORKSPACE
