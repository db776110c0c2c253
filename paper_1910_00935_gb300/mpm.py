"""Python binding of libmpm.so (include/mpm.h) -- argument marshalling only.

Every step of the simulation runs in the library's CUDA kernels; this module turns torch
tensors into device pointers and the current torch stream into a cudaStream_t.  The
library allocates no device memory: `Simulator` allocates the workspace as a torch
uint8 tensor and keeps it alive with the handle.

The functions mpm_* mirror the C entry points one to one.  `MPMSim` is the
torch.autograd.Function of the differentiable simulation: forward runs the tape
(Section 3.2) and returns the state at step T, backward replays it in reverse
(Appendix D) and returns gradients w.r.t. the initial state, E, nu and the actuation
weights.

Importing this module loads the library and raises if it has not been built; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

MPM_OK, MPM_ERR_ARG, MPM_ERR_CUDA, MPM_ERR_OOB = 0, 1, 2, 3
MPM_ERR_NONFINITE, MPM_ERR_TIMEOUT, MPM_ERR_STATE, MPM_ERR_WORKSPACE = 4, 5, 6, 7
MPM_ERR_TOO_LARGE, MPM_ERR_RANGE = 8, 9
MPM_NOALLOC_MAX_NODES = MPM_NOALLOC_MAX_PARTICLES = 1 << 18
MPM_FIXED_COROTATED, MPM_NEO_HOOKEAN, MPM_LIQUID, MPM_MIXED = 0, 1, 3, 4
MPM_LOSS_COM_TARGET, MPM_LOSS_COM_X_DISP = 0, 1
MPM_OPT_USE_GRAPHS, MPM_OPT_SMEM_TILE, MPM_OPT_TILE_CAPACITY, MPM_OPT_PROFILE = 1, 2, 3, 4
MPM_OPT_GATHER_CAPACITY, MPM_OPT_GRID_BLOCKS, MPM_OPT_POLAR_CACHE = 5, 6, 7
MPM_OPT_PERSISTENT, MPM_OPT_BARRIER_TIMEOUT_US, MPM_OPT_BARRIER_TEST_EXTRA = 8, 9, 10
MPM_OPT_PERSISTENT_CHUNK, MPM_OPT_GRID_RECOMPUTE, MPM_OPT_OVERLAP_RESIM = 11, 12, 13
MPM_OPT_BUCKET_SCATTER, MPM_OPT_PAIR_SCATTER, MPM_OPT_SORT_ORDER = 14, 15, 16
KERNEL_CATEGORIES = {1: "p2g", 2: "g2p_p2g", 3: "g2p_p2g_full", 4: "g2p", 5: "grid_clear",
                     6: "adj_g2p", 7: "adj_fused", 8: "adj_p2g", 9: "persistent_step",
                     10: "persistent_adj", 11: "controller"}
MPM_INFO_KERNEL_LAUNCHES, MPM_INFO_N_TOTAL, MPM_INFO_STEPS_RECORDED = 1, 2, 3
MPM_INFO_KEEPS_SEGMENT_GRIDS, MPM_INFO_ACT_PARAMS, MPM_INFO_CKPT_EVERY = 4, 5, 6
MPM_INFO_POLAR_FP64 = 7
MPM_INFO_GATHER_BOXES, MPM_INFO_GATHER_BOX_OVERFLOWS = 8, 9

EXPORTED = ["mpm_workspace_bytes", "mpm_create", "mpm_set_initial", "mpm_forward",
            "mpm_get_state", "mpm_loss", "mpm_backward", "mpm_sync_status", "mpm_set_option",
            "mpm_get_info", "mpm_get_profile", "mpm_last_error", "mpm_destroy",
            "mpm_step_noalloc", "mpm_set_particle_materials", "mpm_initial_p2g_grid",
            "mpm_measure_peak", "mpm_plan_checkpoints"]


class MPMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libmpm error {code}: {msg}")
        self.code = code


class SceneDesc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("n_grid", ctypes.c_int32),
        ("n_scenes", ctypes.c_int32),
        ("n_particles", ctypes.POINTER(ctypes.c_int64)),
        ("dt", ctypes.c_float),
        ("gravity", ctypes.c_float * 3),
        ("wall_cells", ctypes.c_int32),
        ("material", ctypes.c_int32),
        ("rho", ctypes.c_float),
        ("ckpt_every", ctypes.c_int32),
        ("n_groups", ctypes.c_int32),
        ("n_basis", ctypes.c_int32),
        ("act_period", ctypes.c_float),
        ("act_phase", ctypes.c_float),
        ("deterministic_p2g", ctypes.c_int32),
        ("ctrl_hidden", ctypes.c_int32),
        ("ctrl_scale", ctypes.c_float),
        ("ckpt_coarse", ctypes.c_int32),
    ]


_lib = None


def library_path() -> str:
    return os.environ.get("MPM_LIB", _build.LIB)


def lib(load_only: bool = False):
    """Load libmpm.so; raise (never fall back) when it is missing."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libmpm.so not found at {path}: build it with "
                               "`python -m paper_1910_00935_gb300.build`")
        L = ctypes.CDLL(path)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        D = ctypes.POINTER(SceneDesc)
        sig = {
            "mpm_workspace_bytes": (ctypes.c_int, [D, i32, ctypes.POINTER(sz)]),
            "mpm_create": (ctypes.c_int, [D, vp, sz, i32, ctypes.POINTER(vp)]),
            "mpm_set_initial": (ctypes.c_int, [vp] + [vp] * 8 + [vp]),
            "mpm_forward": (ctypes.c_int, [vp, i32, vp]),
            "mpm_get_state": (ctypes.c_int, [vp, vp, vp, vp, vp, vp]),
            "mpm_loss": (ctypes.c_int, [vp, i32, vp, vp, vp, vp, vp]),
            "mpm_backward": (ctypes.c_int, [vp] + [vp] * 11 + [vp]),
            "mpm_sync_status": (ctypes.c_int, [vp]),
            "mpm_set_option": (ctypes.c_int, [vp, i32, i64]),
            "mpm_get_info": (ctypes.c_int, [vp, i32, ctypes.POINTER(i64)]),
            "mpm_get_profile": (ctypes.c_int, [vp, i32, ctypes.POINTER(i64),
                                               ctypes.POINTER(ctypes.c_double)]),
            "mpm_last_error": (ctypes.c_char_p, [vp]),
            "mpm_destroy": (None, [vp]),
            "mpm_step_noalloc": (ctypes.c_int, [D, vp, vp, vp, vp, vp, vp]),
            "mpm_set_particle_materials": (ctypes.c_int, [vp, vp, vp]),
            "mpm_initial_p2g_grid": (ctypes.c_int, [vp, vp, vp]),
            "mpm_measure_peak": (ctypes.c_int, [i32, ctypes.POINTER(ctypes.c_double), vp]),
            "mpm_plan_checkpoints": (ctypes.c_int, [D, i32, sz, ctypes.POINTER(i32),
                                                    ctypes.POINTER(i32), ctypes.POINTER(sz)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


# ----------------------------------------------------------------------------
# one-to-one wrappers of the C entry points
# ----------------------------------------------------------------------------

def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("tensors passed to libmpm must be contiguous")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _check(rc, h=None):
    if rc != MPM_OK:
        msg = lib().mpm_last_error(h)
        raise MPMError(rc, msg.decode() if msg else "")


def make_desc(desc: dict) -> SceneDesc:
    n = list(desc["n_particles"])
    arr = (ctypes.c_int64 * len(n))(*n)
    g = list(desc.get("gravity", (0.0, -9.8, 0.0))) + [0.0, 0.0, 0.0]
    d = SceneDesc(int(desc["dim"]), int(desc["n_grid"]), len(n),
                  ctypes.cast(arr, ctypes.POINTER(ctypes.c_int64)), float(desc["dt"]),
                  (ctypes.c_float * 3)(*g[:3]), int(desc.get("wall_cells", 3)),
                  int(desc.get("material", MPM_FIXED_COROTATED)), float(desc.get("rho", 1.0)),
                  int(desc.get("ckpt_every", 32)), int(desc.get("n_groups", 0)),
                  int(desc.get("n_basis", 0)), float(desc.get("act_period", 50.0)),
                  float(desc.get("act_phase", 0.0)), int(desc.get("deterministic_p2g", 0)),
                  int(desc.get("ctrl_hidden", 0)), float(desc.get("ctrl_scale", 1.0)),
                  int(desc.get("ckpt_coarse", 0)))
    d._keep = arr  # keep the particle-count array alive with the struct
    return d


def mpm_workspace_bytes(desc: SceneDesc, max_steps: int) -> int:
    out = ctypes.c_size_t()
    _check(lib().mpm_workspace_bytes(ctypes.byref(desc), max_steps, ctypes.byref(out)))
    return out.value


def mpm_plan_checkpoints(desc: SceneDesc, max_steps: int, budget_bytes: int):
    """(ckpt_every, ckpt_coarse, workspace bytes) of the fastest schedule within the budget."""
    k, M, b = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_size_t()
    _check(lib().mpm_plan_checkpoints(ctypes.byref(desc), max_steps, budget_bytes, ctypes.byref(k),
                                      ctypes.byref(M), ctypes.byref(b)))
    return k.value, M.value, b.value


def mpm_create(desc: SceneDesc, workspace, workspace_bytes: int, max_steps: int):
    h = ctypes.c_void_p()
    _check(lib().mpm_create(ctypes.byref(desc), _ptr(workspace), workspace_bytes, max_steps,
                            ctypes.byref(h)))
    return h


def mpm_set_initial(h, x0, v0, C0, F0, E, nu, group=None, w=None, stream=None):
    _check(lib().mpm_set_initial(h, _ptr(x0), _ptr(v0), _ptr(C0), _ptr(F0), _ptr(E), _ptr(nu),
                                 _ptr(group), _ptr(w), _stream(stream)), h)


def mpm_set_particle_materials(h, material, stream=None):
    _check(lib().mpm_set_particle_materials(h, _ptr(material), _stream(stream)), h)


def mpm_forward(h, T: int, stream=None):
    _check(lib().mpm_forward(h, T, _stream(stream)), h)


def mpm_get_state(h, x=None, v=None, C=None, F=None, stream=None):
    _check(lib().mpm_get_state(h, _ptr(x), _ptr(v), _ptr(C), _ptr(F), _stream(stream)), h)


def mpm_loss(h, kind, target, loss, dL_dxT, dL_dx0=None, stream=None):
    _check(lib().mpm_loss(h, kind, _ptr(target), _ptr(loss), _ptr(dL_dxT), _ptr(dL_dx0),
                          _stream(stream)), h)


def mpm_backward(h, dL_dx=None, dL_dv=None, dL_dC=None, dL_dF=None, gx0=None, gv0=None,
                 gC0=None, gF0=None, gE=None, gnu=None, gw=None, stream=None):
    _check(lib().mpm_backward(h, _ptr(dL_dx), _ptr(dL_dv), _ptr(dL_dC), _ptr(dL_dF), _ptr(gx0),
                              _ptr(gv0), _ptr(gC0), _ptr(gF0), _ptr(gE), _ptr(gnu), _ptr(gw),
                              _stream(stream)), h)


def mpm_sync_status(h) -> int:
    return lib().mpm_sync_status(h)


def mpm_set_option(h, key: int, value: int):
    _check(lib().mpm_set_option(h, key, value), h)


def mpm_get_info(h, key: int) -> int:
    out = ctypes.c_int64()
    _check(lib().mpm_get_info(h, key, ctypes.byref(out)), h)
    return out.value


def mpm_initial_p2g_grid(h, grid, stream=None):
    _check(lib().mpm_initial_p2g_grid(h, _ptr(grid), _stream(stream)), h)


MPM_PEAK_FP64_FMA, MPM_PEAK_FP32_FMA, MPM_PEAK_RED_F32X4, MPM_PEAK_RED_F32X4_SPREAD = 0, 1, 2, 3


def mpm_measure_peak(kind: int, stream=None) -> float:
    """Measured peak of the current GPU: FLOP/s for MPM_PEAK_FP64_FMA / MPM_PEAK_FP32_FMA,
    float4 reductions per second for MPM_PEAK_RED_F32X4 / MPM_PEAK_RED_F32X4_SPREAD."""
    out = ctypes.c_double()
    _check(lib().mpm_measure_peak(int(kind), ctypes.byref(out), _stream(stream)))
    return out.value


def mpm_get_profile(h, kind: int):
    """(launches, total_ms) of one kernel category while MPM_OPT_PROFILE is on."""
    n, ms = ctypes.c_int64(), ctypes.c_double()
    _check(lib().mpm_get_profile(h, kind, ctypes.byref(n), ctypes.byref(ms)), h)
    return n.value, ms.value


def mpm_last_error(h=None) -> str:
    m = lib().mpm_last_error(h)
    return m.decode() if m else ""


def mpm_destroy(h):
    lib().mpm_destroy(h)


def mpm_step_noalloc(desc: SceneDesc, state_in, E, nu, state_out, device_err=None,
                     stream=None) -> int:
    """One step with no workspace (see include/mpm.h); returns the status code."""
    return lib().mpm_step_noalloc(ctypes.byref(desc), _ptr(state_in), _ptr(E), _ptr(nu),
                                  _ptr(state_out), _ptr(device_err), _stream(stream))


# ----------------------------------------------------------------------------
# convenience object and the autograd Function
# ----------------------------------------------------------------------------

class Simulator:
    """One handle plus its workspace (a torch tensor).  `desc` is a dict with the fields
    of mpm_scene_desc (see include/mpm.h); `max_steps` bounds T."""

    def __init__(self, desc: dict, max_steps: int, device="cuda", workspace_budget=None):
        """workspace_budget (bytes): if given, ckpt_every and ckpt_coarse are chosen by
        mpm_plan_checkpoints for that budget instead of taken from desc."""
        desc = dict(desc)
        if workspace_budget is not None:
            k, M, _ = mpm_plan_checkpoints(make_desc(desc), max_steps, int(workspace_budget))
            desc["ckpt_every"], desc["ckpt_coarse"] = k, M
        self.desc = dict(desc)
        self.dim = int(desc["dim"])
        self.n_scenes = len(desc["n_particles"])
        self.N = int(sum(desc["n_particles"]))
        self._c_desc = make_desc(desc)
        self.ws_bytes = mpm_workspace_bytes(self._c_desc, max_steps)
        self.workspace = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self.h = mpm_create(self._c_desc, self._ws_ptr, self.ws_bytes, max_steps)
        self.device = torch.device(device)
        self.max_steps = int(max_steps)
        self.T = 0

    def close(self):
        if getattr(self, "h", None):
            mpm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, key, value):
        mpm_set_option(self.h, key, value)

    def info(self, key):
        return mpm_get_info(self.h, key)

    def profile(self):
        """{category name: (launches, total_ms)} collected under MPM_OPT_PROFILE."""
        return {name: mpm_get_profile(self.h, k) for k, name in KERNEL_CATEGORIES.items()}

    def _f(self, t, rows=None):
        return None if t is None else t.to(self.device, torch.float32).contiguous()

    def set_initial(self, x0, v0, C0=None, F0=None, E=None, nu=None, group=None, w=None,
                    material=None):
        """material: int32 [N] per-particle material ids (MPM_MIXED scenes only)."""
        self._inputs = [self._f(x0), self._f(v0), self._f(C0), self._f(F0), self._f(E),
                        self._f(nu),
                        None if group is None else group.to(self.device, torch.int32).contiguous(),
                        self._f(w)]
        mpm_set_initial(self.h, *self._inputs)
        if material is not None:
            self._material = material.to(self.device, torch.int32).contiguous()
        if self.desc.get("material") == MPM_MIXED:  # every set-up re-sorts the particles
            mpm_set_particle_materials(self.h, self._material)

    def reload(self):
        """Run the set-up again from the last set_initial inputs (after an option that the
        set-up applies, such as MPM_OPT_SORT_ORDER)."""
        mpm_set_initial(self.h, *self._inputs)
        if self.desc.get("material") == MPM_MIXED:
            mpm_set_particle_materials(self.h, self._material)

    def forward(self, T):
        mpm_forward(self.h, int(T))
        self.T = int(T)

    def state(self):
        d, N = self.dim, self.N
        x = torch.empty(d, N, device=self.device)
        v = torch.empty(d, N, device=self.device)
        C = torch.empty(d * d, N, device=self.device)
        F = torch.empty(d * d, N, device=self.device)
        mpm_get_state(self.h, x, v, C, F)
        return x, v, C, F

    def loss(self, kind, target=None):
        d, N, S = self.dim, self.N, self.n_scenes
        L = torch.empty(S, device=self.device)
        gT = torch.empty(d, N, device=self.device)
        g0 = torch.empty(d, N, device=self.device)
        mpm_loss(self.h, kind, self._f(target), L, gT, g0)
        return L, gT, g0

    def backward(self, dL_dx=None, dL_dv=None, dL_dC=None, dL_dF=None):
        d, N, S = self.dim, self.N, self.n_scenes
        G, K = int(self.desc.get("n_groups", 0)), int(self.desc.get("n_basis", 0))
        n_act = mpm_get_info(self.h, MPM_INFO_ACT_PARAMS)
        # dL/dw [S, G, K] (open loop) or dL/dtheta [S, n_params] (closed-loop controller)
        gw = (torch.zeros(S, n_act, device=self.device) if self.desc.get("ctrl_hidden", 0)
              else torch.zeros(S, G, K, device=self.device))
        out = dict(gx0=torch.empty(d, N, device=self.device),
                   gv0=torch.empty(d, N, device=self.device),
                   gC0=torch.empty(d * d, N, device=self.device),
                   gF0=torch.empty(d * d, N, device=self.device),
                   gE=torch.empty(N, device=self.device), gnu=torch.empty(N, device=self.device),
                   gw=gw)
        mpm_backward(self.h, self._f(dL_dx), self._f(dL_dv), self._f(dL_dC), self._f(dL_dF),
                     out["gx0"], out["gv0"], out["gC0"], out["gF0"], out["gE"], out["gnu"],
                     out["gw"] if n_act else None)
        return out

    def check(self):
        rc = mpm_sync_status(self.h)
        if rc != MPM_OK:
            raise MPMError(rc, mpm_last_error(self.h))


class MPMSim(torch.autograd.Function):
    """(x0, v0, C0, F0, E, nu, w) -> (x_T, v_T, C_T, F_T) through `sim` (a Simulator).
    group is a non-differentiable input passed with the simulator."""

    @staticmethod
    def forward(ctx, sim: Simulator, T: int, group, x0, v0, C0, F0, E, nu, w):
        sim.set_initial(x0, v0, C0, F0, E, nu, group, w)
        sim.forward(T)
        ctx.sim = sim
        return sim.state()

    @staticmethod
    def backward(ctx, gx, gv, gC, gF):
        g = ctx.sim.backward(gx, gv, gC, gF)
        return (None, None, None, g["gx0"], g["gv0"], g["gC0"], g["gF0"], g["gE"], g["gnu"],
                g["gw"])


def simulate(sim: Simulator, T: int, x0, v0, C0, F0, E, nu, group=None, w=None):
    """Differentiable T-step simulation; returns (x_T, v_T, C_T, F_T)."""
    if w is None:
        w = torch.zeros(sim.n_scenes, 0, 0, device=sim.device)
    return MPMSim.apply(sim, T, group, x0, v0, C0, F0, E, nu, w)


def from_scene(scene, max_steps=None, device="cuda"):
    """Simulator for a scene dict made by paper_1910_00935_gb300.scenes, with its initial
    state loaded."""
    desc = scene["desc"]
    sim = Simulator(desc, max_steps or desc["steps"], device)
    a = scene["arrays"]
    G = desc.get("n_groups", 0)
    t = lambda k: torch.as_tensor(a[k])
    sim.set_initial(t("x0"), t("v0"), t("C0"), t("F0"), t("E"), t("nu"),
                    t("group") if G else None, t("w") if G else None,
                    t("material") if desc.get("material") == MPM_MIXED else None)
    return sim
