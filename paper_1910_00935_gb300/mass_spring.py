"""Python binding of the batched differentiable mass-spring systems (include/mass_spring.h):
one-to-one ctypes wrappers of the ms_* entry points, a `MassSprings` owner of the
workspace, and a torch.autograd.Function.  Argument marshalling only: every step runs in
libmpm.so's kernels, and the binding raises (never falls back) when the library is
missing."""
from __future__ import annotations

import ctypes

import torch

from . import mpm as _mpm

EXPORTED = ["ms_workspace_bytes", "ms_create", "ms_forward", "ms_get_state", "ms_backward",
            "ms_sync", "ms_last_error", "ms_destroy"]


class MsDesc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("n_masses", ctypes.c_int32),
        ("n_springs", ctypes.c_int32),
        ("spring_a", ctypes.POINTER(ctypes.c_int32)),
        ("spring_b", ctypes.POINTER(ctypes.c_int32)),
        ("n_systems", ctypes.c_int32),
        ("stiffness", ctypes.c_float),
        ("damping", ctypes.c_float),
        ("dt", ctypes.c_float),
        ("mass", ctypes.c_float),
    ]


_sigs_done = False


def lib():
    global _sigs_done
    L = _mpm.lib()
    if not _sigs_done:
        vp, i32, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t
        D = ctypes.POINTER(MsDesc)
        sig = {
            "ms_workspace_bytes": (ctypes.c_int, [D, i32, ctypes.POINTER(sz)]),
            "ms_create": (ctypes.c_int, [D, vp, sz, i32, ctypes.POINTER(vp)]),
            "ms_forward": (ctypes.c_int, [vp, vp, vp, vp, i32, vp]),
            "ms_get_state": (ctypes.c_int, [vp, i32, vp, vp, vp]),
            "ms_backward": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp]),
            "ms_sync": (ctypes.c_int, [vp]),
            "ms_last_error": (ctypes.c_char_p, [vp]),
            "ms_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _sigs_done = True
    return L


def _check(rc, h=None):
    if rc != _mpm.MPM_OK:
        msg = lib().ms_last_error(h)
        raise _mpm.MPMError(rc, msg.decode() if msg else "")


def make_desc(dim, n_masses, springs, n_systems, stiffness, damping, dt, mass=1.0) -> MsDesc:
    springs = list(springs)
    a = (ctypes.c_int32 * max(len(springs), 1))(*[int(p[0]) for p in springs])
    b = (ctypes.c_int32 * max(len(springs), 1))(*[int(p[1]) for p in springs])
    d = MsDesc(int(dim), int(n_masses), len(springs),
               ctypes.cast(a, ctypes.POINTER(ctypes.c_int32)),
               ctypes.cast(b, ctypes.POINTER(ctypes.c_int32)), int(n_systems), float(stiffness),
               float(damping), float(dt), float(mass))
    d._keep = (a, b)
    return d


def ms_workspace_bytes(desc: MsDesc, steps: int) -> int:
    out = ctypes.c_size_t()
    _check(lib().ms_workspace_bytes(ctypes.byref(desc), int(steps), ctypes.byref(out)))
    return out.value


def _p(t):
    return _mpm._ptr(t)


class MassSprings:
    """n_systems independent mass-spring systems sharing a topology; the workspace is a
    torch CUDA tensor.  Arrays are [rows][n_systems] float32 (rows i*dim + c for masses,
    j for springs), as in include/mass_spring.h."""

    def __init__(self, dim, n_masses, springs, n_systems, stiffness, damping, dt, mass=1.0,
                 steps=1024, device="cuda"):
        self.dim, self.n, self.S = int(dim), int(n_masses), int(n_systems)
        self.springs = list(springs)
        self.device = torch.device(device)
        self.desc = make_desc(dim, n_masses, springs, n_systems, stiffness, damping, dt, mass)
        nbytes = ms_workspace_bytes(self.desc, steps)
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = (self.ws.data_ptr() + 255) // 256 * 256
        h = ctypes.c_void_p()
        _check(lib().ms_create(ctypes.byref(self.desc), base, nbytes, int(steps), ctypes.byref(h)))
        self.h = h
        self.steps = 0

    def _f(self, t):
        return None if t is None else t.to(self.device, torch.float32).contiguous()

    def forward(self, x0, v0, rest, steps, stream=None):
        self._keep = [self._f(x0), self._f(v0), self._f(rest)]
        _check(lib().ms_forward(self.h, *[_p(t) for t in self._keep], int(steps),
                                _mpm._stream(stream)), self.h)
        self.steps = int(steps)

    def state(self, t=None, stream=None):
        t = self.steps - 1 if t is None else int(t)
        x = torch.empty(self.n * self.dim, self.S, device=self.device)
        v = torch.empty_like(x)
        _check(lib().ms_get_state(self.h, t, _p(x), _p(v), _mpm._stream(stream)), self.h)
        return x, v

    def backward(self, dL_dx=None, dL_dv=None, stream=None):
        gx = torch.empty(self.n * self.dim, self.S, device=self.device)
        gv = torch.empty_like(gx)
        gl = torch.empty(max(len(self.springs), 1), self.S, device=self.device)
        seeds = [self._f(dL_dx), self._f(dL_dv)]
        _check(lib().ms_backward(self.h, _p(seeds[0]), _p(seeds[1]), _p(gx), _p(gv), _p(gl),
                                 _mpm._stream(stream)), self.h)
        return gx, gv, gl[:len(self.springs)]

    def sync(self):
        _check(lib().ms_sync(self.h), self.h)

    def close(self):
        if getattr(self, "h", None):
            lib().ms_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MassSpringRun(torch.autograd.Function):
    """(x0, v0, rest) -> (x_T, v_T) of `sys` (a MassSprings) over `steps` states."""

    @staticmethod
    def forward(ctx, sys: MassSprings, steps: int, x0, v0, rest):
        sys.forward(x0, v0, rest, steps)
        ctx.sys = sys
        return sys.state()

    @staticmethod
    def backward(ctx, gx, gv):
        g = ctx.sys.backward(gx.contiguous(), gv.contiguous())
        return None, None, g[0], g[1], g[2]


def triangle_area(x, target=0.2):
    """The example's loss on masses 0, 1, 2 of each system (dim 2; x: [n*2][S]): returns
    (area - target)^2 per system, differentiable in torch."""
    e1 = x[0:2] - x[2:4]
    e2 = x[0:2] - x[4:6]
    area = torch.abs(0.5 * (e1[0] * e2[1] - e1[1] * e2[0]))
    return (area - target) ** 2
