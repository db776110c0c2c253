"""FP64 CPU oracle for the differentiable MLS-MPM step -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  It shares no code with the CUDA path: the arithmetic lives in
``mpm_oracle.c`` (plain serial C, double precision), this module only marshals numpy
arrays through ctypes and loops over independent scenes.

What is pinned and where (each pin is a test under ``tests/test_oracle_*.py``):

* weights / P2G: partition of unity, zero first moment and the dx^2/4 second
  moment of the quadratic B-spline (closed forms);
* P2G + grid_op + G2P: exact affine-field reproduction and linear-momentum
  conservation with gravity and walls off;
* stress: Kirchhoff stress equals dpsi/dF F^T of the textbook energy densities
  (fixed-corotated, neo-Hookean), zero at rest;
* polar: agrees with the SVD-based polar factor of ``numpy.linalg.svd``;
* adjoint: every sub-stage and whole runs against central finite differences of
  the oracle's own forward pass (the adjoint is derived by hand, the forward is
  pinned independently above);
* actuation: closed-form special cases of the sine basis; the closed-loop controller
  against the definition of its inputs and a torch evaluation of its MLP, invariants,
  and finite differences (test_oracle_controller.py).

Sections of the paper followed: Section 3.2 (tape), Section 4.1 and Appendix D
(diffmpm's advance / advance_grad), Appendix C (polar/SVD with a custom gradient).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpm_oracle.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_LIB_OMP = os.path.join(_LIBDIR, "liboracle_omp.so")

OK, ERR_ARG, ERR_MEM, ERR_OOB, ERR_DOMAIN = 0, 1, 2, 3, 4
FIXED_COROTATED, NEO_HOOKEAN, NO_ELASTICITY, LIQUID, MIXED = 0, 1, 2, 3, 4
LOSS_COM_TARGET, LOSS_COM_X_DISP = 0, 1

_lock = threading.Lock()
_lib = None


class OracleError(RuntimeError):
    pass


class Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("n_grid", ctypes.c_int32),
        ("dt", ctypes.c_double),
        ("gravity", ctypes.c_double * 3),
        ("wall_cells", ctypes.c_int32),
        ("material", ctypes.c_int32),
        ("rho", ctypes.c_double),
        ("n_groups", ctypes.c_int32),
        ("n_basis", ctypes.c_int32),
        ("act_period", ctypes.c_double),
        ("act_phase", ctypes.c_double),
        ("particle_material", ctypes.c_void_p),
        ("ctrl_hidden", ctypes.c_int32),
        ("ctrl_scale", ctypes.c_double),
    ]


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile mpm_oracle.c into _build/liboracle.so (plain C, -O3, no -march), or with
    openmp=True into _build/liboracle_omp.so: the same source with -fopenmp, whose particle
    loops run on all host cores (per-thread private grids summed in thread order)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    out = _LIB_OMP if openmp else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O3", "-std=c99", "-fPIC", "-shared"] + (["-fopenmp"] if openmp else [])
            + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def lib():
    """Load the oracle library (ORACLE_LIB overrides the path; the mutation tests use
    it to load deliberately broken copies of the oracle).  ORACLE_OPENMP=1 loads the
    OpenMP build instead of the serial one (a process uses one of the two)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("ORACLE_LIB")
            if not path:
                path = build(openmp=os.environ.get("ORACLE_OPENMP", "0") == "1")
            L = ctypes.CDLL(path)
            P = ctypes.POINTER(Params)
            d = ctypes.POINTER(ctypes.c_double)
            i32 = ctypes.POINTER(ctypes.c_int32)
            I64, I = ctypes.c_int64, ctypes.c_int
            D = ctypes.c_double
            sig = {
                "orc_lame": (None, [I64, d, d, d, d]),
                "orc_lame_adjoint": (None, [I64, d, d, d, d, d, d]),
                "orc_polar": (I, [I, d, d, d]),
                "orc_polar_adjoint": (I, [I, d, d, d]),
                "orc_actuation": (D, [P, d, I, I]),
                "orc_kirchhoff": (I, [P, d, D, D, D, I, d]),
                "orc_kirchhoff_adjoint": (I, [P, d, D, D, D, I, d, d, d, d, d]),
                "orc_p2g": (I, [P, I64, I, d, d, d, d, d, d, i32, d, d, d]),
                "orc_grid_update": (None, [P, d, d, d]),
                "orc_g2p": (I, [P, I64, d, d, d, d, d, d, d]),
                "orc_step": (I, [P, I64, I, d, d, d, d, d, d, i32, d, d, d, d, d]),
                "orc_run": (I, [P, I64, I, d, d, i32, d, d]),
                "orc_step_adjoint": (I, [P, I64, I, d, d, d, d, d, d, i32, d,
                                         d, d, d, d, d, d, d, d, d, d, d]),
                "orc_grad": (I, [P, I64, I, d, d, i32, d, d, d, d, d, d]),
                "orc_com_loss": (I, [I, I64, I, d, d, d, d, d, d]),
                "orc_ms_forward": (I, [I, I, I, i32, i32, d, D, D, D, D, I, d, d]),
                "orc_ms_backward": (I, [I, I, I, i32, i32, d, D, D, D, D, I, d, d, d, d]),
                "orc_ms_area_loss": (I, [I, d, D, d, d]),
                "orc_ctrl_n_inputs": (I, [P]),
                "orc_ctrl_n_params": (I64, [P]),
                "orc_controller": (I, [P, d, I64, I, d, d, i32, d, d]),
                "orc_threads": (I, [I]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


# ----------------------------------------------------------------------------
# marshalling helpers
# ----------------------------------------------------------------------------

def _d(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous, (a.dtype, a.flags)
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    if a is None:
        return None
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != OK:
        names = {ERR_ARG: "bad argument", ERR_MEM: "out of memory",
                 ERR_OOB: "particle stencil left the grid",
                 ERR_DOMAIN: "det F <= 0 or non-finite value"}
        raise OracleError(f"{what}: {names.get(rc, rc)}")


def make_params(dim, n_grid, dt, gravity=(0.0, -9.8, 0.0), wall_cells=3,
                material=FIXED_COROTATED, rho=1.0, n_groups=0, n_basis=0,
                act_period=50.0, act_phase=0.0, ctrl_hidden=0, ctrl_scale=1.0) -> Params:
    g = list(gravity) + [0.0] * (3 - len(gravity))
    p = Params(int(dim), int(n_grid), float(dt), (ctypes.c_double * 3)(*g[:3]),
               int(wall_cells), int(material), float(rho), int(n_groups), int(n_basis),
               float(act_period), float(act_phase))
    p.ctrl_hidden = int(ctrl_hidden)
    p.ctrl_scale = float(ctrl_scale)
    return p


def threads(n: int = 0) -> int:
    """Threads of the oracle's particle loops (1 for the serial build); n > 0 sets it."""
    return int(lib().orc_threads(int(n)))


def n_act_params(params) -> int:
    """Actuation parameters per scene: G*K sine weights (open loop) or the controller's
    theta (closed loop)."""
    if params.n_groups <= 0:
        return 0
    if params.ctrl_hidden > 0:
        return int(lib().orc_ctrl_n_params(ctypes.byref(params)))
    return params.n_groups * params.n_basis


def controller(params, theta, t, x, v, grp):
    """The closed-loop controller at step t on state (x, v): (act[G], inputs u[n_in])."""
    x, v, theta = _f64(x), _f64(v), _f64(theta).reshape(-1)
    n = x.shape[-1]
    act = np.zeros(params.n_groups)
    u = np.zeros(int(lib().orc_ctrl_n_inputs(ctypes.byref(params))))
    _check(lib().orc_controller(ctypes.byref(params), _d(theta), n, int(t), _d(x), _d(v),
                                _i(_grp(grp, n)), _d(act), _d(u)), "controller")
    return act, u


def with_materials(params: Params, material) -> Params:
    """A copy of params whose per-particle material array (MIXED scenes) is `material`
    (int32, indexed like mu and la; kept alive by the returned object)."""
    q = Params.from_buffer_copy(params)
    arr = np.ascontiguousarray(material, dtype=np.int32)
    q.particle_material = arr.ctypes.data
    q._material_ref = arr
    return q


def params_from_desc(desc: dict) -> Params:
    return make_params(desc["dim"], desc["n_grid"], desc["dt"], desc["gravity"],
                       desc["wall_cells"], desc["material"], desc["rho"],
                       desc.get("n_groups", 0), desc.get("n_basis", 0),
                       desc.get("act_period", 50.0), desc.get("act_phase", 0.0),
                       desc.get("ctrl_hidden", 0), desc.get("ctrl_scale", 1.0))


def state_block_len(dim, n):
    return (2 * dim + 2 * dim * dim) * n


def pack_state(x, v, C, F):
    """Concatenate component-major x[d,n], v[d,n], C[d*d,n], F[d*d,n] into one block."""
    return np.ascontiguousarray(np.concatenate(
        [np.asarray(a, np.float64).reshape(-1) for a in (x, v, C, F)]))


def unpack_state(block, dim, n):
    d = dim
    o = 0
    out = []
    for rows in (d, d, d * d, d * d):
        out.append(block[o:o + rows * n].reshape(rows, n))
        o += rows * n
    return tuple(out)


# ----------------------------------------------------------------------------
# thin wrappers of the C functions
# ----------------------------------------------------------------------------

def lame(E, nu):
    E, nu = _f64(E), _f64(nu)
    mu, la = np.empty_like(E), np.empty_like(E)
    lib().orc_lame(E.size, _d(E), _d(nu), _d(mu), _d(la))
    return mu, la


def lame_adjoint(E, nu, mubar, labar):
    E, nu, mubar, labar = map(_f64, (E, nu, mubar, labar))
    Eb, nub = np.empty_like(E), np.empty_like(E)
    lib().orc_lame_adjoint(E.size, _d(E), _d(nu), _d(mubar), _d(labar), _d(Eb), _d(nub))
    return Eb, nub


def polar(F):
    F = _f64(F)
    d = F.shape[0]
    R, S = np.empty_like(F), np.empty_like(F)
    _check(lib().orc_polar(d, _d(F), _d(R), _d(S)), "polar")
    return R, S


def polar_adjoint(F, Rbar):
    F, Rbar = _f64(F), _f64(Rbar)
    Fb = np.empty_like(F)
    _check(lib().orc_polar_adjoint(F.shape[0], _d(F), _d(Rbar), _d(Fb)), "polar_adjoint")
    return Fb


def actuation(params, w, g, t):
    w = _f64(w).reshape(-1)
    return lib().orc_actuation(ctypes.byref(params), _d(w), int(g), int(t))


def kirchhoff(params, F, mu, la, act=0.0, axis=0):
    F = _f64(F)
    tau = np.empty_like(F)
    _check(lib().orc_kirchhoff(ctypes.byref(params), _d(F), mu, la, act, axis, _d(tau)),
           "kirchhoff")
    return tau


def kirchhoff_adjoint(params, F, mu, la, act, axis, taubar):
    F, taubar = _f64(F), _f64(taubar)
    Fb = np.empty_like(F)
    mb, lb, ab = (ctypes.c_double(), ctypes.c_double(), ctypes.c_double())
    rc = lib().orc_kirchhoff_adjoint(
        ctypes.byref(params), _d(F), mu, la, act, axis, _d(taubar), _d(Fb),
        ctypes.cast(ctypes.byref(mb), ctypes.POINTER(ctypes.c_double)),
        ctypes.cast(ctypes.byref(lb), ctypes.POINTER(ctypes.c_double)),
        ctypes.cast(ctypes.byref(ab), ctypes.POINTER(ctypes.c_double)))
    _check(rc, "kirchhoff_adjoint")
    return Fb, mb.value, lb.value, ab.value


def _grp(grp, n):
    if grp is None:
        return None
    return np.ascontiguousarray(grp, dtype=np.int32).reshape(n)


def p2g(params, t, x, v, C, F, mu, la, grp=None, w=None):
    x, v, C, F, mu, la = map(_f64, (x, v, C, F, mu, la))
    n = mu.size
    nn = params.n_grid ** params.dim
    gm = np.empty(nn)
    gp = np.empty(nn * params.dim)
    w = _f64(w).reshape(-1) if w is not None else None
    _check(lib().orc_p2g(ctypes.byref(params), n, t, _d(x), _d(v), _d(C), _d(F), _d(mu),
                         _d(la), _i(_grp(grp, n)), _d(w), _d(gm), _d(gp)), "p2g")
    return gm, gp.reshape(nn, params.dim)


def grid_update(params, gm, gp):
    gm, gp = _f64(gm), _f64(gp)
    gu = np.empty_like(gp)
    lib().orc_grid_update(ctypes.byref(params), _d(gm), _d(gp), _d(gu))
    return gu


def g2p(params, x, F, gu):
    x, F, gu = map(_f64, (x, F, gu))
    n = x.shape[-1]
    x1, v1 = np.empty_like(x), np.empty_like(x)
    C1, F1 = np.empty_like(F), np.empty_like(F)
    _check(lib().orc_g2p(ctypes.byref(params), n, _d(x), _d(F), _d(gu), _d(x1), _d(v1),
                         _d(C1), _d(F1)), "g2p")
    return x1, v1, C1, F1


def step(params, t, x, v, C, F, mu, la, grp=None, w=None):
    x, v, C, F, mu, la = map(_f64, (x, v, C, F, mu, la))
    n = mu.size
    out = [np.empty_like(x), np.empty_like(v), np.empty_like(C), np.empty_like(F)]
    w = _f64(w).reshape(-1) if w is not None else None
    _check(lib().orc_step(ctypes.byref(params), n, t, _d(x), _d(v), _d(C), _d(F), _d(mu),
                          _d(la), _i(_grp(grp, n)), _d(w), *[_d(o) for o in out]), "step")
    return tuple(out)


def run(params, T, x0, v0, C0, F0, mu, la, grp=None, w=None, keep_all=True):
    """T steps from the initial state; returns states[T+1, block] (or the last one)."""
    mu, la = _f64(mu), _f64(la)
    n = mu.size
    blk = state_block_len(params.dim, n)
    states = np.empty((T + 1, blk))
    states[0] = pack_state(x0, v0, C0, F0)
    w = _f64(w).reshape(-1) if w is not None else None
    _check(lib().orc_run(ctypes.byref(params), n, T, _d(mu), _d(la), _i(_grp(grp, n)), _d(w),
                         _d(states)), "run")
    return states if keep_all else states[-1].copy()


def step_adjoint(params, t, state, mu, la, adj_next, grp=None, w=None):
    """Adjoint of one step: returns (adj_state_s, mubar, labar, wbar)."""
    mu, la = _f64(mu), _f64(la)
    n = mu.size
    d = params.dim
    xs, vs, Cs, Fs = [np.ascontiguousarray(a) for a in unpack_state(_f64(state), d, n)]
    xb1, vb1, Cb1, Fb1 = [np.ascontiguousarray(a) for a in unpack_state(_f64(adj_next), d, n)]
    out = [np.empty_like(xs), np.empty_like(vs), np.empty_like(Cs), np.empty_like(Fs)]
    mub, lab = np.zeros(n), np.zeros(n)
    G, K = params.n_groups, params.n_basis
    nw = n_act_params(params)
    wb = np.zeros(max(nw, 1))
    w = _f64(w).reshape(-1) if w is not None else None
    _check(lib().orc_step_adjoint(ctypes.byref(params), n, t, _d(xs), _d(vs), _d(Cs), _d(Fs),
                                  _d(mu), _d(la), _i(_grp(grp, n)), _d(w), _d(xb1), _d(vb1),
                                  _d(Cb1), _d(Fb1), *[_d(o) for o in out], _d(mub), _d(lab),
                                  _d(wb)), "step_adjoint")
    return pack_state(*out), mub, lab, _shape_wbar(params, wb[:nw])


def grad(params, T, states, adj_T, mu, la, grp=None, w=None):
    """Reverse replay of T steps.  Returns (adj_0 block, mubar, labar, wbar[G,K])."""
    mu, la = _f64(mu), _f64(la)
    n = mu.size
    adj = _f64(adj_T).copy()
    mub, lab = np.zeros(n), np.zeros(n)
    nw = n_act_params(params)
    wb = np.zeros(max(nw, 1))
    w = _f64(w).reshape(-1) if w is not None else None
    states = np.ascontiguousarray(states, dtype=np.float64)
    _check(lib().orc_grad(ctypes.byref(params), n, T, _d(mu), _d(la), _i(_grp(grp, n)), _d(w),
                          _d(states), _d(adj), _d(mub), _d(lab), _d(wb)), "grad")
    return adj, mub, lab, _shape_wbar(params, wb[:nw])


def _shape_wbar(params, wb):
    """dL/dw as [G, K] (open loop) or dL/dtheta flat (closed loop)."""
    if params.ctrl_hidden > 0 or wb.size == 0:
        return wb
    return wb.reshape(params.n_groups, params.n_basis)


def com_loss(dim, kind, xT, x0, target=None):
    xT, x0 = _f64(xT), _f64(x0)
    n = xT.shape[-1]
    tgt = _f64(np.zeros(3) if target is None else np.asarray(target, np.float64))
    loss = ctypes.c_double()
    xTb, x0b = np.empty_like(xT), np.empty_like(x0)
    _check(lib().orc_com_loss(dim, n, kind, _d(xT), _d(x0), _d(tgt),
                              ctypes.cast(ctypes.byref(loss), ctypes.POINTER(ctypes.c_double)),
                              _d(xTb), _d(x0b)), "com_loss")
    return loss.value, xTb, x0b


# ----------------------------------------------------------------------------
# whole-scene drivers (a scene is the dict made by the seeded input generator)
# ----------------------------------------------------------------------------

def _scene_slices(scene):
    offs = np.concatenate([[0], np.cumsum(scene["desc"]["n_particles"])])
    return [slice(int(offs[i]), int(offs[i + 1])) for i in range(len(offs) - 1)]


def _scene_inputs(scene, sl, si):
    a = scene["arrays"]
    x0, v0 = a["x0"][:, sl], a["v0"][:, sl]
    C0, F0 = a["C0"][:, sl], a["F0"][:, sl]
    mu, la = lame(a["E"][sl], a["nu"][sl])
    grp = a["group"][sl] if scene["desc"].get("n_groups", 0) > 0 else None
    w = a["w"][si] if scene["desc"].get("n_groups", 0) > 0 else None
    return x0, v0, C0, F0, mu, la, grp, w


def scene_params(scene, sl):
    """Parameters of the scene slice sl (with its per-particle materials when MIXED)."""
    p = params_from_desc(scene["desc"])
    if scene["desc"]["material"] == MIXED:
        p = with_materials(p, scene["arrays"]["material"][sl])
    return p


def simulate(scene, T, keep_all=False):
    """Forward T steps of every scene; returns a list of per-scene state blocks
    (states[T+1] per scene if keep_all, else the final block)."""
    out = []
    for si, sl in enumerate(_scene_slices(scene)):
        x0, v0, C0, F0, mu, la, grp, w = _scene_inputs(scene, sl, si)
        out.append(run(scene_params(scene, sl), T, x0, v0, C0, F0, mu, la, grp, w,
                       keep_all=keep_all))
    return out


def loss_and_grad(scene, T):
    """Loss (sum over scenes) and its gradient w.r.t. the initial state, E, nu and w,
    all in FP64.  Returns dict with loss, per-scene losses, final states, gx0, gv0,
    gC0, gF0 (component-major, concatenated like the inputs), gE, gnu, gw[S,G,K]."""
    desc = scene["desc"]
    d = desc["dim"]
    a = scene["arrays"]
    N = int(sum(desc["n_particles"]))
    g = {k: np.zeros((r, N)) for k, r in (("gx0", d), ("gv0", d), ("gC0", d * d),
                                          ("gF0", d * d))}
    gE, gnu = np.zeros(N), np.zeros(N)
    S = len(desc["n_particles"])
    G, K = desc.get("n_groups", 0), desc.get("n_basis", 0)
    nw = n_act_params(params_from_desc(desc))
    gw = np.zeros((S, nw)) if desc.get("ctrl_hidden", 0) > 0 else np.zeros((S, G, K))
    losses, finals = [], []
    for si, sl in enumerate(_scene_slices(scene)):
        x0, v0, C0, F0, mu, la, grp, w = _scene_inputs(scene, sl, si)
        n = mu.size
        p = scene_params(scene, sl)
        states = run(p, T, x0, v0, C0, F0, mu, la, grp, w, keep_all=True)
        xT = unpack_state(states[-1], d, n)[0]
        tgt = a["target"][si] if "target" in a else None
        L, xTb, x0b = com_loss(d, desc["loss_kind"], xT, x0, tgt)
        adjT = pack_state(xTb, np.zeros((d, n)), np.zeros((d * d, n)), np.zeros((d * d, n)))
        adj0, mub, lab, wb = grad(p, T, states, adjT, mu, la, grp, w)
        gx, gv, gC, gF = unpack_state(adj0, d, n)
        g["gx0"][:, sl] = gx + x0b
        g["gv0"][:, sl] = gv
        g["gC0"][:, sl] = gC
        g["gF0"][:, sl] = gF
        eb, nb = lame_adjoint(a["E"][sl], a["nu"][sl], mub, lab)
        gE[sl], gnu[sl] = eb, nb
        if nw:
            gw[si] = wb
        losses.append(L)
        finals.append(states[-1].copy())
        del states
    return dict(loss=float(sum(losses)), losses=losses, finals=finals, gE=gE, gnu=gnu, gw=gw,
                **g)


# ----------------------------------------------------------------------------
# mass-spring system (Section 2's example, Section 3's tape demonstration)
# ----------------------------------------------------------------------------

def ms_forward(x0, v0, springs, l0, k, alpha, dt, m, steps):
    """States 0..steps-1 of one system: (x, v) each [steps, n, dim].  springs: (a, b) pairs."""
    x0, v0 = _f64(x0), _f64(v0)
    n, dim = x0.shape
    sp = np.ascontiguousarray(springs, dtype=np.int32).reshape(-1, 2)
    sa, sb = np.ascontiguousarray(sp[:, 0]), np.ascontiguousarray(sp[:, 1])
    x = np.zeros((steps, n, dim))
    v = np.zeros((steps, n, dim))
    x[0], v[0] = x0, v0
    _check(lib().orc_ms_forward(dim, n, len(sa), _i(sa), _i(sb), _d(_f64(l0)), float(k),
                                float(alpha), float(dt), float(m), int(steps), _d(x), _d(v)),
           "ms_forward")
    return x, v


def ms_backward(x, springs, l0, k, alpha, dt, m, xb_T, vb_T):
    """Reverse of ms_forward over the recorded positions x [steps, n, dim]: returns
    (dL/dx0, dL/dv0, dL/dl0) given dL/dx, dL/dv of the last state."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    steps, n, dim = x.shape
    sp = np.ascontiguousarray(springs, dtype=np.int32).reshape(-1, 2)
    sa, sb = np.ascontiguousarray(sp[:, 0]), np.ascontiguousarray(sp[:, 1])
    xb = _f64(xb_T).copy()
    vb = _f64(vb_T).copy()
    l0b = np.zeros(len(sa))
    _check(lib().orc_ms_backward(dim, n, len(sa), _i(sa), _i(sb), _d(_f64(l0)), float(k),
                                 float(alpha), float(dt), float(m), int(steps), _d(x), _d(xb),
                                 _d(vb), _d(l0b)), "ms_backward")
    return xb, vb, l0b


def ms_area_loss(x, target=0.2):
    """(L, dL/dx) of the example's triangle-area loss on masses 0, 1, 2 (dim 2)."""
    x = _f64(x)
    loss = ctypes.c_double()
    xb = np.zeros_like(x)
    _check(lib().orc_ms_area_loss(x.shape[0], _d(x), float(target),
                                  ctypes.cast(ctypes.byref(loss), ctypes.POINTER(ctypes.c_double)),
                                  _d(xb)), "ms_area_loss")
    return loss.value, xb
