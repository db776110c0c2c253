"""The oracle's hand-derived adjoint against central finite differences of its forward
pass (whose arithmetic is pinned independently in test_oracle_pins.py).

Adjoint of one step = Appendix D.1's advance_grad (recompute grid, g2p.grad,
grid_op.grad, p2g.grad, actuation/stress adjoint); whole runs = the Section 3.2 tape.
Central differences with a relative step of 1e-6 in FP64 agree with an exact
gradient to ~1e-8 relative, so 1e-6 relative is the pass bar.
"""
import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(777)
EPS = 1e-6


def _params(dim, material, n_grid=16, walls=0, groups=0, basis=0, dt=1e-3,
            gravity=(0.0, -9.8, 0.0)):
    return oracle.make_params(dim, n_grid, dt, gravity, walls, material, 1.0,
                              n_groups=groups, n_basis=basis, act_period=7.0, act_phase=0.3)


def _scene(dim, n_side, n_grid, centre=0.5, rng=RNG, vel=0.5, cmag=2.0, fspread=0.15):
    dx = 1.0 / n_grid
    h = dx / 2
    idx = np.indices((n_side,) * dim).reshape(dim, -1)
    x = centre - n_side * h / 2 + (idx + 0.5) * h + 0.3 * h * rng.uniform(-1, 1, (dim, idx.shape[1]))
    k = x.shape[1]
    v = vel * rng.standard_normal((dim, k))
    C = cmag * rng.standard_normal((dim * dim, k))
    Fm = np.eye(dim)[None] + fspread * rng.standard_normal((k, dim, dim))
    F = np.ascontiguousarray(Fm.reshape(k, -1).T)
    mu = rng.uniform(200, 400, k)
    la = rng.uniform(100, 300, k)
    return [np.ascontiguousarray(a) for a in (x, v, C, F)], mu, la


CASES = [
    (2, oracle.FIXED_COROTATED, 0), (3, oracle.FIXED_COROTATED, 0),
    (2, oracle.NEO_HOOKEAN, 0), (3, oracle.NEO_HOOKEAN, 0),
    (3, oracle.FIXED_COROTATED, 3),  # with actuation
    (2, oracle.NEO_HOOKEAN, 3),
    (2, oracle.LIQUID, 0), (3, oracle.LIQUID, 0),
]


def _dot(a, b):
    return float(np.sum(np.asarray(a) * np.asarray(b)))


@pytest.mark.parametrize("dim,material,groups", CASES)
def test_step_adjoint_matches_fd(dim, material, groups):
    n_grid = 16
    basis = 2 if groups else 0
    P = _params(dim, material, n_grid, groups=groups, basis=basis)
    # the liquid's Tait law is ~gamma = 7 times stiffer than the solids near J = 1 and far
    # stiffer at J ~ 0.7: a smaller spread of F keeps the central differences of the
    # (large) functional above FP64 round-off
    (x, v, C, F), mu, la = _scene(dim, 3, n_grid,
                                  fspread=0.05 if material == oracle.LIQUID else 0.15)
    k = x.shape[1]
    grp = RNG.integers(0, groups, k).astype(np.int32) if groups else None
    w = RNG.standard_normal((groups, basis)) * 20 if groups else None
    t = 3
    state = oracle.pack_state(x, v, C, F)
    adj_next = RNG.standard_normal(state.size)

    def f(st, mu_, la_, w_):
        xs, vs, Cs, Fs = oracle.unpack_state(st, dim, k)
        out = oracle.step(P, t, *[np.ascontiguousarray(a) for a in (xs, vs, Cs, Fs)], mu_, la_,
                          grp, w_)
        return _dot(adj_next, oracle.pack_state(*out))

    adj, mub, lab, wb = oracle.step_adjoint(P, t, state, mu, la, adj_next, grp, w)
    # random directions in state space
    for _ in range(6):
        d = RNG.standard_normal(state.size)
        fd = (f(state + EPS * d, mu, la, w) - f(state - EPS * d, mu, la, w)) / (2 * EPS)
        assert abs(fd - _dot(adj, d)) <= 1e-6 * max(1.0, abs(fd)), (fd, _dot(adj, d))
    # every coordinate of the first particle (x, v, C, F)
    blk = 2 * dim + 2 * dim * dim
    for c in range(blk):
        e = np.zeros(state.size)
        e[c * k] = 1.0
        fd = (f(state + EPS * e, mu, la, w) - f(state - EPS * e, mu, la, w)) / (2 * EPS)
        assert abs(fd - adj[c * k]) <= 1e-6 * max(1.0, abs(fd)), (c, fd, adj[c * k])
    # material parameters (relative step) and actuation weights
    dm = RNG.standard_normal(k)
    em = EPS * 300
    fd_mu = (f(state, mu + em * dm, la, w) - f(state, mu - em * dm, la, w)) / (2 * em)
    assert abs(fd_mu - _dot(mub, dm)) <= 1e-6 * max(1.0, abs(fd_mu))
    fd_la = (f(state, mu, la + em * dm, w) - f(state, mu, la - em * dm, w)) / (2 * em)
    assert abs(fd_la - _dot(lab, dm)) <= 1e-6 * max(1.0, abs(fd_la))
    if groups:
        dw = RNG.standard_normal(w.shape)
        fd_w = (f(state, mu, la, w + EPS * dw) - f(state, mu, la, w - EPS * dw)) / (2 * EPS)
        assert abs(fd_w - _dot(wb, dw)) <= 1e-6 * max(1.0, abs(fd_w))


@pytest.mark.parametrize("dim,material", [(2, oracle.FIXED_COROTATED), (3, oracle.NEO_HOOKEAN),
                                          (3, oracle.FIXED_COROTATED)])
def test_step_adjoint_with_sticky_walls(dim, material):
    """Particles whose stencils reach the 3-node sticky wall (the select of Fig. 3)."""
    n_grid = 16
    P = _params(dim, material, n_grid, walls=3)
    dx = 1.0 / n_grid
    (x, v, C, F), mu, la = _scene(dim, 3, n_grid, centre=3.3 * dx + 0.75 * dx)
    k = x.shape[1]
    state = oracle.pack_state(x, v, C, F)
    adj_next = RNG.standard_normal(state.size)

    def f(st):
        out = oracle.step(P, 0, *[np.ascontiguousarray(a) for a in oracle.unpack_state(st, dim, k)],
                          mu, la)
        return _dot(adj_next, oracle.pack_state(*out))

    adj, *_ = oracle.step_adjoint(P, 0, state, mu, la, adj_next)
    for _ in range(6):
        d = RNG.standard_normal(state.size)
        fd = (f(state + EPS * d) - f(state - EPS * d)) / (2 * EPS)
        assert abs(fd - _dot(adj, d)) <= 1e-6 * max(1.0, abs(fd))


@pytest.mark.parametrize("dim,material,groups", [(2, oracle.FIXED_COROTATED, 0),
                                                 (3, oracle.NEO_HOOKEAN, 0),
                                                 (3, oracle.FIXED_COROTATED, 8)])
def test_run_gradient_matches_fd(dim, material, groups):
    """T-step reverse replay (the tape) against FD of a random linear functional."""
    n_grid = 16
    T = 12
    basis = 4 if groups else 0
    P = _params(dim, material, n_grid, walls=3, groups=groups, basis=basis, dt=5e-4)
    (x, v, C, F), mu, la = _scene(dim, 3 if dim == 3 else 4, n_grid, vel=0.3, cmag=0.5,
                                  fspread=0.05)
    k = x.shape[1]
    grp = (np.arange(k) % groups).astype(np.int32) if groups else None
    w = RNG.standard_normal((groups, basis)) * 30 if groups else None
    s0 = oracle.pack_state(x, v, C, F)
    c = RNG.standard_normal(s0.size)

    def L(st, mu_=mu, la_=la, w_=w):
        xs, vs, Cs, Fs = [np.ascontiguousarray(a) for a in oracle.unpack_state(st, dim, k)]
        return _dot(c, oracle.run(P, T, xs, vs, Cs, Fs, mu_, la_, grp, w_, keep_all=False))

    states = oracle.run(P, T, x, v, C, F, mu, la, grp, w)
    adj0, mub, lab, wb = oracle.grad(P, T, states, c, mu, la, grp, w)
    for _ in range(4):
        d = RNG.standard_normal(s0.size)
        fd = (L(s0 + EPS * d) - L(s0 - EPS * d)) / (2 * EPS)
        assert abs(fd - _dot(adj0, d)) <= 1e-6 * max(1.0, abs(fd))
    dm = RNG.standard_normal(k)
    em = EPS * 300
    fd = (L(s0, mu + em * dm) - L(s0, mu - em * dm)) / (2 * em)
    assert abs(fd - _dot(mub, dm)) <= 1e-6 * max(1.0, abs(fd))
    if groups:
        dw = RNG.standard_normal(w.shape)
        fd = (L(s0, w_=w + EPS * dw) - L(s0, w_=w - EPS * dw)) / (2 * EPS)
        assert abs(fd - _dot(wb, dw)) <= 1e-6 * max(1.0, abs(fd))


def test_lame_adjoint_matches_fd():
    E = RNG.uniform(5e2, 5e3, 50)
    nu = RNG.uniform(0.1, 0.4, 50)
    mb, lb = RNG.standard_normal(50), RNG.standard_normal(50)
    Eb, nub = oracle.lame_adjoint(E, nu, mb, lb)

    def f(E_, nu_):
        mu, la = oracle.lame(E_, nu_)
        return np.sum(mb * mu + lb * la)
    dE = RNG.standard_normal(50)
    fd = (f(E + 1e-3 * dE, nu) - f(E - 1e-3 * dE, nu)) / 2e-3
    assert abs(fd - np.sum(Eb * dE)) <= 1e-8 * abs(fd)
    dn = RNG.standard_normal(50)
    fd = (f(E, nu + 1e-7 * dn) - f(E, nu - 1e-7 * dn)) / 2e-7
    assert abs(fd - np.sum(nub * dn)) <= 1e-6 * abs(fd)


@pytest.mark.parametrize("kind", [oracle.LOSS_COM_TARGET, oracle.LOSS_COM_X_DISP])
def test_com_loss_seed_matches_fd(kind):
    dim, n = 3, 40
    xT = RNG.uniform(0.2, 0.8, (dim, n))
    x0 = RNG.uniform(0.2, 0.8, (dim, n))
    tgt = np.array([0.7, 0.5, 0.5])
    L, gT, g0 = oracle.com_loss(dim, kind, xT, x0, tgt)
    com = xT.mean(1)
    if kind == oracle.LOSS_COM_TARGET:
        assert abs(L - np.sum((com - tgt) ** 2)) < 1e-15
    else:
        assert abs(L + (com[0] - x0.mean(1)[0])) < 1e-15
    d = RNG.standard_normal((dim, n))
    fd = (oracle.com_loss(dim, kind, xT + 1e-6 * d, x0, tgt)[0]
          - oracle.com_loss(dim, kind, xT - 1e-6 * d, x0, tgt)[0]) / 2e-6
    assert abs(fd - np.sum(gT * d)) <= 1e-8
    fd = (oracle.com_loss(dim, kind, xT, x0 + 1e-6 * d, tgt)[0]
          - oracle.com_loss(dim, kind, xT, x0 - 1e-6 * d, tgt)[0]) / 2e-6
    assert abs(fd - np.sum(g0 * d)) <= 1e-8


def test_worked_example_sin_x_squared():
    """Appendix B's worked adjoint: y = sin(x^2) gives xbar = 2 x cos(x^2) ybar.  The
    FD harness used above must reproduce it (pins the harness, not the MPM path)."""
    xs = np.linspace(-1.3, 1.7, 16)
    fd = (np.sin((xs + EPS) ** 2) - np.sin((xs - EPS) ** 2)) / (2 * EPS)
    np.testing.assert_allclose(fd, 2 * xs * np.cos(xs ** 2), rtol=1e-8, atol=1e-9)


# ---------------------------------------------------------------------------
# per-particle materials (a solid and a liquid coupled through one grid)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_mixed_materials_reduce_to_the_uniform_ones(dim):
    """A MIXED step whose particles all carry material m is bitwise the uniform-m step."""
    n_grid = 16
    (x, v, C, F), mu, la = _scene(dim, 3, n_grid, fspread=0.05)
    k = x.shape[1]
    for m in (oracle.FIXED_COROTATED, oracle.NEO_HOOKEAN, oracle.LIQUID):
        Pu = _params(dim, m, n_grid)
        Pm = oracle.with_materials(_params(dim, oracle.MIXED, n_grid), np.full(k, m, np.int32))
        a = oracle.step(Pu, 2, x, v, C, F, mu, la)
        b = oracle.step(Pm, 2, x, v, C, F, mu, la)
        for u, w in zip(a, b):
            np.testing.assert_array_equal(u, w)


@pytest.mark.parametrize("dim", [2, 3])
def test_mixed_step_adjoint_matches_fd(dim):
    """Fixed-corotated and liquid particles interleaved in one grid: the step adjoint
    against central differences (state directions and every coordinate of two particles
    of different materials, and the material parameters)."""
    n_grid = 16
    P0 = _params(dim, oracle.MIXED, n_grid)
    (x, v, C, F), mu, la = _scene(dim, 3, n_grid, fspread=0.05)
    k = x.shape[1]
    mats = np.where(np.arange(k) % 2 == 0, oracle.FIXED_COROTATED, oracle.LIQUID).astype(np.int32)
    P = oracle.with_materials(P0, mats)
    t = 1
    state = oracle.pack_state(x, v, C, F)
    adj_next = RNG.standard_normal(state.size)

    def f(st, mu_=mu, la_=la):
        out = oracle.step(P, t, *[np.ascontiguousarray(a) for a in oracle.unpack_state(st, dim, k)],
                          mu_, la_)
        return _dot(adj_next, oracle.pack_state(*out))

    adj, mub, lab, _ = oracle.step_adjoint(P, t, state, mu, la, adj_next)
    for _ in range(4):
        d = RNG.standard_normal(state.size)
        fd = (f(state + EPS * d) - f(state - EPS * d)) / (2 * EPS)
        assert abs(fd - _dot(adj, d)) <= 1e-6 * max(1.0, abs(fd)), (fd, _dot(adj, d))
    blk = 2 * dim + 2 * dim * dim
    for p in (0, 1):  # one fixed-corotated, one liquid particle
        for c in range(blk):
            e = np.zeros(state.size)
            e[c * k + p] = 1.0
            fd = (f(state + EPS * e) - f(state - EPS * e)) / (2 * EPS)
            assert abs(fd - adj[c * k + p]) <= 1e-6 * max(1.0, abs(fd)), (p, c, fd)
    dm = RNG.standard_normal(k)
    em = EPS * 300
    fd_mu = (f(state, mu + em * dm, la) - f(state, mu - em * dm, la)) / (2 * em)
    assert abs(fd_mu - _dot(mub, dm)) <= 1e-6 * max(1.0, abs(fd_mu))
    fd_la = (f(state, mu, la + em * dm) - f(state, mu, la - em * dm)) / (2 * em)
    assert abs(fd_la - _dot(lab, dm)) <= 1e-6 * max(1.0, abs(fd_la))
