"""Pins of the oracle's closed-loop controller (the neural-network controllers of
Section 4.1: the current state's sensors feed a small MLP whose outputs actuate the
groups at every step).

* forward: the controller's inputs against their plain definition (group means of the
  state, computed here with numpy masks) and its output against the same MLP evaluated
  by torch.nn.functional (a library routine, not the oracle's C);
* invariants: a rigid translation of the body or a permutation of its particles leaves
  the actuation unchanged; a zero controller actuates nothing (the run equals the
  unactuated run exactly);
* adjoint: dL/dtheta and the sensor terms of dL/dx, dL/dv against central finite
  differences of whole runs (the forward pass being pinned above).
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

RNG = np.random.default_rng(4242)
EPS = 1e-6


def _params(dim, G, K, H, scale, n_grid=16, dt=5e-4, walls=3, material=oracle.FIXED_COROTATED):
    return oracle.make_params(dim, n_grid, dt, (0.0, -9.8, 0.0), walls, material, 1.0,
                              n_groups=G, n_basis=K, act_period=9.0, act_phase=0.2,
                              ctrl_hidden=H, ctrl_scale=scale)


def _body(dim, n_side, n_grid, rng, vel=0.3, cmag=0.5, fspread=0.05):
    dx = 1.0 / n_grid
    h = dx / 2
    idx = np.indices((n_side,) * dim).reshape(dim, -1)
    x = 0.5 - n_side * h / 2 + (idx + 0.5) * h + 0.3 * h * rng.uniform(-1, 1, (dim, idx.shape[1]))
    k = x.shape[1]
    v = vel * rng.standard_normal((dim, k))
    C = cmag * rng.standard_normal((dim * dim, k))
    Fm = np.eye(dim)[None] + fspread * rng.standard_normal((k, dim, dim))
    F = np.ascontiguousarray(Fm.reshape(k, -1).T)
    mu = rng.uniform(200, 400, k)
    la = rng.uniform(100, 300, k)
    return [np.ascontiguousarray(a) for a in (x, v, C, F)], mu, la


def _theta(P, rng, s=1.0):
    return s * rng.standard_normal(oracle.n_act_params(P))


def _split(P, th):
    dim, G, K, H = P.dim, P.n_groups, P.n_basis, P.ctrl_hidden
    n_in = K + 2 * dim * G
    o = 0
    W1 = th[o:o + H * n_in].reshape(H, n_in); o += H * n_in
    b1 = th[o:o + H]; o += H
    W2 = th[o:o + G * H].reshape(G, H); o += G * H
    b2 = th[o:o + G]; o += G
    assert o == th.size
    return W1, b1, W2, b2


@pytest.mark.parametrize("dim,G,K,H", [(2, 4, 2, 6), (3, 5, 3, 8), (3, 8, 0, 4)])
def test_controller_forward_against_definition_and_torch(dim, G, K, H):
    P = _params(dim, G, K, H, scale=35.0)
    (x, v, _, _), _, _ = _body(dim, 5 if dim == 2 else 4, 16, RNG)
    n = x.shape[1]
    grp = RNG.integers(-1, G, n).astype(np.int32)   # -1: particles in no group
    grp[grp == G - 1] = 0                            # group G-1 left empty: reads zeros
    th = _theta(P, RNG)
    t = 5
    act, u = oracle.controller(P, th, t, x, v, grp)
    # inputs from their definition
    want = [np.sin(2 * np.pi * k * t / 9.0 + 0.2) for k in range(1, K + 1)]
    com = x.mean(axis=1)
    for g in range(G):
        m = grp == g
        if m.any():
            want += list(x[:, m].mean(axis=1) - com) + list(v[:, m].mean(axis=1))
        else:
            want += [0.0] * (2 * dim)
    np.testing.assert_allclose(u, want, rtol=0, atol=1e-14)
    # the MLP through torch.nn.functional
    W1, b1, W2, b2 = [torch.as_tensor(a) for a in _split(P, th)]
    ut = torch.as_tensor(np.asarray(want))
    h = torch.tanh(torch.nn.functional.linear(ut, W1, b1))
    a = 35.0 * torch.tanh(torch.nn.functional.linear(h, W2, b2))
    np.testing.assert_allclose(act, a.numpy(), rtol=1e-13, atol=1e-12)


def test_controller_is_translation_and_permutation_invariant():
    P = _params(3, 4, 2, 6, scale=20.0)
    (x, v, _, _), _, _ = _body(3, 4, 16, RNG)
    n = x.shape[1]
    grp = (np.arange(n) % 4).astype(np.int32)
    th = _theta(P, RNG)
    a0, _ = oracle.controller(P, th, 3, x, v, grp)
    a1, _ = oracle.controller(P, th, 3, x + np.array([[0.07], [-0.03], [0.11]]), v, grp)
    np.testing.assert_allclose(a1, a0, rtol=0, atol=1e-12)
    perm = RNG.permutation(n)
    a2, _ = oracle.controller(P, th, 3, np.ascontiguousarray(x[:, perm]),
                              np.ascontiguousarray(v[:, perm]), grp[perm])
    np.testing.assert_allclose(a2, a0, rtol=0, atol=1e-12)
    # but not invariant to moving one group against the others
    x3 = x.copy()
    x3[:, grp == 1] += 0.02
    a3, _ = oracle.controller(P, th, 3, x3, v, grp)
    assert np.max(np.abs(a3 - a0)) > 1e-3


@pytest.mark.parametrize("dim", [2, 3])
def test_zero_controller_equals_unactuated_run(dim):
    P = _params(dim, 4, 2, 5, scale=50.0)
    P0 = _params(dim, 0, 0, 0, scale=1.0)
    (x, v, C, F), mu, la = _body(dim, 5 if dim == 2 else 3, 16, RNG)
    grp = (np.arange(x.shape[1]) % 4).astype(np.int32)
    th = np.zeros(oracle.n_act_params(P))
    a = oracle.run(P, 8, x, v, C, F, mu, la, grp, th, keep_all=False)
    b = oracle.run(P0, 8, x, v, C, F, mu, la, keep_all=False)
    assert np.array_equal(a, b)


def _dot(a, b):
    return float(np.sum(np.asarray(a) * np.asarray(b)))


@pytest.mark.parametrize("dim,material", [(2, oracle.FIXED_COROTATED), (3, oracle.NEO_HOOKEAN),
                                          (3, oracle.FIXED_COROTATED)])
def test_controller_run_gradient_matches_fd(dim, material):
    """T steps with the controller in the loop: a random linear functional of the final
    state against central differences in theta, in the state (random directions and one
    group moved against the rest, which only the sensors see) and in v0."""
    G, K, H = 4, 2, 6
    P = _params(dim, G, K, H, scale=40.0, material=material)
    T = 10
    (x, v, C, F), mu, la = _body(dim, 4 if dim == 2 else 3, 16, RNG)
    k = x.shape[1]
    grp = (np.arange(k) % G).astype(np.int32)
    grp[0] = -1  # one particle in no group
    th = _theta(P, RNG, 0.7)
    s0 = oracle.pack_state(x, v, C, F)
    c = RNG.standard_normal(s0.size)

    def L(st, th_=th):
        xs, vs, Cs, Fs = [np.ascontiguousarray(a) for a in oracle.unpack_state(st, dim, k)]
        return _dot(c, oracle.run(P, T, xs, vs, Cs, Fs, mu, la, grp, th_, keep_all=False))

    states = oracle.run(P, T, x, v, C, F, mu, la, grp, th)
    adj0, mub, lab, thb = oracle.grad(P, T, states, c, mu, la, grp, th)
    assert thb.shape == th.shape
    for _ in range(3):
        d = RNG.standard_normal(th.size)
        fd = (L(s0, th + EPS * d) - L(s0, th - EPS * d)) / (2 * EPS)
        assert abs(fd - _dot(thb, d)) <= 1e-6 * max(1.0, abs(fd)), (fd, _dot(thb, d))
    for _ in range(3):
        d = RNG.standard_normal(s0.size)
        fd = (L(s0 + EPS * d) - L(s0 - EPS * d)) / (2 * EPS)
        assert abs(fd - _dot(adj0, d)) <= 1e-6 * max(1.0, abs(fd)), (fd, _dot(adj0, d))
    # group 2 displaced / accelerated against the body: what the sensors measure
    for block in (0, 1):  # x rows, v rows
        d = np.zeros(s0.size)
        for a in range(dim):
            d[(block * dim + a) * k:(block * dim + a + 1) * k][grp == 2] = RNG.standard_normal()
        fd = (L(s0 + EPS * d) - L(s0 - EPS * d)) / (2 * EPS)
        assert abs(fd - _dot(adj0, d)) <= 1e-6 * max(1.0, abs(fd)), (block, fd, _dot(adj0, d))


def test_sensor_path_carries_gradient():
    """The sensor terms are a visible part of dL/dx0 (so a dropped term cannot hide below
    the finite-difference bar): compare against the same run with the state columns of
    W1 zeroed, which makes the controller open-loop."""
    dim, G, K, H = 2, 4, 2, 6
    P = _params(dim, G, K, H, scale=40.0)
    (x, v, C, F), mu, la = _body(dim, 4, 16, RNG)
    k = x.shape[1]
    grp = (np.arange(k) % G).astype(np.int32)
    th = _theta(P, RNG, 0.7)
    c = RNG.standard_normal(oracle.pack_state(x, v, C, F).size)
    states = oracle.run(P, 8, x, v, C, F, mu, la, grp, th)
    adj_a, *_ = oracle.grad(P, 8, states, c, mu, la, grp, th)
    th_open = th.copy()
    W1 = th_open[:H * (K + 2 * dim * G)].reshape(H, -1)
    W1[:, K:] = 0.0
    states_o = oracle.run(P, 8, x, v, C, F, mu, la, grp, th_open)
    adj_o, *_ = oracle.grad(P, 8, states_o, c, mu, la, grp, th_open)
    xv = slice(0, 2 * dim * k)
    rel = np.linalg.norm(adj_a[xv] - adj_o[xv]) / np.linalg.norm(adj_o[xv])
    assert rel > 1e-3, rel
