"""Pins of the FP64 oracle against closed forms, invariants and independent routes.

None of these compares the oracle with itself: each checks a property that the
mathematics of MLS-MPM (Section 4.1 / Appendix D) or of the polar decomposition
(Appendix C) fixes, so that a dropped term, a wrong sign or index, or a transposed
operand in the oracle fails at least one of them.
"""
import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(12345)


def _params(dim, n_grid=16, dt=1e-3, gravity=(0.0, -9.8, 0.0), walls=0,
            material=oracle.FIXED_COROTATED, **kw):
    return oracle.make_params(dim, n_grid, dt, gravity, walls, material, 1.0, **kw)


def _node_positions(dim, n):
    idx = np.indices((n,) * dim).reshape(dim, -1).T  # flat order matches the oracle
    return idx / n


def _random_F(dim, k, spread=0.2, rng=RNG):
    Fs = []
    while len(Fs) < k:
        F = np.eye(dim) + spread * rng.standard_normal((dim, dim))
        if np.linalg.det(F) > 0.2:
            Fs.append(F)
    return np.array(Fs)


def _random_rotation(dim, rng=RNG):
    Q, R = np.linalg.qr(rng.standard_normal((dim, dim)))
    Q = Q @ np.diag(np.sign(np.diag(R)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    return Q


def _soa(mats):
    """list of (d,d) -> component-major (d*d, n)"""
    m = np.asarray(mats)
    return np.ascontiguousarray(m.reshape(m.shape[0], -1).T)


# ---------------------------------------------------------------------------
# quadratic B-spline moments via a single-particle P2G (closed forms)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_weight_moments_single_particle(dim):
    n = 16
    P = _params(dim, n, material=oracle.NO_ELASTICITY)
    dx = 1.0 / n
    m = (0.5 * dx) ** dim
    X = _node_positions(dim, n)
    for _ in range(20):
        xp = RNG.uniform(0.3, 0.7, size=(dim, 1))
        zero = np.zeros((dim, 1))
        C = np.zeros((dim * dim, 1))
        F = _soa([np.eye(dim)])
        gm, gp = oracle.p2g(P, 0, xp, zero, C, F, np.zeros(1), np.zeros(1))
        assert abs(gm.sum() - m) < 1e-14  # partition of unity
        d = X - xp[:, 0][None, :]
        first = (gm[:, None] * d).sum(0)
        assert np.abs(first).max() < 1e-15  # zero first moment
        second = np.einsum("i,ia,ib->ab", gm, d, d)
        np.testing.assert_allclose(second, m * dx * dx / 4 * np.eye(dim), atol=1e-18)
        assert np.all(gp == 0)


def test_bspline_values_at_cell_centre():
    # particle at a node + dx/2 offset pattern: f = 1.0 -> weights (1/8, 3/4, 1/8)
    n = 16
    P = _params(1 + 1, n, material=oracle.NO_ELASTICITY)
    dx = 1.0 / n
    m = (0.5 * dx) ** 2
    xp = np.array([[5 * dx], [7 * dx]])  # X = 5 -> base 4, f = 1
    gm, _ = oracle.p2g(P, 0, xp, np.zeros((2, 1)), np.zeros((4, 1)), _soa([np.eye(2)]),
                       np.zeros(1), np.zeros(1))
    g = gm.reshape(n, n) / m
    np.testing.assert_allclose(g[4:7, 6:9], np.outer([1 / 8, 3 / 4, 1 / 8], [1 / 8, 3 / 4, 1 / 8]),
                               atol=1e-15)
    assert abs(g.sum() - 1) < 1e-14


# ---------------------------------------------------------------------------
# P2G / grid / G2P invariants
# ---------------------------------------------------------------------------

def _blob(dim, n_side, n_grid, centre=0.5, spacing=None, jitter=0.2, rng=RNG):
    dx = 1.0 / n_grid
    h = spacing or dx / 2
    idx = np.indices((n_side,) * dim).reshape(dim, -1)
    x = centre - n_side * h / 2 + (idx + 0.5) * h
    x = x + jitter * h * rng.uniform(-1, 1, size=x.shape)
    return np.ascontiguousarray(x)


@pytest.mark.parametrize("dim,material", [(2, oracle.FIXED_COROTATED), (3, oracle.FIXED_COROTATED),
                                          (2, oracle.NEO_HOOKEAN), (3, oracle.NEO_HOOKEAN),
                                          (2, oracle.LIQUID), (3, oracle.LIQUID)])
def test_momentum_conserved_without_gravity_and_walls(dim, material):
    n_grid = 16
    P = _params(dim, n_grid, dt=1e-3, gravity=(0, 0, 0), walls=0, material=material)
    x = _blob(dim, 4, n_grid)
    k = x.shape[1]
    v = RNG.standard_normal((dim, k))
    C = RNG.standard_normal((dim * dim, k)) * 3
    F = _soa(_random_F(dim, k))
    mu, la = np.full(k, 300.0), np.full(k, 200.0)
    m = (0.5 / n_grid) ** dim
    gm, gp = oracle.p2g(P, 0, x, v, C, F, mu, la)
    np.testing.assert_allclose(gm.sum(), k * m, rtol=1e-13)
    np.testing.assert_allclose(gp.sum(0), m * v.sum(1), rtol=1e-12, atol=1e-15)
    x1, v1, C1, F1 = oracle.step(P, 0, x, v, C, F, mu, la)
    np.testing.assert_allclose(m * v1.sum(1), m * v.sum(1), rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_gravity_free_fall(dim):
    n_grid = 16
    g = (0.3, -9.8, 1.7)[:dim]
    P = _params(dim, n_grid, dt=1e-3, gravity=g + (0.0,) * (3 - dim), walls=0,
                material=oracle.NO_ELASTICITY)
    x = _blob(dim, 3, n_grid)
    k = x.shape[1]
    v0 = np.array([0.4, -0.2, 0.1][:dim])
    v = np.repeat(v0[:, None], k, axis=1)
    x1, v1, C1, F1 = oracle.step(P, 0, x, v, np.zeros((dim * dim, k)), _soa([np.eye(dim)] * k),
                                 np.zeros(k), np.zeros(k))
    exp_v = v0 + 1e-3 * np.array(g)
    np.testing.assert_allclose(v1, np.repeat(exp_v[:, None], k, 1), atol=1e-13)
    np.testing.assert_allclose(x1, x + 1e-3 * v1, atol=1e-15)
    np.testing.assert_allclose(C1, 0, atol=1e-11)


@pytest.mark.parametrize("dim", [2, 3])
def test_affine_field_reproduced(dim):
    n_grid = 16
    P = _params(dim, n_grid, dt=1e-3, gravity=(0, 0, 0), walls=0, material=oracle.NO_ELASTICITY)
    x = _blob(dim, 4, n_grid, jitter=0.45)
    k = x.shape[1]
    A = RNG.standard_normal((dim, dim))
    b = RNG.standard_normal(dim)
    v = A @ x + b[:, None]
    C = np.repeat(A.reshape(-1, 1), k, axis=1)
    F = _random_F(dim, k)
    x1, v1, C1, F1 = oracle.step(P, 0, x, v, C, _soa(F), np.zeros(k), np.zeros(k))
    np.testing.assert_allclose(v1, v, rtol=0, atol=1e-12)
    np.testing.assert_allclose(C1, C, rtol=0, atol=1e-11)
    np.testing.assert_allclose(x1, x + 1e-3 * v, atol=1e-14)
    # F' = (I + dt C') F
    for p in range(k):
        np.testing.assert_allclose(F1[:, p].reshape(dim, dim), (np.eye(dim) + 1e-3 * A) @ F[p],
                                   atol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_sticky_walls_zero_velocity(dim):
    n_grid = 16
    P = _params(dim, n_grid, dt=1e-3, walls=3, material=oracle.NO_ELASTICITY)
    dx = 1.0 / n_grid
    # stencil base 0 -> nodes 0..2, all inside the 3-node wall
    x = np.full((dim, 1), 1.2 * dx)
    v = np.ones((dim, 1))
    x1, v1, C1, F1 = oracle.step(P, 0, x, v, np.zeros((dim * dim, 1)), _soa([np.eye(dim)]),
                                 np.zeros(1), np.zeros(1))
    assert np.all(v1 == 0) and np.all(C1 == 0)
    # one axis clear of the wall: grid nodes with i_k >= n-3 on the far side too
    x = np.full((dim, 1), 0.5)
    x[0, 0] = 1 - 1.2 * dx - dx  # base n-3 -> nodes n-3..n-1, all wall
    x1, v1, *_ = oracle.step(P, 0, x, v, np.zeros((dim * dim, 1)), _soa([np.eye(dim)]),
                             np.zeros(1), np.zeros(1))
    assert np.all(v1 == 0)


def test_out_of_grid_particle_raises():
    P = _params(2, 16)
    x = np.array([[0.5 / 16 * 0.9], [0.5]])  # x/dx < 0.5 -> base -1
    with pytest.raises(oracle.OracleError):
        oracle.step(P, 0, x, np.zeros((2, 1)), np.zeros((4, 1)), _soa([np.eye(2)]),
                    np.ones(1), np.ones(1))


# ---------------------------------------------------------------------------
# polar decomposition vs numpy's SVD
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_polar_matches_svd(dim):
    Fs = _random_F(dim, 2000, spread=0.5)
    for F in Fs:
        R, S = oracle.polar(F)
        U, sig, Vt = np.linalg.svd(F)
        Rsvd = U @ Vt
        np.testing.assert_allclose(R, Rsvd, atol=1e-12)
        np.testing.assert_allclose(R.T @ R, np.eye(dim), atol=1e-13)
        assert abs(np.linalg.det(R) - 1) < 1e-13
        np.testing.assert_allclose(S, S.T, atol=1e-12)
        assert np.all(np.linalg.eigvalsh(0.5 * (S + S.T)) > 0)
        np.testing.assert_allclose(R @ S, F, atol=1e-12)


def test_polar_near_equal_singular_values():
    # sigma_1 = sigma_2 exactly: the polar factor is still unique and smooth
    Q1, Q2 = _random_rotation(3), _random_rotation(3)
    for sig in ([1.0, 1.0, 1.0], [1.1, 1.1, 0.9], [0.8, 1.0, 1.0 + 1e-9]):
        F = Q1 @ np.diag(sig) @ Q2.T
        R, S = oracle.polar(F)
        np.testing.assert_allclose(R, Q1 @ Q2.T, atol=1e-12)


def _svd_polar(F):
    U, s, Vt = np.linalg.svd(F)
    return U @ Vt


@pytest.mark.parametrize("dim", [2, 3])
def test_polar_adjoint_vs_fd_of_numpy_svd(dim):
    eps = 1e-6
    for F in _random_F(dim, 30, spread=0.4):
        Rb = RNG.standard_normal((dim, dim))
        Fb = oracle.polar_adjoint(F, Rb)
        fd = np.zeros_like(F)
        for i in range(dim):
            for j in range(dim):
                E = np.zeros_like(F)
                E[i, j] = eps
                fd[i, j] = (np.sum(Rb * _svd_polar(F + E)) - np.sum(Rb * _svd_polar(F - E))) / (2 * eps)
        np.testing.assert_allclose(Fb, fd, rtol=1e-6, atol=1e-8)


def test_polar_adjoint_at_identity_is_skew():
    Rb = RNG.standard_normal((3, 3))
    Fb = oracle.polar_adjoint(np.eye(3), Rb)
    np.testing.assert_allclose(Fb, 0.5 * (Rb - Rb.T), atol=1e-14)


# ---------------------------------------------------------------------------
# stress = (d psi / d F) F^T of textbook energy densities
# ---------------------------------------------------------------------------

def _psi_fcr(F, mu, la):
    s = np.linalg.svd(F, compute_uv=False)
    J = np.linalg.det(F)
    return mu * np.sum((s - 1) ** 2) + 0.5 * la * (J - 1) ** 2


def _psi_nh(F, mu, la):
    J = np.linalg.det(F)
    d = F.shape[0]
    return 0.5 * mu * (np.sum(F * F) - d) - mu * np.log(J) + 0.5 * la * np.log(J) ** 2


def _psi_liquid(F, mu, la, gamma=7.0):
    """Tait-form weakly compressible liquid energy: kappa (J - J^(1-g)/(1-g)), kappa the
    bulk modulus la + 2 mu / d (no shear energy)."""
    J = np.linalg.det(F)
    kap = la + 2.0 * mu / F.shape[0]
    return kap * (J - J ** (1.0 - gamma) / (1.0 - gamma))


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("material,psi", [(oracle.FIXED_COROTATED, _psi_fcr),
                                          (oracle.NEO_HOOKEAN, _psi_nh),
                                          (oracle.LIQUID, _psi_liquid)])
def test_kirchhoff_is_energy_derivative(dim, material, psi):
    P = _params(dim, material=material)
    mu, la = 417.0, 278.0
    eps = 1e-6
    for F in _random_F(dim, 20, spread=0.3):
        tau = oracle.kirchhoff(P, F, mu, la)
        dpsi = np.zeros_like(F)
        for i in range(dim):
            for j in range(dim):
                E = np.zeros_like(F)
                E[i, j] = eps
                dpsi[i, j] = (psi(F + E, mu, la) - psi(F - E, mu, la)) / (2 * eps)
        np.testing.assert_allclose(tau, dpsi @ F.T, rtol=1e-6, atol=1e-5)


@pytest.mark.parametrize("dim", [2, 3])
def test_stress_zero_at_rest(dim):
    Pf = _params(dim, material=oracle.FIXED_COROTATED)
    Pn = _params(dim, material=oracle.NEO_HOOKEAN)
    R = _random_rotation(dim)
    np.testing.assert_allclose(oracle.kirchhoff(Pf, R, 500.0, 300.0), 0, atol=1e-11)
    np.testing.assert_allclose(oracle.kirchhoff(Pn, np.eye(dim), 500.0, 300.0), 0, atol=1e-13)
    # the liquid carries no shear: zero at any isochoric F (J = 1), rotated or sheared
    Pl = _params(dim, material=oracle.LIQUID)
    shear = np.eye(dim)
    shear[0, 1] = 0.7
    for F in (R, shear, R @ shear):
        np.testing.assert_allclose(oracle.kirchhoff(Pl, F, 500.0, 300.0), 0, atol=1e-11)


@pytest.mark.parametrize("dim", [2, 3])
def test_liquid_stress_is_hydrostatic_tait_pressure(dim):
    """tau = -J p I with the Tait pressure p = kappa (J^-7 - 1): compression pushes out."""
    P = _params(dim, material=oracle.LIQUID)
    mu, la = 417.0, 278.0
    kap = la + 2 * mu / dim
    for F in _random_F(dim, 10, spread=0.3):
        J = np.linalg.det(F)
        tau = oracle.kirchhoff(P, F, mu, la)
        p = kap * (J ** -7.0 - 1.0)
        np.testing.assert_allclose(tau, -J * p * np.eye(dim), rtol=1e-12, atol=1e-9)
    t = oracle.kirchhoff(P, 0.95 ** (1.0 / dim) * np.eye(dim), mu, la)
    assert np.all(np.diag(t) < 0)  # J < 1: negative Kirchhoff stress (positive pressure)


@pytest.mark.parametrize("dim", [2, 3])
def test_liquid_small_strain_limit(dim):
    """Linearised: tau = kappa * gamma * tr(e) I (bulk response only, tangent modulus
    kappa * gamma at J = 1)."""
    P = _params(dim, material=oracle.LIQUID)
    mu, la = 417.0, 278.0
    e = 1e-7 * RNG.standard_normal((dim, dim))
    e = 0.5 * (e + e.T)
    tau = oracle.kirchhoff(P, np.eye(dim) + e, mu, la)
    kap = la + 2 * mu / dim
    np.testing.assert_allclose(tau, 7.0 * kap * np.trace(e) * np.eye(dim), rtol=1e-5, atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("material", [oracle.FIXED_COROTATED, oracle.NEO_HOOKEAN])
def test_small_strain_limit_is_linear_elasticity(dim, material):
    P = _params(dim, material=material)
    mu, la = 417.0, 278.0
    e = 1e-7 * RNG.standard_normal((dim, dim))
    e = 0.5 * (e + e.T)
    tau = oracle.kirchhoff(P, np.eye(dim) + e, mu, la)
    lin = 2 * mu * e + la * np.trace(e) * np.eye(dim)
    np.testing.assert_allclose(tau, lin, rtol=1e-5, atol=1e-12)


# ---------------------------------------------------------------------------
# actuation: closed-form special cases of the sine basis and the fibre stress
# ---------------------------------------------------------------------------

def test_actuation_basis_special_cases():
    P = _params(3, n_groups=2, n_basis=4, act_period=40.0, act_phase=0.0)
    w = np.zeros((2, 4))
    w[1, 1] = 1.0  # k = 2 on group 1
    assert abs(oracle.actuation(P, w, 1, 5)) - 1 < 1e-15  # sin(2 pi 2 5/40) = sin(pi/2)
    assert abs(oracle.actuation(P, w, 1, 5) - 1.0) < 1e-15
    assert abs(oracle.actuation(P, w, 1, 10)) < 1e-15      # sin(pi)
    assert abs(oracle.actuation(P, w, 0, 5)) == 0.0        # other group
    w[1, 0] = 2.0  # k = 1 term: 2 sin(2 pi 5/40) = 2 sin(pi/4)
    assert abs(oracle.actuation(P, w, 1, 5) - (1.0 + np.sqrt(2))) < 1e-14
    Pp = _params(3, n_groups=1, n_basis=1, act_period=40.0, act_phase=np.pi / 2)
    assert abs(oracle.actuation(Pp, np.ones((1, 1)), 0, 0) - 1.0) < 1e-15  # sin(phi)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_actuation_stress_fibre(axis):
    P = _params(3, material=oracle.NO_ELASTICITY)
    tau = oracle.kirchhoff(P, np.eye(3), 0.0, 0.0, act=2.5, axis=axis)
    exp = np.zeros((3, 3))
    exp[axis, axis] = 2.5
    np.testing.assert_allclose(tau, exp, atol=1e-15)
    # pushed forward by a rotation: tau = a (R e)(R e)^T
    R = _random_rotation(3)
    tau = oracle.kirchhoff(P, R, 0.0, 0.0, act=2.5, axis=axis)
    np.testing.assert_allclose(tau, 2.5 * np.outer(R[:, axis], R[:, axis]), atol=1e-14)


def test_lame_closed_form():
    mu, la = oracle.lame(np.array([1e3, 5e3]), np.array([0.2, 0.3]))
    np.testing.assert_allclose(mu, [1e3 / 2.4, 5e3 / 2.6], rtol=1e-15)
    np.testing.assert_allclose(la, [1e3 * 0.2 / (1.2 * 0.6), 5e3 * 0.3 / (1.3 * 0.4)], rtol=1e-15)


# ---------------------------------------------------------------------------
# the stress term of P2G is dt times the grid force -dPsi/dx_i
# ---------------------------------------------------------------------------

def _bspline(f):
    return np.array([0.5 * (1.5 - f) ** 2, 0.75 - (f - 1) ** 2, 0.5 * (f - 0.5) ** 2])


@pytest.mark.parametrize("material,psi", [(oracle.FIXED_COROTATED, _psi_fcr),
                                          (oracle.NEO_HOOKEAN, _psi_nh)])
def test_p2g_stress_momentum_is_minus_energy_gradient(material, psi):
    """MLS-MPM (Hu et al. 2018): with v = C = 0 the grid momentum after P2G is dt f_i,
    f_i = -dPsi/dxhat_i, Psi = sum_p V0 psi(F_p(xhat)), F_p(xhat) = (I + sum_i
    (xhat_i - x_i) g_ip^T) F_p, g_ip = (4/dx^2) W_ip (x_i - x_p).  The stress P = dpsi/dF
    is taken by central differences of the textbook energy, not from the oracle."""
    dim, n_grid, dt = 2, 16, 1e-3
    P = _params(dim, n_grid, dt=dt, gravity=(0, 0, 0), walls=0, material=material)
    dx = 1.0 / n_grid
    V0 = (0.5 * dx) ** dim
    mu, la = 300.0, 200.0
    x = _blob(dim, 2, n_grid)
    k = x.shape[1]
    Fs = _random_F(dim, k, spread=0.1)
    gm, gp = oracle.p2g(P, 0, x, np.zeros((dim, k)), np.zeros((dim * dim, k)), _soa(Fs),
                        np.full(k, mu), np.full(k, la))
    force = np.zeros((n_grid ** dim, dim))
    eps = 1e-6
    for p in range(k):
        Fp = Fs[p]
        dpsi = np.zeros((dim, dim))
        for i in range(dim):
            for j in range(dim):
                E = np.zeros((dim, dim))
                E[i, j] = eps
                dpsi[i, j] = (psi(Fp + E, mu, la) - psi(Fp - E, mu, la)) / (2 * eps)
        X = x[:, p] / dx
        base = np.floor(X - 0.5).astype(int)
        f = X - base
        w = [_bspline(f[a]) for a in range(dim)]
        for o0 in range(3):
            for o1 in range(3):
                W = w[0][o0] * w[1][o1]
                dpos = (np.array([o0, o1]) - f) * dx
                g = 4.0 / dx ** 2 * W * dpos
                node = (base[0] + o0) * n_grid + base[1] + o1
                force[node] -= V0 * (dpsi @ Fp.T) @ g
    np.testing.assert_allclose(gp, dt * force, rtol=1e-6, atol=1e-14)


@pytest.mark.parametrize("material", [oracle.FIXED_COROTATED, oracle.NEO_HOOKEAN, oracle.LIQUID])
def test_stretched_block_contracts(material):
    dim, n_grid = 2, 32
    P = _params(dim, n_grid, dt=1e-4, gravity=(0, 0, 0), walls=0, material=material)
    x = _blob(dim, 8, n_grid, jitter=0.0)
    k = x.shape[1]
    for s, sign in ((1.1, -1), (0.9, 1)):
        F = _soa([s * np.eye(dim)] * k)
        _, v1, _, _ = oracle.step(P, 0, x, np.zeros((dim, k)), np.zeros((dim * dim, k)), F,
                                  np.full(k, 400.0), np.full(k, 300.0))
        radial = np.sum(v1 * (x - x.mean(1, keepdims=True)))
        assert sign * radial > 0
