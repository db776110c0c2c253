"""Pins of the oracle's mass-spring system (the paper's introductory example, Section 2,
and the tape demonstration of Section 3): Hooke's springs with the example's 1e-4 length
guard, semi-implicit Euler with damping exp(-dt alpha).

* closed form: with k = 0 the motion is free damped drift, v_t = s^t v0,
  x_t = x0 + dt v0 (s + s^2 + ... + s^t);
* invariants: internal spring forces conserve the total momentum (alpha = 0) and the
  centre of mass moves uniformly; a rigid translation of the initial positions translates
  every state;
* the spring force against a central difference of the energy whose gradient the guarded
  Hooke force is (forces are minus its gradient);
* adjoint: dL/d(x0, v0, l0) of whole runs against central finite differences; the area
  loss's gradient likewise;
* the demonstration: gradient descent on the rest lengths with the area loss shrinks the
  loss (the paper's final lengths depend on constants it does not state, so only the
  behaviour is pinned).
"""
import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(99)
TRI = [(0, 1), (0, 2), (1, 2)]
X_TRI = np.array([[0.0, 0.0], [0.0, 0.1], [0.1, 0.0]])


def _system(n=5, dim=2, rng=RNG):
    x0 = rng.uniform(0.0, 0.3, (n, dim))
    v0 = rng.normal(0.0, 0.2, (n, dim))
    springs = [(i, j) for i in range(n) for j in range(i + 1, n) if (i + j) % 2 == 1 or j == i + 1]
    l0 = np.array([np.linalg.norm(x0[a] - x0[b]) for a, b in springs]) * rng.uniform(0.7, 1.3, len(springs))
    return x0, v0, springs, l0


def test_free_damped_drift_closed_form():
    x0, v0, springs, l0 = _system()
    dt, alpha, T = 2e-3, 3.0, 50
    x, v = oracle.ms_forward(x0, v0, springs, l0, 0.0, alpha, dt, 1.0, T)
    s = np.exp(-dt * alpha)
    for t in (1, 7, T - 1):
        np.testing.assert_allclose(v[t], s ** t * v0, rtol=0, atol=1e-14)
        geo = sum(s ** i for i in range(1, t + 1))
        np.testing.assert_allclose(x[t], x0 + dt * v0 * geo, rtol=0, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_momentum_conserved_and_translation_equivariant(dim):
    x0, v0, springs, l0 = _system(6, dim)
    x, v = oracle.ms_forward(x0, v0, springs, l0, 50.0, 0.0, 1e-3, 2.0, 200)
    p = v.sum(axis=1)
    np.testing.assert_allclose(p, np.broadcast_to(p[0], p.shape), rtol=0, atol=1e-11)
    com = x.mean(axis=1)
    t = np.arange(x.shape[0])[:, None]
    np.testing.assert_allclose(com, com[0] + 1e-3 * t * v0.mean(axis=0), rtol=0, atol=1e-11)
    shift = RNG.normal(size=dim)
    x2, v2 = oracle.ms_forward(x0 + shift, v0, springs, l0, 50.0, 0.0, 1e-3, 2.0, 200)
    np.testing.assert_allclose(x2, x + shift, rtol=0, atol=1e-11)
    np.testing.assert_allclose(v2, v, rtol=0, atol=1e-11)


def test_spring_force_is_minus_the_energy_gradient():
    """One step from rest with dt = 1, m = 1, alpha = 0 gives v_1 = f(x_0); f must be minus
    the gradient of the energy whose gradient the guarded Hooke force is: with r = |d|,
    k (r + e - l0) d / (r + e) = phi'(r) d / r for phi(r) = k (r^2/2 - l0 r + l0 e ln(r + e)),
    e = 1e-4 (at e = 0 this is the textbook (k/2)(r - l0)^2 up to a constant)."""
    x0, _, springs, l0 = _system()
    k = 7.0
    _, v = oracle.ms_forward(x0, np.zeros_like(x0), springs, l0, k, 0.0, 1.0, 1.0, 2)

    def energy(x):
        e = 1e-4
        return sum(k * (0.5 * r * r - l * r + l * e * np.log(r + e))
                   for r, l in ((np.linalg.norm(x[a] - x[b]), l) for (a, b), l in zip(springs, l0)))

    h = 1e-6
    grad = np.zeros_like(x0)
    for i in range(x0.shape[0]):
        for c in range(x0.shape[1]):
            e = np.zeros_like(x0)
            e[i, c] = h
            grad[i, c] = (energy(x0 + e) - energy(x0 - e)) / (2 * h)
    np.testing.assert_allclose(v[1], -grad, rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("dim,alpha", [(2, 5.0), (3, 0.0)])
def test_adjoint_matches_finite_differences(dim, alpha):
    x0, v0, springs, l0 = _system(5, dim)
    k, dt, m, T = 40.0, 2e-3, 1.5, 120
    cx = RNG.normal(size=x0.shape)
    cv = RNG.normal(size=x0.shape)

    def L(x0_, v0_, l0_):
        x, v = oracle.ms_forward(x0_, v0_, springs, l0_, k, alpha, dt, m, T)
        return float(np.sum(cx * x[-1]) + np.sum(cv * v[-1]))

    x, _ = oracle.ms_forward(x0, v0, springs, l0, k, alpha, dt, m, T)
    gx, gv, gl = oracle.ms_backward(x, springs, l0, k, alpha, dt, m, cx, cv)
    eps = 1e-6
    for _ in range(3):
        for which in range(3):
            d = RNG.normal(size=(x0, v0, l0)[which].shape)
            args_p = [x0, v0, l0]
            args_m = [x0, v0, l0]
            args_p[which] = args_p[which] + eps * d
            args_m[which] = args_m[which] - eps * d
            fd = (L(*args_p) - L(*args_m)) / (2 * eps)
            an = float(np.sum((gx, gv, gl)[which] * d))
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (which, fd, an)


def test_area_loss_gradient():
    x = X_TRI + RNG.normal(0, 0.02, X_TRI.shape)
    L, g = oracle.ms_area_loss(x, 0.2)
    eps = 1e-7
    for i in range(3):
        for c in range(2):
            e = np.zeros_like(x)
            e[i, c] = eps
            fd = (oracle.ms_area_loss(x + e, 0.2)[0] - oracle.ms_area_loss(x - e, 0.2)[0]) / (2 * eps)
            assert abs(fd - g[i, c]) <= 1e-6 * max(1.0, abs(fd))
    # a right triangle with legs 0.1: area 0.005
    L0, _ = oracle.ms_area_loss(X_TRI, 0.2)
    assert abs(L0 - (0.005 - 0.2) ** 2) <= 1e-15


def test_rest_length_optimisation_reduces_the_loss():
    """Section 3's demonstration: gradient descent on the three rest lengths (initially
    0.1, 0.1, 0.14) towards a triangle of area 0.2 at the last step."""
    k, alpha, dt, m, T = 100.0, 10.0, 2e-3, 1.0, 400
    l0 = np.array([0.1, 0.1, 0.14])
    losses = []
    for _ in range(40):
        x, _ = oracle.ms_forward(X_TRI, np.zeros((3, 2)), TRI, l0, k, alpha, dt, m, T)
        L, xb = oracle.ms_area_loss(x[-1], 0.2)
        _, _, gl = oracle.ms_backward(x, TRI, l0, k, alpha, dt, m, xb, np.zeros((3, 2)))
        losses.append(L)
        l0 = l0 - 2.0 * gl
    assert losses[-1] < 0.05 * losses[0], (losses[0], losses[-1])
    assert np.all(l0 > np.array([0.1, 0.1, 0.14]))  # the springs lengthen to expand the triangle
