"""Batched mass-spring systems (include/mass_spring.h; the paper's Section 2 example and
Section 3 tape demonstration) on the GPU against the FP64 oracle: recorded states, the
reverse pass (dL/dx0, dL/dv0, dL/drest of random linear functionals of the last state),
and the rest-length optimisation of the triangle through torch.autograd."""
import numpy as np
import pytest

from mpm_testlib import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TRI = [(0, 1), (0, 2), (1, 2)]


@pytest.fixture(scope="module")
def ms():
    from paper_1910_00935_gb300 import build, mass_spring
    build.build()
    return mass_spring


def _batch(S, n, dim, rng):
    """S systems of n masses: jittered copies of one random shape, springs between
    neighbours and across, rest lengths scaled per system."""
    springs = [(i, j) for i in range(n) for j in range(i + 1, n) if (i + j) % 2 == 1 or j == i + 1]
    base = rng.uniform(0.0, 0.3, (n, dim))
    x0 = base[None] + rng.normal(0, 0.01, (S, n, dim))
    v0 = rng.normal(0, 0.2, (S, n, dim))
    l0 = np.stack([[np.linalg.norm(x0[s, a] - x0[s, b]) for a, b in springs] for s in range(S)])
    l0 *= rng.uniform(0.7, 1.3, l0.shape)
    return springs, x0, v0, l0


def _rows(a):  # [S, n, dim] -> [n*dim, S] float32
    S = a.shape[0]
    return torch.as_tensor(np.ascontiguousarray(a.reshape(S, -1).T), dtype=torch.float32)


def _unrows(t, n, dim):
    a = t.detach().cpu().numpy().astype(np.float64)
    return a.T.reshape(-1, n, dim)


@pytest.mark.parametrize("dim,alpha,n", [(2, 5.0, 5), (3, 0.0, 5),   # shared-memory rows
                                         (2, 5.0, 4), (3, 1.0, 4)])  # register rows (<= 4 masses, springs)
def test_states_and_gradients_match_oracle(ms, dim, alpha, n):
    import oracle
    rng = np.random.default_rng(7 + dim + n)
    S, T = 300, 160
    k, dt, m = 40.0, 2e-3, 1.5
    springs, x0, v0, l0 = _batch(S, n, dim, rng)
    sim = ms.MassSprings(dim, n, springs, S, k, alpha, dt, m, steps=T)
    sim.forward(_rows(x0).cuda(), _rows(v0).cuda(),
                torch.as_tensor(np.ascontiguousarray(l0.T), dtype=torch.float32).cuda(), T)
    xT, vT = sim.state()
    xm, _ = sim.state(T // 2)
    cx = rng.normal(size=(S, n, dim))
    cv = rng.normal(size=(S, n, dim))
    gx, gv, gl = sim.backward(_rows(cx).cuda(), _rows(cv).cuda())
    sim.sync()
    gx, gv = _unrows(gx, n, dim), _unrows(gv, n, dim)
    gl = gl.cpu().numpy().T.astype(np.float64)
    ox, ov, om, ogx, ogv, ogl = [], [], [], [], [], []
    for s in range(S):
        X, V = oracle.ms_forward(x0[s], v0[s], springs, l0[s], k, alpha, dt, m, T)
        a, b, c = oracle.ms_backward(X, springs, l0[s], k, alpha, dt, m, cx[s], cv[s])
        ox.append(X[-1]); ov.append(V[-1]); om.append(X[T // 2])
        ogx.append(a); ogv.append(b); ogl.append(c)
    assert rel_l2(_unrows(xT, n, dim), np.array(ox)) <= 1e-5
    assert rel_l2(_unrows(xm, n, dim), np.array(om)) <= 1e-5
    assert rel_l2(_unrows(vT, n, dim), np.array(ov)) <= 1e-4
    assert rel_l2(gx, np.array(ogx)) <= 1e-3
    assert rel_l2(gv, np.array(ogv)) <= 1e-3
    assert rel_l2(gl, np.array(ogl)) <= 1e-3
    sim.close()


def test_triangle_rest_length_optimisation(ms):
    """Section 3's demonstration on 64 copies of the triangle (rest lengths 0.1, 0.1, 0.14
    towards area 0.2 at the last step), through torch.autograd; the same gradient-descent
    run in the FP64 oracle ends at the same rest lengths."""
    import oracle
    k, alpha, dt, m, T, lr, iters = 100.0, 10.0, 2e-3, 1.0, 400, 2.0, 25
    S = 64
    x_tri = np.array([[0.0, 0.0], [0.0, 0.1], [0.1, 0.0]])
    sim = ms.MassSprings(2, 3, TRI, S, k, alpha, dt, m, steps=T)
    x0 = _rows(np.broadcast_to(x_tri, (S, 3, 2)).copy()).cuda()
    v0 = torch.zeros_like(x0)
    rest = torch.tensor([0.1, 0.1, 0.14], device="cuda")[:, None].repeat(1, S).contiguous()
    losses = []
    for _ in range(iters):
        r = rest.clone().requires_grad_(True)
        xT, vT = ms.MassSpringRun.apply(sim, T, x0, v0, r)
        L = ms.triangle_area(xT).sum()
        L.backward()
        losses.append(float(L.detach()) / S)
        rest = (rest - lr * r.grad).detach().contiguous()
    sim.close()
    l0 = np.array([0.1, 0.1, 0.14])
    for _ in range(iters):
        X, _ = oracle.ms_forward(x_tri, np.zeros((3, 2)), TRI, l0, k, alpha, dt, m, T)
        Lo, xb = oracle.ms_area_loss(X[-1], 0.2)
        _, _, g = oracle.ms_backward(X, TRI, l0, k, alpha, dt, m, xb, np.zeros((3, 2)))
        l0 = l0 - lr * g
    assert losses[-1] < 0.1 * losses[0]
    got = rest.cpu().numpy().astype(np.float64)
    assert rel_l2(got, np.broadcast_to(l0[:, None], got.shape)) <= 1e-3


def test_errors(ms):
    from paper_1910_00935_gb300 import mpm
    sim = ms.MassSprings(2, 3, TRI, 8, 1.0, 0.0, 1e-3, 1.0, steps=10)
    with pytest.raises(mpm.MPMError) as e:
        sim.backward()
    assert e.value.code == mpm.MPM_ERR_STATE
    x0 = torch.zeros(6, 8, device="cuda")
    with pytest.raises(mpm.MPMError) as e:
        sim.forward(x0, x0, torch.ones(3, 8, device="cuda"), 11)
    assert e.value.code == mpm.MPM_ERR_STATE
    sim.forward(x0, x0, torch.ones(3, 8, device="cuda"), 1)  # state 0 only
    x, v = sim.state(0)
    sim.sync()
    assert torch.equal(x, x0)
    sim.close()
