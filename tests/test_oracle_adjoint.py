"""Pins of the adjoint oracle (oracle/adjoint_oracle.py): every derivative it forms is
compared with central finite differences of acac_oracle's residual, energy and
time stepping, which the other oracle tests pin to the paper; plus the closed form
of dF/dU^n when U^{n+1} = U^n."""
import numpy as np
import pytest

from oracle import acac_oracle as O
from oracle import adjoint_oracle as A
from workloads import BC_NEUMANN, BC_PERIODIC, Params, initial_fields, perturbed_pair

H = 1e-6


def _soa(X):
    return np.concatenate([X[0].ravel(), X[1].ravel()])


def _unsoa(x, shape):
    n = x.size // 2
    return x[:n].reshape(shape), x[n:].reshape(shape)


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
@pytest.mark.parametrize("dim,n", [(2, (9, 7, 1)), (3, (5, 4, 4))])
def test_step_jacobians_match_central_differences(bc, dim, n):
    """J1 = dF/dU^{n+1} and J0 = dF/dU^n against central differences of F in random
    directions."""
    p = Params(dim=dim, n=n, bc=bc)
    X1, X0 = perturbed_pair(p, 7, u_mean=0.45, amp=0.1, step_amp=0.02)
    dt = 2e-3
    J1, J0 = A.jacobians(p, X1, X0, dt)
    F = lambda a, b: _soa(O.residual(p, a, b, dt))
    x1, x0 = _soa(X1), _soa(X0)
    rng = np.random.default_rng(3)
    for _ in range(2):
        w = rng.standard_normal(x1.size)
        fd1 = (F(_unsoa(x1 + H * w, p.shape), X0) - F(_unsoa(x1 - H * w, p.shape), X0)) / (2 * H)
        fd0 = (F(X1, _unsoa(x0 + H * w, p.shape)) - F(X1, _unsoa(x0 - H * w, p.shape))) / (2 * H)
        assert np.linalg.norm(fd1 - J1 @ w) <= 1e-6 * np.linalg.norm(fd1)
        assert np.linalg.norm(fd0 - J0 @ w) <= 1e-6 * np.linalg.norm(fd0)


def test_step_jacobians_agree_with_the_interleaved_jacobian():
    """J1 in the [u | v] layout is acac_oracle.jacobian permuted."""
    p = Params(n=(8, 6, 1))
    X1, X0 = perturbed_pair(p, 2, u_mean=0.4, amp=0.05, step_amp=0.01)
    J1, _ = A.jacobians(p, X1, X0, 1e-3)
    Ji = O.jacobian(p, X1, X0, 1e-3)
    perm = O._interleave_perm(p.ncells)          # interleaved index -> [u | v] index
    Jb = np.zeros((2 * p.ncells, 2 * p.ncells))
    Jb[np.ix_(perm, perm)] = Ji.toarray()
    np.testing.assert_allclose(J1.toarray(), Jb, rtol=1e-13, atol=1e-10)


def test_step_jacobians_at_zero_increment():
    """With U^{n+1} = U^n, sigma = 0 and the series is even in sigma, so the two
    Jacobians differ only in the time difference: J1 - J0 = 2 I / dt exactly."""
    p = Params(n=(7, 6, 1), bc=BC_NEUMANN)
    u, v = initial_fields(p, 5, 0.45, 0.1)
    dt = 1e-3
    J1, J0 = A.jacobians(p, (u, v), (u, v), dt)
    D = (J1 - J0).toarray()
    np.testing.assert_allclose(D, 2.0 / dt * np.eye(D.shape[0]), rtol=0, atol=1e-9)


def test_parameter_derivatives_match_central_differences():
    p = Params(n=(8, 9, 1), bc=BC_PERIODIC)
    X1, X0 = perturbed_pair(p, 11, u_mean=0.42, amp=0.08, step_amp=0.02)
    dt = 1e-3
    dF = A.dF_dparams(p, X1, X0, dt)
    for name in A.PARAMS:
        val = getattr(p, name)
        hp = H * val
        fp = _soa(O.residual(p.replace(**{name: val + hp}), X1, X0, dt))
        fm = _soa(O.residual(p.replace(**{name: val - hp}), X1, X0, dt))
        fd = (fp - fm) / (2 * hp)
        assert np.linalg.norm(fd - dF[name]) <= 1e-6 * np.linalg.norm(fd), name


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
def test_loss_gradient_matches_central_differences(bc):
    p = Params(n=(9, 8, 1), bc=bc)
    X = initial_fields(p, 21, 0.4, 0.1)
    T = initial_fields(p, 22, 0.5, 0.1)
    dX, dP = A.loss_grad(p, X, T, 1.0, 0.7)
    L = lambda q, x: A.loss(q, _unsoa(x, p.shape), T, 1.0, 0.7)
    x = _soa(X)
    rng = np.random.default_rng(4)
    w = rng.standard_normal(x.size)
    # fourth-order central difference at h = 1e-4: truncation ~h^4, rounding ~eps |L| / h, both
    # far below the tolerance (a second-order difference at 1e-6 carries ~1e-6 rounding noise)
    h = 1e-4
    fd = (8.0 * (L(p, x + h * w) - L(p, x - h * w)) - (L(p, x + 2 * h * w) - L(p, x - 2 * h * w))) / (12.0 * h)
    assert fd == pytest.approx(float(dX @ w), rel=1e-8)
    for name in A.PARAMS:
        val = getattr(p, name)
        fd = (L(p.replace(**{name: val + H * val}), x) - L(p.replace(**{name: val - H * val}), x)) / (2 * H * val)
        assert fd == pytest.approx(dP[name], rel=1e-7, abs=1e-12), name


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
def test_adjoint_gradient_matches_central_differences(bc):
    """Three fixed-dt steps (checkpoint every 2, so one segment is recomputed): the
    adjoint gradient of L with respect to the coefficients and, in a random
    direction, the initial fields agrees with central differences of the forward
    loss (dense Newton solves to 1e-11)."""
    p = Params(n=(8, 7, 1), bc=bc, newton_rtol=1e-11, newton_atol=1e-13)
    U0 = initial_fields(p, 31, 0.42, 0.06)
    T = initial_fields(p, 131, 0.45, 0.06)
    dt, K = 2e-3, 3
    L0, du, dv, grad = A.adjoint_gradient(p, U0, K, dt, T, 1.0, 2.0, every=2)
    assert L0 == pytest.approx(A.forward_loss(p, U0, K, dt, T, 1.0, 2.0), rel=1e-13)
    for name in A.PARAMS:
        val = getattr(p, name)
        h = H * val
        fd = (A.forward_loss(p.replace(**{name: val + h}), U0, K, dt, T, 1.0, 2.0)
              - A.forward_loss(p.replace(**{name: val - h}), U0, K, dt, T, 1.0, 2.0)) / (2 * h)
        assert grad[name] == pytest.approx(fd, rel=1e-6, abs=1e-10), name
    rng = np.random.default_rng(5)
    wu, wv = rng.standard_normal(p.shape), rng.standard_normal(p.shape)
    s = 1e-6
    fd = (A.forward_loss(p, (U0[0] + s * wu, U0[1] + s * wv), K, dt, T, 1.0, 2.0)
          - A.forward_loss(p, (U0[0] - s * wu, U0[1] - s * wv), K, dt, T, 1.0, 2.0)) / (2 * s)
    assert float(np.sum(du * wu) + np.sum(dv * wv)) == pytest.approx(fd, rel=1e-6)
