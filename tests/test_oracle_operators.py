"""Pins of the oracle's difference operators, energy and variational derivative:
closed forms on Fourier modes, the summation-by-parts identity (Eq. summation),
semi-positivity of A~ (Eq. neq:02) and the discrete variational-derivative
identity (Eq. DVD)."""
import numpy as np
import pytest

from oracle import acac_oracle as O
from workloads import BC_NEUMANN, BC_PERIODIC, Params, perturbed_pair


def _params(dim, bc, n=(12, 10, 8)):
    return Params(dim=dim, n=n, L=(1.0, 0.8, 1.3), bc=bc, ras_parts=(2, 2, 2))


def _centres(p):
    axes = [(np.arange(p.n[d]) + 0.5) * p.L[d] / p.n[d] for d in range(p.dim)]
    mesh = np.meshgrid(*axes[::-1], indexing="ij")     # slowest axis first
    return mesh[::-1]                                   # x, y, (z)


@pytest.mark.parametrize("dim", [2, 3])
def test_laplacian_cosine_mode_closed_form(dim):
    """Periodic: Delta_h cos(2 pi k.x) = -sum_d (4/h_d^2) sin^2(pi k_d h_d) cos(.)"""
    p = _params(dim, BC_PERIODIC)
    g = O.grid_for(p)
    xs = _centres(p)
    k = [2, 1, 3][:dim]
    phase = sum(2 * np.pi * k[d] * xs[d] / p.L[d] for d in range(dim))
    mode = np.cos(phase)
    kh2 = sum(4.0 / g.h[d] ** 2 * np.sin(np.pi * k[d] * g.h[d] / p.L[d]) ** 2
              for d in range(dim))
    np.testing.assert_allclose(g.lap(mode), -kh2 * mode, rtol=0, atol=1e-9 * kh2)


def test_laplacian_neumann_cosine_mode():
    """Neumann: cos(pi m x / L) at cell centres is an eigenvector of the
    ghost-rule Laplacian with eigenvalue -(4/h^2) sin^2(pi m h / (2L))."""
    p = _params(2, BC_NEUMANN)
    g = O.grid_for(p)
    x, y = _centres(p)
    m = 3
    mode = np.cos(np.pi * m * x / p.L[0])
    lam = 4.0 / g.h[0] ** 2 * np.sin(np.pi * m * g.h[0] / (2 * p.L[0])) ** 2
    np.testing.assert_allclose(g.lap(mode), -lam * mode, rtol=0, atol=1e-9 * lam)


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
@pytest.mark.parametrize("dim", [2, 3])
def test_summation_by_parts(bc, dim):
    """-sum phi [D c~ D psi] = 1/2 sum (c~_{+} D+phi D+psi + c~_{-} D-phi D-psi),
    per direction and summed, with the ghost rule of Sec. 2 (Eq. summation)."""
    p = _params(dim, bc)
    g = O.grid_for(p)
    rng = np.random.default_rng(11)
    phi, psi = rng.standard_normal(p.shape), rng.standard_normal(p.shape)
    c = rng.uniform(0.0, 1.0, p.shape)
    lhs = -np.sum(phi * g.mob_div(c, psi))
    rhs = 0.0
    for d in range(dim):
        axis = dim - 1 - d
        dpp, dmp = O._dplus_dminus(phi, p, d)
        dps, dms = O._dplus_dminus(psi, p, d)
        if bc == BC_PERIODIC:
            cn, cp = np.roll(c, -1, axis), np.roll(c, 1, axis)
        else:
            n = p.shape[axis]
            cn = np.take(c, np.minimum(np.arange(n) + 1, n - 1), axis=axis)
            cp = np.take(c, np.maximum(np.arange(n) - 1, 0), axis=axis)
        cplus, cminus = 0.5 * (c + cn), 0.5 * (c + cp)
        rhs += 0.5 * np.sum(cplus * dpp * dps + cminus * dmp * dms)
    assert lhs == pytest.approx(rhs, rel=1e-12)


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
def test_A11_symmetric_semipositive(bc):
    """A11 = -div c grad is symmetric and <phi, A11 phi> >= 0 for c >= 0 (Eq. neq:02)."""
    p = _params(2, bc)
    g = O.grid_for(p)
    rng = np.random.default_rng(5)
    c = rng.uniform(0.0, 0.0625, p.shape)
    for _ in range(5):
        a, b = rng.standard_normal(p.shape), rng.standard_normal(p.shape)
        Aa, Ab = -g.mob_div(c, a), -g.mob_div(c, b)
        assert np.sum(a * Aa) >= 0.0
        assert np.sum(b * Aa) == pytest.approx(np.sum(a * Ab), rel=1e-12)
        # Cauchy–Schwarz in the A11 inner product
        assert abs(np.sum(b * Aa)) <= np.sqrt(np.sum(a * Aa) * np.sum(b * Ab)) * (1 + 1e-12)


def test_energy_closed_forms():
    """Constant state: E = (e1 + e2)|Omega|.  A cosine mode adds the gradient
    energy gamma/2 * eps^2 k_h^2 / 2 * |Omega| exactly (Eqs. relations, freeenergy)."""
    p = _params(2, BC_PERIODIC)
    u0, v0 = 0.4, 0.1
    area = p.L[0] * p.L[1]
    bulk = (0.5 * p.alpha * u0 * (1 - u0) - 0.5 * p.beta * v0 ** 2
            + p.theta * (O.Phi(u0 + v0) + O.Phi(u0 - v0)))
    u = np.full(p.shape, u0)
    v = np.full(p.shape, v0)
    assert O.energy(p, u, v) == pytest.approx(bulk * area, rel=1e-14)
    x, y = _centres(p)
    eps, k = 1e-3, 2
    du = eps * np.cos(2 * np.pi * k * x / p.L[0])
    hx = p.L[0] / p.n[0]
    kh2 = 4.0 / hx ** 2 * np.sin(np.pi * k * hx / p.L[0]) ** 2
    grad = 0.5 * p.gamma * eps ** 2 * kh2 / 2 * area
    e_bulk_mode = np.sum(0.5 * p.alpha * (u0 + du) * (1 - u0 - du) - 0.5 * p.beta * v0 ** 2
                         + p.theta * (O.Phi(u0 + du + v0) + O.Phi(u0 + du - v0))) * hx * (p.L[1] / p.n[1])
    assert O.energy(p, u + du, v) == pytest.approx(e_bulk_mode + grad, rel=1e-13)


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
@pytest.mark.parametrize("dim", [2, 3])
def test_dvd_identity_exact_G2(bc, dim):
    """E~(U1) - E~(U0) = <G~ . (U1 - U0)> with the exact quotient G2 (Eq. DVD, D2)."""
    p = _params(dim, bc, n=(9, 7, 6))
    g = O.grid_for(p)
    (X1, X0) = perturbed_pair(p, 21, u_mean=0.45, amp=0.1, step_amp=0.05)
    Gu, Gv = O.G_tilde(p, g, *X1, *X0, exact=True)
    vol = g.cell_volume
    lhs = O.energy(p, *X1) - O.energy(p, *X0)
    rhs = np.sum(Gu * (X1[0] - X0[0]) + Gv * (X1[1] - X0[1])) * vol
    assert lhs == pytest.approx(rhs, rel=1e-10, abs=1e-14)


def test_series_G2_close_to_exact_G2():
    """G2^S differs from the exact G2 only by the series remainder R^S (Eq. D2-1)."""
    p = _params(2, BC_PERIODIC)
    g = O.grid_for(p)
    (X1, X0) = perturbed_pair(p, 3, u_mean=0.5, amp=0.1, step_amp=0.02)
    Gs = O.G_tilde(p, g, *X1, *X0)
    Ge = O.G_tilde(p, g, *X1, *X0, exact=True)
    # |sigma/zeta| <= 0.02/0.3 here, so the S=10 remainder is far below round-off of Ge
    for a, b in zip(Gs, Ge):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-10)
