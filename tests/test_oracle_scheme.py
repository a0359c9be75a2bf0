"""Pins of the oracle's residual, Jacobian, ILU(0), Schwarz/GMRES solve, Newton
iteration and time stepping against closed forms, finite differences, a dense
direct solve and the invariants the paper proves (Theorem 2.3, mass)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import acac_oracle as O
from workloads import (BC_NEUMANN, BC_PERIODIC, DT_ADAPTIVE, Params, initial_fields,
                       perturbed_pair, random_vector)


def _F(p, X0, dt):
    def f(x):
        return O.interleave(*O.residual(p, O.deinterleave(x, p.shape), X0, dt))
    return f


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
@pytest.mark.parametrize("dim,n", [(2, (8, 7, 1)), (3, (5, 4, 6))])
def test_jacobian_matches_central_differences(bc, dim, n):
    p = Params(dim=dim, n=n, bc=bc, ras_parts=(2, 2, 2))
    X1, X0 = perturbed_pair(p, 4, u_mean=0.45, amp=0.1, step_amp=0.01)
    dt = 3e-3
    J = O.jacobian(p, X1, X0, dt)
    f = _F(p, X0, dt)
    x = O.interleave(*X1)
    rng = np.random.default_rng(1)
    for _ in range(3):
        w = rng.standard_normal(x.size)
        h = 1e-6
        fd = (f(x + h * w) - f(x - h * w)) / (2 * h)
        assert np.linalg.norm(fd - J @ w) <= 1e-6 * np.linalg.norm(fd)
    # pattern: the full 2x2-block radius-2 stencil, 13 (2D) / 25 (3D) blocks per interior cell
    nblk = 13 if dim == 2 else 25
    if bc == BC_PERIODIC and min(n[:dim]) >= 5:
        assert J.nnz == 4 * nblk * np.prod(n[:dim])


def test_steady_state_and_v_zero_invariance():
    """Constant u with v = 0 is a fixed point: F(U, U) = 0, zero Newton iterations;
    v = 0 stays exactly 0 (G_v = 0 when p = q)."""
    p = Params(n=(12, 12, 1), ras_parts=(2, 2, 1))
    u = np.full(p.shape, 0.37)
    v = np.zeros(p.shape)
    Fu, Fv = O.residual(p, (u, v), (u, v), 1e-2)
    assert np.max(np.abs(Fu)) == 0.0 and np.max(np.abs(Fv)) == 0.0
    X, info = O.nks_solve(p, (u, v), 1e-2)
    assert info.status == O.OK and info.newton_its == 0
    rng = np.random.default_rng(2)
    u = 0.4 + 0.05 * rng.uniform(-1, 1, p.shape)
    X, info = O.nks_solve(p.replace(newton_rtol=1e-12), (u, v), 1e-3)
    assert info.status == O.OK and np.max(np.abs(X[1])) == 0.0


def test_u_v_symmetry():
    """(u, v) -> (u, -v) maps the scheme onto itself."""
    p = Params(n=(10, 10, 1), ras_parts=(2, 2, 1), newton_rtol=1e-12)
    u, v = initial_fields(p, 9, 0.45, 0.05)
    Xa, ia = O.nks_solve(p, (u, v), 2e-3)
    Xb, ib = O.nks_solve(p, (u, -v), 2e-3)
    np.testing.assert_allclose(Xa[0], Xb[0], rtol=0, atol=1e-13)
    np.testing.assert_allclose(Xa[1], -Xb[1], rtol=0, atol=1e-13)


@pytest.mark.parametrize("which", ["u", "v"])
def test_linear_mode_growth_factor(which):
    """A small Fourier mode on a constant state (u0, 0) is multiplied per step by
    (1 - dt lam/2)/(1 + dt lam/2), with k_h^2 = sum (4/h^2) sin^2(pi k h) and
      u-mode: lam = c0 k_h^2 (-alpha + 2 theta/(u0(1-u0)) + gamma k_h^2),
      v-mode: lam = (c0/rho)(-beta + 2 theta/(u0(1-u0)) + gamma k_h^2),  c0 = u0(1-u0)/4."""
    p = Params(n=(16, 16, 1), ras_parts=(2, 2, 1), newton_rtol=1e-6, newton_atol=1e-12,
               gmres_rtol=1e-12, gamma=2e-3, rho=0.5)
    u0, eps, k, dt = 0.35, 1e-7, 2, 5e-3
    h = 1.0 / 16
    x = (np.arange(16) + 0.5) * h
    mode = np.cos(2 * np.pi * k * x)[None, :] * np.ones((16, 1))
    kh2 = 4.0 / h ** 2 * math.sin(math.pi * k * h) ** 2
    c0 = u0 * (1 - u0) / 4
    if which == "u":
        U = (u0 + eps * mode, np.zeros(p.shape))
        lam = c0 * kh2 * (-p.alpha + 2 * p.theta / (u0 * (1 - u0)) + p.gamma * kh2)
    else:
        U = (np.full(p.shape, u0), eps * mode)
        lam = c0 / p.rho * (-p.beta + 2 * p.theta / (u0 * (1 - u0)) + p.gamma * kh2)
    X, info = O.nks_solve(p, U, dt)
    assert info.status == O.OK
    comp = 0 if which == "u" else 1
    amp = np.sum((X[comp] - (u0 if which == "u" else 0.0)) * mode) / np.sum(mode * mode)
    expect = eps * (1 - dt * lam / 2) / (1 + dt * lam / 2)
    assert amp == pytest.approx(expect, rel=1e-5)


def test_ilu0_defining_property():
    """ILU(0): (L U)_ij = A_ij on the pattern of A; exact LU when no fill is possible."""
    p = Params(n=(8, 8, 1), ras_parts=(2, 2, 1), ras_overlap=1)
    X1, X0 = perturbed_pair(p, 6)
    J = O.jacobian(p, X1, X0, 1e-3)
    ras = O.RAS(p, J)
    s = ras.subs[0]
    n = s.diag.size
    F = sp.csr_matrix((s.data, s.indices, s.indptr), shape=(n, n)).toarray()
    pat = sp.csr_matrix((np.ones_like(s.data), s.indices, s.indptr), shape=(n, n)).toarray() > 0
    Lm = np.tril(F, -1) + np.eye(n)
    Um = np.triu(F)
    A = J[s.idx][:, s.idx].toarray()
    prod = Lm @ Um
    assert np.max(np.abs((prod - A)[pat])) <= 1e-12 * np.max(np.abs(A))
    assert np.any(np.abs((prod - A)[~pat]) > 0)        # fill was dropped somewhere
    # tridiagonal: ILU(0) = LU, so the solve is exact
    m = 50
    rng = np.random.default_rng(0)
    T = sp.diags([rng.uniform(-1, 0, m - 1), rng.uniform(3, 4, m), rng.uniform(-1, 0, m - 1)],
                 [-1, 0, 1], format="csr")
    T.sort_indices()
    sub = O.Subdomain(cells=np.arange(m), owned=np.ones(m, bool), box=(m,))
    sub.indptr, sub.indices = T.indptr.astype(np.int32), T.indices.astype(np.int32)
    sub.data, sub.diag = T.data.copy(), np.zeros(m, np.int32)
    lib = O._lib()
    assert lib.oracle_ilu0_factor(m, O._iptr(sub.indptr), O._iptr(sub.indices),
                                  O._dptr(sub.data), O._iptr(sub.diag)) == 0
    b = rng.standard_normal(m)
    x = O.RAS.solve_local(None, sub, b)
    np.testing.assert_allclose(T @ x, b, rtol=0, atol=1e-13)


def test_subdomain_boxes():
    """Near-equal boxes (first N mod P one larger), extended by delta layers,
    wrapped when periodic, clipped at Neumann walls; owned parts partition the grid."""
    assert O.partition_1d(10, 3) == [(0, 4), (4, 7), (7, 10)]
    for bc in (BC_PERIODIC, BC_NEUMANN):
        p = Params(n=(13, 15, 1), bc=bc, ras_parts=(3, 2, 1), ras_overlap=2)
        subs = O.subdomains(p)
        owned = np.concatenate([s.cells[s.owned] for s in subs])
        assert np.array_equal(np.sort(owned), np.arange(13 * 15))
        s0 = subs[0]
        if bc == BC_PERIODIC:
            assert s0.box == (5 + 4, 8 + 4)
            assert s0.cells[0] == (15 - 2) * 13 + (13 - 2)     # wrapped corner
        else:
            assert s0.box == (5 + 2, 8 + 2)
            assert s0.cells[0] == 0
    with pytest.raises(ValueError):             # a periodic box may not wrap onto itself
        O.subdomains(Params(n=(13, 11, 1), ras_parts=(3, 2, 1), ras_overlap=2))


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
def test_gmres_schwarz_solution_matches_dense_solve(kind, bc):
    p = Params(n=(16, 16, 1), bc=bc, ras_parts=(2, 2, 1), ras_overlap=1, ras_type=kind)
    X1, X0 = perturbed_pair(p, 8, u_mean=0.45, amp=0.05, step_amp=1e-3)
    J = O.jacobian(p, X1, X0, 2e-3)
    b = O.interleave(*random_vector(p, 3))
    prec = O.RAS(p, J, {0: "left", 1: "as", 2: "right"}[kind])
    res = O.gmres(lambda w: J @ w, prec.apply, b, 1e-11, 0.0, restart=30, maxit=500)
    assert res.converged
    xd = np.linalg.solve(J.toarray(), b)
    assert np.linalg.norm(res.x - xd) <= 1e-9 * np.linalg.norm(xd)
    assert np.linalg.norm(J @ res.x - b) <= 1.5e-11 * np.linalg.norm(b)


def test_block_jacobi_limits_agree():
    """delta = 0: left-RAS, AS and right-RAS all reduce to block Jacobi."""
    p = Params(n=(12, 12, 1), ras_parts=(3, 2, 1), ras_overlap=0)
    X1, X0 = perturbed_pair(p, 2)
    J = O.jacobian(p, X1, X0, 1e-3)
    r = O.interleave(*random_vector(p, 4))
    zs = [O.RAS(p, J, k).apply(r) for k in ("left", "as", "right")]
    np.testing.assert_allclose(zs[0], zs[1], rtol=0, atol=1e-14)
    np.testing.assert_allclose(zs[0], zs[2], rtol=0, atol=1e-14)


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
def test_nks_root_equals_dense_newton_root(bc):
    p = Params(n=(16, 16, 1), bc=bc, ras_parts=(2, 2, 1), ras_overlap=1,
               newton_rtol=1e-12, gmres_rtol=1e-8)
    u, v = initial_fields(p, 5, 0.5, 0.05)
    Xa, ia = O.nks_solve(p, (u, v), 2e-3, "nks")
    Xb, ib = O.nks_solve(p, (u, v), 2e-3, "dense")
    assert ia.status == ib.status == O.OK
    for a, b in zip(Xa, Xb):
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
def test_energy_dissipation_and_mass(bc):
    """Theorem 2.3: E~ non-increasing at every accepted step; sum u conserved."""
    p = Params(n=(24, 24, 1), bc=bc, ras_parts=(3, 3, 1), ras_overlap=1, dt0=5e-3)
    u, v = initial_fields(p, 12, 0.45, 0.05)
    st = O.Stepper(p)
    E, M = O.energy(p, u, v), O.mass(p, u)
    for _ in range(6):
        X, info = st.step(u, v)
        assert info.status == O.OK
        assert info.energy <= E + 1e-14 * abs(E)
        assert abs(info.mass - M) <= 1e-12 * abs(M)
        E = info.energy
        u, v = X


def test_adaptive_dt_predictor_formula():
    """Eq. sencondt: dt~ = max(dt_min, dt_max / sqrt(1 + eta X_d'^2))."""
    p = Params(n=(4, 4, 1), dt_mode=DT_ADAPTIVE, dt0=1e-4, dt_min=1e-5, dt_max=1e-1, eta0=100.0)
    st = O.Stepper(p)
    u = np.full(p.shape, 0.4)
    v = np.zeros(p.shape)
    assert st.predict(u, v) == 1e-4
    st.prev, st.dt_prev = (u - 1e-3, v), 1e-3
    xd = math.sqrt(16 * 1e-6) / 1e-3
    assert st.predict(u, v) == pytest.approx(max(1e-5, 1e-1 / math.sqrt(1 + 100 * xd * xd)),
                                             rel=1e-15)
    st.prev = (u - 1.0, v)
    assert st.predict(u, v) == 1e-5


def test_divergence_paths():
    """Fixed dt: divergence is an error.  Adaptive: dt / sqrt 2 and eta * 2 per retry,
    dt below dt_min is an underflow error."""
    p = Params(n=(12, 12, 1), ras_parts=(2, 2, 1), newton_maxit=1, newton_rtol=1e-14,
               newton_atol=0.0)
    u, v = initial_fields(p, 1, 0.5, 0.05)
    X, info = O.Stepper(p).step(u, v)
    assert info.status == O.E_DIVERGED
    pa = p.replace(dt_mode=DT_ADAPTIVE, dt0=1e-3, dt_min=2e-4, eta0=10.0)
    st = O.Stepper(pa)
    X, info = st.step(u, v)
    assert info.status == O.E_DT_UNDERFLOW
    assert info.divergences == 5            # 1e-3 / sqrt(2)^k >= 2e-4 for k <= 4
    assert st.eta == 10.0 * 2 ** 5
    bad = u.copy()
    bad[0, 0] = 1.2
    X, info = O.Stepper(p).step(bad, v)
    assert info.status == O.E_DOMAIN


def _e1_initial(p):
    """Sec. 4.1 A: u = 0.4(sin^2(2 pi x) + cos^2(2 pi y)) + 0.1,
    v = 0.4(sin^2(2 pi x) - cos^2(2 pi y))."""
    h = 1.0 / p.n[0]
    x = (np.arange(p.n[0]) + 0.5) * h
    y = (np.arange(p.n[1]) + 0.5) * h
    X, Y = np.meshgrid(x, y)
    u = 0.4 * (np.sin(2 * np.pi * X) ** 2 + np.cos(2 * np.pi * Y) ** 2) + 0.1
    v = 0.4 * (np.sin(2 * np.pi * X) ** 2 - np.cos(2 * np.pi * Y) ** 2)
    return u, v


def _run(p, T, dt, mode="midpoint"):
    u, v = _e1_initial(p)
    for _ in range(int(round(T / dt))):
        X, info = O.nks_solve(p, (u, v), dt, "nks", mode)
        assert info.status == O.OK
        u, v = X
    return u, v


def _paper_coeffs(n):
    # Sec. 4.1 A coefficients
    return Params(n=(n, n, 1), alpha=4.0, beta=2.0, gamma=0.005, theta=0.1, rho=0.001,
                  ras_parts=(2, 2, 1), ras_overlap=1, newton_rtol=1e-12, gmres_rtol=1e-10)


@pytest.mark.parametrize("mode,order", [("midpoint", 2.0), ("explicit", 1.0)])
def test_temporal_order(mode, order):
    """Fig. 1(b): second order in time with the midpoint mobility; the mobility
    frozen at U^n drops to first order (Sec. 2, trapezoidal rule reading)."""
    p = _paper_coeffs(16)
    T = 4e-3
    sols = [_run(p, T, dt, mode) for dt in (1e-3, 5e-4, 2.5e-4)]
    e1 = np.linalg.norm(sols[0][0] - sols[1][0]) + np.linalg.norm(sols[0][1] - sols[1][1])
    e2 = np.linalg.norm(sols[1][0] - sols[2][0]) + np.linalg.norm(sols[1][1] - sols[2][1])
    rate = math.log2(e1 / e2)
    assert abs(rate - order) < 0.25, rate


def test_spatial_order():
    """Fig. 1(a): second order in space (self-convergence, 2x2 cell averages)."""
    T, dt = 2e-3, 2.5e-4
    sols = {n: _run(_paper_coeffs(n), T, dt) for n in (16, 32, 64)}

    def coarsen(a):
        return 0.25 * (a[0::2, 0::2] + a[1::2, 0::2] + a[0::2, 1::2] + a[1::2, 1::2])

    def err(nc, nf):
        uc, vc = sols[nc]
        uf, vf = sols[nf]
        return math.sqrt(np.mean((uc - coarsen(uf)) ** 2 + (vc - coarsen(vf)) ** 2))

    rate = math.log2(err(16, 32) / err(32, 64))
    assert abs(rate - 2.0) < 0.3, rate
