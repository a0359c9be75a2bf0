"""Adjoint of the implicit step on the GPU against the adjoint oracle
(oracle/adjoint_oracle.py, pinned to central differences of the forward oracle), and
the end-to-end gradient against central differences of the GPU's own forward loss."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import acac_oracle as O
from oracle import adjoint_oracle as A
from tests._helpers import dev, host, lib_built, need_cuda, soa, stencil_J_to_csr
from workloads import BC_NEUMANN, BC_PERIODIC, C5, Params, initial_fields, perturbed_pair

pytestmark = pytest.mark.gpu


def _soa_matrix(Ji, N):
    """Interleaved CSR (index 2c + dof) -> the [u | v] layout."""
    perm = np.empty(2 * N, dtype=np.int64)
    perm[0::2] = np.arange(N)
    perm[1::2] = N + np.arange(N)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(2 * N)
    P = sp.csr_matrix((np.ones(2 * N), (perm, np.arange(2 * N))), shape=(2 * N, 2 * N))
    return (P @ Ji @ P.T).tocsr()


CASES = [(2, (20, 17, 1), (2, 2, 1), BC_PERIODIC), (2, (19, 22, 1), (2, 3, 1), BC_NEUMANN),
         (3, (9, 8, 10, 1)[:3], (2, 2, 2), BC_NEUMANN)]


@pytest.mark.parametrize("dim,n,parts,bc", CASES)
def test_jacobian_x0_and_transposed_product(dim, n, parts, bc):
    """dF/dX0 in stencil storage equals the oracle's J0; J^T w equals the CSR transpose
    product (FP64, 1e-12 relative)."""
    need_cuda()
    P = lib_built()
    import torch
    p = Params(dim=dim, n=n, bc=bc, ras_parts=parts)
    X1, X0 = perturbed_pair(p, 3, u_mean=0.45, amp=0.08, step_amp=0.01)
    dt = 2e-3
    N = p.ncells
    with P.Solver(p) as s:
        J = torch.empty(4 * s.nslot * N, dtype=torch.float64, device="cuda")
        s.jacobian_x0(dev(soa(*X1)), dev(soa(*X0)), dt, J)
        J0g = _soa_matrix(stencil_J_to_csr(host(J), p), N)
        _, J0o = A.jacobians(p, X1, X0, dt)
        D = (J0g - J0o).toarray()
        assert np.abs(D).max() <= 1e-12 * np.abs(J0o.toarray()).max()
        w = np.random.default_rng(1).standard_normal(2 * N)
        y = torch.empty(2 * N, dtype=torch.float64, device="cuda")
        s.spmv_t(J, dev(w), y)
        ref = J0o.T @ w
        assert np.linalg.norm(host(y) - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
def test_loss_and_gradient(bc):
    need_cuda()
    P = lib_built()
    import torch
    p = Params(n=(33, 29, 1), bc=bc, ras_parts=(2, 2, 1))
    X = initial_fields(p, 8, 0.4, 0.08)
    T = initial_fields(p, 9, 0.5, 0.08)
    with P.Solver(p) as s:
        dX = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
        L, g = s.loss(dev(soa(*X)), dev(soa(*T)), 1.0, 0.6, dX)
    Lo = A.loss(p, X, T, 1.0, 0.6)
    dXo, go = A.loss_grad(p, X, T, 1.0, 0.6)
    assert L == pytest.approx(Lo, rel=1e-12)
    assert np.linalg.norm(host(dX) - dXo) <= 1e-12 * np.linalg.norm(dXo)
    for i, name in enumerate(A.PARAMS):
        assert g[i] == pytest.approx(go[name], rel=1e-11, abs=1e-15), name


@pytest.mark.parametrize("ras_type", [0, 1, 2])
def test_adjoint_step_matches_dense_solve(ras_type):
    """One adjoint step: lambda^n = -J0^T J1^{-T} lambda^{n+1} and -mu^T dF/dp against a
    dense solve (GMRES on J1^T to 1e-12)."""
    need_cuda()
    P = lib_built()
    p = Params(n=(24, 20, 1), ras_parts=(3, 2, 1), ras_overlap=1, ras_type=ras_type)
    X1, X0 = perturbed_pair(p, 12, u_mean=0.42, amp=0.06, step_amp=0.01)
    dt = 1e-3
    lam1 = np.random.default_rng(6).standard_normal(2 * p.ncells)
    with P.Solver(p) as s:
        lam0 = dev(np.zeros(2 * p.ncells))
        g, its = s.adjoint_step(dev(soa(*X1)), dev(soa(*X0)), dt, dev(lam1), lam0, rtol=1e-12)
    J1, J0 = A.jacobians(p, X1, X0, dt)
    mu = np.linalg.solve(J1.toarray().T, lam1)
    ref = -(J0.T @ mu)
    assert its > 0
    assert np.linalg.norm(host(lam0) - ref) <= 1e-9 * np.linalg.norm(ref)
    dF = A.dF_dparams(p, X1, X0, dt)
    for i, name in enumerate(A.PARAMS):
        assert g[i] == pytest.approx(-float(mu @ dF[name]), rel=1e-9), name


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
def test_adjoint_gradient_matches_dense_oracle(bc):
    """Seven steps at 16^2 with a checkpoint every 5 (a full and a partial segment):
    loss and every gradient entry against the oracle's dense adjoint."""
    need_cuda()
    P = lib_built()
    import torch
    p = Params(n=(16, 16, 1), bc=bc, ras_parts=(2, 2, 1), ras_overlap=1, newton_rtol=1e-12, newton_atol=1e-14)
    U0 = initial_fields(p, 41, 0.42, 0.05)
    T = initial_fields(p, 141, 0.45, 0.05)
    dt, K = 1e-3, 7
    Lo, duo, dvo, go = A.adjoint_gradient(p, U0, K, dt, T, 1.0, 1.5, every=5)
    with P.Solver(p) as s:
        L, du, dv, g, its = s.adjoint(dev(U0[0].ravel()), dev(U0[1].ravel()), K, dt, dev(T[0].ravel()),
                                      dev(T[1].ravel()), 1.0, 1.5, every=5, rtol=1e-12)
    torch.cuda.synchronize()
    assert L == pytest.approx(Lo, rel=1e-11)
    x, xo = soa(host(du), host(dv)), soa(duo, dvo)
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)
    for i, name in enumerate(A.PARAMS):
        assert g[i] == pytest.approx(go[name], rel=1e-8), name


def test_adjoint_c5_matches_central_differences():
    """The 512^2 adjoint workload (20 steps at dt = 1e-3, checkpoint every 5, loss = final
    energy + misfit): dL/d(alpha, beta, theta, gamma) and dL/dU0 in a random direction
    against central differences (relative step 1e-6) of the forward loss, to 1e-5."""
    need_cuda()
    P = lib_built()
    import torch
    w = C5
    p = w.params.replace(newton_rtol=1e-11, newton_atol=1e-14)
    u0, v0 = w.fields()
    ut, vt = w.target()
    U0, V0, UT, VT = (dev(a.ravel()) for a in (u0, v0, ut, vt))
    with P.Solver(p) as s:
        L, du, dv, g, its = s.adjoint(U0, V0, w.steps, p.dt0, UT, VT, w.w_energy, w.w_misfit, every=w.every,
                                      rtol=1e-11)

        def fwd(q, a, b):
            s.set_coeffs(0, q.alpha, q.beta, q.theta, q.gamma, q.rho)
            X = torch.cat([a, b])
            Y = torch.empty_like(X)
            for _ in range(w.steps):
                s.nks_solve(X, q.dt0, Y)
                X, Y = Y, X
            val, _ = s.loss(X, torch.cat([UT, VT]), w.w_energy, w.w_misfit, torch.empty_like(X))
            return val

        assert fwd(p, U0, V0) == pytest.approx(L, rel=1e-12)
        for i, name in enumerate(A.PARAMS):
            val = getattr(p, name)
            h = 1e-6 * val
            fd = (fwd(p.replace(**{name: val + h}), U0, V0) - fwd(p.replace(**{name: val - h}), U0, V0)) / (2 * h)
            assert g[i] == pytest.approx(fd, rel=1e-5), name
        s.set_coeffs(0, p.alpha, p.beta, p.theta, p.gamma, p.rho)
        rng = np.random.default_rng(7)
        wu, wv = dev(rng.standard_normal(p.ncells)), dev(rng.standard_normal(p.ncells))
        h = 1e-6
        fd = (fwd(p, U0 + h * wu, V0 + h * wv) - fwd(p, U0 - h * wu, V0 - h * wv)) / (2 * h)
        ad = float((du * wu).sum() + (dv * wv).sum())
        assert ad == pytest.approx(fd, rel=1e-5)


def test_autograd_function():
    """implicit_loss through torch.autograd: backward gives the adjoint's gradients, and
    the forward-only call (no gradient needed) gives the same loss."""
    need_cuda()
    P = lib_built()
    import torch
    from paper_2007_04560_gb300.autograd import implicit_loss
    p = Params(n=(32, 32, 1), ras_parts=(2, 2, 1), newton_rtol=1e-12, newton_atol=1e-14)
    u0, v0 = (dev(a) for a in initial_fields(p, 51, 0.42, 0.05))
    ut, vt = (dev(a) for a in initial_fields(p, 151, 0.45, 0.05))
    coeffs = torch.tensor([p.alpha, p.beta, p.theta, p.gamma], dtype=torch.float64, device="cuda",
                          requires_grad=True)
    u0.requires_grad_(True)
    v0.requires_grad_(True)
    with P.Solver(p) as s:
        L = implicit_loss(s, u0, v0, coeffs, 6, 1e-3, ut, vt, 1.0, 2.0, every=4, rtol=1e-12)
        L.backward()
        with torch.no_grad():
            L2 = implicit_loss(s, u0.detach(), v0.detach(), coeffs.detach(), 6, 1e-3, ut, vt, 1.0, 2.0)
        Lr, dur, dvr, gr, _ = s.adjoint(u0.detach().reshape(-1), v0.detach().reshape(-1), 6, 1e-3,
                                        ut.reshape(-1), vt.reshape(-1), 1.0, 2.0, every=3, rtol=1e-12)
    assert float(L.detach()) == pytest.approx(Lr, rel=1e-13) and float(L2) == pytest.approx(Lr, rel=1e-12)
    np.testing.assert_allclose(host(coeffs.grad), gr, rtol=1e-9)
    assert np.linalg.norm(host(u0.grad).ravel() - host(dur)) <= 1e-9 * np.linalg.norm(host(dur))
    assert np.linalg.norm(host(v0.grad).ravel() - host(dvr)) <= 1e-9 * np.linalg.norm(host(dvr))
