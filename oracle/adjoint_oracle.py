"""CPU FP64 oracle of the adjoint (reverse-mode derivative) of the implicit DVD time
step, for gradients of a loss of the final state with respect to the initial fields
and the coefficients alpha, beta, theta, gamma.

TEST INFRASTRUCTURE ONLY, like acac_oracle: only the tests, the smoke check and the
benchmark's CPU legs may import it; the CUDA library shares no code with it.

The paper solves forward only.  The adjoint here is the plain chain rule applied to
the scheme as acac_oracle defines it (scheme NSOA-1 of Sec. 2 at a fixed dt):

  step n:   F(U^{n+1}, U^n; p) = 0,  n = 0..K-1,   loss  L(U^K; p).

With lambda^K = dL/dU^K, going backwards, for every step
  J1^T mu = lambda^{n+1},        J1 = dF/dU^{n+1} at (U^{n+1}, U^n)
  lambda^n = -J0^T mu,           J0 = dF/dU^n
  dL/dp   += -mu^T dF/dp,
and dL/dU^0 = lambda^0, dL/dp = the sum plus the explicit dL/dp of the loss.  The
linear solves are dense (small grids only).

Loss: L = w_E E~(U^K) + (w_M / 2) sum_cells [(u - u*)^2 + (v - v*)^2] dx dy, with E~
the discrete free energy of Eq. freeenergy.

Vectors are in the state layout [u | v] (each field flattened, x fastest).

Parity pins: tests/test_oracle_adjoint.py compares every derivative here with central
finite differences of acac_oracle's residual, energy and time stepping.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from oracle import acac_oracle as O

PARAMS = ("alpha", "beta", "theta", "gamma")


# --------------------------------------------------------------------------- one step
def jacobians(p, X1, X0, dt, g=None):
    """(J1, J0) = (dF/dX1, dF/dX0) as sparse 2N x 2N matrices in the [u | v] layout,
    by the chain rule on acac_oracle.residual.

    X0 enters F through the time difference (-1/dt on the diagonal), through
    G1 and G3 exactly as X1 does (they depend on u1 + u0), through the mobility at
    the midpoint (again as X1 does), and through G2^S = theta (phi + psi, phi - psi)
    with phi = phi^S(zeta, sigma): zeta = (p1 + p0)/2 moves by +1/2 and
    sigma = (p1 - p0)/2 by -1/2 when p0 grows, so d phi/d p0 = (d_zeta - d_sigma)/2
    while d phi/d p1 = (d_zeta + d_sigma)/2."""
    g = g or O.grid_for(p)
    N = g.N
    u1, v1 = X1
    u0, v0 = X0
    I = sp.identity(N, format="csr")
    diag = lambda a: sp.diags(np.asarray(a).ravel(), format="csr")
    ub, vb = 0.5 * (u1 + u0), 0.5 * (v1 + v0)
    c = O.mobility(ub, vb).ravel()
    cu = (0.5 * (1.0 - 2.0 * ub) * (0.25 - vb * vb)).ravel()     # dc/du1 = dc/du0
    cv = (0.5 * ub * (1.0 - ub) * (-2.0 * vb)).ravel()           # dc/dv1 = dc/dv0
    Gu, Gv = (a.ravel() for a in O.G_tilde(p, g, u1, v1, u0, v0))
    zp, sp_, zq, sq, omp, omq = O._pq(u1, v1, u0, v0)
    dzp, dsp = O.dphi_S(zp, sp_, p.taylor_S, omp)
    dzq, dsq = O.dphi_S(zq, sq, p.taylor_S, omq)
    out = []
    for sgn, tsign in ((1.0, 1.0), (-1.0, -1.0)):      # X1, then X0
        A = (p.theta * 0.5 * (dzp + sgn * dsp)).ravel()   # theta d phi / d p
        B = (p.theta * 0.5 * (dzq + sgn * dsq)).ravel()   # theta d psi / d q
        dGu_du = diag(-0.5 * p.alpha + A + B) - 0.5 * p.gamma * g.Lap
        dGu_dv = diag(A - B)
        dGv_du = diag(A - B)
        dGv_dv = diag(-0.5 * p.beta + A + B) - 0.5 * p.gamma * g.Lap
        Juu = tsign * I / dt
        Juv = sp.csr_matrix((N, N))
        for d in range(p.dim):
            h = g.h[d]
            gradG = diag(g.Df[d] @ Gu / h)
            cface = diag(g.Af[d] @ c)
            Juu = Juu - g.Dv[d] @ (gradG @ g.Af[d] @ diag(cu) + cface @ g.Df[d] @ dGu_du / h) / h
            Juv = Juv - g.Dv[d] @ (gradG @ g.Af[d] @ diag(cv) + cface @ g.Df[d] @ dGu_dv / h) / h
        Jvu = (diag(Gv * cu) + diag(c) @ dGv_du) / p.rho
        Jvv = tsign * I / dt + (diag(Gv * cv) + diag(c) @ dGv_dv) / p.rho
        out.append(sp.bmat([[Juu, Juv], [Jvu, Jvv]], format="csr"))
    return out[0], out[1]


def dF_dparams(p, X1, X0, dt, g=None):
    """{name: dF/dp} for p in alpha, beta, theta, gamma, each a [u | v] vector.

    F_u = (u1-u0)/dt - div(c~ grad G_u) and F_v = (v1-v0)/dt + c G_v / rho, where
    c does not depend on the coefficients and G~ is linear in each of them:
      dG/dalpha = (-(u1+u0-1)/2, 0),          dG/dbeta  = (0, -(v1+v0)/2),
      dG/dtheta = (phi + psi, phi - psi),     dG/dgamma = -(Delta(u1+u0), Delta(v1+v0))/2."""
    g = g or O.grid_for(p)
    u1, v1 = X1
    u0, v0 = X0
    c = O.mobility_state(u1, v1, u0, v0)
    zp, sp_, zq, sq, omp, omq = O._pq(u1, v1, u0, v0)
    phi = O.phi_S(zp, sp_, p.taylor_S, omp)
    psi = O.phi_S(zq, sq, p.taylor_S, omq)
    zero = np.zeros(p.shape)
    dG = {
        "alpha": (-0.5 * (u1 + u0 - 1.0), zero),
        "beta": (zero, -0.5 * (v1 + v0)),
        "theta": (phi + psi, phi - psi),
        "gamma": (-0.5 * (g.lap(u1) + g.lap(u0)), -0.5 * (g.lap(v1) + g.lap(v0))),
    }
    out = {}
    for name, (gu, gv) in dG.items():
        fu = -g.mob_div(c, gu)
        fv = c * gv / p.rho
        out[name] = np.concatenate([fu.ravel(), fv.ravel()])
    return out


# --------------------------------------------------------------------------- loss
def loss(p, X, target, w_energy=1.0, w_misfit=1.0):
    """w_E E~(X) + (w_M/2) sum [(u - u*)^2 + (v - v*)^2] dx dy."""
    u, v = X
    ut, vt = target
    vol = O.grid_for(p).cell_volume
    mis = 0.5 * vol * float(np.sum((u - ut) ** 2) + np.sum((v - vt) ** 2))
    return w_energy * O.energy(p, u, v) + w_misfit * mis


def loss_grad(p, X, target, w_energy=1.0, w_misfit=1.0):
    """(dL/dX as a [u | v] vector, {name: dL/dp}) of loss() at X.

    E~ = sum e~ dx dy with e~ = alpha/2 u(1-u) - beta/2 v^2 + theta(Phi(u+v) + Phi(u-v))
    + gamma/4 sum_d ((D+ u)^2 + (D- u)^2 + (D+ v)^2 + (D- v)^2) (Eq. relations).  Each
    face difference appears once as a D+ and once as a D- term, so the gradient part
    of E~ is (gamma/2) sum over faces of the squared differences, whose derivative in
    u at a cell is -gamma [Delta u] there; Phi'(z) = ln z - ln(1-z)."""
    g = O.grid_for(p)
    u, v = X
    ut, vt = target
    vol = g.cell_volume
    pp, qq = u + v, u - v
    mp, mq = O.one_minus_pq(u, v)                  # 1 - p, 1 - q (accurate near p, q -> 1)
    lp = np.log(pp) - np.log(mp)
    lq = np.log(qq) - np.log(mq)
    dEu = 0.5 * p.alpha * (1.0 - 2.0 * u) + p.theta * (lp + lq) - p.gamma * g.lap(u)
    dEv = -p.beta * v + p.theta * (lp - lq) - p.gamma * g.lap(v)
    du = vol * (w_energy * dEu + w_misfit * (u - ut))
    dv = vol * (w_energy * dEv + w_misfit * (v - vt))
    grad_terms = 0.0
    for phi in (u, v):
        for d in range(p.dim):
            dp, dm = O._dplus_dminus(phi, p, d)
            grad_terms = grad_terms + 0.25 * (dp * dp + dm * dm)
    dp_ = {
        "alpha": w_energy * vol * float(np.sum(0.5 * u * (1.0 - u))),
        "beta": w_energy * vol * float(np.sum(-0.5 * v * v)),
        "theta": w_energy * vol * float(np.sum(O.Phi(pp, mp) + O.Phi(qq, mq))),
        "gamma": w_energy * vol * float(np.sum(grad_terms)),
    }
    return np.concatenate([du.ravel(), dv.ravel()]), dp_


# --------------------------------------------------------------------------- K steps
def forward(p, U0, nsteps, dt, linear="dense"):
    """States U^0..U^K of K fixed-dt steps (each the Newton root of F = 0)."""
    q = p.replace(dt_mode=0, dt0=dt)
    states = [(U0[0].copy(), U0[1].copy())]
    for _ in range(nsteps):
        X, info = O.nks_solve(q, states[-1], dt, linear)
        if info.status != O.OK:
            raise RuntimeError("forward step failed: %s" % info.reason)
        states.append(X)
    return states


def forward_loss(p, U0, nsteps, dt, target, w_energy=1.0, w_misfit=1.0, linear="dense"):
    X = forward(p, U0, nsteps, dt, linear)[-1]
    return loss(p, X, target, w_energy, w_misfit)


def adjoint_gradient(p, U0, nsteps, dt, target, w_energy=1.0, w_misfit=1.0, every=5,
                     linear="dense"):
    """(loss, dL/du0, dL/dv0, {name: dL/dp}) by the adjoint recursion of the module
    docstring, with dense solves of J1^T mu = lambda.  The forward states are kept at
    every `every`-th step and the others recomputed segment by segment on the way
    back, as the GPU implementation does."""
    q = p.replace(dt_mode=0, dt0=dt)
    g = O.grid_for(q)
    ckpt = {}
    X = (U0[0].copy(), U0[1].copy())
    for n in range(nsteps):
        if n % every == 0:
            ckpt[n] = X
        X, info = O.nks_solve(q, X, dt, linear)
        if info.status != O.OK:
            raise RuntimeError("forward step failed: %s" % info.reason)
    L = loss(q, X, target, w_energy, w_misfit)
    lam, grad = loss_grad(q, X, target, w_energy, w_misfit)
    for start in sorted(ckpt, reverse=True):
        end = min(start + every, nsteps)
        seg = forward(q, ckpt[start], end - start, dt, linear)
        for n in range(end - 1, start - 1, -1):
            X1, X0 = seg[n + 1 - start], seg[n - start]
            J1, J0 = jacobians(q, X1, X0, dt, g)
            mu = np.linalg.solve(J1.toarray().T, lam)
            lam = -(J0.T @ mu)
            dF = dF_dparams(q, X1, X0, dt, g)
            for name in PARAMS:
                grad[name] -= float(mu @ dF[name])
    N = g.N
    return L, lam[:N].reshape(q.shape), lam[N:].reshape(q.shape), grad
