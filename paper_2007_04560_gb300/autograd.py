"""torch.autograd wrapper of the library's adjoint (acac_adjoint in include/acac.h).

`implicit_loss(solver, u0, v0, coeffs, ...)` returns L(U^K): the loss of the state after
K fixed-dt implicit steps of the scheme, L = w_E E~(U^K) + (w_M/2) |U^K - U*|^2 dx dy.
Its backward pass yields dL/du0, dL/dv0 and dL/d(alpha, beta, theta, gamma) from the
library's checkpointed adjoint recursion (transposed-Jacobian GMRES per step).

Argument marshalling only: the forward steps, the loss and the adjoint all run in
libacac.so's kernels.  When no input needs a gradient, only the forward steps and
the loss are computed.
"""
from __future__ import annotations

import torch

from . import acac as _A


class _ImplicitLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, v0, coeffs, solver, nsteps, dt, u_target, v_target, w_energy, w_misfit, every, rtol):
        c = [float(x) for x in coeffs.detach().cpu().tolist()]
        rho = float(solver.params.rho)
        solver.set_coeffs(0, c[0], c[1], c[2], c[3], rho)
        if any(ctx.needs_input_grad[:3]):
            L, du, dv, g, _ = solver.adjoint(u0.detach().contiguous(), v0.detach().contiguous(), nsteps, dt,
                                             u_target.contiguous(), v_target.contiguous(), w_energy, w_misfit,
                                             every, rtol)
            ctx.save_for_backward(du, dv, torch.tensor(g, dtype=coeffs.dtype, device=coeffs.device))
        else:
            n = u0.numel()
            X = torch.cat([u0.detach().reshape(-1), v0.detach().reshape(-1)])
            Y = torch.empty_like(X)
            for _ in range(nsteps):
                solver.nks_solve(X, dt, Y)
                X, Y = Y, X
            T = torch.cat([u_target.reshape(-1), v_target.reshape(-1)])
            L, _ = solver.loss(X, T, w_energy, w_misfit, torch.empty_like(X))
            assert X.numel() == 2 * n
        return torch.tensor(L, dtype=torch.float64, device=u0.device)

    @staticmethod
    def backward(ctx, gL):
        du, dv, g = ctx.saved_tensors
        return (gL * du, gL * dv, gL.to(g.device) * g) + (None,) * 9


def implicit_loss(solver, u0, v0, coeffs, nsteps, dt, u_target, v_target, w_energy=1.0, w_misfit=1.0,
                  every=5, rtol=1e-10):
    """L(U^K) after `nsteps` steps of size dt from (u0, v0) (float64 CUDA tensors of the
    grid's shape), with coeffs = tensor([alpha, beta, theta, gamma]) (float64; rho is
    the solver's).  Differentiable in u0, v0 and coeffs.  The solver must be an FP64,
    batch-1 handle; its coefficients are set from coeffs."""
    return _ImplicitLoss.apply(u0, v0, coeffs, solver, int(nsteps), float(dt), u_target, v_target,
                               float(w_energy), float(w_misfit), int(every), float(rtol))
