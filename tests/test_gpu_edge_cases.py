"""GPU path against the CPU FP64 oracle where the discrete variational derivative is
hardest: near pure phases (u + v or u - v within 1e-8..1e-3 of 0 or 1, v near +-1/2)
and at large series ratios |sigma/zeta|, |sigma/(1 - zeta)| up to 0.7 (Lemma 2.2,
Eq. D2-1; the admissible set of Sec. 2), element by element on the same seeded inputs.

These inputs drive the kernels' warp-uniform choice of the number of series terms
through every case (a handful of terms where the ratios are tiny, all S terms where a
ratio reaches 1/2), the logarithm at arguments within 1e-8 of 0 and of 1, and the
float Jacobian of the mixed form at derivatives of order 1e8.

Tolerances as in the other parity tests: single evaluations within 1e-12 of the
largest entry (FP64) or 1e-5 (float Jacobian action), the energy within 1e-13
relative.  Newton solves near pure phases stop on an absolute residual of 1e-10 (the
residual's rounding floor there is about 1e-12, below the relative target), and the
roots agree within 1e-9 (FP64) / 1e-8 (mixed) relative L2.
"""
import numpy as np
import pytest

from oracle import acac_oracle as O
from tests._helpers import (dev, host, interleaved_to_soa, lib_built, need_cuda, soa,
                            soa_to_interleaved, stencil_J_to_csr)
from workloads import (BC_NEUMANN, BC_PERIODIC, PREC_MIXED, Params, near_pure_pair, near_pure_state,
                       random_vector)

pytestmark = pytest.mark.gpu

GRIDS = [((37, 29, 1), (3, 2, 1)), ((64, 48, 1), (4, 3, 1))]
# the paper's Sec. 4.1 coefficients with a smaller theta: the near-pure states below are
# then close to equilibrium, so that one implicit step stays near the pure phase
NEAR = dict(alpha=4.0, beta=2.0, gamma=0.005, rho=1.0)


@pytest.fixture(scope="module")
def P():
    need_cuda()
    return lib_built()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _ratios(X1, X0):
    """max |sigma/zeta|, |sigma/(1 - zeta)| over p = u + v and q = u - v."""
    out = 0.0
    for sgn in (1.0, -1.0):
        a1, a0 = X1[0] + sgn * X1[1], X0[0] + sgn * X0[1]
        z, s = 0.5 * (a1 + a0), 0.5 * (a1 - a0)
        out = max(out, float(np.max(np.abs(s / z))), float(np.max(np.abs(s / (1.0 - z)))))
    return out


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
@pytest.mark.parametrize("grid", GRIDS)
def test_residual_energy_near_pure(P, bc, grid):
    import torch
    n, parts = grid
    p = Params(n=n, bc=bc, ras_parts=parts)
    X1, X0 = near_pure_pair(p, 51)
    dt = 2e-3
    Fo = soa(*O.residual(p, X1, X0, dt))
    with P.Solver(p) as s:
        F = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
        fn = s.residual(dev(soa(*X1)), dev(soa(*X0)), dt, F)
        e, m = s.energy(dev(X0[0].ravel()), dev(X0[1].ravel()))
        torch.cuda.synchronize()
    assert _rel(host(F), Fo) <= 1e-12
    assert fn == pytest.approx(np.linalg.norm(Fo), rel=1e-12)
    assert e == pytest.approx(O.energy(p, *X0), rel=1e-13)
    assert m == pytest.approx(O.mass(p, X0[0]), rel=1e-14)


@pytest.mark.parametrize("ratio_max", [1e-4, 0.05, 0.3, 0.7])
def test_residual_series_term_counts(P, ratio_max):
    """Ratios capped at 1e-4 .. 0.7: the kernels sum from a few up to all S terms (per
    warp); every case agrees with the oracle's S-term sum."""
    import torch
    p = Params(n=(64, 48, 1), ras_parts=(4, 3, 1))
    X1, X0 = near_pure_pair(p, 53, frac=0.3, ratio_max=ratio_max)
    dt = 1e-3
    Fo = soa(*O.residual(p, X1, X0, dt))
    with P.Solver(p) as s:
        F = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
        s.residual(dev(soa(*X1)), dev(soa(*X0)), dt, F)
        torch.cuda.synchronize()
    assert _rel(host(F), Fo) <= 1e-12


def test_residual_energy_near_pure_3d(P):
    import torch
    p = Params(dim=3, n=(12, 11, 10), L=(1.0, 0.9, 1.1), bc=BC_NEUMANN, ras_parts=(2, 2, 2))
    X1, X0 = near_pure_pair(p, 55)
    dt = 2e-3
    Fo = soa(*O.residual(p, X1, X0, dt))
    with P.Solver(p) as s:
        F = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
        s.residual(dev(soa(*X1)), dev(soa(*X0)), dt, F)
        e, m = s.energy(dev(X1[0].ravel()), dev(X1[1].ravel()))
        torch.cuda.synchronize()
    assert _rel(host(F), Fo) <= 1e-12
    assert e == pytest.approx(O.energy(p, *X1), rel=1e-13)
    assert m == pytest.approx(O.mass(p, X1[0]), rel=1e-14)


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
@pytest.mark.parametrize("grid", GRIDS)
def test_jacobian_jvp_near_pure(P, bc, grid):
    import torch
    n, parts = grid
    p = Params(n=n, bc=bc, ras_parts=parts)
    X1, X0 = near_pure_pair(p, 57)
    dt = 2e-3
    Jo = O.jacobian(p, X1, X0, dt)
    w = soa(*random_vector(p, 59))
    yo = interleaved_to_soa(Jo @ soa_to_interleaved(w))
    with P.Solver(p) as s:
        J = torch.empty(52 * p.ncells, dtype=torch.float64, device="cuda")
        s.jacobian(dev(soa(*X1)), dev(soa(*X0)), dt, J)
        y1 = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
        y2 = torch.empty_like(y1)
        s.spmv(J, dev(w), y1)
        s.jvp(dev(soa(*X1)), dev(soa(*X0)), dt, dev(w), y2)
        torch.cuda.synchronize()
        Jg = stencil_J_to_csr(host(J), p)
    D = (Jg - Jo).tocoo()
    assert np.max(np.abs(D.data), initial=0.0) <= 1e-12 * np.max(np.abs(Jo.data))
    assert _rel(host(y1), yo) <= 1e-12
    assert _rel(host(y2), yo) <= 1e-12


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
@pytest.mark.parametrize("grid", GRIDS + [((130, 17, 1), (4, 2, 1))])
def test_jvp_fp32_near_pure(P, bc, grid):
    """Mixed form's tiled float Jacobian action near pure phases (derivatives of the
    logarithm up to 1e8) against the FP64 oracle: 1e-5 of max |J w|."""
    import torch
    n, parts = grid
    p = Params(n=n, bc=bc, ras_parts=parts, precision=PREC_MIXED)
    X1, X0 = near_pure_pair(p, 61)
    dt = 2e-3
    Jo = O.jacobian(p, X1, X0, dt)
    w = soa(*random_vector(p, 63))
    yo = interleaved_to_soa(Jo @ soa_to_interleaved(w))
    with P.Solver(p) as s:
        y = torch.empty(2 * p.ncells, dtype=torch.float32, device="cuda")
        s.jvp(dev(soa(*X1)), dev(soa(*X0)), dt, dev(w, torch.float32), y)
        torch.cuda.synchronize()
    assert _rel(host(y), yo) <= 1e-5


# (theta, eps_p, eps_q, dt, flip): start states 1e-8 .. 1e-3 from the pure phase, steps whose
# series ratios reach 0.3 .. 0.55 (checked below)
NKS_CASES = [(0.02, 1e-8, 1e-8, 1e-2, False), (0.1, 1e-6, 1e-4, 1e-4, True), (0.02, 1e-3, 1e-3, 1e-1, False)]


def _nks_near_pure(P, case, bc, precision):
    import torch
    theta, ep, eq, dt, flip = case
    base = Params(n=(48, 40, 1), L=(0.75, 0.625, 1.0), bc=bc, ras_parts=(3, 2, 1), ras_overlap=2,
                  theta=theta, newton_rtol=1e-12, newton_atol=1e-10, **NEAR)
    U0 = near_pure_state(base, 71, ep, eq, flip=flip)
    Xo, io = O.nks_solve(base.replace(gmres_rtol=1e-8), U0, dt)
    assert io.status == 0
    pg = base.replace(precision=precision, gmres_rtol=1e-8 if precision == 0 else 1e-6)
    with P.Solver(pg) as s:
        U1 = torch.empty(2 * pg.ncells, dtype=torch.float64, device="cuda")
        ig = s.nks_solve(dev(soa(*U0)), dt, U1)
        Xg = host(U1)
    return U0, Xo, io, Xg, ig


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
@pytest.mark.parametrize("case", NKS_CASES)
def test_nks_step_near_pure_fp64(P, case, bc):
    U0, Xo, io, Xg, ig = _nks_near_pure(P, case, bc, 0)
    xo = soa(*Xo)
    assert ig.status == 0
    assert np.linalg.norm(Xg - xo) <= 1e-9 * np.linalg.norm(xo)
    assert abs(ig.newton_its - io.newton_its) <= 1
    assert _ratios(Xo, U0) >= 0.25                 # the step really moved far in the series
    n = Xg.size // 2
    pq = np.concatenate([Xg[:n] + Xg[n:], Xg[:n] - Xg[n:]])
    assert pq.min() > 0.0 and pq.max() < 1.0


@pytest.mark.parametrize("case", NKS_CASES)
def test_nks_step_near_pure_mixed(P, case):
    U0, Xo, io, Xg, ig = _nks_near_pure(P, case, BC_PERIODIC, PREC_MIXED)
    xo = soa(*Xo)
    assert ig.status == 0
    assert np.linalg.norm(Xg - xo) <= 1e-8 * np.linalg.norm(xo)
