"""Subdomain solves with fill (ILU(1), ILU(2), exact LU; Sec. 4.2, Table 2) through the
C ABI against the oracle: the Schwarz preconditioner (three restriction / extension
types, 2D and 3D, both boundary conditions) and the Newton root of a time step.

Tolerances: the preconditioner goes through the factorization and both triangular sweeps
(1e-10 relative, FP64; 2e-4 in FP32 against the FP64 oracle); roots at 1e-9 relative L2
with Newton iterated to 1e-12 on both sides."""
import numpy as np
import pytest

from oracle import acac_oracle as O
from tests._helpers import dev, host, interleaved_to_soa, lib_built, need_cuda, soa, soa_to_interleaved
from workloads import (BC_NEUMANN, BC_PERIODIC, DT_ADAPTIVE, PREC_MIXED, SUB_ILU1, SUB_ILU2, SUB_LU, Params,
                       initial_fields, perturbed_pair, random_vector)

pytestmark = pytest.mark.gpu

CASES = [  # dim, n, parts, bc, overlap
    (2, (30, 22, 1), (3, 2, 1), BC_PERIODIC, 1),
    (2, (26, 21, 1), (2, 3, 1), BC_NEUMANN, 2),
    (3, (10, 9, 8), (2, 2, 2), BC_NEUMANN, 1),
]
KIND = {0: "left", 1: "as", 2: "right"}


@pytest.fixture(scope="module")
def P():
    need_cuda()
    return lib_built()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _apply_pair(P, p, seed=13):
    import torch
    X1, X0 = perturbed_pair(p, seed, u_mean=0.45, amp=0.05, step_amp=2e-3)
    dt = 2e-3
    Jo = O.jacobian(p, X1, X0, dt)
    r = soa(*random_vector(p, seed + 4))
    zo = interleaved_to_soa(O.RAS(p, Jo, KIND[p.ras_type]).apply(soa_to_interleaved(r)))
    kd = torch.float32 if p.precision == PREC_MIXED else torch.float64
    nslot = 25 if p.dim == 3 else 13
    with P.Solver(p) as s:
        J = torch.empty(4 * nslot * p.ncells, dtype=kd, device="cuda")
        s.jacobian(dev(soa(*X1)), dev(soa(*X0)), dt, J)
        s.ras_factor(J)
        z = torch.empty(2 * p.ncells, dtype=kd, device="cuda")
        s.ras_apply(dev(r).to(kd), z)
        torch.cuda.synchronize()
        return host(z.double()), zo


@pytest.mark.parametrize("solver", [SUB_ILU1, SUB_ILU2, SUB_LU])
@pytest.mark.parametrize("ras_type", [0, 1, 2])
@pytest.mark.parametrize("case", CASES)
def test_apply_matches_oracle(P, case, ras_type, solver):
    dim, n, parts, bc, delta = case
    p = Params(dim=dim, n=n, bc=bc, ras_parts=parts, ras_overlap=delta, ras_type=ras_type,
               subdomain_solver=solver)
    z, zo = _apply_pair(P, p)
    assert _rel(z, zo) <= 1e-10


@pytest.mark.parametrize("solver", [SUB_ILU1, SUB_ILU2, SUB_LU])
def test_apply_mixed_precision(P, solver):
    dim, n, parts, bc, delta = CASES[1]
    p = Params(dim=dim, n=n, bc=bc, ras_parts=parts, ras_overlap=delta, subdomain_solver=solver,
               precision=PREC_MIXED)
    z, zo = _apply_pair(P, p)
    assert _rel(z, zo) <= 2e-4


def test_lu_one_box_inverts(P):
    """One subdomain covering a Neumann domain: the LU preconditioner is inv(J)."""
    import torch
    p = Params(n=(14, 11, 1), bc=BC_NEUMANN, ras_parts=(1, 1, 1), ras_overlap=0, subdomain_solver=SUB_LU)
    X1, X0 = perturbed_pair(p, 3, u_mean=0.45, amp=0.05, step_amp=2e-3)
    Jo = O.jacobian(p, X1, X0, 2e-3)
    r = soa(*random_vector(p, 9))
    with P.Solver(p) as s:
        J = torch.empty(52 * p.ncells, dtype=torch.float64, device="cuda")
        s.jacobian(dev(soa(*X1)), dev(soa(*X0)), 2e-3, J)
        s.ras_factor(J)
        z = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
        s.ras_apply(dev(r), z)
        torch.cuda.synchronize()
        zi = soa_to_interleaved(host(z))
    res = Jo @ zi - soa_to_interleaved(r)
    assert np.linalg.norm(res) <= 1e-11 * np.linalg.norm(r)


@pytest.mark.parametrize("case,solver", [(CASES[0], SUB_ILU1), (CASES[1], SUB_LU), (CASES[2], SUB_ILU2)])
def test_nks_root(P, case, solver):
    import torch
    dim, n, parts, bc, delta = case
    p = Params(dim=dim, n=n, bc=bc, ras_parts=parts, ras_overlap=delta, subdomain_solver=solver,
               newton_rtol=1e-12, gmres_rtol=1e-8)
    U0 = initial_fields(p, 3, 0.45, 0.05)
    Xo, io = O.nks_solve(p, U0, 3e-3)
    with P.Solver(p) as s:
        U1 = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
        ig = s.nks_solve(dev(soa(*U0)), 3e-3, U1)
        xg = host(U1)
    xo = soa(*Xo)
    assert io.status == 0 and ig.status == 0
    assert np.linalg.norm(xg - xo) <= 1e-9 * np.linalg.norm(xo)
    assert ig.newton_its == io.newton_its


def test_fill_reduces_gmres_iterations(P):
    """Table 2's trend: more fill, fewer GMRES iterations per Newton (LU fewest)."""
    import torch
    its = {}
    for solver in (0, SUB_ILU1, SUB_ILU2, SUB_LU):
        p = Params(n=(48, 48, 1), bc=BC_NEUMANN, ras_parts=(3, 3, 1), ras_overlap=1, ras_type=1,
                   subdomain_solver=solver, newton_rtol=1e-10, gmres_rtol=1e-8)
        U0 = initial_fields(p, 5, 0.45, 0.05)
        with P.Solver(p) as s:
            U1 = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
            ig = s.nks_solve(dev(soa(*U0)), 2e-3, U1)
            assert ig.status == 0
            its[solver] = ig.gmres_its / ig.newton_its
    assert its[SUB_LU] <= its[SUB_ILU2] <= its[SUB_ILU1] <= its[0]
    assert its[SUB_LU] < its[0]


def test_adjoint_rejects_fill_solvers(P):
    import torch
    from paper_2007_04560_gb300.acac import AcacError
    p = Params(n=(16, 16, 1), ras_parts=(2, 2, 1), subdomain_solver=SUB_ILU1)
    u, v = initial_fields(p, 1, 0.45, 0.05)
    with P.Solver(p) as s:
        with pytest.raises(AcacError):
            s.adjoint(dev(u.ravel()), dev(v.ravel()), 2, 1e-3, dev(u.ravel()), dev(v.ravel()), every=1)


def test_apply_mixed_precision_3d(P):
    dim, n, parts, bc, delta = CASES[2]
    p = Params(dim=dim, n=n, bc=bc, ras_parts=parts, ras_overlap=delta, subdomain_solver=SUB_ILU2,
               precision=PREC_MIXED)
    z, zo = _apply_pair(P, p)
    assert _rel(z, zo) <= 2e-4


@pytest.mark.parametrize("solver", [SUB_ILU1, SUB_LU])
def test_graph_replay_matches_direct_launches(P, solver):
    """With a fill solver, GMRES iterations replayed from captured graphs give bit-identical
    steps to direct launches."""
    import torch
    p = Params(n=(40, 32, 1), bc=BC_NEUMANN, ras_parts=(3, 2, 1), ras_overlap=1, dt_mode=DT_ADAPTIVE, dt0=1e-4,
               dt_min=1e-5, dt_max=1e-1, eta0=1e4, subdomain_solver=solver)
    u, v = initial_fields(p, 7, 0.45, 0.05)
    out = []
    for graphs in (0, 1):
        ug, vg = dev(u.ravel()), dev(v.ravel())
        with P.Solver(p.replace(graphs=graphs)) as s:
            infos = [s.step(ug, vg) for _ in range(3)]
        torch.cuda.synchronize()
        out.append((host(ug), host(vg), [(i.dt, i.gmres_its, i.newton_its) for i in infos]))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


def test_ensemble_member_equals_single_handle(P):
    """Member m of an ensemble with ILU(1) subdomain solves is bit-identical to a batch-1
    handle stepping the same member."""
    import torch
    p1 = Params(n=(32, 24, 1), ras_parts=(2, 2, 1), ras_overlap=1, subdomain_solver=SUB_ILU1,
                precision=PREC_MIXED)
    fields = [initial_fields(p1, 40 + m, 0.45, 0.05) for m in range(2)]
    u = np.stack([f[0] for f in fields])
    v = np.stack([f[1] for f in fields])
    ug, vg = dev(u.ravel()), dev(v.ravel())
    with P.Solver(p1.replace(batch=2)) as s:
        for _ in range(2):
            s.step(ug, vg)
    torch.cuda.synchronize()
    gu, gv = host(ug).reshape(2, -1), host(vg).reshape(2, -1)
    for m in range(2):
        su, sv = dev(fields[m][0].ravel()), dev(fields[m][1].ravel())
        with P.Solver(p1) as one:
            for _ in range(2):
                one.step(su, sv)
        torch.cuda.synchronize()
        assert np.array_equal(host(su), gu[m]) and np.array_equal(host(sv), gv[m]), m
