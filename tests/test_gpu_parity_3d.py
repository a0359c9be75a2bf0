"""3D GPU path against the CPU oracle (same tolerances as the 2D parity tests):
25-point radius-2 stencil, boxes of the 3D Schwarz decomposition, wavefront level
i + 2j + 3k, both boundary conditions."""
import numpy as np
import pytest

from oracle import acac_oracle as O
from tests._helpers import (dev, host, interleaved_to_soa, lib_built, need_cuda, soa,
                            soa_to_interleaved, stencil_J_to_csr)
from workloads import BC_NEUMANN, BC_PERIODIC, Params, initial_fields, perturbed_pair, random_vector

pytestmark = pytest.mark.gpu

# periodic boxes must not wrap onto themselves: width <= N - 2.  The first two have a
# different spacing per axis, the last two equal spacing (the kernels' one-scaling form of
# the Laplacians and face sums)
ANISO, CUBE = (1.0, 0.9, 1.1), (1.0, 1.0, 1.0)
CASES = [(BC_PERIODIC, (12, 11, 10), (2, 2, 2), ANISO), (BC_NEUMANN, (10, 9, 11), (2, 2, 3), ANISO),
         (BC_PERIODIC, (12, 12, 12), (2, 2, 2), CUBE), (BC_NEUMANN, (10, 10, 10), (2, 2, 2), CUBE)]


@pytest.fixture(scope="module")
def P():
    need_cuda()
    return lib_built()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _p(bc, n, parts, L=ANISO, **kw):
    return Params(dim=3, n=n, L=L, bc=bc, ras_parts=parts, ras_overlap=1, **kw)


@pytest.mark.parametrize("bc,n,parts,L", CASES)
def test_residual_energy_3d(P, bc, n, parts, L):
    import torch
    p = _p(bc, n, parts, L)
    X1, X0 = perturbed_pair(p, 5, u_mean=0.45, amp=0.05, step_amp=2e-3)
    dt = 2e-3
    Fo = soa(*O.residual(p, X1, X0, dt))
    with P.Solver(p) as s:
        F = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
        fn = s.residual(dev(soa(*X1)), dev(soa(*X0)), dt, F)
        e, m = s.energy(dev(X1[0].ravel()), dev(X1[1].ravel()))
        torch.cuda.synchronize()
    assert _rel(host(F), Fo) <= 1e-12
    assert fn == pytest.approx(np.linalg.norm(Fo), rel=1e-12)
    assert e == pytest.approx(O.energy(p, *X1), rel=1e-13)
    assert m == pytest.approx(O.mass(p, X1[0]), rel=1e-14)


@pytest.mark.parametrize("bc,n,parts,L", CASES)
def test_jacobian_spmv_jvp_3d(P, bc, n, parts, L):
    import torch
    p = _p(bc, n, parts, L)
    X1, X0 = perturbed_pair(p, 7, u_mean=0.45, amp=0.05, step_amp=2e-3)
    dt = 2e-3
    Jo = O.jacobian(p, X1, X0, dt)
    w = soa(*random_vector(p, 9))
    yo = interleaved_to_soa(Jo @ soa_to_interleaved(w))
    with P.Solver(p) as s:
        J = torch.empty(100 * p.ncells, dtype=torch.float64, device="cuda")
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


@pytest.mark.parametrize("ras_type", [0, 1, 2])
@pytest.mark.parametrize("bc,n,parts,L", CASES)
def test_ras_apply_3d(P, bc, n, parts, L, ras_type):
    import torch
    p = _p(bc, n, parts, L, ras_type=ras_type)
    X1, X0 = perturbed_pair(p, 13, u_mean=0.45, amp=0.05, step_amp=2e-3)
    dt = 2e-3
    Jo = O.jacobian(p, X1, X0, dt)
    r = soa(*random_vector(p, 17))
    zo = interleaved_to_soa(O.RAS(p, Jo, {0: "left", 1: "as", 2: "right"}[ras_type]).apply(
        soa_to_interleaved(r)))
    with P.Solver(p) as s:
        J = torch.empty(100 * p.ncells, dtype=torch.float64, device="cuda")
        s.jacobian(dev(soa(*X1)), dev(soa(*X0)), dt, J)
        s.ras_factor(J)
        z = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
        s.ras_apply(dev(r), z)
        torch.cuda.synchronize()
    assert _rel(host(z), zo) <= 1e-10


@pytest.mark.parametrize("bc,n,parts,L", CASES)
def test_nks_root_and_steps_3d(P, bc, n, parts, L):
    import torch
    p = _p(bc, n, parts, L, newton_rtol=1e-12, gmres_rtol=1e-8, dt0=2e-3)
    u, v = initial_fields(p, 3, 0.45, 0.05)
    st = O.Stepper(p)
    uo, vo = u.copy(), v.copy()
    ug, vg = dev(u.ravel()), dev(v.ravel())
    E = O.energy(p, u, v)
    M = O.mass(p, u)
    with P.Solver(p) as s:
        for k in range(3):
            Xo, io = st.step(uo, vo)
            uo, vo = Xo
            ig = s.step(ug, vg)
            torch.cuda.synchronize()
            xg, xo = soa(host(ug), host(vg)), soa(uo, vo)
            assert np.linalg.norm(xg - xo) <= 1e-9 * np.linalg.norm(xo), k
            assert ig.newton_its == io.newton_its
            assert ig.energy <= E + 1e-14 * abs(E)
            assert abs(ig.mass - M) <= 1e-12 * abs(M)
            E = ig.energy


def test_mixed_precision_root_3d(P):
    p = _p(BC_NEUMANN, (12, 12, 12), (2, 2, 2), newton_rtol=1e-8, precision=1)
    U0 = initial_fields(p, 4, 0.45, 0.05)
    import torch
    Xo, io = O.nks_solve(p.replace(precision=0, newton_rtol=1e-12), U0, 2e-3)
    with P.Solver(p) as s:
        U1 = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
        ig = s.nks_solve(dev(soa(*U0)), 2e-3, U1)
    xo = soa(*Xo)
    assert ig.status == 0
    assert np.linalg.norm(host(U1) - xo) <= 1e-8 * np.linalg.norm(xo)
