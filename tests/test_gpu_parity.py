"""GPU path (libacac.so through the C ABI) against the CPU FP64 oracle, element
by element on the same seeded inputs.

Tolerances (FP64 path): both sides evaluate the same formulas in double with a
different order of operations, so single evaluations agree to a few hundred ulp
of the largest term (1e-12 relative is used); quantities that go through the ILU
triangular sweeps or a Krylov solve are compared at 1e-10; Newton roots and time
steps at 1e-9 relative L2 per step (the stated FP64 parity bar), with both sides
iterating Newton to rtol 1e-12 so that both reach the same root.
"""
import math

import numpy as np
import pytest

from oracle import acac_oracle as O
from tests._helpers import (dev, host, interleaved_to_soa, lib_built, need_cuda, soa,
                            soa_to_interleaved, stencil_J_to_csr)
from workloads import (BC_NEUMANN, BC_PERIODIC, C1, DT_ADAPTIVE, PREC_FP64, PREC_MIXED, Params,
                       initial_fields, perturbed_pair, random_vector)

pytestmark = pytest.mark.gpu

GRIDS = [((37, 29, 1), (3, 2, 1)), ((64, 64, 1), (4, 4, 1))]


@pytest.fixture(scope="module")
def P():
    need_cuda()
    return lib_built()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
@pytest.mark.parametrize("grid", GRIDS)
def test_residual(P, bc, grid):
    import torch
    n, parts = grid
    p = Params(n=n, bc=bc, ras_parts=parts)
    X1, X0 = perturbed_pair(p, 31, u_mean=0.45, amp=0.05, step_amp=2e-3)
    dt = 2e-3
    Fo = soa(*O.residual(p, X1, X0, dt))
    with P.Solver(p) as s:
        F = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
        fn = s.residual(dev(soa(*X1)), dev(soa(*X0)), dt, F)
        torch.cuda.synchronize()
    assert _rel(host(F), Fo) <= 1e-12
    assert fn == pytest.approx(np.linalg.norm(Fo), rel=1e-12)


def test_table_log_accuracy(P):
    """The residual / energy logarithm against the library log: within 2 ulp over
    (1e-300, 1e300), and within 2 ulp of ln 2 absolute on (1/2, 2)."""
    import torch
    from paper_2007_04560_gb300.acac import acac_log
    rng = np.random.default_rng(0)
    xs = np.concatenate([10.0 ** rng.uniform(-300, 300, 200000), rng.uniform(0.0, 1.0, 200000),
                         1.0 + rng.uniform(-1e-3, 1e-3, 100000), rng.uniform(0.5, 2.0, 100000),
                         np.array([1.0, 2.0, 0.5, 1e-308, 3.0, 1.0 - 2 ** -53, 1.0 + 2 ** -52])])
    xs = xs[xs > 0]
    x = torch.tensor(xs, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    acac_log(x, y)
    ref = torch.log(x)
    torch.cuda.synchronize()
    err = (y - ref).abs()
    ulp = torch.abs(torch.nextafter(ref, torch.full_like(ref, float("inf"))) - ref)
    assert float((err / ulp).max()) <= 2.0
    near1 = (x > 0.5) & (x < 2.0)
    assert float(err[near1].max()) <= 2.3e-16


def test_residual_domain_error(P):
    import torch
    p = Params(n=(16, 16, 1))
    X1, X0 = perturbed_pair(p, 1)
    u1 = X1[0].copy()
    u1[3, 4] = 1.5
    with P.Solver(p) as s:
        F = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
        with pytest.raises(P.AcacError) as e:
            s.residual(dev(soa(u1, X1[1])), dev(soa(*X0)), 1e-3, F)
        assert e.value.status == -3


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
def test_energy_and_mass(P, bc):
    p = Params(n=(37, 29, 1), bc=bc, ras_parts=(3, 2, 1))
    u, v = initial_fields(p, 5, 0.4, 0.08)
    with P.Solver(p) as s:
        e, m = s.energy(dev(u.ravel()), dev(v.ravel()))
    assert e == pytest.approx(O.energy(p, u, v), rel=1e-13)
    assert m == pytest.approx(O.mass(p, u), rel=1e-14)


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
@pytest.mark.parametrize("grid", GRIDS)
def test_jacobian_spmv_jvp(P, bc, grid):
    import torch
    n, parts = grid
    p = Params(n=n, bc=bc, ras_parts=parts)
    X1, X0 = perturbed_pair(p, 7, u_mean=0.45, amp=0.05, step_amp=2e-3)
    dt = 2e-3
    Jo = O.jacobian(p, X1, X0, dt)
    w = soa(*random_vector(p, 9))
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
def test_jvp_fp32(P, bc, grid):
    """Mixed form: the fused tiled FP32 Jacobian action against the FP64 oracle J w.
    FP32 arithmetic on O(1) inputs: 1e-5 of max |J w|."""
    import torch
    n, parts = grid
    p = Params(n=n, bc=bc, ras_parts=parts, precision=PREC_MIXED)
    X1, X0 = perturbed_pair(p, 29, u_mean=0.45, amp=0.05, step_amp=2e-3)
    dt = 2e-3
    Jo = O.jacobian(p, X1, X0, dt)
    w = soa(*random_vector(p, 31))
    yo = interleaved_to_soa(Jo @ soa_to_interleaved(w))
    with P.Solver(p) as s:
        y = torch.empty(2 * p.ncells, dtype=torch.float32, device="cuda")
        s.jvp(dev(soa(*X1)), dev(soa(*X0)), dt, dev(w, torch.float32), y)
        torch.cuda.synchronize()
    assert _rel(host(y), yo) <= 1e-5


@pytest.mark.parametrize("window", [2, 1])
@pytest.mark.parametrize("ras_type", [0, 1, 2])
@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
@pytest.mark.parametrize("grid", GRIDS)
def test_ras_apply(P, bc, grid, ras_type, window):
    """ILU(0) of every A_k and the Schwarz sum (left-RAS, AS, right-RAS), with the whole box
    vector in shared memory (window = 2) and with the level-window kernel (window = 1)."""
    import torch
    n, parts = grid
    p = Params(n=n, bc=bc, ras_parts=parts, ras_overlap=2 if n[0] == 64 else 1, ras_type=ras_type,
               ras_window=window)
    X1, X0 = perturbed_pair(p, 13, u_mean=0.45, amp=0.05, step_amp=2e-3)
    dt = 2e-3
    Jo = O.jacobian(p, X1, X0, dt)
    r = soa(*random_vector(p, 17))
    zo = interleaved_to_soa(O.RAS(p, Jo, {0: "left", 1: "as", 2: "right"}[ras_type]).apply(
        soa_to_interleaved(r)))
    with P.Solver(p) as s:
        J = torch.empty(52 * p.ncells, dtype=torch.float64, device="cuda")
        s.jacobian(dev(soa(*X1)), dev(soa(*X0)), dt, J)
        s.ras_factor(J)
        z = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
        s.ras_apply(dev(r), z)
        torch.cuda.synchronize()
    assert _rel(host(z), zo) <= 1e-10


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
def test_gmres_solution(P, bc):
    import torch
    p = Params(n=(37, 29, 1), bc=bc, ras_parts=(3, 2, 1), gmres_rtol=1e-12, gmres_atol=0.0)
    X1, X0 = perturbed_pair(p, 19, u_mean=0.45, amp=0.05, step_amp=2e-3)
    dt = 2e-3
    Jo = O.jacobian(p, X1, X0, dt)
    b = soa(*random_vector(p, 23))
    xd = interleaved_to_soa(np.linalg.solve(Jo.toarray(), soa_to_interleaved(b)))
    oracle = O.gmres(lambda w: Jo @ w, O.RAS(p, Jo).apply, soa_to_interleaved(b), 1e-12, 0.0)
    with P.Solver(p) as s:
        x = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
        its, res, st = s.gmres(dev(soa(*X1)), dev(soa(*X0)), dt, dev(b), x)
    xg = host(x)
    assert np.linalg.norm(xg - xd) <= 1e-10 * np.linalg.norm(xd)
    assert abs(its - oracle.its) <= 2


def _nks_pair(P, p, U0, dt):
    import torch
    Xo, io = O.nks_solve(p, U0, dt)
    with P.Solver(p) as s:
        U1 = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
        ig = s.nks_solve(dev(soa(*U0)), dt, U1)
        return Xo, io, host(U1), ig


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
@pytest.mark.parametrize("grid", GRIDS)
def test_nks_root(P, bc, grid):
    n, parts = grid
    p = Params(n=n, bc=bc, ras_parts=parts, newton_rtol=1e-12, gmres_rtol=1e-8)
    U0 = initial_fields(p, 3, 0.45, 0.05)
    Xo, io, Xg, ig = _nks_pair(P, p, U0, 3e-3)
    xo = soa(*Xo)
    assert io.status == 0 and ig.status == 0
    assert np.linalg.norm(Xg - xo) <= 1e-9 * np.linalg.norm(xo)
    assert ig.newton_its == io.newton_its


def test_steps_match_oracle_tight():
    """C1 workload (64x64 periodic, fixed dt 1e-3) with Newton rtol 1e-12 on both sides:
    every step's fields within 1e-9 relative L2, energy non-increasing, mass conserved."""
    need_cuda()
    P = lib_built()
    import torch
    p = C1.params.replace(newton_rtol=1e-12)
    u, v = C1.fields()
    st = O.Stepper(p)
    uo, vo = u.copy(), v.copy()
    ug, vg = dev(u.ravel()), dev(v.ravel())
    E0, M0 = O.energy(p, u, v), O.mass(p, u)
    with P.Solver(p) as s:
        for k in range(C1.steps):
            Xo, io = st.step(uo, vo)
            uo, vo = Xo
            ig = s.step(ug, vg)
            torch.cuda.synchronize()
            xg, xo = soa(host(ug), host(vg)), soa(uo, vo)
            assert np.linalg.norm(xg - xo) <= 1e-9 * np.linalg.norm(xo), k
            assert ig.energy <= E0 + 1e-14 * abs(E0)
            assert abs(ig.mass - M0) <= 1e-12 * abs(M0)
            assert ig.energy == pytest.approx(io.energy, rel=1e-12)
            E0 = ig.energy


@pytest.mark.parametrize("precision,tol", [(PREC_FP64, 1e-9), (PREC_MIXED, 1e-8)])
def test_steps_with_gmres_restarts_match_oracle(precision, tol):
    """C1 at dt = 1e-2 with GMRES restarted every 4 iterations (about 60 iterations per
    Newton step, so every solve restarts many times from r = b - J x with b = -F): each step's
    fields within 1e-9 (FP64) / 1e-8 (mixed) relative L2 of the oracle's at Newton rtol 1e-12,
    with the oracle's Newton iteration count."""
    need_cuda()
    P = lib_built()
    import torch
    p = C1.params.replace(dt0=1e-2, gmres_restart=4, newton_rtol=1e-12, precision=precision)
    u, v = C1.fields()
    st = O.Stepper(p)
    uo, vo = u.copy(), v.copy()
    ug, vg = dev(u.ravel()), dev(v.ravel())
    with P.Solver(p) as s:
        for k in range(2):
            Xo, io = st.step(uo, vo)
            uo, vo = Xo
            ig = s.step(ug, vg)
            torch.cuda.synchronize()
            xg, xo = soa(host(ug), host(vg)), soa(uo, vo)
            assert np.linalg.norm(xg - xo) <= tol * np.linalg.norm(xo), k
            assert ig.newton_its == io.newton_its
            assert ig.gmres_its > 8 * ig.newton_its    # restarts taken


def test_steps_match_oracle_config_tolerance():
    """C1 exactly as configured (Newton rtol 1e-8): roots agree to the size the
    Newton tolerance leaves (1e-8 relative per step plus accumulation over 10 steps)."""
    need_cuda()
    P = lib_built()
    import torch
    p = C1.params
    u, v = C1.fields()
    st = O.Stepper(p)
    uo, vo = u.copy(), v.copy()
    ug, vg = dev(u.ravel()), dev(v.ravel())
    M0 = O.mass(p, u)
    with P.Solver(p) as s:
        for k in range(C1.steps):
            Xo, io = st.step(uo, vo)
            uo, vo = Xo
            ig = s.step(ug, vg)
            torch.cuda.synchronize()
            xg, xo = soa(host(ug), host(vg)), soa(uo, vo)
            assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo), k
            assert abs(ig.mass - M0) <= 1e-12 * abs(M0)
            assert ig.newton_its == io.newton_its


def test_adaptive_steps_match_oracle():
    """Adaptive dt (Eq. sencondt): same dt sequence and fields as the oracle."""
    need_cuda()
    P = lib_built()
    import torch
    p = Params(n=(48, 40, 1), ras_parts=(3, 2, 1), ras_overlap=2, dt_mode=DT_ADAPTIVE, dt0=1e-4,
               dt_min=1e-5, dt_max=1e-1, eta0=10.0, newton_rtol=1e-12)
    u, v = initial_fields(p, 1, 0.4, 0.05)
    st = O.Stepper(p)
    uo, vo = u.copy(), v.copy()
    ug, vg = dev(u.ravel()), dev(v.ravel())
    with P.Solver(p) as s:
        for k in range(6):
            Xo, io = st.step(uo, vo)
            uo, vo = Xo
            ig = s.step(ug, vg)
            torch.cuda.synchronize()
            assert ig.dt == pytest.approx(io.dt, rel=1e-9)
            assert ig.t == pytest.approx(io.t, rel=1e-9)
            xg, xo = soa(host(ug), host(vg)), soa(uo, vo)
            assert np.linalg.norm(xg - xo) <= 1e-9 * np.linalg.norm(xo), k


def test_mixed_precision_root():
    """Mixed path (FP32 Jacobian, Krylov, ILU; FP64 residual and update) reaches the
    FP64 oracle's root within 1e-8 relative at equal Newton tolerance."""
    need_cuda()
    P = lib_built()
    p = Params(n=(64, 64, 1), ras_parts=(4, 4, 1), newton_rtol=1e-8, precision=PREC_MIXED)
    U0 = initial_fields(p, 3, 0.45, 0.05)
    Xo, io = O.nks_solve(p.replace(precision=0, newton_rtol=1e-12), U0, 2e-3)
    Xo8, io8 = O.nks_solve(p.replace(precision=0), U0, 2e-3)
    Xo_, io_, Xg, ig = _nks_pair(P, p, U0, 2e-3)
    xo = soa(*Xo)
    assert ig.status == 0
    assert np.linalg.norm(Xg - xo) <= 1e-8 * np.linalg.norm(xo)
    assert ig.fnorm <= 1e-8 * ig.fnorm0


def test_error_paths():
    need_cuda()
    P = lib_built()
    import torch
    with pytest.raises(P.AcacError) as e:
        P.Solver(Params(n=(3, 64, 1)))
    assert e.value.status == -1
    with pytest.raises(P.AcacError):
        P.Solver(Params(n=(16, 16, 1), ras_parts=(2, 2, 1), ras_overlap=4))   # box wraps
    p = Params(n=(16, 16, 1), ras_parts=(2, 2, 1), newton_maxit=1, newton_rtol=1e-14, newton_atol=0.0)
    u, v = initial_fields(p, 1, 0.5, 0.05)
    with P.Solver(p) as s:
        ug, vg = dev(u.ravel()), dev(v.ravel())
        info = s.step(ug, vg, check=False)
        assert info.status == -4
        assert np.array_equal(host(ug), u.ravel())          # unchanged on error
    pa = p.replace(dt_mode=DT_ADAPTIVE, dt0=1e-3, dt_min=2e-4, eta0=10.0)
    with P.Solver(pa) as s:
        info = s.step(dev(u.ravel()), dev(v.ravel()), check=False)
        assert info.status == -5 and info.divergences == 5
    bad = u.copy()
    bad[0, 0] = 1.2
    with P.Solver(Params(n=(16, 16, 1), ras_parts=(2, 2, 1))) as s:
        info = s.step(dev(bad.ravel()), dev(v.ravel()), check=False)
        assert info.status == -3


def test_step_host_matches_device():
    need_cuda()
    P = lib_built()
    import torch
    p = C1.params
    u, v = C1.fields()
    with P.Solver(p) as s1, P.Solver(p) as s2:
        ug, vg = dev(u.ravel()), dev(v.ravel())
        uh, vh = u.ravel().copy(), v.ravel().copy()
        for _ in range(2):
            s1.step(ug, vg)
            s2.step_host(uh, vh)
        torch.cuda.synchronize()
        assert np.array_equal(host(ug), uh) and np.array_equal(host(vg), vh)


@pytest.mark.parametrize("precision", [0, 1])
def test_window_apply_steps_match_whole_box(P, precision):
    """Time steps with the level-window apply equal those with the whole-box apply up to
    rounding (the two sum the same products in the same order: bit-identical)."""
    import torch
    p = Params(n=(96, 80, 1), ras_parts=(3, 2, 1), ras_overlap=2, dt_mode=DT_ADAPTIVE, dt0=1e-4, dt_min=1e-5,
               dt_max=1e-1, eta0=1e4, precision=precision)
    u, v = initial_fields(p, 9, 0.4, 0.05)
    out = []
    for window in (2, 1):
        ug, vg = dev(u.ravel()), dev(v.ravel())
        with P.Solver(p.replace(ras_window=window)) as s:
            infos = [s.step(ug, vg) for _ in range(3)]
        torch.cuda.synchronize()
        out.append((host(ug), host(vg), [(i.dt, i.gmres_its) for i in infos]))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


@pytest.mark.parametrize("ras_type", [1, 2])
@pytest.mark.parametrize("case", ["2d-box", "2d-window", "3d", "2d-ilu1", "3d-float"])
def test_additive_extension_is_deterministic(P, ras_type, case):
    """AS and right-RAS add the values of the overlapping boxes per grid cell in a fixed order
    (the apply writes them by box cell, one pass sums them): repeated applies of one
    factorization give bit-identical results, in every apply kernel."""
    import torch
    from workloads import SUB_ILU1
    kw = dict(ras_type=ras_type)
    if case.startswith("3d"):
        p = Params(dim=3, n=(18, 16, 14), bc=BC_NEUMANN, ras_parts=(2, 2, 2), ras_overlap=2,
                   precision=PREC_MIXED if case == "3d-float" else 0, **kw)
    else:
        p = Params(n=(64, 48, 1), bc=BC_PERIODIC, ras_parts=(4, 3, 1), ras_overlap=2,
                   ras_window=1 if case == "2d-window" else 2, subdomain_solver=SUB_ILU1 if case == "2d-ilu1" else 0,
                   **kw)
    X1, X0 = perturbed_pair(p, 23, u_mean=0.45, amp=0.05, step_amp=2e-3)
    dt = 2e-3
    ft = torch.float32 if p.precision == PREC_MIXED else torch.float64
    nslot = 25 if p.dim == 3 else 13
    with P.Solver(p) as s:
        J = torch.empty(nslot * 4 * p.ncells, dtype=ft, device="cuda")
        s.jacobian(dev(soa(*X1)), dev(soa(*X0)), dt, J)
        s.ras_factor(J)
        r = dev(soa(*random_vector(p, 29)), ft)
        outs = []
        for _ in range(3):
            z = torch.empty(2 * p.ncells, dtype=ft, device="cuda")
            s.ras_apply(r, z)
            outs.append(host(z))
        torch.cuda.synchronize()
    assert np.all(np.isfinite(outs[0])) and np.abs(outs[0]).max() > 0
    assert all(np.array_equal(outs[0], o) for o in outs[1:])
