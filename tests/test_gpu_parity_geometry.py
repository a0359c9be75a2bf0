"""GPU path against the CPU FP64 oracle at the Schwarz box geometry of the timed
workloads, on full-size grids (the oracle takes about a minute per solve here).

* 1024^2 periodic with 16 x 16 boxes and overlap 2 (68^2 extended boxes, the whole-box
  apply kernel): one FP64 time step of the 1024^2 workload from its seeded initial state.
* 1024^2 periodic with 8 x 8 boxes and overlap 2: extended boxes of 132^2 cells, for which
  the launch plan picks the level-window apply kernel in both precisions (the whole box
  vector needs 296 KB in double, 148 KB in float: more than two CTAs per SM can hold).
  One Newton solve in FP64 and one in the mixed form against the same oracle root.
* 964^2 periodic with 8 x 8 boxes and overlap 2: extended boxes of 124 and 125 cells per
  direction, exactly the boxes of the 2048^2 workload (17 x 17 boxes of 120-121 owned
  cells), again with the level-window apply; the same two solves.
* Three mixed-precision time steps of the 64^2 workload against the FP64 oracle's steps.

Tolerances: FP64 roots within 1e-9 relative L2 (both sides iterate Newton to rtol 1e-12
so that both reach the same root), mixed within 1e-8 at the workload's Newton tolerance.
"""
import numpy as np
import pytest

from oracle import acac_oracle as O
from tests._helpers import dev, host, lib_built, need_cuda, soa
from workloads import C1, C2, C3, PREC_FP64, PREC_MIXED, H64, initial_fields

pytestmark = pytest.mark.gpu

_ROOTS = {}


@pytest.fixture(scope="module")
def P():
    need_cuda()
    return lib_built()


def _boxes132():
    """1024^2 on [0,16]^2 (h = 1/64), 8 x 8 boxes of 128^2 owned cells, overlap 2."""
    return C3.params.replace(n=(1024, 1024, 1), L=(1024 * H64, 1024 * H64, 1.0), ras_parts=(8, 8, 1),
                             ras_overlap=2, dt_mode=0, dt0=1e-4)


def _boxes124():
    """964^2 on [0, 964/64]^2 (h = 1/64), 8 x 8 boxes of 120-121 owned cells, overlap 2: the
    extended boxes (124 and 125 cells per direction) of the 2048^2 workload's 17 x 17 boxes."""
    return C3.params.replace(n=(964, 964, 1), L=(964 * H64, 964 * H64, 1.0), ras_parts=(8, 8, 1),
                             ras_overlap=2, dt_mode=0, dt0=1e-4)


def _oracle_root(key, p, U0, dt):
    if key not in _ROOTS:
        X, info = O.nks_solve(p.replace(precision=PREC_FP64, newton_rtol=1e-12), U0, dt)
        assert info.status == 0
        _ROOTS[key] = (soa(*X), info)
    return _ROOTS[key]


def test_fp64_step_1024_boxes68(P):
    """One adaptive-workload time step (its first, dt = dt0 = 1e-4) at 1024^2 with the
    configured 16 x 16 boxes, overlap 2: FP64 fields within 1e-9, energy and mass."""
    import torch
    p = C2.params.replace(newton_rtol=1e-12)
    u, v = C2.fields()
    Xo, io = O.Stepper(p).step(u, v)
    xo = soa(*Xo)
    ug, vg = dev(u.ravel()), dev(v.ravel())
    with P.Solver(p) as s:
        ig = s.step(ug, vg)
        torch.cuda.synchronize()
    xg = soa(host(ug), host(vg))
    assert ig.status == 0 and ig.dt == io.dt
    assert np.linalg.norm(xg - xo) <= 1e-9 * np.linalg.norm(xo)
    assert ig.newton_its == io.newton_its
    assert ig.energy == pytest.approx(io.energy, rel=1e-12)
    assert abs(ig.mass - io.mass) <= 1e-12 * abs(io.mass)


@pytest.mark.parametrize("precision", [PREC_FP64, PREC_MIXED])
def test_nks_1024_boxes132(P, precision):
    """One Newton solve at dt = 1e-4 from the 2048^2 workload's initial-state recipe on
    1024^2 with 132^2 extended boxes (the level-window apply): FP64 within 1e-9 of the
    oracle root, the mixed form (Newton rtol 1e-8, as the workload) within 1e-8."""
    import torch
    p = _boxes132()
    U0 = initial_fields(p, C3.seed, C3.u_mean, C3.amp)
    xo, io = _oracle_root("boxes132", p, U0, p.dt0)
    pg = p.replace(precision=precision, newton_rtol=1e-12 if precision == PREC_FP64 else 1e-8)
    with P.Solver(pg) as s:
        U1 = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
        ig = s.nks_solve(dev(soa(*U0)), p.dt0, U1)
        xg = host(U1)
    assert ig.status == 0
    tol = 1e-9 if precision == PREC_FP64 else 1e-8
    assert np.linalg.norm(xg - xo) <= tol * np.linalg.norm(xo)
    if precision == PREC_FP64:
        assert ig.newton_its == io.newton_its
    else:
        assert ig.fnorm <= 1e-8 * ig.fnorm0


@pytest.mark.parametrize("precision", [PREC_FP64, PREC_MIXED])
def test_nks_964_boxes124(P, precision):
    """One Newton solve at dt = 1e-4 with the 2048^2 workload's box shapes (124 / 125 cells
    per direction, the level-window apply): FP64 within 1e-9 of the oracle root, the mixed
    form (Newton rtol 1e-8) within 1e-8."""
    import torch
    p = _boxes124()
    U0 = initial_fields(p, C3.seed, C3.u_mean, C3.amp)
    xo, io = _oracle_root("boxes124", p, U0, p.dt0)
    pg = p.replace(precision=precision, newton_rtol=1e-12 if precision == PREC_FP64 else 1e-8)
    with P.Solver(pg) as s:
        U1 = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
        ig = s.nks_solve(dev(soa(*U0)), p.dt0, U1)
        xg = host(U1)
    assert ig.status == 0
    tol = 1e-9 if precision == PREC_FP64 else 1e-8
    assert np.linalg.norm(xg - xo) <= tol * np.linalg.norm(xo)
    if precision == PREC_FP64:
        assert ig.newton_its == io.newton_its
    else:
        assert ig.fnorm <= 1e-8 * ig.fnorm0


def test_mixed_steps_64_match_fp64_oracle(P):
    """Three time steps of the 64^2 workload (fixed dt 1e-3, Newton rtol 1e-8) in the mixed
    form against the FP64 oracle's steps: fields within 1e-8 relative L2 per step, mass
    conserved to 1e-12, energy non-increasing."""
    import torch
    p = C1.params
    u, v = C1.fields()
    st = O.Stepper(p)
    uo, vo = u.copy(), v.copy()
    ug, vg = dev(u.ravel()), dev(v.ravel())
    M0 = O.mass(p, u)
    E0 = O.energy(p, u, v)
    with P.Solver(p.replace(precision=PREC_MIXED)) as s:
        for k in range(3):
            Xo, io = st.step(uo, vo)
            uo, vo = Xo
            ig = s.step(ug, vg)
            torch.cuda.synchronize()
            xg, xo = soa(host(ug), host(vg)), soa(uo, vo)
            assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo), k
            assert abs(ig.mass - M0) <= 1e-12 * abs(M0)
            assert ig.energy <= E0 + 1e-14 * abs(E0)
            E0 = ig.energy
