"""Ensembles (params.batch = B > 1): B independent problems with their own
coefficients and time steps in one handle.  Each member must match the oracle
stepping that member alone, and must equal bit for bit what a batch-1 handle
computes for the same member (the members share no arithmetic)."""
import numpy as np
import pytest

from oracle import acac_oracle as O
from tests._helpers import dev, host, lib_built, need_cuda, soa
from workloads import DT_ADAPTIVE, E32, PREC_FP64, PREC_MIXED, Params, initial_fields

pytestmark = pytest.mark.gpu

THETAS = (0.25, 0.3, 0.35)


def _members(p, seeds):
    return [initial_fields(p, s, 0.4, 0.05) for s in seeds]


def _stack(fields):
    u = np.ascontiguousarray(np.stack([f[0] for f in fields]))
    v = np.ascontiguousarray(np.stack([f[1] for f in fields]))
    return u, v


@pytest.mark.parametrize("adaptive", [False, True])
def test_ensemble_members_match_oracle(adaptive):
    """Three 40x32 periodic members with theta 0.25 / 0.3 / 0.35 (FP64): after each of
    four steps every member's fields, dt and energy agree with the oracle's
    single-member run (1e-9 relative L2 at Newton rtol 1e-12)."""
    need_cuda()
    P = lib_built()
    import torch
    kw = dict(dt_mode=DT_ADAPTIVE, dt0=1e-4, dt_min=1e-5, dt_max=1e-1, eta0=10.0) if adaptive else dict(dt0=1e-3)
    p1 = Params(n=(40, 32, 1), ras_parts=(2, 2, 1), ras_overlap=1, newton_rtol=1e-12, **kw)
    B = len(THETAS)
    fields = _members(p1, (11, 12, 13))
    u, v = _stack(fields)
    ug, vg = dev(u.ravel()), dev(v.ravel())
    steppers = [O.Stepper(p1.replace(theta=t)) for t in THETAS]
    states = [(f[0].copy(), f[1].copy()) for f in fields]
    with P.Solver(p1.replace(batch=B)) as s:
        for m, t in enumerate(THETAS):
            s.set_coeffs(m, p1.alpha, p1.beta, t, p1.gamma, p1.rho)
        for k in range(4):
            infos = s.step(ug, vg)
            torch.cuda.synchronize()
            assert len(infos) == B
            gu = host(ug).reshape(B, -1)
            gv = host(vg).reshape(B, -1)
            for m in range(B):
                X, io = steppers[m].step(*states[m])
                states[m] = X
                xo = soa(*X)
                xg = soa(gu[m], gv[m])
                assert infos[m].status == 0
                assert np.linalg.norm(xg - xo) <= 1e-9 * np.linalg.norm(xo), (k, m)
                assert infos[m].dt == pytest.approx(io.dt, rel=1e-9)
                assert infos[m].energy == pytest.approx(O.energy(steppers[m].p, *X), rel=1e-10, abs=1e-13)
        # the members really had different coefficients
        e, _ = s.energy(ug, vg)
        assert len(set(np.round(e, 12))) == B


def test_ensemble_member_equals_single_handle():
    """Mixed precision, adaptive: member m of a four-member ensemble is bit-identical
    to a batch-1 handle stepping the same member with the same theta."""
    need_cuda()
    P = lib_built()
    import torch
    p1 = Params(n=(64, 48, 1), ras_parts=(4, 3, 1), ras_overlap=2, dt_mode=DT_ADAPTIVE, dt0=1e-4,
                dt_min=1e-5, dt_max=1e-1, eta0=1e4, precision=PREC_MIXED)
    thetas = (0.26, 0.29, 0.31, 0.34)
    B = len(thetas)
    fields = _members(p1, (21, 22, 23, 24))
    u, v = _stack(fields)
    ug, vg = dev(u.ravel()), dev(v.ravel())
    with P.Solver(p1.replace(batch=B)) as s:
        for m, t in enumerate(thetas):
            s.set_coeffs(m, p1.alpha, p1.beta, t, p1.gamma, p1.rho)
        ens = [s.step(ug, vg) for _ in range(3)]
    torch.cuda.synchronize()
    gu, gv = host(ug).reshape(B, -1), host(vg).reshape(B, -1)
    for m in (0, 3):
        su, sv = dev(fields[m][0].ravel()), dev(fields[m][1].ravel())
        with P.Solver(p1.replace(theta=thetas[m])) as one:
            solo = [one.step(su, sv) for _ in range(3)]
        torch.cuda.synchronize()
        assert np.array_equal(host(su), gu[m]) and np.array_equal(host(sv), gv[m]), m
        for k in range(3):
            assert solo[k].dt == ens[k][m].dt and solo[k].gmres_its == ens[k][m].gmres_its


def test_ensemble_step_host_and_errors():
    """Host entry point of an ensemble, per-member coefficients validation, and the
    component entry points refusing an ensemble handle."""
    need_cuda()
    P = lib_built()
    import torch
    from paper_2007_04560_gb300 import acac as A
    p1 = Params(n=(32, 32, 1), ras_parts=(2, 2, 1), ras_overlap=1)
    fields = _members(p1, (31, 32))
    u, v = _stack(fields)
    with P.Solver(p1.replace(batch=2)) as s:
        with pytest.raises(A.AcacError):
            s.set_coeffs(2, 3.0, 1.0, 0.3, 1e-3, 1.0)
        with pytest.raises(A.AcacError):
            s.set_coeffs(0, 3.0, 1.0, -0.3, 1e-3, 1.0)
        uh, vh = u.copy().ravel(), v.copy().ravel()
        infos = s.step_host(uh, vh)
        assert [i.status for i in infos] == [0, 0]
        X = dev(np.zeros(2 * 32 * 32))
        with pytest.raises(A.AcacError):
            s.residual(X, X, 1e-3, X)
    for m in range(2):
        (uo, vo), _ = O.Stepper(p1).step(*fields[m])
        xg = soa(uh.reshape(2, -1)[m], vh.reshape(2, -1)[m])
        xo = soa(uo, vo)
        assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)


def test_ensemble_workload_runs():
    """The 32 x 256^2 ensemble (theta ~ U(0.25, 0.35)): two steps, every member
    admissible, mass conserved per member, energies differ across members."""
    need_cuda()
    P = lib_built()
    import torch
    w = E32
    u, v = w.fields()
    ug, vg = dev(u.ravel()), dev(v.ravel())
    B = w.members
    th = w.thetas()
    with P.Solver(w.params) as s:
        for m in range(B):
            s.set_coeffs(m, w.params.alpha, w.params.beta, th[m], w.params.gamma, w.params.rho)
        _, m0 = s.energy(ug, vg)
        for _ in range(2):
            infos = s.step(ug, vg)
        torch.cuda.synchronize()
        _, m1 = s.energy(ug, vg)
    assert all(i.status == 0 for i in infos)
    np.testing.assert_allclose(m1, m0, rtol=1e-11)
    assert len(set(np.round([i.energy for i in infos], 10))) > B // 2


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_matches_direct_launches(precision):
    """GMRES iterations replayed from captured CUDA graphs give bit-identical steps to
    direct launches (same kernels, same order), with profiling on and off."""
    need_cuda()
    P = lib_built()
    import torch
    p = Params(n=(64, 48, 1), ras_parts=(4, 3, 1), ras_overlap=2, dt_mode=DT_ADAPTIVE, dt0=1e-4,
               dt_min=1e-5, dt_max=1e-1, eta0=1e4, precision=precision)
    u, v = initial_fields(p, 5, 0.4, 0.05)
    out = []
    for graphs in (0, 1):
        ug, vg = dev(u.ravel()), dev(v.ravel())
        with P.Solver(p.replace(graphs=graphs)) as s:
            infos = [s.step(ug, vg) for _ in range(2)]
            s.profile(True)
            infos += [s.step(ug, vg) for _ in range(2)]
            stats = s.kernel_stats()
            s.profile(False)
            infos += [s.step(ug, vg)]
        torch.cuda.synchronize()
        out.append((host(ug), host(vg), [(i.dt, i.gmres_its, i.newton_its) for i in infos], stats))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]
    # the same launches are counted, and replayed kernels are timed
    for k in ("ras_apply", "gs_dot", "gs_update"):
        assert out[0][3][k][0] == out[1][3][k][0] > 0, k
        assert out[1][3][k][1] > 0, k


def test_autotune_picks_a_valid_partition():
    """acac_autotune returns one of its candidates (valid for acac_create), the time of
    its trial steps, and leaves the input state unchanged; the tuned solver then steps
    to the oracle's result."""
    need_cuda()
    P = lib_built()
    import torch
    from paper_2007_04560_gb300.acac import acac_autotune
    p = Params(n=(96, 80, 1), ras_parts=(2, 2, 1), ras_overlap=1, newton_rtol=1e-12)
    u, v = initial_fields(p, 61, 0.4, 0.05)
    ug, vg = dev(u.ravel()), dev(v.ravel())
    best, ms, nc = acac_autotune(p, ug, vg, trial_steps=2)
    torch.cuda.synchronize()
    assert nc >= 4 and ms > 0
    assert np.array_equal(host(ug), u.ravel()) and np.array_equal(host(vg), v.ravel())
    assert best.ras_overlap in (1, 2)
    with P.Solver(best) as s:
        s.step(ug, vg)
    (uo, vo), _ = O.Stepper(p).step(u, v)
    xo = soa(uo, vo)
    assert np.linalg.norm(soa(host(ug), host(vg)) - xo) <= 1e-9 * np.linalg.norm(xo)


def test_ensemble_one_launch_per_kernel():
    """The members are solved in lockstep: one Schwarz apply launch per Arnoldi step for
    the whole ensemble (not one per member), so an eight-member step launches the apply
    about as often as its slowest member iterates, far fewer times than the members'
    iterations summed."""
    need_cuda()
    P = lib_built()
    import torch
    p1 = Params(n=(64, 48, 1), ras_parts=(4, 3, 1), ras_overlap=2, precision=PREC_MIXED, dt0=1e-3)
    B = 8
    fields = _members(p1, tuple(range(50, 50 + B)))
    u, v = _stack(fields)
    ug, vg = dev(u.ravel()), dev(v.ravel())
    with P.Solver(p1.replace(batch=B)) as s:
        for m in range(B):
            s.set_coeffs(m, p1.alpha, p1.beta, 0.25 + 0.01 * m, p1.gamma, p1.rho)
        s.step(ug, vg)
        s.profile(True)
        infos = s.step(ug, vg)
        stats = s.kernel_stats()
        s.profile(False)
    torch.cuda.synchronize()
    its = [i.gmres_its for i in infos]
    newton = max(i.newton_its for i in infos)
    applies = stats["ras_apply"][0]
    assert min(its) >= 2
    # the Arnoldi steps of the slowest member, plus at most a restart length of steps
    # launched past convergence per Newton iteration before the host looks
    assert applies <= max(its) + newton * p1.gmres_restart
    assert applies < sum(its) / 2, (applies, its)


def test_ensemble_3d_member_equals_single_handle():
    """3D Neumann members with uneven boxes (17 cells split 2 ways, overlap 2), mixed
    precision: member m of a two-member ensemble is bit-identical to a batch-1 handle."""
    need_cuda()
    P = lib_built()
    import torch
    from workloads import BC_NEUMANN
    p1 = Params(dim=3, n=(17, 16, 15), bc=BC_NEUMANN, ras_parts=(2, 2, 2), ras_overlap=2, precision=PREC_MIXED,
                dt0=1e-3)
    fields = _members(p1, (71, 72))
    u, v = _stack(fields)
    ug, vg = dev(u.ravel()), dev(v.ravel())
    thetas = (0.27, 0.33)
    with P.Solver(p1.replace(batch=2)) as s:
        for m, t in enumerate(thetas):
            s.set_coeffs(m, p1.alpha, p1.beta, t, p1.gamma, p1.rho)
        ens = [s.step(ug, vg) for _ in range(2)]
    torch.cuda.synchronize()
    gu, gv = host(ug).reshape(2, -1), host(vg).reshape(2, -1)
    for m in range(2):
        su, sv = dev(fields[m][0].ravel()), dev(fields[m][1].ravel())
        with P.Solver(p1.replace(theta=thetas[m])) as one:
            solo = [one.step(su, sv) for _ in range(2)]
        torch.cuda.synchronize()
        assert np.array_equal(host(su), gu[m]) and np.array_equal(host(sv), gv[m]), m
        assert [i.gmres_its for i in solo] == [e[m].gmres_its for e in ens]


def test_ensemble_member_retry_matches_single_handle():
    """Adaptive steps where the members' Newton solves diverge at different times (a very
    large dt0 and dt_max with theta spread): each member retries with its own dt while the
    others wait, and still equals a batch-1 handle bit for bit, dt and divergence count
    included."""
    need_cuda()
    P = lib_built()
    import torch
    p1 = Params(n=(48, 40, 1), ras_parts=(3, 2, 1), ras_overlap=1, dt_mode=DT_ADAPTIVE, dt0=5.0, dt_min=1e-6,
                dt_max=5.0, eta0=1.0, newton_maxit=4)
    thetas = (0.22, 0.3, 0.38)
    B = len(thetas)
    fields = _members(p1, (81, 82, 83))
    u, v = _stack(fields)
    ug, vg = dev(u.ravel()), dev(v.ravel())
    with P.Solver(p1.replace(batch=B)) as s:
        for m, t in enumerate(thetas):
            s.set_coeffs(m, p1.alpha, p1.beta, t, p1.gamma, p1.rho)
        ens = [s.step(ug, vg, check=False) for _ in range(2)]
    torch.cuda.synchronize()
    gu, gv = host(ug).reshape(B, -1), host(vg).reshape(B, -1)
    for m in range(B):
        su, sv = dev(fields[m][0].ravel()), dev(fields[m][1].ravel())
        with P.Solver(p1.replace(theta=thetas[m])) as one:
            solo = [one.step(su, sv, check=False) for _ in range(2)]
        torch.cuda.synchronize()
        assert np.array_equal(host(su), gu[m]) and np.array_equal(host(sv), gv[m]), m
        for k in range(2):
            a, b = solo[k], ens[k][m]
            assert (a.status, a.dt, a.divergences, a.gmres_its, a.newton_its) == \
                   (b.status, b.dt, b.divergences, b.gmres_its, b.newton_its), (m, k)
    assert sum(e.divergences for e in ens[0]) > 0   # the retry path was taken


@pytest.mark.parametrize("precision", [PREC_FP64, PREC_MIXED])
def test_stationary_member_keeps_its_state(precision):
    """A uniform state u = 1/2, v = 0 is a fixed point of the scheme (F(X0) = 0 exactly: G is
    uniform and p = q), so its Newton solve ends before the first iteration and the root is
    the start state itself.  Beside a member that iterates (adaptive steps, so the
    predictor's change of state is 0 for one member and not for the other) the stationary
    member keeps its fields bit for bit with zero Newton iterations, the other matches a
    batch-1 handle bit for bit, and a batch-1 handle on the stationary state agrees."""
    need_cuda()
    P = lib_built()
    import torch
    p1 = Params(n=(48, 40, 1), ras_parts=(3, 2, 1), ras_overlap=1, dt_mode=DT_ADAPTIVE, dt0=1e-3, dt_min=1e-5,
                dt_max=1e-1, eta0=1e4, precision=precision)
    uf, vf = initial_fields(p1, 31, 0.4, 0.05)
    uc, vc = np.full_like(uf, 0.5), np.zeros_like(vf)
    u, v = _stack([(uc, vc), (uf, vf)])
    ug, vg = dev(u.ravel()), dev(v.ravel())
    with P.Solver(p1.replace(batch=2)) as s:
        ens = [s.step(ug, vg) for _ in range(3)]
    torch.cuda.synchronize()
    gu, gv = host(ug).reshape(2, -1), host(vg).reshape(2, -1)
    assert np.array_equal(gu[0], uc.ravel()) and np.array_equal(gv[0], vc.ravel())
    assert all(e[0].newton_its == 0 and e[0].status == 0 for e in ens)
    assert ens[-1][0].dt == pytest.approx(p1.dt_max)            # no change of state: the largest dt
    assert ens[0][0].energy == pytest.approx(O.energy(p1, uc, vc), rel=1e-12)
    assert all(e[1].newton_its >= 1 for e in ens)
    su, sv = dev(uf.ravel()), dev(vf.ravel())
    with P.Solver(p1) as one:
        solo = [one.step(su, sv) for _ in range(3)]
    torch.cuda.synchronize()
    assert np.array_equal(host(su), gu[1]) and np.array_equal(host(sv), gv[1])
    assert [(a.dt, a.newton_its, a.gmres_its) for a in solo] == [(e[1].dt, e[1].newton_its, e[1].gmres_its)
                                                               for e in ens]
    cu, cv = dev(uc.ravel()), dev(vc.ravel())
    with P.Solver(p1) as one:
        infos = [one.step(cu, cv) for _ in range(2)]
    torch.cuda.synchronize()
    assert np.array_equal(host(cu), uc.ravel()) and np.array_equal(host(cv), vc.ravel())
    assert [i.newton_its for i in infos] == [0, 0]


def test_autotune_ensemble():
    """acac_autotune on an ensemble: times the whole ensemble per candidate, returns a
    partition acac_create accepts, and leaves the members' fields unchanged."""
    need_cuda()
    P = lib_built()
    import torch
    from paper_2007_04560_gb300.acac import acac_autotune
    p1 = Params(n=(64, 48, 1), ras_parts=(2, 2, 1), ras_overlap=1, precision=PREC_MIXED, dt0=1e-3, batch=3)
    fields = _members(p1, (91, 92, 93))
    u, v = _stack(fields)
    ug, vg = dev(u.ravel()), dev(v.ravel())
    best, ms, nc = acac_autotune(p1, ug, vg, trial_steps=1)
    torch.cuda.synchronize()
    assert nc >= 2 and ms > 0 and best.batch == 3
    assert np.array_equal(host(ug), u.ravel()) and np.array_equal(host(vg), v.ravel())
    with P.Solver(best) as s:
        infos = s.step(ug, vg)
    assert [i.status for i in infos] == [0, 0, 0]
