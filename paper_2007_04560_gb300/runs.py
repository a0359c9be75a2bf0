"""The paper's numerical experiments, run through the library on one GPU.

    python -m paper_2007_04560_gb300.runs convergence --kind space [...]   (Sec. 4.1 A, Fig. 1a)
    python -m paper_2007_04560_gb300.runs convergence --kind time  [...]   (Sec. 4.1 A, Fig. 1b)
    python -m paper_2007_04560_gb300.runs long --bc neumann|periodic [...] (Sec. 4.1 A, Figs. 2-4)
    python -m paper_2007_04560_gb300.runs schwarz [--dim 2|3] [...]        (Sec. 4.2, Table 3)
    python -m paper_2007_04560_gb300.runs subdomain [--dim 2|3] [...]      (Sec. 4.2, Table 2)

Each prints one JSON document (or, for `long`, one JSON line per step with --jsonl) with
what the paper plots or tabulates.  Coefficients and tolerances are those of the paper's
Sec. 4 (workloads.PAPER_COEF, workloads.PAPER_TOL); the initial states are the paper's
(the smooth state of Sec. 4.1 A, or 0.55 + U(-0.05, 0.05), U(-0.05, 0.05) drawn from a
seeded generator).  Every time step is libacac.so's acac_step.

Error of the convergence study (Sec. 4.1 A): relative l2 over both fields against the
reference solution; a finer reference field is compared after averaging each block of
fine cells onto the coarse cell that contains it (cell-centred grids do not share points).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _params(**kw):
    from workloads import PAPER_COEF, PAPER_TOL, Params
    base = dict(PAPER_COEF)
    base.update(PAPER_TOL)
    base.update(kw)
    return Params(**base)


def _solver(p):
    from paper_2007_04560_gb300 import acac as A
    return A.Solver(p)


def _parts(n, box=32):
    return max(2, n // box)


def _fixed_run(p, u0, v0, nsteps):
    """(u, v) after nsteps fixed-dt steps (float64 CUDA tensors) and the last report."""
    import torch
    u = torch.tensor(u0.ravel(), device="cuda")
    v = torch.tensor(v0.ravel(), device="cuda")
    s = _solver(p)
    info = None
    for _ in range(nsteps):
        info = s.step(u, v)
    s.close()
    torch.cuda.synchronize()
    return u.view(p.shape), v.view(p.shape), info


def _block_average(a, r):
    """Mean over r x r blocks of a 2D tensor."""
    import torch
    ny, nx = a.shape
    return a.reshape(ny // r, r, nx // r, r).mean(dim=(1, 3)) if r > 1 else a.clone()


def _rel_l2(u, v, ur, vr):
    import torch
    num = torch.sum((u - ur) ** 2) + torch.sum((v - vr) ** 2)
    den = torch.sum(ur ** 2) + torch.sum(vr ** 2)
    return float(torch.sqrt(num / den))


def convergence(kind="space", ns=(16, 32, 64), nref=128, dt=5e-5, dts=(8e-4, 4e-4, 2e-4, 1e-4),
                dtref=2.5e-5, T=3.2e-3, n=64, newton_rtol=1e-10, box=8, ref_solver=0, ref_overlap=1,
                ref_box=None, ref_newton_atol=None):
    """Relative l2 errors against the reference run and the observed orders (Fig. 1).

    space: grids ns at fixed dt, reference grid nref, all to time T;
    time:  grid n, time steps dts, reference time step dtref, all to time T.
    The space reference may take its own subdomain solver, overlap and box size (ILU(0)
    boxes do not converge on the paper's 1024^2 reference) and an absolute Newton
    tolerance (the rounding floor of F grows with 1/dt and the cell count)."""
    from workloads import BC_PERIODIC, sinusoidal_fields
    out = {"kind": kind, "T": T, "coefficients": "Sec. 4.1", "newton_rtol": newton_rtol, "rows": []}
    t0 = time.perf_counter()
    if kind == "space":
        steps = int(round(T / dt))
        rb = ref_box or box
        pr = _params(n=(nref, nref, 1), bc=BC_PERIODIC, dt0=dt, ras_parts=(_parts(nref, rb), _parts(nref, rb), 1),
                     newton_rtol=newton_rtol, subdomain_solver=ref_solver, ras_overlap=ref_overlap)
        if ref_newton_atol is not None:
            pr = pr.replace(newton_atol=ref_newton_atol)
        t1 = time.perf_counter()
        ur, vr, _ = _fixed_run(pr, *sinusoidal_fields(pr), steps)
        out["reference"] = {"n": nref, "subdomain_solver": ref_solver, "overlap": ref_overlap, "box": rb,
                            "newton_atol": pr.newton_atol, "seconds": time.perf_counter() - t1}
        base = _params(n=(nref, nref, 1), bc=BC_PERIODIC, dt0=dt, newton_rtol=newton_rtol)
        prev = None
        for m in ns:
            p = base.replace(n=(m, m, 1), ras_parts=(_parts(m, box), _parts(m, box), 1))
            try:
                u, v, info = _fixed_run(p, *sinusoidal_fields(p), steps)
            except Exception as exc:   # a coarse grid that fails keeps the (costly) reference's rows
                out["rows"].append({"n": m, "error": str(exc)})
                continue
            r = nref // m
            e = _rel_l2(u, v, _block_average(ur, r), _block_average(vr, r))
            row = {"n": m, "l2": e, "newton_last_step": info.newton_its}
            if prev:
                row["order"] = math.log(prev[1] / e) / math.log(m / prev[0])
            out["rows"].append(row)
            prev = (m, e)
        out.update({"nref": nref, "dt": dt, "steps": steps})
    else:
        p = _params(n=(n, n, 1), bc=BC_PERIODIC, ras_parts=(_parts(n, box), _parts(n, box), 1), newton_rtol=newton_rtol)
        ur, vr, _ = _fixed_run(p.replace(dt0=dtref), *sinusoidal_fields(p), int(round(T / dtref)))
        prev = None
        for d in dts:
            u, v, info = _fixed_run(p.replace(dt0=d), *sinusoidal_fields(p), int(round(T / d)))
            e = _rel_l2(u, v, ur, vr)
            row = {"dt": d, "l2": e, "newton_last_step": info.newton_its}
            if prev:
                row["order"] = math.log(prev[1] / e) / math.log(prev[0] / d)
            out["rows"].append(row)
            prev = (d, e)
        out.update({"n": n, "dtref": dtref})
    out["seconds"] = time.perf_counter() - t0
    return out


def long_run(bc="neumann", n=128, t_end=1e4, seed=0, dt_min=1e-4, dt_max=10.0, eta=1e4, dt0=1e-4,
             max_steps=200000, parts=8, every=1, sink=None, L=2.0, subdomain_solver=0, overlap=1,
             max_seconds=None):
    """The long adaptive runs of Sec. 4.1 A (Figs. 2-4): 0.55 + U(-0.05, 0.05) /
    U(-0.05, 0.05) on n^2 cells of [0, L]^2, adaptive dt (eta, dt_min, dt_max) until t_end.
    L = 2 keeps h = 1/64 (on the unit square at 128^2 the subdomain ILU(0) does not
    converge from the random initial state with Neumann walls).  subdomain_solver / overlap:
    the Schwarz subdomain solve (ILU(0), ILU(1), ILU(2), LU) and overlap; max_seconds stops
    the run early.  Calls sink(record) every `every` steps (and at the last); returns the
    summary: steps, time, dt range, energy monotonicity, mass drift."""
    import torch
    from workloads import BC_NEUMANN, BC_PERIODIC, DT_ADAPTIVE, initial_fields
    p = _params(n=(n, n, 1), L=(L, L, 1.0), bc=BC_NEUMANN if bc == "neumann" else BC_PERIODIC, dt_mode=DT_ADAPTIVE,
                dt0=dt0, dt_min=dt_min, dt_max=dt_max, eta0=eta, ras_parts=(parts, parts, 1), ras_overlap=overlap,
                subdomain_solver=subdomain_solver)
    u0, v0 = initial_fields(p, seed, 0.55, 0.05)
    u = torch.tensor(u0.ravel(), device="cuda")
    v = torch.tensor(v0.ravel(), device="cuda")
    s = _solver(p)
    e0, m0 = s.energy(u, v)
    t, k, e_prev = 0.0, 0, e0
    increases, max_rise = 0, 0.0
    dts = []
    div = 0
    t0 = time.perf_counter()
    while t < t_end and k < max_steps and (max_seconds is None or time.perf_counter() - t0 < max_seconds):
        info = s.step(u, v)
        k += 1
        t = info.t
        dts.append(info.dt)
        div += info.divergences
        if info.energy > e_prev:
            increases += 1
            max_rise = max(max_rise, (info.energy - e_prev) / abs(e_prev))
        e_prev = info.energy
        if sink and (k % every == 0 or t >= t_end):
            sink({"step": k, "t": t, "dt": info.dt, "energy": info.energy, "mass": info.mass,
                  "newton": info.newton_its, "gmres": info.gmres_its, "divergences": info.divergences,
                  "eta": info.eta})
    torch.cuda.synchronize()
    s.close()
    return {"bc": bc, "n": n, "L": L, "subdomain_solver": ["ILU(0)", "ILU(1)", "ILU(2)", "LU"][subdomain_solver],
            "overlap": overlap, "boxes": [parts, parts], "eta0": eta, "dt_bounds": [dt_min, dt_max],
            "steps": k, "t": t, "t_end": t_end, "seconds": time.perf_counter() - t0,
            "dt_min_seen": min(dts), "dt_max_seen": max(dts), "energy0": e0, "energy_end": e_prev,
            "energy_increases": increases, "max_relative_rise": max_rise, "mass_drift": abs(info.mass - m0) / abs(m0),
            "divergences": div}


def schwarz_table(dim=2, steps=10, dt=1e-4, seed=0, L=2.0):
    """Sec. 4.2, Tables 2-3: the first `steps` steps at fixed dt on 128^2 (24 subdomains,
    6 x 4) or 128^3 (512 subdomains, 8 x 8 x 8) cells of [0, L]^d, homogeneous Neumann,
    0.55 + U(-0.05, 0.05) / U(-0.05, 0.05), per preconditioner variant: total Newton
    iterations, GMRES iterations per Newton, time.  The section does not state the domain;
    L = 2 (h = 1/64) gives the iteration counts the tables print, while on the unit square
    the subdomain ILU(0) of these box sizes does not converge."""
    import torch
    from workloads import BC_NEUMANN, initial_fields
    if dim == 2:
        base = _params(n=(128, 128, 1), L=(L, L, 1.0), bc=BC_NEUMANN, dt0=dt, ras_parts=(6, 4, 1))
    else:
        base = _params(dim=3, n=(128, 128, 128), L=(L, L, L), bc=BC_NEUMANN, dt0=dt, ras_parts=(8, 8, 8))
    u0, v0 = initial_fields(base, seed, 0.55, 0.05)
    variants = [("classical-AS", 1, 0, 1), ("classical-AS", 1, 1, 1), ("classical-AS", 1, 2, 1),
                ("left-RAS", 0, 1, 1), ("left-RAS", 0, 2, 1), ("right-RAS", 2, 1, 1), ("right-RAS", 2, 2, 1),
                ("classical-AS, ILU(0) without reuse", 1, 1, 0)]
    rows = []
    for name, ras_type, delta, reuse in variants:
        p = base.replace(ras_type=ras_type, ras_overlap=delta, ilu_reuse=reuse)
        u = torch.tensor(u0.ravel(), device="cuda")
        v = torch.tensor(v0.ravel(), device="cuda")
        s = _solver(p)
        s.step(u.clone(), v.clone())          # warm-up (first-use costs), not counted
        torch.cuda.synchronize()
        newton = gmres = 0
        t0 = time.perf_counter()
        for _ in range(steps):
            info = s.step(u, v)
            newton += info.newton_its
            gmres += info.gmres_its
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        s.close()
        rows.append({"preconditioner": name, "delta": delta, "ilu_reuse": bool(reuse), "total_newton": newton,
                     "gmres_per_newton": gmres / max(newton, 1), "seconds": el})
    return {"dim": dim, "grid": list(base.shape[::-1]), "subdomains": list(base.ras_parts[:dim]), "steps": steps,
            "dt": dt, "rows": rows}


def subdomain_table(dim=2, steps=10, dt=1e-4, seed=0, L=2.0, precision=None):
    """Sec. 4.2, Table 2: classical AS with overlap 1 and the subdomain solvers ILU(0),
    ILU(1), ILU(2), LU (factored at every Newton iteration) and ILU(0) with reuse, on the
    workload of schwarz_table; per solver total Newton iterations, GMRES iterations per
    Newton and time.  precision: PREC_FP64 (default in 2D) or PREC_MIXED (default in 3D,
    where the LU factors of the 512 boxes take ~50 GB in float)."""
    import torch
    from workloads import BC_NEUMANN, PREC_FP64, PREC_MIXED, SUB_ILU0, SUB_ILU1, SUB_ILU2, SUB_LU, initial_fields
    if precision is None:
        precision = PREC_FP64 if dim == 2 else PREC_MIXED
    if dim == 2:
        base = _params(n=(128, 128, 1), L=(L, L, 1.0), bc=BC_NEUMANN, dt0=dt, ras_parts=(6, 4, 1))
    else:
        base = _params(dim=3, n=(128, 128, 128), L=(L, L, L), bc=BC_NEUMANN, dt0=dt, ras_parts=(8, 8, 8))
    base = base.replace(ras_type=1, ras_overlap=1, precision=precision)
    u0, v0 = initial_fields(base, seed, 0.55, 0.05)
    variants = [("ILU(0)", SUB_ILU0, 0), ("ILU(1)", SUB_ILU1, 0), ("ILU(2)", SUB_ILU2, 0),
                ("ILU(0)-reuse", SUB_ILU0, 1), ("LU", SUB_LU, 0)]     # the costly one last
    rows = []
    for name, solver, reuse in variants:
        p = base.replace(subdomain_solver=solver, ilu_reuse=reuse)
        u = torch.tensor(u0.ravel(), device="cuda")
        v = torch.tensor(v0.ravel(), device="cuda")
        s = _solver(p)
        s.step(u.clone(), v.clone())          # warm-up (first-use costs), not counted
        torch.cuda.synchronize()
        newton = gmres = 0
        t0 = time.perf_counter()
        for _ in range(steps):
            info = s.step(u, v)
            newton += info.newton_its
            gmres += info.gmres_its
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        s.close()
        rows.append({"subdomain_solver": name, "total_newton": newton, "gmres_per_newton": gmres / max(newton, 1),
                     "seconds": el})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)      # progress
    return {"dim": dim, "grid": list(base.shape[::-1]), "subdomains": list(base.ras_parts[:dim]), "steps": steps,
            "dt": dt, "preconditioner": "classical AS, overlap 1",
            "precision": "fp64" if precision == PREC_FP64 else "mixed", "rows": rows}


def main(argv=None):
    from paper_2007_04560_gb300 import build
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("convergence")
    c.add_argument("--kind", choices=["space", "time"], default="space")
    c.add_argument("--ns", default="16,32,64")
    c.add_argument("--nref", type=int, default=128)
    c.add_argument("--dt", type=float, default=5e-5)
    c.add_argument("--n", type=int, default=64)
    c.add_argument("--dts", default="8e-4,4e-4,2e-4,1e-4")
    c.add_argument("--dtref", type=float, default=2.5e-5)
    c.add_argument("--T", type=float, default=3.2e-3)
    c.add_argument("--box", type=int, default=8, help="owned cells per subdomain box and direction")
    c.add_argument("--ref-solver", choices=["ilu0", "ilu1", "ilu2", "lu"], default="ilu0",
                   help="subdomain solver of the space reference run")
    c.add_argument("--ref-overlap", type=int, default=1)
    c.add_argument("--ref-box", type=int, default=None)
    c.add_argument("--ref-newton-atol", type=float, default=None)
    lr = sub.add_parser("long")
    lr.add_argument("--bc", choices=["neumann", "periodic"], default="neumann")
    lr.add_argument("--n", type=int, default=128)
    lr.add_argument("--t-end", type=float, default=1e4)
    lr.add_argument("--seed", type=int, default=0)
    lr.add_argument("--every", type=int, default=10)
    lr.add_argument("--jsonl", action="store_true")
    lr.add_argument("--L", type=float, default=2.0, help="domain [0, L]^2")
    lr.add_argument("--subdomain-solver", choices=["ilu0", "ilu1", "ilu2", "lu"], default="ilu0")
    lr.add_argument("--overlap", type=int, default=1)
    lr.add_argument("--parts", type=int, default=8, help="Schwarz boxes per direction")
    lr.add_argument("--max-seconds", type=float, default=None)
    sw = sub.add_parser("schwarz")
    sw.add_argument("--dim", type=int, choices=[2, 3], default=2)
    sw.add_argument("--steps", type=int, default=10)
    sd = sub.add_parser("subdomain")
    sd.add_argument("--dim", type=int, choices=[2, 3], default=2)
    sd.add_argument("--steps", type=int, default=10)
    sd.add_argument("--precision", choices=["fp64", "mixed"], default=None)
    args = ap.parse_args(argv)
    build.build()
    if args.cmd == "convergence":
        solvers = {"ilu0": 0, "ilu1": 1, "ilu2": 2, "lu": 3}
        res = convergence(args.kind, tuple(int(x) for x in args.ns.split(",")), args.nref, args.dt,
                          tuple(float(x) for x in args.dts.split(",")), args.dtref, args.T, args.n, box=args.box,
                          ref_solver=solvers[args.ref_solver], ref_overlap=args.ref_overlap, ref_box=args.ref_box,
                          ref_newton_atol=args.ref_newton_atol)
    elif args.cmd == "long":
        sink = (lambda r: print(json.dumps(r), flush=True)) if args.jsonl else None
        res = long_run(args.bc, args.n, args.t_end, args.seed, every=args.every, sink=sink, L=args.L,
                       subdomain_solver=["ilu0", "ilu1", "ilu2", "lu"].index(args.subdomain_solver),
                       overlap=args.overlap, parts=args.parts, max_seconds=args.max_seconds)
    elif args.cmd == "subdomain":
        prec = None if args.precision is None else (0 if args.precision == "fp64" else 1)
        res = subdomain_table(args.dim, args.steps, precision=prec)
    else:
        res = schwarz_table(args.dim, args.steps)
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
