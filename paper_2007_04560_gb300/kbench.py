"""Component timings of the time step on one workload grid.

    python -m paper_2007_04560_gb300.kbench [--workload NAME] [--precision fp64|mixed]
                                             [--reps R] [--components a,b,...]
                                             [--ras-window W] [--subdomain-solver ilu0|ilu1|ilu2|lu]
                                             [--grid NX NY] [--parts PX PY]
    python -m paper_2007_04560_gb300.kbench --probe      (FP64 / FP32 multiply-add rates)

Each component is one C-ABI entry point applied to seeded synthetic inputs of the
workload's grid (a state pair near the workload's initial state, a random direction):

    residual   acac_residual        F(X1) (passes A and B, norm)
    jacobian   acac_jacobian        linearisation + assembly
    spmv       acac_spmv            assembled J w
    jvp        acac_jvp             matrix-free J w (its linearisation is timed separately
                                    by the handle's per-kernel counters)
    ras_factor acac_ras_factor      subdomain ILU(0)
    ras_apply  acac_ras_apply       Schwarz preconditioner
    energy     acac_energy          E~ and mass

The handle's per-kernel CUDA-event counters give each kernel's average duration and its
algorithmic bytes, printed per component.  Also a convenient target for a profiler:
every component runs --reps times after one warm-up call, in the order listed.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

COMPONENTS = ("residual", "jacobian", "spmv", "jvp", "ras_factor", "ras_apply", "energy", "nks")


def main(argv=None):
    import numpy as np
    import torch

    from paper_2007_04560_gb300 import acac as A
    from paper_2007_04560_gb300 import build
    from workloads import PREC_FP64, PREC_MIXED, WORKLOADS, perturbed_pair, random_vector

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="2d-1024x1024-periodic-fp64-adaptive", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed"])
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--components", default=",".join(COMPONENTS))
    ap.add_argument("--ras-window", type=int, default=None, choices=[0, 1, 2],
                    help="2D Schwarz apply variant (params.ras_window)")
    ap.add_argument("--subdomain-solver", default=None, choices=["ilu0", "ilu1", "ilu2", "lu"],
                    help="subdomain solve of the Schwarz preconditioner (params.subdomain_solver)")
    ap.add_argument("--grid", type=int, nargs=2, default=None, metavar=("NX", "NY"),
                    help="2D grid in place of the workload's (same mesh spacing)")
    ap.add_argument("--parts", type=int, nargs=2, default=None, metavar=("PX", "PY"),
                    help="Schwarz boxes per direction in place of the workload's")
    ap.add_argument("--probe", action="store_true",
                    help="only measure the FP64 and FP32 multiply-add rates (acac_peak_probe)")
    args = ap.parse_args(argv)
    if args.probe:
        build.build()
        for kind, name, iters in ((0, "fp64", 4000), (1, "fp32", 200000), (2, "fp64 16 lanes", 4000),
                                  (3, "fp64 8 lanes", 4000), (6, "fp64 1 lane", 4000)):
            for rep in range(3):
                tf, ms = A.acac_peak_probe(kind, iters)
                print("probe %s rep %d: %.4f TFLOP/s (%.3f ms)" % (name, rep, tf, ms))
        return
    build.build()
    w = WORKLOADS[args.workload]
    p = w.params.replace(batch=1)
    if args.precision:
        p = p.replace(precision=PREC_MIXED if args.precision == "mixed" else PREC_FP64)
    if args.ras_window is not None:
        p = p.replace(ras_window=args.ras_window)
    if args.subdomain_solver is not None:
        p = p.replace(subdomain_solver=["ilu0", "ilu1", "ilu2", "lu"].index(args.subdomain_solver))
    if args.grid is not None:
        h = p.L[0] / p.n[0]
        p = p.replace(n=(args.grid[0], args.grid[1], 1), L=(args.grid[0] * h, args.grid[1] * h, 1.0))
    if args.parts is not None:
        p = p.replace(ras_parts=(args.parts[0], args.parts[1], 1))
    comps = [c for c in args.components.split(",") if c]
    for c in comps:
        if c not in COMPONENTS:
            raise SystemExit("unknown component %r" % c)
    N = p.ncells
    X1, X0 = perturbed_pair(p, w.seed, u_mean=w.u_mean, amp=w.amp, step_amp=1e-4)
    x1 = torch.tensor(np.concatenate([X1[0].ravel(), X1[1].ravel()]), device="cuda")
    x0 = torch.tensor(np.concatenate([X0[0].ravel(), X0[1].ravel()]), device="cuda")
    dt = p.dt0
    s = A.Solver(p)
    kd = s.kdtype
    wv = torch.tensor(np.concatenate([a.ravel() for a in random_vector(p, w.seed + 7)]), device="cuda").to(kd)
    y = torch.empty_like(wv)
    F = torch.empty_like(x1)
    J = torch.empty(4 * s.nslot * N, dtype=kd, device="cuda")
    s.jacobian(x1, x0, dt, J)
    s.ras_factor(J)
    calls = {
        "residual": lambda: s.residual(x1, x0, dt, F),
        "jacobian": lambda: s.jacobian(x1, x0, dt, J),
        "spmv": lambda: s.spmv(J, wv, y),
        "jvp": lambda: s.jvp(x1, x0, dt, wv, y),
        "ras_factor": lambda: s.ras_factor(J),
        "ras_apply": lambda: s.ras_apply(wv, y),
        "energy": lambda: s.energy(x1[:N], x1[N:]),
        # one Newton solve from X0 at dt (every kernel of the step's solve, including pass A
        # writing the linearisation cache and the Gram-Schmidt kernels)
        "nks": lambda: s.nks_solve(x0, dt, F),
    }
    print("workload %s, %s, %d cells, %d reps" % (w.name, "mixed" if p.precision == PREC_MIXED else "fp64", N,
                                                  args.reps))
    for c in comps:
        calls[c]()
        torch.cuda.synchronize()
        s.profile(True)
        for _ in range(args.reps):
            calls[c]()
        torch.cuda.synchronize()
        for k, (n, ms, b, f) in s.kernel_stats().items():
            if n and ms > 0:
                print("  %-10s %-11s %4d launches  %9.1f us/launch  %8.1f GB/s algorithmic" % (
                    c, k, n, 1e3 * ms / n, b / (ms * 1e-3) / 1e9))
    s.close()


if __name__ == "__main__":
    main()
