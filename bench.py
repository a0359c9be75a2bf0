#!/usr/bin/env python
"""Benchmark of the Newton–Krylov–Schwarz time step of the energy-stable DVD scheme
for the coupled Allen–Cahn / Cahn–Hilliard system on GB300.

One bench step = one accepted time step (acac_step): residual, Jacobian /
linearisation, Schwarz-ILU(0) factorization and application, GMRES, Newton line
search, energy / mass and the adaptive-dt predictor.

Default workload: 2D 2048x2048 periodic on [0,32]^2 (mesh spacing h = 1/64), adaptive
dt from 1e-4 in [1e-5, 1e-1], RAS 17x17 overlap 2 ILU(0) (289 boxes of 124-125 cells per
direction),
seeded random initial fields (u = 0.4 + 0.05 U(-1,1), v = 0.05 U(-1,1), seed 2),
Newton rtol 1e-8.  `value` is the FP64 form's rate; the mixed-precision form (FP32
Jacobian, Krylov vectors and ILU; FP64 residual, Newton update, energy and dt
estimator) runs the same steps from the same initial state in the same process and
is reported in the `mixed` object with its speed-up over FP64 and the relative L2
difference of its fields from the FP64 fields.  The working set (state, Krylov basis,
ILU factors: several GB) is far larger than L2, so no flush is needed.

Prints one JSON line (rank 0).  --impl reference times the CPU FP64 oracle on the
host instead (a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import C3_FP64, PREC_FP64, PREC_MIXED, WORKLOADS, initial_fields  # noqa: E402

FP64_DERIVED_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # SMs x DFMA/clk/SM x 2 flop x max SM clock
FP32_DERIVED_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FALLBACK_HBM_GBS = 6800.0

# DRAM bytes (read + write) per box cell of the Schwarz kernels, from one-kernel ncu captures
# of the current kernels on a 964^2 grid with 8x8 boxes of the same 124-125 cells as the 2048^2
# workloads (one box per SM; profiles/ras_factor_2d-boxes124.md,
# profiles/ras_apply_win_2d-boxes124.md): a launch's traffic is this x its box cells (the
# traffic grows with the box cells).  Keyed by (kernel class, precision, width of the
# narrowest extended box).  A kernel changed after its capture must be removed from this table.
TRAFFIC_PER_BOX_CELL = {
    ("ras_factor", PREC_FP64, 124): 866.94e6 / 992016,
    ("ras_factor", PREC_MIXED, 124): 381.76e6 / 992016,
    ("ras_apply", PREC_FP64, 124): 505.17e6 / 992016,
    ("ras_apply", PREC_MIXED, 124): 249.47e6 / 992016,
}
# DRAM bytes per grid cell of cell kernels, from captures at the 2048^2 grid itself (or, where
# that held too much on the device, at the workload's mesh on a smaller grid whose traffic per
# cell matches): keyed by (kernel class, precision).
TRAFFIC_PER_CELL = {}
# Residual pass A has two forms in one kernel class: the first evaluation of each Newton solve
# (at the start state) and the trial evaluations.  DRAM bytes per cell of each, (first, trial),
# from one ncu capture of both at 2048^2 (profiles/residual_g_forms_2d-2048x2048-mixed.md); a
# launch's traffic is the mix of the two over the timed launches (one first evaluation per
# Newton solve).  The capture predates the kernel's launch bound (three blocks per SM), which
# changed its register allocation only (the float-cache form no longer spills 8 bytes).
TRAFFIC_PASS_A = {
    PREC_MIXED: (296.11e6 / 4194304, 377.58e6 / 4194304),
}


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback 6.8 TB/s (no MEASURED_PEAKS.json)"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id):
        self.device_id = device_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.device_id)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names[1:], parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def smi_index():
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if vis:
        return vis.split(",")[int(os.environ.get("LOCAL_RANK", "0"))]
    return os.environ.get("LOCAL_RANK", "0")


def smi_index():
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if vis:
        return vis.split(",")[int(os.environ.get("LOCAL_RANK", "0"))]
    return os.environ.get("LOCAL_RANK", "0")


# ------------------------------------------------------------------ CPU oracle sample
# The oracle needs about four minutes of one host core for one 2048^2 step, so it is timed on
# a bounded piece of the same workload: a PIECE x PIECE periodic grid with the same mesh
# spacing, coefficients, tolerances and Schwarz box geometry (boxes of the same owned width
# and overlap, hence the same 132^2 extended boxes at 2048^2), stepped at dt = dt_min, the
# step size of the timed GPU steps once the predictor has settled.  Its cost per step is
# proportional to the number of cells at fixed box geometry and iteration counts, so the
# piece's rate is scaled by piece cells / workload cells.
PIECE = 512


def piece_params(w):
    """A square periodic piece of about PIECE^2 cells with the workload's mesh spacing and
    its Schwarz boxes: an integer number of the workload's owned box widths per side, so
    the piece's extended boxes have the workload's sizes."""
    p = w.params.replace(batch=1, precision=PREC_FP64)
    own = p.n[0] / p.ras_parts[0]                       # owned box width of the workload
    parts = max(2, min(p.ras_parts[0], int(round(min(PIECE, p.n[0]) / own))))
    n = int(round(parts * own))
    h = p.L[0] / p.n[0]
    return p.replace(n=(n, n, 1), L=(n * h, n * h, 1.0), ras_parts=(parts, parts, 1), dt_mode=0, dt0=p.dt_min)


def oracle_worker(spec):
    """One oracle process of the CPU sample: build the piece, print 'ready', then for every
    'go' line on stdin take one time step from the piece's initial state and print the
    step's monotonic start / end times and iteration counts."""
    from oracle import acac_oracle as O
    d = json.loads(spec)
    w = WORKLOADS[d["workload"]]
    p = piece_params(w)
    u, v = initial_fields(p, int(d["seed"]), w.u_mean, w.amp)
    O.build_lib()
    print("ready", flush=True)
    for line in sys.stdin:
        if line.strip() != "go":
            break
        st = O.Stepper(p)
        t0 = time.monotonic()
        X, info = st.step(u, v)
        t1 = time.monotonic()
        print(json.dumps({"t0": t0, "t1": t1, "newton": info.newton_its, "gmres": info.gmres_its,
                          "status": info.status}), flush=True)


class OracleSample:
    """`procs` oracle processes, each stepping its own seeded piece; one round = every
    process takes one step at the same moment.  Piece steps per second of a round, times
    piece cells / workload cells, is the oracle's rate in workload steps per second."""

    def __init__(self, w, procs):
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
                   CUDA_VISIBLE_DEVICES="")
        self.w = w
        self.p = piece_params(w)
        self.procs = []
        for i in range(procs):
            spec = json.dumps({"workload": w.name, "seed": 1000 * w.seed + i})
            self.procs.append(subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-worker", spec],
                                               stdin=subprocess.PIPE, stdout=subprocess.PIPE, text=True, env=env))
        for pr in self.procs:
            if pr.stdout.readline().strip() != "ready":
                raise RuntimeError("oracle worker failed to start")

    def round(self):
        for pr in self.procs:
            pr.stdin.write("go\n")
            pr.stdin.flush()
        res = [json.loads(pr.stdout.readline()) for pr in self.procs]
        wall = max(r["t1"] for r in res) - min(r["t0"] for r in res)
        scale = self.p.ncells / self.w.params.ncells
        return len(res) * scale / wall, wall, res

    def close(self):
        for pr in self.procs:
            try:
                pr.stdin.write("quit\n")
                pr.stdin.flush()
                pr.stdin.close()
                pr.wait(timeout=30)
            except Exception:
                pr.kill()


def cpu_baseline(w, repeats=3):
    """The oracle as it stands, on the host: single-threaded, and one process per host core
    (at most the number of pieces that tile the workload grid), median of `repeats` rounds."""
    ncpu = os.cpu_count() or 1
    p = piece_params(w)
    tiles = max(1, w.params.ncells // p.ncells)
    out = {"unit": "steps/s", "kind": "oracle", "nproc": ncpu}
    for label, procs in (("single", 1), ("all_cores", min(ncpu, tiles))):
        sm = OracleSample(w, procs)
        try:
            rounds = [sm.round() for _ in range(repeats)]
        finally:
            sm.close()
        rates = sorted(r[0] for r in rounds)
        med = rates[len(rates) // 2]
        its = rounds[0][2][0]
        out[label] = {"value": med, "cores": procs, "round_seconds": [round(r[1], 3) for r in rounds],
                      "newton": its["newton"], "gmres": its["gmres"]}
    out["value"] = out["all_cores"]["value"]
    out["cores"] = out["all_cores"]["cores"]
    out["sample"] = (
        "FP64 NumPy/SciPy + C ILU(0) oracle on %dx%d periodic pieces of the workload (same h, coefficients, "
        "tolerances and Schwarz boxes of %d to %d cells per side with overlap %d), one time step at dt = dt_min = %g from seeded "
        "initial states, scaled by piece/workload cells (1/%.2f); median of %d rounds.  single: one process; "
        "all_cores: %d processes at once, one piece each (the pieces are not coupled, so this bounds a "
        "multi-core oracle from above); nproc = %d" % (
            p.n[0], p.n[1], p.n[0] // p.ras_parts[0] + 2 * p.ras_overlap,
            -(-p.n[1] // p.ras_parts[1]) + 2 * p.ras_overlap,
            p.ras_overlap, p.dt0, w.params.ncells / p.ncells, repeats, out["all_cores"]["cores"], ncpu))
    return out


# ------------------------------------------------------------------ roofline
def fp64_peak(probe):
    if probe:
        return probe, "measured: acac_peak_probe DFMA rate in this run"
    return FP64_DERIVED_TFLOPS, "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz"


# kernel classes whose arithmetic is double in both precision forms (residual, energy)
FP64_CLASSES = {"residual_g", "residual_f", "energy"}


def roofline(stats, precision, hbm, probe_fp64, box_cells, box_w, share_stats=None, cells=None, n_first=None):
    name, (n, ms, b, f) = max(stats.items(), key=lambda kv: kv[1][1])
    if n == 0 or ms <= 0:
        return None
    gbs = b / (ms * 1e-3) / 1e9
    tflops = f / (ms * 1e-3) / 1e12
    hbm_gbs, hbm_src = hbm
    if precision == PREC_FP64 or name in FP64_CLASSES:
        fpeak, fsrc = fp64_peak(probe_fp64)
    else:
        fpeak, fsrc = FP32_DERIVED_TFLOPS, "derived: 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz"
    per = TRAFFIC_PER_BOX_CELL.get((name, precision, box_w))
    traffic = per * box_cells if per is not None else None
    if traffic is None and cells and (name, precision) in TRAFFIC_PER_CELL:
        traffic = TRAFFIC_PER_CELL[(name, precision)] * cells
    if traffic is None and cells and name == "residual_g" and precision in TRAFFIC_PASS_A and n_first:
        first, trial = TRAFFIC_PASS_A[precision]
        k = min(n_first, n)
        traffic = cells * (k * first + (n - k) * trial) / n
    intensity = f / b if b > 0 else 0.0
    ridge = fpeak * 1e12 / (hbm_gbs * 1e9)
    out = {"kernel": name, "launches": n, "avg_launch_us": ms * 1e3 / n, "share_of_kernel_time": None,
           "traffic": traffic, "bytes_per_launch": b / n, "flops_per_launch": f / n}
    if f > 0 and intensity > ridge:
        out.update({"bound": "alu", "achieved": tflops, "peak": fpeak, "unit": "TFLOP/s", "frac": tflops / fpeak,
                    "peak_source": fsrc, "hbm_achieved_gbs": gbs})
    else:
        out.update({"bound": "hbm", "achieved": gbs, "peak": hbm_gbs, "unit": "GB/s", "frac": gbs / hbm_gbs,
                    "peak_source": hbm_src, "tflops_achieved": tflops})
    src = share_stats if share_stats is not None else stats
    tot = sum(v[1] for v in src.values())
    out["share_of_kernel_time"] = src[name][1] / tot if tot > 0 else None
    return out


def rank_barrier(world):
    """Barrier over the job's ranks (no-op for one rank)."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device):
    """Maximum of x over all ranks: the job's time is its slowest rank's."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return x


def job_rate(world, members, steps, seconds):
    """Whole-job throughput: every rank advances `members` problems by `steps` steps."""
    return world * members * steps / seconds


def twin_of(name):
    """The workload of the other precision form, if there is one."""
    for a, b in (("-fp64-", "-mixed-"), ("-mixed-", "-fp64-")):
        if a in name and name.replace(a, b) in WORKLOADS:
            return name.replace(a, b)
    return None


def run_mine(args, rank, world):
    import numpy as np
    import torch
    import paper_2007_04560_gb300 as P
    from paper_2007_04560_gb300 import build
    from paper_2007_04560_gb300.acac import acac_peak_probe

    build.build()
    w = WORKLOADS[args.workload]
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    u0, v0 = w.fields()
    B = int(w.params.batch)                  # ensemble members (1: one problem)
    N = w.params.ncells

    def barrier():
        rank_barrier(world)

    def report(info):
        """Per-step report; an ensemble reports member 0's iterations and dt."""
        return (info[0] if isinstance(info, list) else info).as_dict()

    def timed_form(wl):
        """W warm-up steps and K timed steps of workload wl on the device (inputs resident in
        HBM).  Returns the timing, the kernel statistics and the final fields."""
        p = wl.params
        s = P.Solver(p, stream)
        if B > 1:
            th = wl.thetas()
            for m in range(B):
                s.set_coeffs(m, p.alpha, p.beta, float(th[m]), p.gamma, p.rho)
        u = torch.tensor(u0.ravel(), device=dev)
        v = torch.tensor(v0.ravel(), device=dev)
        for _ in range(args.warmup - 1):
            s.step(u, v)
        # the last warm-up step times every kernel class; the timed region then times only
        # the class that took the most time there (two events per timed launch cost host time)
        s.profile(True)
        s.step(u, v)
        warm_stats = s.kernel_stats()
        dominant = max(warm_stats.items(), key=lambda kv: kv[1][1])[0]
        s.profile(True, kernels=[dominant])
        infos = []
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            infos.append(report(s.step(u, v)))
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
        stats = s.kernel_stats()
        s.close()
        return {"ms": ms, "stats": stats, "warm_stats": warm_stats, "dominant": dominant, "infos": infos,
                "u": u.cpu().numpy(), "v": v.cpu().numpy(), "params": p}

    def e2e_form(wl):
        """Same steps through the C ABI with host buffers: H2D of the state, the step and the
        D2H of the result inside the timed region, every step."""
        p = wl.params
        s2 = P.Solver(p, stream)
        if B > 1:
            th = wl.thetas()
            for m in range(B):
                s2.set_coeffs(m, p.alpha, p.beta, float(th[m]), p.gamma, p.rho)
        uh = torch.tensor(u0.ravel()).pin_memory()
        vh = torch.tensor(v0.ravel()).pin_memory()
        for _ in range(args.warmup):
            s2.step_host(uh, vh)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            s2.step_host(uh, vh)
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t0, world, dev)
        barrier()
        s2.close()
        return {"value": job_rate(world, B, args.steps, el), "unit": "steps/s" if B == 1 else "member-steps/s",
                "h2d_bytes_per_step": 16 * N * B, "d2h_bytes_per_step": 16 * N * B}

    def box_geometry(p):
        """(extended width of the narrowest box, cells of all boxes): per axis the owned
        widths add up to n and every box adds the overlap on each side (not on a wall's
        side, with Neumann walls)."""
        if p.dim != 2:
            return None, None
        wb = p.n[0] // p.ras_parts[0] + 2 * p.ras_overlap
        ends = 0 if p.bc == 0 else 1     # periodic: every box overlaps on both sides
        ext = [p.n[a] + 2 * p.ras_overlap * (p.ras_parts[a] - ends) for a in (0, 1)]
        return wb, ext[0] * ext[1]

    def summary(res, prec):
        infos = res["infos"]
        nits = sum(i["newton_its"] for i in infos)
        bw, bc = box_geometry(res["params"])
        return {
            "iterations": {"newton_per_step": nits / len(infos),
                           "gmres_per_newton": sum(i["gmres_its"] for i in infos) / max(1, nits),
                           "dt_first": infos[0]["dt"], "dt_last": infos[-1]["dt"], "t_end": infos[-1]["t"]},
            # one first evaluation of pass A per Newton solve: per step, plus one per retry
            "roofline": roofline(res["stats"], prec, hbm_peak(), probe_fp64, bc, bw, res["warm_stats"],
                                 res["params"].ncells * int(res["params"].batch),
                                 len(infos) + sum(i["divergences"] for i in infos)),
            "kernels": {k: {"launches": v[0], "ms": round(v[1], 4),
                            "gbs": (v[2] / (v[1] * 1e-3) / 1e9) if v[1] > 0 else None}
                        for k, v in res["stats"].items() if v[0] > 0},
            "kernels_timed": "timed region: events around %s launches only; last warm-up step, every class: %s" % (
                res["dominant"], {k: round(v[1], 3) for k, v in res["warm_stats"].items() if v[0] > 0}),
        }

    sampler = ClockSampler(smi_index())
    sampler.start()
    probe_fp64, probe_ms = acac_peak_probe(0, 4000)
    main = timed_form(w)
    twin_name = None if args.no_twin else twin_of(w.name)
    twin = timed_form(WORKLOADS[twin_name]) if twin_name else None
    clocks = sampler.stop()
    e2e = None if args.no_e2e else e2e_form(w)
    twin_e2e = None if (args.no_e2e or twin is None) else e2e_form(WORKLOADS[twin_name])

    if rank != 0:
        return None
    prec = w.params.precision
    steps_per_s = job_rate(world, B, args.steps, main["ms"] * 1e-3)
    launches = int(sum(v[0] for v in main["stats"].values()))
    p = w.params
    h = p.L[0] / p.n[0]
    sm = summary(main, prec)
    out = {
        "metric": "NKS time steps/s (one accepted implicit time step per step)" if B == 1 else
                  "ensemble member time steps/s (every member takes one accepted implicit step per step)",
        "value": steps_per_s,
        "unit": "steps/s" if B == 1 else "member-steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": main["ms"] / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if prec == PREC_FP64 else "f64 residual/update + f32 krylov/jacobian/ilu",
        "data": "synthetic (seeded uniform perturbation of a constant state)",
        "config": {"workload": w.name, "grid": list(p.shape[::-1]),
                   "domain": [[0.0, float(x)] for x in p.L[:p.dim]], "h": h,
                   "bc": "periodic" if p.bc == 0 else "neumann",
                   "precision": "fp64" if prec == PREC_FP64 else "mixed",
                   "unknowns": 2 * N * B, "members": B,
                   "ras": "%s overlap %d ILU(0) left-RAS" % ("x".join(str(x) for x in p.ras_parts[:p.dim]),
                                                           p.ras_overlap),
                   "newton_rtol": p.newton_rtol, "gmres_rtol": p.gmres_rtol,
                   "dt_mode": "adaptive" if p.dt_mode == 1 else "fixed",
                   "l2": "inputs larger than L2 (no flush)", "parallelism": "replicas" if world > 1 else "1 GPU"},
        "unknowns_steps_per_s": steps_per_s * 2 * N,   # per member for an ensemble
        "iterations": sm["iterations"],
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": sm["roofline"],
        "fp64_probe": {"tflops": probe_fp64, "ms": probe_ms,
                       "derived_tflops_at_2070mhz": FP64_DERIVED_TFLOPS},
        "kernels": sm["kernels"],
        "kernels_timed": sm["kernels_timed"],
    }
    if twin is not None:
        tp = twin["params"].precision
        tsm = summary(twin, tp)
        tval = job_rate(world, B, args.steps, twin["ms"] * 1e-3)
        xf = np.concatenate([main["u"], main["v"]])
        xt = np.concatenate([twin["u"], twin["v"]])
        key = "mixed" if tp == PREC_MIXED else "fp64"
        out[key] = {
            "workload": twin_name, "value": tval, "unit": out["unit"], "ms_per_step": twin["ms"] / args.steps,
            "ratio_vs_fp64": (tval / steps_per_s) if tp == PREC_MIXED else (steps_per_s / tval),
            "rel_l2_vs_fp64_fields": float(np.linalg.norm(xt - xf) / np.linalg.norm(xf)),
            "fields_compared": "after %d warm-up + %d timed steps from the same initial state" % (args.warmup,
                                                                                               args.steps),
            "e2e": twin_e2e,
            "gpu_launches": int(sum(v[0] for v in twin["stats"].values())),
            "iterations": tsm["iterations"], "roofline": tsm["roofline"], "kernels": tsm["kernels"],
            "kernels_timed": tsm["kernels_timed"],
        }
    if not args.no_extras and world == 1:
        out["other_workloads"] = other_workloads(P, stream, dev, args.extra_steps)
    if not args.no_cpu_baseline and world == 1 or (not args.no_cpu_baseline and rank == 0):
        try:
            out["cpu_baseline"] = cpu_baseline(w)
        except Exception as e:                                   # reported, not fatal
            out["cpu_baseline"] = {"value": None, "unit": "steps/s", "cores": 0, "kind": "oracle",
                                   "sample": "failed: %s" % str(e)[-200:]}
    return out


def other_workloads(P, stream, dev, steps):
    """The other configurations, briefly (device-timed, inputs resident in HBM, 3 warm-up
    steps then `steps` timed ones): 3D 128^3 Neumann in both precision forms, the 32 x 256^2
    ensemble, and one gradient of the 512^2 adjoint workload (20 steps forward and back)."""
    import torch
    from workloads import C4, C4_FP64, C5, E32
    res = []

    def stepped(w):
        p = w.params
        s = P.Solver(p, stream)
        if p.batch > 1:
            th = w.thetas()
            for m in range(p.batch):
                s.set_coeffs(m, p.alpha, p.beta, float(th[m]), p.gamma, p.rho)
        u0, v0 = w.fields()
        u = torch.tensor(u0.ravel(), device=dev)
        v = torch.tensor(v0.ravel(), device=dev)
        for _ in range(3):
            s.step(u, v)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = [s.step(u, v) for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        s.close()
        ms = e0.elapsed_time(e1) / steps
        first = [i[0] if isinstance(i, list) else i for i in infos]
        B = int(p.batch)
        return {"workload": w.name, "value": 1000.0 * B / ms, "unit": "steps/s" if B == 1 else "member-steps/s",
                "ms_per_step": ms, "steps": steps, "warmup": 3,
                "ras": "%s overlap %d" % ("x".join(str(x) for x in p.ras_parts[:p.dim]), p.ras_overlap),
                "newton_per_step": sum(i.newton_its for i in first) / steps,
                "gmres_per_step": sum(i.gmres_its for i in first) / steps,
                "dt_last": first[-1].dt}

    for w in (C4, C4_FP64, E32):
        try:
            res.append(stepped(w))
        except Exception as e:                                   # reported, not fatal
            res.append({"workload": w.name, "error": str(e)[-200:]})
    try:
        p = C5.params
        u0, v0 = C5.fields()
        ut, vt = C5.target()
        t = lambda a: torch.tensor(a.ravel(), device=dev)
        with P.Solver(p, stream) as s:
            s.adjoint(t(u0), t(v0), C5.steps, p.dt0, t(ut), t(vt), C5.w_energy, C5.w_misfit, C5.every)  # warm-up
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L, _, _, g, its = s.adjoint(t(u0), t(v0), C5.steps, p.dt0, t(ut), t(vt), C5.w_energy, C5.w_misfit,
                                        C5.every)
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        res.append({"workload": C5.name, "value": 1000.0 / ms, "unit": "gradients/s", "ms_per_gradient": ms,
                    "gradient": "loss after %d fixed-dt steps w.r.t. u0, v0, alpha, beta, theta, gamma "
                                "(checkpoint every %d)" % (C5.steps, C5.every),
                    "adjoint_gmres_its": its, "loss": L})
    except Exception as e:
        res.append({"workload": C5.name, "error": str(e)[-200:]})
    return res


def run_reference(args, rank, world):
    """The oracle on the host cores, on the same workload: each bench step is one round of
    the bounded sample (one oracle process per host core, one piece each); the rate is the
    mean over the timed rounds.  At most 1 warm-up and 3 timed rounds are run."""
    if rank != 0:
        return None
    w = WORKLOADS[args.workload]
    warm, steps = min(args.warmup, 1), min(args.steps, 3)
    ncpu = os.cpu_count() or 1
    p = piece_params(w)
    tiles = max(1, w.params.ncells // p.ncells)
    procs = min(ncpu, tiles)
    try:
        sm = OracleSample(w, procs)
        try:
            for _ in range(warm):
                sm.round()
            rounds = [sm.round() for _ in range(steps)]
        finally:
            sm.close()
    except Exception as e:
        return {"impl": "reference", "unavailable": "oracle run failed: " + str(e)[-200:].replace("\n", " ")}
    sec = sum(1.0 / r[0] for r in rounds)          # workload-step equivalents take 1/rate each
    val = steps / sec
    sample = ("FP64 oracle on %d concurrent %dx%d periodic pieces of the workload (same h, coefficients, tolerances "
              "and Schwarz box geometry), one step each at dt = dt_min per round, scaled by piece/workload cells; "
              "%d timed rounds after %d warm-up (bounded: --steps/--warmup capped at 3/1); nproc = %d" % (
                  procs, p.n[0], p.n[1], steps, warm, ncpu))
    return {"impl": "reference", "metric": "NKS time steps/s (one accepted implicit time step per step)",
            "value": val, "unit": "steps/s", "n_gpus": world, "steps": steps, "warmup": warm,
            "ms_per_step": sec * 1e3 / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded uniform perturbation of a constant state)",
            "config": {"workload": w.name, "grid": list(w.params.shape[::-1])},
            "cpu_baseline": {"value": val, "unit": "steps/s", "cores": procs, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    if len(sys.argv) == 3 and sys.argv[1] == "--oracle-worker":
        oracle_worker(sys.argv[2])
        return
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default=C3_FP64.name, choices=sorted(WORKLOADS))
    ap.add_argument("--no-twin", action="store_true", help="skip the other precision form")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other workloads' brief timings")
    ap.add_argument("--extra-steps", type=int, default=10)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            dist.init_process_group("nccl")
        out = run_mine(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
