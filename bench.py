#!/usr/bin/env python
"""Benchmark of the Newton–Krylov–Schwarz time step of the energy-stable DVD scheme
for the coupled Allen–Cahn / Cahn–Hilliard system on GB300.

One bench step = one accepted time step (acac_step): residual, Jacobian /
linearisation, Schwarz-ILU(0) factorization and application, GMRES, Newton line
search, energy / mass and the adaptive-dt predictor.

Default workload: 2D 1024x1024 periodic, FP64, adaptive dt from 1e-4 in
[1e-5, 1e-1], RAS 16x16 overlap 2 ILU(0), seeded random initial fields
(u = 0.4 + 0.05 U(-1,1), v = 0.05 U(-1,1), seed 1).  The working set (state,
Krylov basis, ILU factors: ~1 GB) is far larger than L2, so no flush is needed.

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

from workloads import C2, PREC_FP64, PREC_MIXED, WORKLOADS  # noqa: E402

FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # SMs x DFMA/clk/SM x 2 flop x max SM clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FALLBACK_HBM_GBS = 6800.0

# DRAM bytes (read + write) per launch from one ncu capture of the current kernels on the
# 1024^2 workload: FP64 from the launch list of this benchmark's own run
# (profiles/launches_2d-1024x1024-periodic-fp64.md), FP32 apply from
# profiles/ras_apply_2d-1024x1024.md.  A kernel changed after its capture must be removed.
TRAFFIC = {
    ("2d-1024x1024-periodic-fp64-adaptive", "ras_apply", PREC_FP64): 552.4e6,
    ("2d-1024x1024-periodic-fp64-adaptive", "ras_apply", PREC_MIXED): 282.9e6,
    ("2d-1024x1024-periodic-fp64-adaptive", "ras_factor", PREC_FP64): 975.9e6,
}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


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


def cpu_baseline(workload_name, precision, steps=1):
    """Time the CPU oracle as it stands, single-threaded, on one time step of the
    workload (run in a fresh process)."""
    code = (
        "import sys, time, json; sys.path.insert(0, %r)\n"
        "from workloads import WORKLOADS\n"
        "from oracle import acac_oracle as O\n"
        "w = WORKLOADS[%r]\n"
        "one = hasattr(w, 'member_params')  # an ensemble: time member 0\n"
        "p = (w.member_params(0) if one else w.params).replace(precision=0)\n"
        "u, v = w.member_fields(0) if one else w.fields()\n"
        "st = O.Stepper(p)\n"
        "t = time.perf_counter()\n"
        "for k in range(%d):\n"
        "    X, info = st.step(u, v)\n"
        "    u, v = X\n"
        "el = time.perf_counter() - t\n"
        "print(json.dumps({'seconds': el, 'steps': %d, 'newton': info.newton_its, 'gmres': info.gmres_its}))\n"
    ) % (ROOT, workload_name, steps, steps)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        return {"error": r.stderr[-400:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def roofline(stats, precision, hbm_gbs, peak_src, workload, share_stats=None):
    name, (n, ms, b, f) = max(stats.items(), key=lambda kv: kv[1][1])
    if n == 0 or ms <= 0:
        return None
    gbs = b / (ms * 1e-3) / 1e9
    tflops = f / (ms * 1e-3) / 1e12
    fpeak = FP64_PEAK_TFLOPS if precision == PREC_FP64 else FP32_PEAK_TFLOPS
    traffic = TRAFFIC.get((workload, name, precision))
    intensity = f / b if b > 0 else 0.0
    ridge = fpeak * 1e12 / (hbm_gbs * 1e9)
    out = {"kernel": name, "launches": n, "avg_launch_us": ms * 1e3 / n, "share_of_kernel_time": None,
           "traffic": traffic}
    if f > 0 and intensity > ridge:
        out.update({"bound": "alu", "achieved": tflops, "peak": fpeak, "unit": "TFLOP/s",
                    "frac": tflops / fpeak,
                    "peak_source": "derived: 152 SMs x %s/clk x 2 flop x 2.07 GHz" %
                                   ("2 DFMA" if precision == PREC_FP64 else "128 FFMA"),
                    "hbm_achieved_gbs": gbs})
    else:
        out.update({"bound": "hbm", "achieved": gbs, "peak": hbm_gbs, "unit": "GB/s", "frac": gbs / hbm_gbs,
                    "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                    else "fallback 6.8 TB/s", "tflops_achieved": tflops})
    # share of GPU kernel time: from a run in which every class was timed
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


def run_mine(args, rank, world):
    import numpy as np
    import torch
    import paper_2007_04560_gb300 as P
    from paper_2007_04560_gb300 import build

    build.build()
    w = WORKLOADS[args.workload]
    prec = w.params.precision if args.precision is None else (PREC_MIXED if args.precision == "mixed" else PREC_FP64)
    p = w.params.replace(precision=prec)
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    u0, v0 = w.fields()
    N = p.ncells
    B = int(p.batch)                       # ensemble members (1: one problem)

    def set_member_coeffs(solver):
        if B > 1:
            th = w.thetas()
            for m in range(B):
                solver.set_coeffs(m, p.alpha, p.beta, float(th[m]), p.gamma, p.rho)

    def report(info):
        """Per-step report; an ensemble reports member 0's iterations and dt."""
        return (info[0] if isinstance(info, list) else info).as_dict()

    def barrier():
        rank_barrier(world)

    # ---- device-resident timed region
    s = P.Solver(p, stream)
    set_member_coeffs(s)
    u = torch.tensor(u0.ravel(), device=dev)
    v = torch.tensor(v0.ravel(), device=dev)
    for _ in range(args.warmup - 1):
        s.step(u, v)
    # the last warm-up step times every kernel class; the timed region then times only
    # the class that took the most time there (two events per timed launch cost host
    # time, which an ensemble's host-driven members feel)
    s.profile(True)
    s.step(u, v)
    warm_stats = s.kernel_stats()
    dominant = max(warm_stats.items(), key=lambda kv: kv[1][1])[0]
    s.profile(True, kernels=[dominant])
    sampler = ClockSampler(smi_index())
    sampler.start()
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
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    stats = s.kernel_stats()
    s.close()
    ms = max_over_ranks(ms, world, dev)
    launches = int(sum(v[0] for v in stats.values()))

    # ---- end to end through the C ABI with host buffers (H2D + step + D2H per step)
    e2e = None
    if not args.no_e2e:
        s2 = P.Solver(p, stream)
        set_member_coeffs(s2)
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
        e2e = {"value": job_rate(world, B, args.steps, el), "unit": "steps/s" if B == 1 else "member-steps/s",
               "h2d_bytes_per_step": 16 * N * B, "d2h_bytes_per_step": 16 * N * B}

    if rank != 0:
        return None
    hbm, src = peaks()
    steps_per_s = job_rate(world, B, args.steps, ms * 1e-3)
    out = {
        "metric": "NKS time steps/s (one accepted implicit time step per step)" if B == 1 else
                  "ensemble member time steps/s (every member takes one accepted implicit step per step)",
        "value": steps_per_s,
        "unit": "steps/s" if B == 1 else "member-steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if prec == PREC_FP64 else "f64 residual/update + f32 krylov/jacobian/ilu",
        "data": "synthetic (seeded uniform perturbation of a constant state)",
        "config": {"workload": w.name, "grid": list(p.shape[::-1]), "bc": "periodic" if p.bc == 0 else "neumann",
                   "precision": "fp64" if prec == PREC_FP64 else "mixed",
                   "unknowns": 2 * N * B, "members": B, "ras": "%dx%d overlap %d ILU(0) left-RAS" % (p.ras_parts[0], p.ras_parts[1],
                                                                                 p.ras_overlap),
                   "dt_mode": "adaptive" if p.dt_mode == 1 else "fixed",
                   "l2": "inputs larger than L2 (no flush)", "parallelism": "replicas" if world > 1 else "1 GPU"},
        "unknowns_steps_per_s": steps_per_s * 2 * N,   # per member for an ensemble
        "iterations": {"newton_per_step": sum(i["newton_its"] for i in infos) / len(infos),
                       "gmres_per_newton": sum(i["gmres_its"] for i in infos) / max(1, sum(i["newton_its"] for i in infos)),
                       "dt_first": infos[0]["dt"], "dt_last": infos[-1]["dt"], "t_end": infos[-1]["t"]},
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": roofline(stats, prec, hbm, src, w.name, warm_stats),
        "kernels": {k: {"launches": v[0], "ms": round(v[1], 4), "gbs": (v[2] / (v[1] * 1e-3) / 1e9) if v[1] > 0 else None}
                    for k, v in stats.items() if v[0] > 0},
        "kernels_timed": "timed region: events around %s launches only; last warm-up step, every class: %s" % (
            dominant, {k: round(v[1], 3) for k, v in warm_stats.items() if v[0] > 0}),
    }
    if not args.no_cpu_baseline and world == 1 or (not args.no_cpu_baseline and rank == 0):
        cb = cpu_baseline(w.name, prec, 1)
        if "seconds" in cb:
            out["cpu_baseline"] = {"value": cb["steps"] / cb["seconds"], "unit": "steps/s", "cores": 1,
                                   "kind": "oracle",
                                   "sample": "first time step of the same workload, single-threaded NumPy/SciPy + C ILU(0) "
                                             "oracle, %.1f s" % cb["seconds"]}
        else:
            out["cpu_baseline"] = {"value": None, "unit": "steps/s", "cores": 1, "kind": "oracle",
                                   "sample": "failed: " + cb.get("error", "")[-200:]}
    return out


def run_reference(args, rank, world):
    """The oracle on the host cores, on the same workload: each bench step is one
    oracle time step; W warm-up steps are run and not timed."""
    if rank != 0:
        return None
    w = WORKLOADS[args.workload]
    # Bounded sample: one oracle time step of this workload takes about a minute on
    # one host core, so at most 1 warm-up and 2 timed steps are run.
    warm, steps = min(args.warmup, 1), min(args.steps, 2)
    code = (
        "import sys, time, json; sys.path.insert(0, %r)\n"
        "from workloads import WORKLOADS\n"
        "from oracle import acac_oracle as O\n"
        "w = WORKLOADS[%r]\n"
        "one = hasattr(w, 'member_params')  # an ensemble: time member 0\n"
        "p = (w.member_params(0) if one else w.params).replace(precision=0)\n"
        "u, v = w.member_fields(0) if one else w.fields()\n"
        "st = O.Stepper(p)\n"
        "for k in range(%d):\n"
        "    X, info = st.step(u, v); u, v = X\n"
        "t = time.perf_counter()\n"
        "for k in range(%d):\n"
        "    X, info = st.step(u, v); u, v = X\n"
        "print(json.dumps({'seconds': time.perf_counter() - t}))\n"
    ) % (ROOT, w.name, warm, steps)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=3600)
    if res.returncode != 0:
        return {"impl": "reference", "unavailable": "oracle run failed: " + res.stderr[-200:].replace("\n", " ")}
    sec = json.loads(res.stdout.strip().splitlines()[-1])["seconds"]
    val = steps / sec
    return {"impl": "reference", "metric": "NKS time steps/s (one accepted implicit time step per step)",
            "value": val, "unit": "steps/s", "n_gpus": world, "steps": steps, "warmup": warm,
            "ms_per_step": sec * 1e3 / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded uniform perturbation of a constant state)",
            "config": {"workload": w.name, "grid": list(w.params.shape[::-1])},
            "cpu_baseline": {"value": val, "unit": "steps/s", "cores": 1, "kind": "oracle",
                             "sample": "%d oracle time steps after %d warm-up step(s) of the same workload "
                                       "(bounded: --steps/--warmup capped at 2/1), single-threaded" % (steps, warm)},
            "e2e": {"value": val, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default=C2.name, choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
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
