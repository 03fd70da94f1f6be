#!/usr/bin/env python
"""Benchmark of the GB300 BMG eigensolver: converged eigenpairs per second.

Workload: the unit sphere (icosahedron refined 6 times, 40962 vertices), 6 levels,
k = 64 seeded Gaussian test vectors, the 49 lowest eigenpairs (l = 0..6),
multicolour symmetric Gauss-Seidel smoothing, FP64, tolerance 1e-10.  One step is
one complete BFMG solve (levels 2..6, every cycle until convergence); a pair counts
as converged when its relative residual ||A u - lambda M u|| / (||A||_1 ||u||) is at
most 1e-8.  The hierarchy (meshes, matrices, transfers, colourings, Galerkin
operators) is built before the timed region and stays resident in HBM; L2 is flushed
(a 256 MiB write) before every timed step, outside the timed interval.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank solves its own
replica (different X0 seed): weak scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "converged eigenpairs/s at rel residual 1e-8; smoother SpMM HBM GB/s vs peak"
UNIT = "eigenpairs/s"
CONV_TOL = 1e-8
WL = dict(name="sphere40962_k64_mcsgs_fp64", refinements=6, levels=6, k=64, n_wanted=49, sigma=0.0,
          tol=1e-10, smoother="mcsgs", nu=1, omega=1.0, seed=1002)
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (vector and tensor) nominal peak


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def run_oracle_solve(H, X0):
    from oracle import bmg as obmg
    opt = obmg.Options(smoother=WL["smoother"], nu=WL["nu"], omega=WL["omega"])
    t0 = time.perf_counter()
    res = obmg.bfmg(H, X0, WL["k"], WL["n_wanted"], WL["sigma"], WL["tol"], opt)
    dt = time.perf_counter() - t0
    conv = int((res.resid[:WL["n_wanted"]] <= CONV_TOL).sum())
    return conv, dt, res


def oracle_hierarchy():
    from oracle import bmg as obmg
    from paper_1511_07042_gb300 import inputs
    v, t = inputs.icosahedron()
    return obmg.build_hierarchy(v, t, WL["levels"])


def cpu_baseline():
    """The oracle, as it stands, on one full solve of the same workload (10-20 s)."""
    from paper_1511_07042_gb300 import inputs
    H = oracle_hierarchy()
    X0 = inputs.gaussian_block(inputs.n_vertices(2), WL["k"], WL["seed"])
    conv, dt, _ = run_oracle_solve(H, X0)
    return {"value": conv / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "one complete FP64 oracle BFMG solve of the same workload (%d pairs converged "
                      "in %.1f s; NumPy/SciPy, BLAS pool of %d threads, sparse products single-threaded)"
                      % (conv, dt, os.cpu_count())}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1511_07042_gb300 import inputs
    from oracle import bmg as obmg
    v, t = inputs.icosahedron()
    Hs = obmg.build_hierarchy(v, t, 3)
    for _ in range(args.warmup):       # warm-up on the 642-vertex problem
        obmg.bfmg(Hs, inputs.gaussian_block(162, 20, 1001), 20, 16, 0.0, 1e-10)
    H = oracle_hierarchy()
    X0 = inputs.gaussian_block(inputs.n_vertices(2), WL["k"], WL["seed"])
    total_conv, total_t, steps = 0, 0.0, 0
    budget = 170.0
    for _ in range(args.steps):
        conv, dt, _ = run_oracle_solve(H, X0)
        total_conv += conv
        total_t += dt
        steps += 1
        if total_t + dt > budget:
            break
    value = total_conv / total_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WL["name"], "vertices": inputs.n_vertices(6),
                                            "levels": WL["levels"], "k": WL["k"],
                                            "n_wanted": WL["n_wanted"], "tol": WL["tol"],
                                            "smoother": WL["smoother"], "requested_steps": args.steps},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "%d complete FP64 oracle BFMG solves (stops early past %.0f s)"
                                       % (steps, budget)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def dominant_roofline(prof, hbm_peak, peak_kind):
    """Roofline of the kernel class with the largest device time in the timed region."""
    name, d = max(prof.items(), key=lambda kv: kv[1]["ms"])
    if d["launches"] == 0 or d["ms"] <= 0:
        return None, name
    per_launch_s = d["ms"] * 1e-3 / d["launches"]
    b = d["bytes"] / d["launches"]
    fl = d["flops"] / d["launches"]
    t_mem = b / (hbm_peak * 1e9)
    t_alu = fl / (FP64_NOMINAL_TFLOPS * 1e12)
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        try:
            from paper_1511_07042_gb300 import build as B
            with open(tfile) as fh:
                tj = json.load(fh)
            ent = tj.get(name)
            if ent and ent.get("sources") == B._stamp(B._sources()):
                traffic = ent["bytes_per_launch"]
        except Exception:
            traffic = None
    if t_alu >= t_mem:
        ach = fl / per_launch_s / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_NOMINAL_TFLOPS, "traffic": traffic, "kernel": name,
                "peak_source": "nominal FP64 (1.25 TFLOP/s at 2070 MHz, 152 SMs)",
                "algorithmic_flops_per_launch": fl, "algorithmic_bytes_per_launch": b,
                "launches": d["launches"], "avg_launch_us": per_launch_s * 1e6}
    else:
        ach = b / per_launch_s / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "traffic": traffic, "kernel": name,
                "peak_source": peak_kind + " copy bandwidth",
                "algorithmic_flops_per_launch": fl, "algorithmic_bytes_per_launch": b,
                "launches": d["launches"], "avg_launch_us": per_launch_s * 1e6}
    return roof, name


def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1511_07042_gb300 import bmg, inputs

    dev = torch.device("cuda", local)
    v, t = inputs.icosahedron()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prob = bmg.Problem(v, t, WL["refinements"])
    prob.hierarchy(WL["levels"])
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    n2, nL = inputs.n_vertices(2), inputs.n_vertices(WL["refinements"])
    k, nw = WL["k"], WL["n_wanted"]
    X0 = inputs.gaussian_block(n2, k, WL["seed"] + rank)
    X0d = torch.from_numpy(X0).to(dev)
    Ud = torch.empty((nL, nw), dtype=torch.float64, device=dev)
    opt = bmg.options(smoother=WL["smoother"], nu=WL["nu"], omega=WL["omega"])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        ev, _, rs, info = prob.solve(X0d, k, nw, WL["sigma"], WL["tol"], opt, evecs_device=Ud)
        return int((rs <= CONV_TOL).sum()), info

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    bmg.profile_reset()
    bmg.profile_enable(True)
    launches0 = bmg.launch_count()
    conv_total, ms_total, cycles = 0, 0.0, []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c, info = step()
        e1.record(stream)
        e1.synchronize()
        ms_total += e0.elapsed_time(e1)
        conv_total += c
        cycles.append(info.total_cycles)
    torch.cuda.synchronize()
    launches = bmg.launch_count() - launches0
    bmg.profile_enable(False)
    prof = bmg.profile_read()
    clocks = sampler.stop()
    if dist:
        dist.barrier()

    # end to end through the public call with host buffers (pinned X0 in, pinned
    # eigenvectors, values and residuals out), wall clock around each step
    X0h = torch.from_numpy(X0).pin_memory()
    Uh_t = torch.empty((nL, nw), dtype=torch.float64).pin_memory()
    e2e_total, e2e_conv = 0.0, 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        ta = time.perf_counter()
        ev, _, rs, info = prob.solve_host(X0h, Uh_t, k, nw, WL["sigma"], WL["tol"], opt)
        e2e_total += time.perf_counter() - ta
        e2e_conv += int((rs <= CONV_TOL).sum())

    tmax = torch.tensor([ms_total, e2e_total], dtype=torch.float64, device=dev)
    csum = torch.tensor([conv_total, e2e_conv], dtype=torch.float64, device=dev)
    if dist:
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(csum, op=dist.ReduceOp.SUM)
    ms_max, e2e_max = float(tmax[0]), float(tmax[1])
    value = float(csum[0]) / (ms_max * 1e-3)
    e2e_value = float(csum[1]) / e2e_max
    hbm_peak, peak_kind = load_peaks()
    roof, dom = dominant_roofline(prof, hbm_peak, peak_kind)
    if rank == 0:
        cpu = cpu_baseline() if world == 1 else None
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WL["name"], "vertices": nL, "levels": WL["levels"], "k": k,
                           "n_wanted": nw, "tol": WL["tol"], "smoother": WL["smoother"],
                           "parallelism": "replicas" if world > 1 else "single",
                           "l2": "flushed (256 MiB write) before every step, outside the timed interval",
                           "setup_s": setup_s, "cycles_per_solve": cycles[-1] if cycles else None},
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(X0.nbytes),
                        "d2h_bytes_per_step": int(nL * nw * 8 + 2 * nw * 8)},
                "gpu_launches": int(launches),
                "roofline": roof,
                "kernels": {n: {"ms": d["ms"], "launches": d["launches"]} for n, d in prof.items()},
                "cpu_baseline": cpu,
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
