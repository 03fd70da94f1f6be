#!/usr/bin/env python
"""Benchmark of the GB300 BMG eigensolver: converged eigenpairs per second.

Workload (the largest configuration that fits one GPU): the unit sphere, icosahedron
refined 8 times (655362 vertices), 8 levels, k = 128 seeded Gaussian test vectors
(seed 1004), the 100 lowest eigenpairs (l = 0..9), damped Jacobi (nu = 2, omega = 2/3),
8 cycles on each intermediate level, tolerance 1e-8, plain float64 arithmetic (the
Gram products and the Ritz-vector expansion on the tensor cores from exact digit
slices).  One step is one complete BFMG solve (levels 2..8, every cycle until every
wanted pair meets the tolerance); a pair counts as converged when its relative
residual ||A u - lambda M u|| / (||A||_1 ||u||) is at most 1e-8.  The hierarchy
(meshes, matrices, transfers, Galerkin operators) is built before the timed region
and stays resident in HBM; every block (671 MB) is larger than L2, and L2 is also
flushed (a 256 MiB write) before every timed step, outside the timed interval.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-extras]

Prints one JSON line (rank 0).  Rank 0 also adds objects measured after the timed
region: "kernels_finest" (SpMM and Jacobi sweep on the finest level, per arithmetic),
"precision_form" (the same workload with float32 blocks), "sphere40962" (the 6-level
40962-vertex workload), "batched_form" (32 perturbed spheres x 2 shifts, float32 and
float64 blocks) and "interior" (the 163842-vertex perturbed sphere at shift 110).
With N > 1 (torchrun) every rank solves its own replica (different X0 seed): weak
scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
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
WL = dict(name="sphere655362_k128_jacobi_fp64", refinements=8, levels=8, k=128, n_wanted=100, sigma=0.0,
          tol=1e-8, smoother="jacobi", nu=2, omega=2.0 / 3.0, seed=1004, cycles_intermediate=8)
# BFMG cycles per level (levels 2..8) of the FP64 oracle on this workload, from a
# complete oracle solve (166 s on 8 host cores); the GPU solve runs the same counts.
ORACLE_CYCLES = [8, 8, 8, 8, 8, 8, 9]
WL_C2 = dict(name="sphere40962_k64_mcsgs_fp64", refinements=6, levels=6, k=64, n_wanted=49, sigma=0.0,
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


def whole_job(ms_total, e2e_s, conv, e2e_conv, dist=None, device="cpu"):
    """Whole-job figures over the replicas: the slowest rank's device time and end-to-end
    wall time (max over ranks) and the converged pairs of all ranks (sum).  Returns
    (ms_max, e2e_max_s, pairs/s, end-to-end pairs/s)."""
    import torch
    tmax = torch.tensor([ms_total, e2e_s], dtype=torch.float64, device=device)
    csum = torch.tensor([conv, e2e_conv], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(csum, op=dist.ReduceOp.SUM)
    ms_max, e2e_max = float(tmax[0]), float(tmax[1])
    return ms_max, e2e_max, float(csum[0]) / (ms_max * 1e-3), float(csum[1]) / e2e_max


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


# ------------------------------------------------------------- CPU oracle ----
def oracle_sample():
    """The oracle, as it stands, on a bounded sample of the workload: its hierarchy
    (built first, untimed), then one BMG cycle on each level 2..8 from a prolongated
    Gaussian block.  The full solve's time is estimated from these per-cycle times
    and the oracle's own cycle counts per level (ORACLE_CYCLES).  Returns
    (estimated pairs/s, sample seconds, per-level seconds, cores)."""
    from oracle import bmg as obmg
    from paper_1511_07042_gb300 import inputs
    v, t = inputs.icosahedron()
    H = obmg.build_hierarchy(v, t, WL["levels"], colour=False)
    opt = obmg.Options(smoother=WL["smoother"], nu=WL["nu"], omega=WL["omega"],
                       cycles_intermediate=WL["cycles_intermediate"])
    X = inputs.gaussian_block(inputs.n_vertices(2), WL["k"], WL["seed"])
    per_level = []
    for f in range(2, WL["levels"] + 1):
        if f > 2:
            X = H.P[f] @ X
        t0 = time.perf_counter()
        obmg.cycle(H, f, X, WL["sigma"], WL["k"], WL["n_wanted"], WL["tol"], opt, smooth_if_converged=True)
        per_level.append(time.perf_counter() - t0)
    est = sum(c * s for c, s in zip(ORACLE_CYCLES, per_level))
    return WL["n_wanted"] / est, sum(per_level), per_level, os.cpu_count()


def cpu_baseline():
    value, sample_s, per_level, cores = oracle_sample()
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "one oracle BMG cycle on each level 2..8 of the same workload (%.1f s; finest level "
                      "%.1f s), scaled by the oracle's own cycles per level %s to a full solve of %.0f s; "
                      "NumPy/SciPy, BLAS pool of %d threads, sparse products single-threaded"
                      % (sample_s, per_level[-1], ORACLE_CYCLES,
                         sum(c * s for c, s in zip(ORACLE_CYCLES, per_level)), cores)}


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
    values, samples, steps, budget, t_all = [], [], 0, 150.0, 0.0
    for _ in range(args.steps):
        value, sample_s, per_level, cores = oracle_sample()
        values.append(value)
        samples.append(sample_s)
        steps += 1
        t_all += sample_s
        if t_all + sample_s > budget:
            break
    values.sort()
    value = values[len(values) // 2]
    est_s = WL["n_wanted"] / value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * est_s,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WL["name"], "vertices": inputs.n_vertices(8),
                                            "levels": WL["levels"], "k": WL["k"], "n_wanted": WL["n_wanted"],
                                            "tol": WL["tol"], "smoother": WL["smoother"],
                                            "requested_steps": args.steps},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "per step: one oracle BMG cycle on each level 2..8 (median %.1f s), "
                                       "scaled by the oracle's cycles per level %s to a full solve; median "
                                       "over %d steps (stops early past %.0f s)"
                                       % (sorted(samples)[len(samples) // 2], ORACLE_CYCLES, steps, budget)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ ours ----
def class_table(prof, hbm_peak):
    """Per kernel class: device ms, launches, algorithmic GB/s and TFLOP/s."""
    out = {}
    for n, d in prof.items():
        if d["ms"] > 0:
            out[n] = {"ms": d["ms"], "launches": d["launches"],
                      "gbs": d["bytes"] / (d["ms"] * 1e-3) / 1e9,
                      "tflops": d["flops"] / (d["ms"] * 1e-3) / 1e12}
    return out


# The source file that defines each kernel whose DRAM traffic is recorded.
TRAFFIC_SOURCE = {"row_update_kernel": "ops.cu", "spmm_am_kernel": "ops.cu",
                  "gram_tc_kernel": "tc.cu", "expand_tc_kernel": "tc.cu"}


def traffic_stamp(name):
    """Stamp of a kernel's code: the names and contents of its source file, every
    library header and the public header, and the compile flags (the stamp the
    traffic lines carry; independent of where the tree sits)."""
    from paper_1511_07042_gb300 import build as B
    files = [os.path.join(B.CSRC, TRAFFIC_SOURCE[name])]
    files += sorted(os.path.join(B.CSRC, f) for f in os.listdir(B.CSRC) if f.endswith((".cuh", ".h")))
    files += [os.path.join(B.INCLUDE, "bmg.h")]
    h = hashlib.sha256()
    for p in files:
        h.update(os.path.basename(p).encode())
        with open(p, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(B.ARCH + B.FLAGS).encode())
    return h.hexdigest()[:16]


def read_traffic(name):
    """DRAM bytes per launch of a kernel from the committed ncu summary
    (profiles/traffic_sphere655362_k128.txt: lines 'kernel bytes_per_launch stamp'),
    valid only while the kernel's code matches the stamp the counters were taken on."""
    path = os.path.join(ROOT, "profiles", "traffic_sphere655362_k128.txt")
    try:
        stamp = traffic_stamp(name)
        with open(path) as fh:
            for line in fh:
                f = line.split()
                if len(f) == 3 and f[0] == name and f[2] == stamp:
                    return float(f[1])
    except Exception:
        return None
    return None


# Kernel classes of the library's profiler that are one kernel each (the smoother
# sweeps and the residuals are both row_update_kernel launches); dense_eig (about 15
# kernels per call) and small are aggregates and are reported on their own.
SINGLE_KERNELS = {"row_update_kernel": ("smooth_sweep", "residual"), "spmm_am_kernel": ("spmm_am",),
                  "gram_tc_kernel": ("gram",), "expand_tc_kernel": ("expand",)}


def class_roofline(name, d, hbm_peak, peak_kind):
    """Roofline of one kernel (or class) from its summed profiler record: float64
    arithmetic against the nominal FP64 peak when its algorithmic flops take longer
    there than its bytes at the HBM peak, else against the HBM peak."""
    if d["launches"] == 0 or d["ms"] <= 0:
        return None
    per_launch_s = d["ms"] * 1e-3 / d["launches"]
    b = d["bytes"] / d["launches"]
    fl = d["flops"] / d["launches"]
    traffic = read_traffic(name)
    common = {"traffic": traffic, "kernel": name, "algorithmic_flops_per_launch": fl,
              "algorithmic_bytes_per_launch": b, "launches": d["launches"], "avg_launch_us": per_launch_s * 1e6}
    if fl / (FP64_NOMINAL_TFLOPS * 1e12) >= b / (hbm_peak * 1e9):
        ach = fl / per_launch_s / 1e12
        out = {"bound": "alu", "achieved": ach, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
               "frac": ach / FP64_NOMINAL_TFLOPS, "peak_source": "nominal FP64 (1.25 TFLOP/s at 2070 MHz, 152 SMs)"}
    else:
        ach = b / per_launch_s / 1e9
        out = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
               "peak_source": peak_kind + " copy bandwidth"}
    out.update(common)
    return out


def dominant_roofline(prof, hbm_peak, peak_kind):
    """Roofline of the single kernel with the largest device time in the timed region."""
    merged = {}
    for kern, classes in SINGLE_KERNELS.items():
        d = {"ms": 0.0, "launches": 0, "bytes": 0.0, "flops": 0.0}
        for c in classes:
            for key in d:
                d[key] += prof.get(c, {}).get(key, 0)
        merged[kern] = d
    name, d = max(merged.items(), key=lambda kv: kv[1]["ms"])
    return class_roofline(name, d, hbm_peak, peak_kind)


def kernels_finest(bmg, prob, torch, hbm_peak, reps=10):
    """SpMM [AX | MX] and one Jacobi sweep on the finest level (655362 rows, k = 128),
    float64 and float32 blocks, timed per launch by the kernel-class profiler (CUDA
    events on the launching stream).  Algorithmic bytes: the CSR pattern and values
    once, the block read once and written once (SpMM: two outputs)."""
    L = WL["levels"]
    n = prob.sizes(WL["refinements"])[0]
    out = {}
    for prec, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        ld = 128
        X = torch.randn((n, ld), dtype=dt, device="cuda")
        AX, MX, W = torch.empty_like(X), torch.empty_like(X), torch.empty_like(X)
        s = torch.zeros(ld, dtype=dt, device="cuda")
        spmm = prob.spmm if prec == "fp64" else prob.spmm_f32
        smooth = prob.smooth if prec == "fp64" else prob.smooth_f32
        for _ in range(2):
            spmm(L, L, X, 128, AX, MX)
            smooth(L, L, X, None, s, 128, "jacobi", 1, 2.0 / 3.0, W)
        torch.cuda.synchronize()
        bmg.profile_reset()
        bmg.profile_enable(True)
        for _ in range(reps):
            spmm(L, L, X, 128, AX, MX)
            smooth(L, L, X, None, s, 128, "jacobi", 1, 2.0 / 3.0, W)
        torch.cuda.synchronize()
        bmg.profile_enable(False)
        prof = bmg.profile_read()
        for cls, key in (("spmm_am", "spmm"), ("smooth_sweep", "jacobi")):
            d = prof[cls]
            gbs = d["bytes"] / (d["ms"] * 1e-3) / 1e9
            tfl = d["flops"] / (d["ms"] * 1e-3) / 1e12
            ent = {"us_per_launch": 1e3 * d["ms"] / d["launches"], "gbs": gbs, "frac_of_hbm_peak": gbs / hbm_peak,
                   "tflops": tfl, "bytes_per_launch": d["bytes"] / d["launches"]}
            if prec == "fp64":
                ent["frac_of_fp64_peak"] = tfl / FP64_NOMINAL_TFLOPS
                ent["bound"] = "fp64 alu (about 1 flop per byte against 0.18 at the GB300 FP64/HBM ratio)"
            else:
                ent["bound"] = "hbm"
            out["%s_%s" % (key, prec)] = ent
        del X, AX, MX, W
    return out


def solve_timed(bmg, prob, X0, wl, opt, steps, torch):
    ms, conv, info, ev = 0.0, 0, None, None
    for _ in range(steps):
        torch.cuda.synchronize()
        ta = time.perf_counter()
        ev, _, rs, info = prob.solve(X0, wl["k"], wl["n_wanted"], wl["sigma"], wl["tol"], opt, evecs=False)
        ms += (time.perf_counter() - ta) * 1e3
        conv += int((rs <= CONV_TOL).sum())
    return ms / steps, conv / (ms * 1e-3), info, ev


def precision_form_extra(bmg, prob, inputs, np, torch, steps, fp64_ms, fp64_ev):
    """The headline workload with float32 blocks (float64 Grams from float32 digit
    products, float64 eigensolve and hand-over), beside the plain float64 solve;
    per-eigenvalue error against the oracle's reference values of this workload."""
    X0 = inputs.gaussian_block(inputs.n_vertices(2), WL["k"], WL["seed"])
    ref = np.loadtxt(os.path.join(ROOT, "tests", "golden", "sphere655362_k128_mixed_oracle_eigs.txt"))[:, 1]
    opt = bmg.options(smoother=WL["smoother"], nu=WL["nu"], omega=WL["omega"], precision="fp32",
                      cycles_intermediate=WL["cycles_intermediate"])
    prob.solve(X0, WL["k"], WL["n_wanted"], WL["sigma"], WL["tol"], opt, evecs=False)   # warm-up
    ms, pairs_s, info, ev = solve_timed(bmg, prob, X0, WL, opt, steps, torch)

    def errs(e):
        d = np.abs(np.sort(e) - np.sort(ref)) / np.maximum(np.abs(ref), 1.0)
        return float(d.max()), float(np.median(d))
    e32, m32 = errs(ev)
    e64, m64 = errs(fp64_ev)
    return {"workload": WL["name"].replace("fp64", "fp32"), "eigenpairs_per_s": pairs_s, "ms_per_solve": ms,
            "cycles": info.total_cycles, "fp32_cycles": info.fp32_cycles,
            "max_rel_eig_err_vs_oracle": e32, "median_rel_eig_err_vs_oracle": m32,
            "fp64_max_rel_eig_err_vs_oracle": e64, "fp64_median_rel_eig_err_vs_oracle": m64,
            "speedup_over_fp64": fp64_ms / ms, "timing": "host wall clock around each solve, %d solves" % steps}


def c2_extra(bmg, inputs, torch, steps):
    """The 6-level 40962-vertex workload (k = 64, 49 pairs, MC-SGS, tol 1e-10, FP64)."""
    v, t = inputs.icosahedron()
    prob = bmg.Problem(v, t, WL_C2["refinements"])
    prob.hierarchy(WL_C2["levels"])
    X0 = inputs.gaussian_block(inputs.n_vertices(2), WL_C2["k"], WL_C2["seed"])
    opt = bmg.options(smoother=WL_C2["smoother"], nu=WL_C2["nu"], omega=WL_C2["omega"])
    for _ in range(2):
        prob.solve(X0, WL_C2["k"], WL_C2["n_wanted"], 0.0, WL_C2["tol"], opt, evecs=False)
    ms, pairs_s, info, _ = solve_timed(bmg, prob, X0, WL_C2, opt, steps, torch)
    prob.close()
    return {"workload": WL_C2["name"], "eigenpairs_per_s": pairs_s, "ms_per_solve": ms,
            "cycles": info.total_cycles, "timing": "host wall clock around each solve, %d solves" % steps}


def batched_form_extra(bmg, inputs, np, torch):
    """32 seeded perturbed spheres (refinements 4..7) x shifts {0, U(20, 200)}, k=32,
    24 wanted, tol 1e-8, all 64 jobs in one batched call: float32 blocks and, on the
    same jobs, float64 blocks."""
    descs = inputs.batch_instances()
    v, t = inputs.icosahedron()
    probs = []
    for d in descs:
        p = bmg.Problem(v, t, d["refinements"], d["amplitude"], d["coefs"])
        p.hierarchy(d["refinements"])
        probs.append(p)
    jobs = [(i, s) for i, d in enumerate(descs) for s in d["sigmas"]]
    X0s = [inputs.gaussian_block(inputs.n_vertices(2), 32, descs[i]["x0_seed"] + (s != 0.0)) for i, s in jobs]
    out = {"workload": "32 perturbed spheres x 2 shifts, k=32, 24 wanted", "jobs": len(jobs),
           "vertices_total": int(sum(inputs.n_vertices(descs[i]["refinements"]) for i, _ in jobs))}
    for prec in ("fp32", "fp64"):
        opt = bmg.options(precision=prec, max_cycles=100)
        args = ([probs[i] for i, _ in jobs], [s for _, s in jobs], X0s, 32, 24, 1e-8, opt)
        bmg.solve_batched(*args)   # warm-up (also creates the per-job workspaces)
        torch.cuda.synchronize()
        ta = time.perf_counter()
        ev, _, rs, infos, code = bmg.solve_batched(*args)
        dt = time.perf_counter() - ta
        conv_pairs = int(sum(int((r <= CONV_TOL).sum()) for r in rs))
        conv_jobs = [q for q in range(len(jobs)) if infos[q].converged]
        out[prec] = {"converged_pairs_per_s": conv_pairs / dt, "ms": dt * 1e3, "converged_pairs": conv_pairs,
                     "converged_jobs": len(conv_jobs),
                     "converged_jobs_sigma0": sum(1 for q in conv_jobs if jobs[q][1] == 0.0)}
    out["fp32_over_fp64"] = out["fp32"]["converged_pairs_per_s"] / out["fp64"]["converged_pairs_per_s"]
    out["note"] = ("interior shifts far above the 42-vertex coarse space do not converge with the method (the "
                   "FP64 oracle stalls the same way, tests/test_oracle_interior.py); they stop at the 100-cycle cap")
    for p in probs:
        p.close()
    return out


def interior_extra(bmg, inputs, np):
    """The interior workload: perturbed sphere r = 1 + 0.1 sum c_lm Y_lm (seed 1003),
    163842 vertices, 7 levels, k = 48, 21 pairs nearest sigma = 110, 40-cycle cap:
    damped Jacobi (the workload's smoother) and five multicolour Kaczmarz sweeps (the
    paper's smoother for interior problems, Sec. 5.3)."""
    wl = inputs.WORKLOADS["bumpy163842_k48_s110"]
    v, t = inputs.icosahedron()
    prob = bmg.Problem(v, t, wl["refinements"], wl["amplitude"], inputs.sh_coefficients(wl["coef_seed"]))
    prob.hierarchy(wl["refinements"])
    X0 = inputs.gaussian_block(inputs.n_vertices(2), wl["k"], wl["seed"])
    out = {"workload": "bumpy163842_k48_s110"}
    for name, kw in (("jacobi", dict(smoother=wl["smoother"], nu=wl["nu"], omega=wl["omega"])),
                     ("kaczmarz5", dict(smoother="kaczmarz", nu=5, omega=1.0))):
        ta = time.perf_counter()
        ev, _, rs, info = prob.solve(X0, wl["k"], wl["n_wanted"], wl["sigma"], wl["tol"],
                                     bmg.options(max_cycles=40, **kw), evecs=False)
        dt = time.perf_counter() - ta
        out[name] = {"converged": bool(info.converged), "cycles": info.total_cycles, "max_resid": float(rs.max()),
                     "ritz_min": float(np.min(ev)), "ritz_max": float(np.max(ev)), "ms": dt * 1e3}
    prob.close()
    out["oracle_verdict"] = ("the FP64 oracle does not reach the cluster either: on the same surface at refinement 4 "
                             "(LAPACK and Sylvester inertia put the 21 eigenvalues nearest 110 in [99.6, 119.5]) its "
                             "Ritz values settle far below it with Jacobi and MC-SGS, and five Kaczmarz sweeps crawl "
                             "(residual 3e-4 after 200 cycles) with pairs outside the cluster "
                             "(tests/test_oracle_interior.py)")
    return out


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
    opt = bmg.options(smoother=WL["smoother"], nu=WL["nu"], omega=WL["omega"],
                      cycles_intermediate=WL["cycles_intermediate"])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        ev, _, rs, info = prob.solve(X0d, k, nw, WL["sigma"], WL["tol"], opt, evecs_device=Ud)
        return int((rs <= CONV_TOL).sum()), info, ev

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = bmg.launch_count()
    conv_total, ms_total, cycles, last_ev = 0, 0.0, [], None
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c, info, last_ev = step()
        e1.record(stream)
        e1.synchronize()
        ms_total += e0.elapsed_time(e1)
        conv_total += c
        cycles.append(info.total_cycles)
    torch.cuda.synchronize()
    launches = bmg.launch_count() - launches0
    clocks = sampler.stop()
    if dist:
        dist.barrier()
    # per-kernel-class device times (CUDA events on the launching stream) over a
    # second pass of the same steps: the events cost host time per launch, so the
    # headline above is timed without them
    bmg.profile_reset()
    bmg.profile_enable(True)
    for _ in range(args.steps):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    bmg.profile_enable(False)
    prof = bmg.profile_read()

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

    ms_max, e2e_max, value, e2e_value = whole_job(ms_total, e2e_total, conv_total, e2e_conv, dist, dev)
    hbm_peak, peak_kind = load_peaks()
    roof = dominant_roofline(prof, hbm_peak, peak_kind)
    dense_roof = class_roofline("dense_eig", prof["dense_eig"], hbm_peak, peak_kind)
    extras = {}
    if rank == 0 and not args.no_extras:
        del Ud, Uh_t, flush
        extras["kernels_finest"] = kernels_finest(bmg, prob, torch, hbm_peak)
        extras["precision_form"] = precision_form_extra(bmg, prob, inputs, np, torch, max(2, min(args.steps, 3)),
                                                        ms_total / args.steps, last_ev)
        prob.close()
        extras["sphere40962"] = c2_extra(bmg, inputs, torch, max(3, min(args.steps, 5)))
        extras["batched_form"] = batched_form_extra(bmg, inputs, np, torch)
        extras["interior"] = interior_extra(bmg, inputs, np)
    if rank == 0:
        cpu = cpu_baseline() if world == 1 else None
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WL["name"], "vertices": nL, "levels": WL["levels"], "k": k,
                           "n_wanted": nw, "tol": WL["tol"], "smoother": WL["smoother"], "nu": WL["nu"],
                           "cycles_intermediate": WL["cycles_intermediate"], "tensor_cores": True,
                           "parallelism": "replicas" if world > 1 else "single",
                           "l2": "inputs larger than L2 (671 MB per block); L2 also flushed (256 MiB write) "
                                 "before every step, outside the timed interval",
                           "setup_s": setup_s, "cycles_per_solve": cycles[-1] if cycles else None},
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(X0.nbytes),
                        "d2h_bytes_per_step": int(nL * nw * 8 + 2 * nw * 8)},
                "gpu_launches": int(launches),
                "roofline": roof,
                "roofline_dense_eig": dense_roof,
                "dense_eig_share": prof["dense_eig"]["ms"] / max(sum(v["ms"] for v in prof.values()), 1e-9),
                "kernel_classes": class_table(prof, hbm_peak),
                "kernel_timing": "per-class CUDA events over a second pass of the same steps",
                "cpu_baseline": cpu,
                "clocks": clocks}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_case(args):
    """Small fixed cases for profiler captures (no timing line of the metric):
    precision_r7 -- one precision-form solve, icosphere refined 7 times (163842
    vertices), 7 levels, k=128, 100 pairs, tol 1e-8, Jacobi nu=2, float32 blocks;
    fp64_r7 -- the same in plain float64 (enriched problems of n = 170);
    tc_163842 -- two tensor-core Grams and two expansions, 163842 x 128, float64 then
    float32 blocks (seeded Gaussian data);
    rows_655362 -- the SpMM [AX | MX] and one Jacobi sweep on the finest level of the
    655362-vertex sphere, k = 128, float64 then float32 blocks."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1511_07042_gb300 import bmg, inputs
    cases = ("precision_r7", "fp64_r7", "tc_163842", "rows_655362")
    if args.case not in cases:
        raise SystemExit("unknown case %s (one of %s)" % (args.case, ", ".join(cases)))
    if args.case == "tc_163842":
        gen = torch.Generator(device="cuda").manual_seed(7)
        n, k = 163842, 128
        for dt in (torch.float64, torch.float32):
            X = torch.randn((n, k), dtype=dt, device="cuda", generator=gen)
            Y = torch.randn((n, k), dtype=dt, device="cuda", generator=gen)
            Yx = torch.randn((k, k), dtype=torch.float64, device="cuda", generator=gen)
            U = torch.empty_like(X)
            G = torch.empty((k, k), dtype=torch.float64, device="cuda")
            gram = bmg.gram_tc if dt == torch.float64 else bmg.gram_tc_f32
            for _ in range(2):
                gram(X, Y, k, G)
                bmg.expand(None, X, Yx, k, U, True)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "ok": True}), flush=True)
        return 0
    if args.case == "rows_655362":
        v, t = inputs.icosahedron()
        prob = bmg.Problem(v, t, 8)
        prob.hierarchy(8)
        n = prob.sizes(8)[0]
        gen = torch.Generator(device="cuda").manual_seed(7)
        for dt in (torch.float64, torch.float32):
            X = torch.randn((n, 128), dtype=dt, device="cuda", generator=gen)
            AX, MX, W = torch.empty_like(X), torch.empty_like(X), torch.empty_like(X)
            s = torch.zeros(128, dtype=dt, device="cuda")
            spmm = prob.spmm if dt == torch.float64 else prob.spmm_f32
            smooth = prob.smooth if dt == torch.float64 else prob.smooth_f32
            for _ in range(2):
                spmm(8, 8, X, 128, AX, MX)
                smooth(8, 8, X, None, s, 128, "jacobi", 1, 2.0 / 3.0, W)
            del X, AX, MX, W
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "ok": True}), flush=True)
        return 0
    v, t = inputs.icosahedron()
    prob = bmg.Problem(v, t, 7)
    prob.hierarchy(7)
    X0 = inputs.gaussian_block(inputs.n_vertices(2), 128, 1004)
    opt = bmg.options(smoother="jacobi", nu=2, omega=2.0 / 3.0,
                      precision="fp32" if args.case == "precision_r7" else "fp64", cycles_intermediate=8)
    torch.cuda.synchronize()
    ta = time.perf_counter()
    ev, _, rs, info = prob.solve(X0, 128, 100, 0.0, 1e-8, opt, evecs=False)
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "ms": (time.perf_counter() - ta) * 1e3, "converged": info.converged,
                      "cycles": info.total_cycles, "fp32_cycles": info.fp32_cycles}), flush=True)
    return 0 if info.converged else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the measurements after the timed region")
    ap.add_argument("--case", default=None,
                    help="profiling case: precision_r7 | fp64_r7 | tc_163842 | rows_655362")
    args = ap.parse_args()
    if args.case:
        return run_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
