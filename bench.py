"""Throughput of the IB-FE-IPCS time step on GB300.

A step is one full IPCS time step (tentative-velocity BiCGStab, BCE-IB force
solve and correction, pressure-increment PCG with the multigrid V-cycle,
velocity-correction PCG) of the default workload: the synthetic aorta-like
vessel (arched, tapered, three branches) on a 256x256x384 coarse grid with two
refinement levels in a band around the wall and domain reduction (56 M active
leaf cells, 204k wall points, cardiac inflow waveform of peak Re 1500,
dt = 5e-4), mixed precision (FP32 Krylov iterations inside FP64 defect
correction).  Metric: active leaf cells x steps / second.  The same line
carries the plain FP64 GPU path timed on the same steps (`fp64`), the
continuously batched serving run against the FP64 path one request at a time
(`serve`), the dominant kernel's roofline and the CPU oracle on a bounded slab
of the same workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                    [--precision mixed|fp64] [--workload NAME] [--serve N | --no-serve]

Under torchrun each rank runs an independent replica on its own GPU (the path
has no exchange step between problems): value = all ranks' cell-steps / the
slowest rank's time.  --impl reference times the CPU oracle instead (rank 0).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "IPCS cell-steps/s at 1e-6 vs plain FP64 GPU path; %HBM peak; serve p50/p99"
UNIT = "cell-steps/s"
FALLBACK_HBM_GBS = 6800.0


DEFAULT_WORKLOAD = "aorta_256x256x384_L2"


def workload(name):
    import workloads as W
    if name == "cylinder_64x64x256_L1":
        return W.cylinder_refined_64x64x256()
    if name == "cylinder_16x16x64":
        return W.cylinder_uniform_16x16x64()
    if name == "aneurysm_128x128x256_L2":
        return W.aneurysm_128x128x256_L2()
    if name == "aorta_256x256x384_L2":
        return W.aorta_256x256x384_L2()
    raise SystemExit(f"unknown workload {name}")


def apply_variant(case, args):
    """The viscous form and the inlet condition of the timed workload."""
    case["viscous"] = args.viscous
    if args.inlet == "pressure":
        p = case["ports"][0]
        if p["kind"] != "inlet":
            raise SystemExit("--inlet pressure needs a workload whose first port is a velocity inlet")
        f = 16.0 * case["nu"] * case["extent"][p["axis"]] / p["radius"] ** 2
        p.update(kind="pinlet", a0=p["a0"] * f, a=tuple(v * f for v in p["a"]), b=tuple(v * f for v in p["b"]))
    return case


def job_aggregate(t_local, units_per_step, steps, world, dist=None, device="cuda"):
    """Replicas: every rank steps its own problem; the job's time is the
    slowest rank's (max over ranks) and its value the units of all ranks over
    that time.  Returns (time, value per second of that time unit)."""
    import torch
    t = float(t_local)
    if dist is not None and world > 1:
        tt = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return t, units_per_step * steps * world / t


def moving_wall(case, device):
    """Wall motion for --moving: every point oscillates along x with amplitude
    0.4 finest cells and period 25 steps, wall velocity the time derivative.
    Returns n -> (X, U_B) at t = (n + 1) dt as CUDA tensors."""
    import math
    import torch
    X0 = torch.tensor(case["X"], dtype=torch.float64, device=device)
    hf = case["extent"][0] / (case["n"][0] * 2 ** case["max_level"])
    amp, period, dt = 0.4 * hf, 25 * case["dt"], case["dt"]
    w = 2.0 * math.pi / period

    def at(n):
        t = (n + 1) * dt
        X = X0.clone()
        X[:, 0] += amp * math.sin(w * t)
        UB = torch.zeros_like(X0)
        UB[:, 0] = amp * w * math.cos(w * t)
        return X, UB
    return at


def sample_case(name):
    """Bounded sample of the workload for the CPU oracle: the same cross-section,
    grid, bands and point density over a slab of the tube's length."""
    import workloads as W
    if name == "cylinder_64x64x256_L1":
        return (W.cylinder_refined_slab_64x64x16(),
                "64x64x16 coarse-cell slab of the same tube (16 of 256 cells in z, 2000 points), 2 steps")
    if name == "aneurysm_128x128x256_L2":
        return (W.aneurysm_slab_128x128x16_L2(nz=4),
                "128x128x4 coarse-cell slab of the aneurysm through the sac centre (4 of 256 cells in z)")
    if name == "aorta_256x256x384_L2":
        # 4 of 384 coarse cells in z across the two straight limbs (z = -3):
        # each limb gets an inlet on the slab's low face and an outlet on its high face
        c = W.aorta_256x256x384_L2()
        h = c["extent"][2] / c["n"][2]
        k0 = int((-3.0 - c["origin"][2]) / h)
        return (_slab(c, k0, 4, [(-3.0, 1.0), (3.0, None)]),
                "256x256x4 coarse-cell slab of the aorta across its two straight limbs (4 of 384 cells in z)")
    return workload(name), "full workload"


def _slab(c, k0, nz, tubes):
    """A slab of nz coarse cells of a case from coarse layer k0: the wall
    points there, the inside mask cut to the slab, and for each z-aligned tube
    (x centre, radius or None for the largest wall distance there) a velocity
    inlet on the slab's low face and an outlet on its high face."""
    import numpy as np
    import workloads as W
    h = c["extent"][2] / c["n"][2]
    z0 = c["origin"][2] + k0 * h
    keep = (c["X"][:, 2] >= z0) & (c["X"][:, 2] <= z0 + nz * h)
    X = c["X"][keep].copy()
    ports = []
    for x0, r in tubes:
        if r is None:
            near = np.abs(X[:, 0] - x0) < 2.0
            r = float(np.hypot(X[near, 0] - x0, X[near, 1]).max())
        ports.append(W._port(2, 0, (x0, 0.0, z0), r, W.INLET, a0=1.0))
        ports.append(W._port(2, 1, (x0, 0.0, z0 + nz * h), r, W.OUTLET))
    return W._case(c["name"] + "_slab", (c["origin"][0], c["origin"][1], z0), (c["extent"][0], c["extent"][1], nz * h),
                   (c["n"][0], c["n"][1], nz), X, c["dS"][keep], np.ascontiguousarray(c["inside"][k0:k0 + nz]),
                   ports, c["nu"], c["dt"], 2, c["max_level"], c["refine_band"], c["reduce_band"])


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# algorithmic bytes per stored node copy and launch, by profiling class
# (FP32 values in the mixed path's inner solves, FP64 otherwise; meta = 2 B)
def class_bytes(cls, vb, multigrid=False):
    """Algorithmic bytes per stored valid node slot of one launch of a kernel class."""
    return {
        0: 4 * vb + 2,                 # Poisson CG stencil: read z, p_old, meta; write p_new, q
        1: (6 if multigrid else 7) * vb + 2,   # CG update: x rw, r rw, p, q read, meta (+ D^-1 read, z write)
        2: 3 * vb,                     # p = z + beta p: z read, p rw
        3: 12 * vb + 2,                # mass CG stencil, 3 comps: read z, p_old; write p_new, q
        4: 3 * 6 * vb + vb + 2,        # mass CG update, 3 components + D^-1
        5: 3 * 3 * vb,                 # mass direction update
        6: 15 * vb + 6 * vb + 2,       # momentum apply: 15 coefficients, 3 in, 3 out
        7: 3 * 7 * vb + 2,             # BiCGStab x, r update: x rw, ph, sh, s, t, rh read, r write (3 comps)
        8: 3 * 5 * vb + vb + 2,        # BiCGStab p update: r, v read, p rw, ph write (3 comps), D^-1
        9: 2 * vb + 2,                 # V-cycle stencil apply: read x, meta; write q
        10: 5 * vb + 2,                # V-cycle smoothing update: read z, r, q, D^-1, meta; write z
    }.get(cls)


def timed_class_bandwidth(dms, dn, vb, multigrid, n_valid, peak):
    """Per timed class with a byte model (every class but the V-cycle
    transfers), the achieved fraction of `peak`, and over all of them together
    the algorithmic bytes per step over their time: dms / dn are the
    milliseconds and launches per class, n_valid the valid node slots."""
    ks = [k for k in CLASS_NAMES if dn[k] > 0 and class_bytes(k, vb, multigrid) is not None]
    frac = {}
    total_b = total_ms = 0.0
    for k in ks:
        b = class_bytes(k, vb, multigrid) * n_valid * dn[k]
        frac[CLASS_NAMES[k]] = round(b / (dms[k] / 1e3) / 1e9 / peak, 3) if dms[k] > 0 else None
        total_b += b
        total_ms += dms[k]
    gbs = total_b / (total_ms / 1e3) / 1e9 if total_ms > 0 else None
    return {"gbs": gbs, "frac": gbs / peak if gbs else None,
            "time_share": total_ms / sum(dms) if sum(dms) > 0 else None, "per_class_frac": frac}


CLASS_NAMES = {0: "k_poisson_cg (p = z + beta p, q = K p, fused p.q)", 1: "k_cg_update<Poisson>",
               2: "k_cg_p<Poisson>", 3: "k_apply15<mass> (fused p = z + beta p, p.q)", 4: "k_cg_update<mass>",
               5: "k_cg_p<mass>",
               6: "momentum apply, 15 coefficients, 3 comps (k_apply15_mom32 on the mixed path)",
               7: "k_bcgv_xr<momentum>",
               8: "k_bcgv_p<momentum>", 9: "k_poisson_cg<apply> (V-cycle smoothing stencil)",
               10: "k_mg_c_smooth (V-cycle smoothing update)", 11: "V-cycle transfers and coarse levels"}


TUNE_CACHE = os.path.join(ROOT, "paper_2007_02082_gb300", "tune_cache.json")


def resolve_tune(case, precision, args, local_rank):
    """Launch choices of the timed handles: the autotuner's cached choice for
    the workload's class (--tune cache, the default), a fresh tuning run that
    updates the cache (--tune run), or the library's defaults (--tune off)."""
    from paper_2007_02082_gb300 import tune as T
    if args.tune == "off":
        return None, {"source": "library defaults", "choice": dict(T.DEFAULTS)}
    cache = T.TuneCache(TUNE_CACHE)
    if args.tune == "run":
        cache.table.pop(_tune_key(case, precision, local_rank), None)
    choice, key, hit, timings = T.tune_case(case, precision, cache=cache, device=local_rank, steps=3, warmup=2)
    return choice, {"source": "cache" if hit else "tuned now", "key": key, "choice": choice,
                    "candidates": [{"overrides": o, "ms_per_step": t} for o, t in timings] or None}


def _tune_key(case, precision, local_rank):
    from paper_2007_02082_gb300 import IBGrid
    from paper_2007_02082_gb300 import tune as T
    h = IBGrid(case, precision=precision, device=local_rank, deferred=True)
    k = T.class_key(h.ib_grid_info(), precision, case["max_level"])
    h.close()
    return k


def run_native(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2007_02082_gb300 import IBGrid, load_library

    torch.cuda.set_device(local_rank)
    load_library(build_if_missing=True)
    case = apply_variant(workload(args.workload), args)
    tune, tune_meta = resolve_tune(case, args.precision, args, local_rank)
    args.tune_choice = tune
    g = IBGrid(case, precision=args.precision, device=local_rank, poisson_pc=args.poisson_pc, tune=tune)
    info0 = g.ib_grid_info()
    cells = info0["n_leaf_cells"]
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod

    wall = moving_wall(case, f"cuda:{local_rank}") if args.moving else None
    nstep = [0]
    rebuild_ms = [0.0]

    def step():
        if wall is not None:
            X, UB = wall(nstep[0])
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.ib_set_points(X, UB)
            e1.record(stream)
            e1.synchronize()
            rebuild_ms[0] += e0.elapsed_time(e1)
        g.ipcs_step(1)
        nstep[0] += 1

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    rebuild_ms[0] = 0.0
    i1 = g.ib_grid_info()
    clocks = ClockSampler(local_rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        flush.zero_()                     # evict the working set from L2 between steps
        if args.nvtx:
            torch.cuda.nvtx.range_push("ipcs_step")
        step()
        if args.nvtx:
            torch.cuda.nvtx.range_pop()
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    if dist:
        dist.barrier()
    ck = clocks.stop()
    i2 = g.ib_grid_info()
    launches = i2["kernel_launches"] - i1["kernel_launches"]
    ms, value = job_aggregate(ms / 1e3, cells, args.steps, world, dist)
    ms *= 1e3

    # Kernels inside the step graph cannot be bracketed by events, so the same
    # step is replayed eagerly on a second handle (same stream, same kernels,
    # same order) with CUDA events around every solver kernel launch.
    gp = IBGrid(case, precision=args.precision, device=local_rank, profile=True, poisson_pc=args.poisson_pc,
                tune=tune)
    for _ in range(max(1, args.warmup)):
        gp.ipcs_step(1)
    j1 = gp.ib_grid_info()
    prof_steps = max(1, min(args.steps, 3))
    for _ in range(prof_steps):
        flush.zero_()
        if args.nvtx:   # kernels of a graph with conditional nodes are not profiled by ncu: use this range
            torch.cuda.nvtx.range_push("ipcs_step_eager")
        gp.ipcs_step(1)
        if args.nvtx:
            torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    j2 = gp.ib_grid_info()
    gp.close()
    dms = [j2["prof_ms"][k] - j1["prof_ms"][k] for k in range(12)]
    dn = [j2["prof_launches"][k] - j1["prof_launches"][k] for k in range(12)]
    mgon = info0["mg_levels"] > 0
    vb = 4 if args.precision == "mixed" else 8
    dom = max((k for k in CLASS_NAMES if dn[k] > 0 and class_bytes(k, vb) is not None), key=lambda k: dms[k])
    prof_share = {CLASS_NAMES[k]: round(dms[k] / max(sum(dms), 1e-30), 4) for k in CLASS_NAMES if dn[k] > 0}
    prof_us = {CLASS_NAMES[k]: round(1e3 * dms[k] / dn[k], 1) for k in CLASS_NAMES if dn[k] > 0}
    prof_ms_step = {CLASS_NAMES[k]: round(dms[k] / prof_steps, 3) for k in CLASS_NAMES if dn[k] > 0}
    per_launch_bytes = class_bytes(dom, vb, mgon) * info0["n_valid_slots"]
    avg_ms = dms[dom] / dn[dom]
    achieved = per_launch_bytes / (avg_ms / 1e3) / 1e9
    peak, peak_src = peaks()
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        try:
            tj = json.load(open(tfile))
            key = f"{args.workload}:{args.precision}:{dom}"
            if args.viscous != "grad" or args.inlet != "velocity":
                key += f":{args.viscous}:{args.inlet}"
            traffic = tj.get(key)
        except Exception:
            traffic = None

    # end to end through the public API with host buffers: per step, set the
    # state from pinned host memory, step, read the state back
    N = info0["n_nodes"]
    hu = torch.empty((N, 3), dtype=torch.float64, pin_memory=True).numpy()
    hp = torch.empty((N,), dtype=torch.float64, pin_memory=True).numpy()
    hu[:] = g.ib_fields_get("U")
    hp[:] = g.ib_fields_get("P")
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(e2e_steps):
        g.ib_fields_set("U", hu)
        g.ib_fields_set("P", hp)
        g.ipcs_step(1)
        g.ib_fields_get("U", out=hu)        # straight into the pinned buffers
        g.ib_fields_get("P", out=hp)
    torch.cuda.synchronize()
    te = time.perf_counter() - te
    te, e2e_value = job_aggregate(te, cells, e2e_steps, world, dist)
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": int(hu.nbytes + hp.nbytes), "d2h_bytes_per_step": int(hu.nbytes + hp.nbytes)}

    # the plain FP64 GPU path on the same steps from the same start, timed with
    # CUDA events like the timed region, and the accuracy of the mixed path
    # against it (outside the timed region)
    fp64 = None
    if args.accuracy_steps > 0 and args.precision == "mixed":
        fp64 = fp64_comparison(case, args, local_rank, wall, flush, stream)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32-inner/f64-outer" if args.precision == "mixed" else "f64",
        "data": "synthetic (seeded analytic geometry)",
        "config": {"workload": case["name"], "grid": list(case["n"]), "max_level": case["max_level"],
                   "leaf_cells": cells, "nodes": info0["n_nodes"], "points": info0["n_points"],
                   "precision": args.precision,
                   "poisson_pc": (f"multigrid V(2,2), {info0['mg_levels']} levels, coarsest {info0['mg_coarsest']}"
                                  if info0["mg_levels"] else "jacobi"),
                   "viscous": args.viscous, "inlet": args.inlet,
                   "moving": ("wall oscillating along x, amplitude 0.4 finest cells, period 25 steps; "
                              f"device rebuild {rebuild_ms[0] / args.steps:.3f} ms per step, inside the timed step")
                   if wall is not None else None,
                   "l2": "flushed between steps (256 MB write)",
                   "launch_choices": tune_meta,
                   "parallelism": f"replicas x{world}"},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "kernel": CLASS_NAMES[dom], "peak_source": peak_src,
                     "avg_launch_us": avg_ms * 1e3, "bytes_per_launch": per_launch_bytes,
                     "timing": "CUDA events around each launch, eager replay of the same step",
                     "solver_kernel_time_share": prof_share, "solver_kernel_avg_us": prof_us,
                     "solver_kernel_ms_per_step": prof_ms_step,
                     "timed_classes": timed_class_bandwidth(dms, dn, vb, mgon, info0["n_valid_slots"], peak)},
        "clocks": ck,
        "e2e": e2e,
        "iters_last_step": {k: i2[k] for k in ("iters_mom", "iters_ib", "iters_p", "iters_corr", "outer_mom",
                                              "outer_p", "outer_corr")},
        "fp64": fp64,
        "fp64_ms_per_step": fp64["fp64_ms_per_step"] if fp64 else None,
        "mixed_vs_fp64_speedup": fp64["speedup"] if fp64 else None,
    }
    if args.wss:
        X = torch.tensor(case["X"], dtype=torch.float64, device=f"cuda:{local_rank}")
        if args.moving:
            X = wall(nstep[0] - 1)[0]
        nrm = torch.zeros_like(X)
        r = torch.sqrt(X[:, 0] ** 2 + X[:, 1] ** 2)
        nrm[:, 0], nrm[:, 1] = X[:, 0] / r, X[:, 1] / r
        w = torch.empty(X.shape[0], dtype=torch.float64, device=X.device)
        gr = torch.empty((X.shape[0], 3, 3), dtype=torch.float64, device=X.device)
        for _ in range(2):
            g.lib.ib_wss(g.h, nrm.data_ptr(), w.data_ptr(), gr.data_ptr(), 1)
        reps = 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            g.lib.ib_wss(g.h, nrm.data_ptr(), w.data_ptr(), gr.data_ptr(), 1)
        e1.record(stream)
        torch.cuda.synchronize()
        out["wss"] = {"ms": e0.elapsed_time(e1) / reps, "points": int(X.shape[0]),
                      "max": float(w.max()), "mean": float(w.mean()),
                      "method": "second-order DC-PSE over finest-level fluid nodes within 3.5 finest spacings"}
    g.close()
    return out


def fp64_comparison(case, args, local_rank, wall, flush, stream):
    """The mixed path and the plain FP64 GPU path stepped from the same start
    for args.accuracy_steps steps, each step timed with CUDA events on the
    library's stream (L2 flushed before each); returns the per-step times,
    the speed-up and the relative L2 distance of U and P after the last step."""
    import numpy as np
    import torch
    from paper_2007_02082_gb300 import IBGrid
    n = args.accuracy_steps
    res = {}
    fields = {}
    for prec in ("mixed", "fp64"):
        h = IBGrid(case, precision=prec, device=local_rank, poisson_pc=args.poisson_pc,
                   tune=getattr(args, "tune_choice", None) if prec == "mixed" else None)
        cells = h.ib_grid_info()["n_leaf_cells"]
        ms = 0.0
        for k in range(n):
            if wall is not None:            # the same wall motion on both paths
                X, UB = wall(k)
                h.ib_set_points(X, UB)
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.ipcs_step(1)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        res[prec] = ms / n
        fields[prec] = {f: h.ib_fields_get(f) for f in ("U", "P")}
        h.close()
    acc = {"rel_l2_" + f.lower(): float(np.linalg.norm(fields["mixed"][f] - fields["fp64"][f])
                                        / max(np.linalg.norm(fields["fp64"][f]), 1e-300)) for f in ("U", "P")}
    return {"steps": n, "from": "rest (the same start on both paths)", "mixed_ms_per_step": res["mixed"],
            "fp64_ms_per_step": res["fp64"], "fp64_cell_steps_per_s": cells / (res["fp64"] / 1e3),
            "speedup": res["fp64"] / res["mixed"], **acc, "tolerance": 1e-6,
            "within": bool(max(acc.values()) <= 1e-6),
            "accuracy_against": "plain FP64 GPU path, same start (each path matches the FP64 oracle: "
                                "FP64 <= 1e-10, mixed <= 1e-6, in the parity tests)"}


def run_oracle_sample(name, steps=1):
    """Time the CPU oracle (as it stands) on a bounded sample of the workload."""
    from oracle import ibfe
    case, desc = sample_case(name)
    o = ibfe.Oracle(case)
    cells = int(len(o.mesh.leaf_corner))
    c = time.process_time()
    t = time.perf_counter()
    o.run(steps)
    t = time.perf_counter() - t
    c = time.process_time() - c
    # the oracle's numpy / scipy calls may run library threads: the cores it
    # used are measured as the process CPU time over the wall time
    return {"value": cells * steps / t, "unit": UNIT, "cores": max(1, round(c / t)), "kind": "oracle",
            "sample": f"{desc}, {steps} step(s): {cells} leaf cells, {t:.1f} s wall, {c:.1f} s CPU "
                      f"(numpy / scipy library threads on {os.cpu_count()} host cores; cores = CPU / wall)"}


def run_serving(n_req, steps, seed=5):
    """Serving comparison on a reduced config-5 stream (the full mix is 256
    requests x 200 steps of 32^3-128^3 active leaf cells): seeded vessels of
    32^3-96^3 active leaf cells, 0-2 levels, Poisson arrivals at 0.8 x the
    batched path's capacity, measured first on the same requests all arriving
    at once.  The continuously batched mixed path and the plain FP64 path one
    request at a time serve the same arrivals."""
    import workloads as W
    from paper_2007_02082_gb300.serve import serve, serve_one_at_a_time
    base = W.serving_requests(n_req=n_req, rate=None, seed=seed, steps=steps, cells_lo=32 ** 3,
                              cells_hi=96 ** 3)
    # capacity of the batched path: the whole stream at t = 0
    cal = serve([(0.0, c) for _, c in base], precision="mixed", epoch_steps=10).summary()
    capacity = n_req / cal["makespan_s"]
    lam = 0.8 * capacity
    stream = [(t / lam, c) for t, c in base]      # unit-rate arrivals scaled to rate lam
    b = serve(stream, precision="mixed", epoch_steps=10).summary()
    o = serve_one_at_a_time(stream, precision="fp64").summary()
    return {"requests": n_req, "steps": steps, "capacity_req_per_s": capacity, "rate_req_per_s": lam,
            "batched_mixed": b, "one_at_a_time_fp64": o,
            "p99_speedup": o["p99_s"] / b["p99_s"], "throughput_speedup": b["cell_steps_per_s"] / o["cell_steps_per_s"],
            "stream": "seeded Poisson arrivals at 0.8 x the measured capacity of the batched path; straight, bent "
                      "and aneurysmal tubes, R 0.3-1.0, L 3-10, coarse spacing sized for 32^3-96^3 active leaf "
                      "cells, 0-2 levels, nu 0.01-0.05; mixed path at the 1e-6 accuracy of the parity tests"}


def parse_tune(text):
    """Launch choices given as "key=value,key=value" (keys of the library's
    tune array); empty text gives None (the library's defaults)."""
    if not text:
        return None
    out = {}
    for item in text.split(","):
        k, _, v = item.partition("=")
        out[k.strip()] = int(v)
    return out


def run_batch_gaps(n_req, seed=5, tune=None):
    """How busy the GPU is inside a batched serving step: a batch of n_req
    serving requests steps through its captured graph (CUDA events, mean of 5
    steps), then steps once eagerly inside the NVTX range 'batch_step_eager'
    (a launch-list capture of that range gives the sum of the kernels'
    durations).  Returns the graph time per step and the kernel launches per
    step; the gaps are the graph time minus the kernels' summed durations."""
    import torch
    import workloads as W
    from paper_2007_02082_gb300 import IBBatch, IBGrid
    stream = W.serving_requests(n_req=n_req, rate=None, seed=seed, steps=40, cells_lo=32 ** 3, cells_hi=96 ** 3)
    out = {}
    for mode in ("graph", "eager"):
        mem = [IBGrid(c, precision="mixed", deferred=True, profile=(mode == "eager"), tune=tune) for _, c in stream]
        b = IBBatch(mem)
        b.step(2)
        torch.cuda.synchronize()
        k0 = b.info(0)["kernel_launches"]
        if mode == "graph":
            st = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.nvtx.range_push("batch_step_graph")
            e0.record(st)
            b.step(5)
            e1.record(st)
            torch.cuda.nvtx.range_pop()
            torch.cuda.synchronize()
            out["graph_ms_per_step"] = e0.elapsed_time(e1) / 5
            out["launches_per_step"] = (b.info(0)["kernel_launches"] - k0) / 5
            out["cells"] = sum(b.info(i)["n_leaf_cells"] for i in range(len(mem)))
        else:
            torch.cuda.nvtx.range_push("batch_step_eager")
            b.step(1)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
            out["eager_launches_per_step"] = b.info(0)["kernel_launches"] - k0
        b.close()
        for m in mem:
            m.close()
    out["requests"] = n_req
    out["tune"] = tune
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--poisson-pc", default="multigrid", choices=["multigrid", "jacobi"])
    ap.add_argument("--accuracy-steps", type=int, default=10,
                    help="steps of the timed mixed vs plain FP64 comparison reported under 'fp64' (0: skip)")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--viscous", default="grad", choices=["grad", "sym"],
                    help="viscous form: nu (grad u, grad v) or the symmetric 2 nu (eps(u), eps(v))")
    ap.add_argument("--inlet", default="velocity", choices=["velocity", "pressure"],
                    help="drive the tube by its inlet velocity or by the inlet pressure that gives the same "
                         "Poiseuille peak (16 nu L / R^2 per unit of peak speed)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tune", default="cache", choices=["cache", "run", "off"],
                    help="launch choices: the autotuner's cached choice for the workload class (tuning it when "
                         "the class is new), a fresh tuning run, or the library defaults")
    ap.add_argument("--wss", action="store_true",
                    help="also time the wall shear stress at the wall points (ib_wss, device buffers) after the "
                         "timed steps; tubes along z, radial normals")
    ap.add_argument("--moving", action="store_true",
                    help="move the wall every step (ib_set_points: device rebuild of the IB structures), "
                         "timed with the step")
    ap.add_argument("--nvtx", action="store_true",
                    help="wrap each timed step in an NVTX range 'ipcs_step' and each eagerly replayed step "
                         "in 'ipcs_step_eager'")
    ap.add_argument("--serve", type=int, default=24,
                    help="requests of the serving comparison run after the timed steps (0: skip)")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-steps", type=int, default=40)
    ap.add_argument("--batch-gaps", type=int, default=0,
                    help="only time a batch of this many serving requests (graph step, and one eager step in the "
                         "NVTX range 'batch_step_eager' for a launch-list capture) and print the result")
    ap.add_argument("--batch-tune", default="",
                    help="launch choices of the --batch-gaps members, e.g. 'mg_persist=2,poisson_kernel=3'")
    args = ap.parse_args()

    if args.batch_gaps:
        from paper_2007_02082_gb300 import load_library
        load_library(build_if_missing=True)
        print(json.dumps({"batch_gaps": run_batch_gaps(args.batch_gaps, tune=parse_tune(args.batch_tune))}))
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        cb = run_oracle_sample(args.workload, steps=max(1, min(args.steps, 2)))
        v = cb["value"]
        out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded analytic geometry)",
               "config": {"workload": args.workload, "precision": "f64 oracle"},
               "cpu_baseline": dict(cb, value=v),
               "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    out = run_native(args, rank, world, local_rank)
    if args.serve and not args.no_serve and rank == 0 and world == 1:
        out["serve"] = run_serving(args.serve, args.serve_steps)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = run_oracle_sample(args.workload)
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
