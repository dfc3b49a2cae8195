"""Continuous batching of IB-FE-IPCS simulations on one GPU.

Requests (a seeded vessel geometry, its grid and a number of time steps)
arrive on the wall clock.  A pool of setup threads builds each request's grid
(host side) and its device state snapshot as soon as it arrives, at most
`max_ready` of them ahead of admission.  The serving loop admits ready
requests while the device memory they would hold fits the budget (the batch
engine's footprint of every member plus the state snapshot that every built
request keeps), steps
all admitted requests together in one batch (one captured graph per step over
their concatenated bricks, reductions segmented per request), and between
epochs of a few steps lets finished requests leave and new ones join.  A
request's result is bitwise the same alone and in the mix.

The comparison path runs the same stream one request at a time, each on its own
standalone handle, in arrival order.
"""
from __future__ import annotations

import concurrent.futures as cf
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import IBBatch, IBGrid

# device bytes per stored node slot of a batch (fields, FP64 work, coefficients:
# FP64 planes on the FP64 path, compact FP32 pairs on the mixed path; in mixed
# precision the FP32 Krylov work; the multigrid levels and transfers), per Lagrangian row (in mixed precision with the force solve's
# FP64 product, FP32 work and FP32 Jacobi diagonal), per nonzero of A_F
# (column, FP64 value, FP32 copy if mixed), per entry of the coarsest
# multigrid level's dense inverse (in the Krylov precision), and per problem
# (solver states, reduction buffers, small tables)
BYTES_PER_SLOT = {"mixed": 560, "fp64": 660}
BYTES_PER_ROW = {"mixed": 1400 + 24 + 84 + 4, "fp64": 1400}
BYTES_PER_NNZ = {"mixed": 16, "fp64": 12}
BYTES_PER_CINV = {"mixed": 4, "fp64": 8}
BYTES_PER_PROBLEM = 1 << 20


@dataclass
class Request:
    rid: int
    arrival: float              # seconds after the start of the run
    case: dict
    steps: int
    handle: IBGrid = None
    cells: int = 0
    footprint: int = 0          # estimated bytes of the request inside a batch engine
    snap_bytes: int = 0         # device bytes of its state snapshot (held until it leaves)
    t_ready: float = 0.0
    t_admit: float = 0.0
    t_done: float = 0.0
    done_steps: int = 0
    status: int = 0


def footprint(info, precision):
    """Estimated device bytes of one problem inside a batch engine."""
    nc = int(info.get("mg_coarsest", 0)) if info.get("mg_levels", 0) else 0
    return int(info["n_slots"] * BYTES_PER_SLOT[precision]
               + ((info["n_points"] + 255) // 256 * 256) * BYTES_PER_ROW[precision]
               + BYTES_PER_NNZ[precision] * info["af_nnz"] + BYTES_PER_CINV[precision] * nc * nc
               + BYTES_PER_PROBLEM)


@dataclass
class ServeResult:
    latencies: list = field(default_factory=list)    # arrival -> result, seconds
    cell_steps: int = 0
    makespan: float = 0.0
    epochs: int = 0
    batch_sizes: list = field(default_factory=list)
    statuses: list = field(default_factory=list)
    footprint_scale: float = 1.0     # measured / estimated batch bytes (admission correction)

    def summary(self):
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "cell_steps_per_s": self.cell_steps / max(self.makespan, 1e-12), "makespan_s": self.makespan,
                "requests": len(self.latencies), "epochs": self.epochs,
                "mean_batch": float(np.mean(self.batch_sizes)) if self.batch_sizes else 0.0,
                "failed": int(sum(1 for s in self.statuses if s)), "footprint_scale": self.footprint_scale}


def serve(stream, precision="mixed", hbm_budget=150 * 2 ** 30, max_members=64, epoch_steps=10, setup_workers=4,
          keep=None, max_ready=None):
    """Run a request stream [(arrival_s, case)] through the continuous batcher.
    `keep(rid, handle)` may read a finished request's fields.

    Admission counts, against `hbm_budget`, the batch footprint of every
    member (footprint(), scaled up whenever a batch engine reports more device
    bytes than the estimate of its members) plus the device snapshot of every
    built request, admitted or waiting.  At most `max_ready` requests
    (default: max_members) are built ahead of admission, so the snapshots of
    waiting requests stay bounded."""
    reqs = [Request(k, float(a), c, int(c.get("steps", 200))) for k, (a, c) in enumerate(stream)]
    out = ServeResult()
    t0 = time.perf_counter()
    now = lambda: time.perf_counter() - t0
    slots = threading.BoundedSemaphore(max_ready or max_members)
    scale = [1.0]          # measured / estimated batch bytes, at least 1

    def setup(r):
        # wait for the arrival and for a free slot in the ready backlog, then
        # build the grid and the state snapshot
        dt = r.arrival - now()
        if dt > 0:
            time.sleep(dt)
        slots.acquire()
        r.handle = IBGrid(r.case, precision=precision, deferred=True)
        info = r.handle.ib_grid_info()
        r.cells = info["n_leaf_cells"]
        r.footprint = footprint(info, precision)
        r.snap_bytes = int(info.get("device_bytes", 0))
        r.t_ready = now()
        return r

    pool = cf.ThreadPoolExecutor(max_workers=setup_workers)
    futures = [pool.submit(setup, r) for r in reqs]
    pending = list(futures)
    ready, active, finished = [], [], 0
    batch = None
    members_key = None
    while finished < len(reqs):
        still = []
        for f in pending:
            if f.done():
                ready.append(f.result())
            else:
                still.append(f)
        pending = still
        ready.sort(key=lambda r: r.arrival)
        # every built request holds its snapshot; members add their batch share
        used = sum(r.snap_bytes for r in ready) + sum(r.snap_bytes + scale[0] * r.footprint for r in active)
        while ready and len(active) < max_members and used + scale[0] * ready[0].footprint <= hbm_budget:
            r = ready.pop(0)
            r.t_admit = now()
            active.append(r)
            used += scale[0] * r.footprint
            slots.release()
        if not active:
            if ready:    # a single request larger than the budget still runs alone
                r = ready.pop(0)
                r.t_admit = now()
                active.append(r)
                slots.release()
            else:
                time.sleep(0.002)
                continue
        key = tuple(r.rid for r in active)
        if key != members_key:
            if batch is not None:
                batch.close()
            batch = IBBatch([r.handle for r in active])
            members_key = key
            est = sum(r.footprint for r in active)
            measured = int(batch.info(0).get("device_bytes", 0))
            if est > 0 and measured > scale[0] * est:
                scale[0] = measured / est
        k = min(epoch_steps, min(r.steps - r.done_steps for r in active))
        st = batch.step(k)
        out.epochs += 1
        out.batch_sizes.append(len(active))
        leaving = []
        for r, s in zip(active, st):
            r.done_steps += k
            out.cell_steps += r.cells * k
            if s:
                r.status = int(s)
            if r.done_steps >= r.steps or r.status:
                r.t_done = now()
                leaving.append(r)
        if leaving:
            if keep is not None:
                for r in leaving:
                    keep(r.rid, r.handle)
            batch.close()
            batch = None
            members_key = None
            for r in leaving:
                active.remove(r)
                r.handle.close()
                r.handle = None
                out.latencies.append(r.t_done - r.arrival)
                out.statuses.append(r.status)
                finished += 1
    if batch is not None:
        batch.close()
    pool.shutdown(wait=True)
    out.makespan = now()
    out.footprint_scale = scale[0]
    return out


def serve_one_at_a_time(stream, precision="fp64", keep=None):
    """The comparison path: each request alone on a standalone handle, in
    arrival order, set up when it arrives (or when the previous one ends)."""
    out = ServeResult()
    t0 = time.perf_counter()
    now = lambda: time.perf_counter() - t0
    for rid, (arrival, case) in enumerate(stream):
        dt = arrival - now()
        if dt > 0:
            time.sleep(dt)
        g = IBGrid(case, precision=precision)
        cells = g.ib_grid_info()["n_leaf_cells"]
        steps = int(case.get("steps", 200))
        status = 0
        try:
            g.ipcs_step(steps)
        except Exception as e:       # a failed solve ends the request
            status = getattr(e, "status", -1)
        if keep is not None:
            keep(rid, g)
        g.close()
        out.latencies.append(now() - arrival)
        out.statuses.append(status)
        out.cell_steps += cells * steps
        out.epochs += 1
        out.batch_sizes.append(1)
    out.makespan = now()
    return out
