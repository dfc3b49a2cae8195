"""Autotuner of the library's launch choices (ib_grid_desc.tune).

The choices change speed, not the method: the Poisson stencil kernel (staged
asynchronously or register-pipelined), the bricks per CTA of the streaming
Krylov kernels, the size below which multigrid levels run in one CTA per
problem, and the damped-Jacobi sweeps of the V-cycle (a symmetric
preconditioner for any sweep count, so the solution is the same to the
solver tolerance; the iteration count and the time per step change).

A workload class is keyed by precision, refinement depth and the order of
magnitude of its storage (log2 of the node slots): problems of one class
share the best choice.  tune_case() times each candidate on the problem
itself (captured step graphs, L2 flushed between steps, CUDA events) and
keeps the fastest; TuneCache stores the choice per class in a JSON file, so
a serving loop or a benchmark tunes a class once.
"""
from __future__ import annotations

import json
import math
import os

DEFAULTS = {"poisson_kernel": 1, "stream_chunk": 8, "mg_small": 8192, "mg_sweeps": 2, "mg_persist": 1}

# candidates, each a set of overrides of the defaults; the first is the default
CANDIDATES = [
    {},
    {"poisson_kernel": 2},
    {"poisson_kernel": 3},
    {"stream_chunk": 4},
    {"mg_small": 2048},
    {"mg_small": 32768},
    {"mg_sweeps": 1},
    {"mg_sweeps": 3},
    {"mg_persist": 2},
]


def class_key(info, precision, max_level):
    """Workload class of a problem: precision, levels, log2 of its slots."""
    return f"{precision}:L{int(max_level)}:s{int(round(math.log2(max(int(info['n_slots']), 1))))}"


def choose(timings):
    """The fastest candidate of [(overrides, ms_per_step)]; ties keep the
    earlier candidate.  Returns the full choice (defaults plus overrides)."""
    best = None
    for over, ms in timings:
        if ms is None or not math.isfinite(ms):
            continue
        if best is None or ms < best[1]:
            best = (over, ms)
    if best is None:
        raise ValueError("no candidate ran")
    return dict(DEFAULTS, **best[0]), best[1]


class TuneCache:
    """Choices per workload class, kept in a JSON file."""

    def __init__(self, path=None):
        self.path = path
        self.table = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.table = json.load(f)

    def get(self, key):
        e = self.table.get(key)
        return dict(e["choice"]) if e else None

    def put(self, key, choice, ms, timings):
        self.table[key] = {"choice": dict(choice), "ms_per_step": float(ms),
                           "candidates": [{"overrides": o, "ms_per_step": t} for o, t in timings]}
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.table, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def time_candidate(case, precision, overrides, steps=3, warmup=2, device=0, poisson_pc="multigrid"):
    """ms per step of the captured step graph under the given launch choices."""
    import torch
    from . import IBGrid
    g = IBGrid(case, precision=precision, device=device, poisson_pc=poisson_pc, tune=overrides)
    try:
        stream = torch.cuda.current_stream()
        flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=f"cuda:{device}")
        for _ in range(warmup):
            g.ipcs_step(1)
        ms = 0.0
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.ipcs_step(1)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        return ms / steps
    finally:
        g.close()


def tune_case(case, precision="mixed", cache=None, candidates=None, steps=3, warmup=2, device=0, timer=None):
    """Best launch choices for the class of `case`: from the cache when the
    class is known, else by timing every candidate on the case.  `timer`
    replaces the GPU timing (overrides -> ms per step).  Returns (choice,
    key, from_cache, timings)."""
    from . import IBGrid
    probe = IBGrid(case, precision=precision, device=device, deferred=True)
    key = class_key(probe.ib_grid_info(), precision, case["max_level"])
    probe.close()
    if cache is not None:
        hit = cache.get(key)
        if hit is not None:
            return hit, key, True, []
    cands = CANDIDATES if candidates is None else candidates
    run = timer or (lambda over: time_candidate(case, precision, over, steps=steps, warmup=warmup, device=device))
    timings = [(over, run(over)) for over in cands]
    choice, ms = choose(timings)
    if cache is not None:
        cache.put(key, choice, ms, timings)
    return choice, key, False, timings
