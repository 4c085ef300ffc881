"""Autotuner: picks the library options that run a given pattern fastest.

The options that change performance but not the result are the supernode
amalgamation (relax_small, relax_zeros: front sizes and tree height), the
factor policy of wide fronts (column-block owners, CTA clusters, tile DAG or
per-panel launches) and the solve schedule (persistent or one launch per level).  For
one sparsity pattern, shift count, RHS count and precision, `autotune` times
every candidate on the GPU with CUDA events (factor + solve, a few
repetitions after a warm-up) and returns the fastest.  Results are cached in
a JSON file (path from $PISP_TUNE_CACHE, or the `cache` argument) keyed by a
hash of the pattern and the call shape.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os

import numpy as np

RELAX = [(8, 0.05), (4, 0.0), (16, 0.10), (32, 0.20)]
POLICIES = [0, 1, 2, 3]
SCHEDULES = [0, 1]


def candidates():
    for (rs, rz), fp, sch in itertools.product(RELAX, POLICIES, SCHEDULES):
        yield dict(relax_small=rs, relax_zeros=rz, factor_policy=fp, solve_schedule=sch)


def _key(sizes, row_ptr, col, K, R, precision, sweeps) -> str:
    h = hashlib.sha256()
    for a in (np.asarray(sizes, np.int64), np.asarray(row_ptr, np.int64), np.asarray(col, np.int32)):
        h.update(np.ascontiguousarray(a).tobytes())
    return f"{h.hexdigest()[:24]}-K{K}-R{R}-{precision}-s{sweeps}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def autotune(sizes, row_ptr, col, values, D, t, b, precision="fp32", sweeps=2, reps=5,
             cache: str | None = None, options=None) -> dict:
    """Fastest options for this pattern / call shape: {"options": {...}, "ms": ..., "all": [...]}."""
    import torch

    from .solver import Solver

    cache = cache or os.environ.get("PISP_TUNE_CACHE")
    R = b.shape[1] if b.dim() == 2 else 1
    key = _key(sizes, row_ptr, col, len(t), R, precision, sweeps)
    if cache:
        hit = _load(cache).get(key)
        if hit:
            return hit
    results = []
    x = torch.empty_like(b)
    for opts in (options or list(candidates())):
        s = Solver(sizes, row_ptr, col, **opts)
        for _ in range(2):
            s.factor(values, D, t, precision)
            s.solve(b, sweeps=sweeps, out=x)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(reps):
            s.factor(values, D, t, precision)
            s.solve(b, sweeps=sweeps, out=x)
        ev[1].record()
        ev[1].synchronize()
        results.append({"options": opts, "ms": ev[0].elapsed_time(ev[1]) / reps})
        s.close()
    best = min(results, key=lambda r: r["ms"])
    out = {"options": best["options"], "ms": best["ms"], "all": results}
    if cache:
        data = _load(cache)
        data[key] = out
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1)
        os.replace(tmp, cache)
    return out
