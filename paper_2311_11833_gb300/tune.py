"""Autotuner: picks the library options that run a given pattern fastest.

The options that change performance but not the result:

* the tiling of the persistent solve -- resident CTAs per SM (register
  budget 128 / 80 / 64 per thread), shifts per segment task of a narrow
  front (one task per shift, or one task for a group of shifts that pays
  the front's dependency wait and structure loads once) and the widest front
  one 32-lane segment takes before a whole CTA does;
* the supernode amalgamation (relax_small, relax_zeros: front sizes and
  tree height) and the factor policy (column-block owners per level, CTA
  clusters, tile DAG, per-panel launches, or the whole factorisation in one
  launch, at 2 or 3 resident CTAs per SM);
* the solve schedule (persistent or one launch per level).

For one sparsity pattern, shift count, RHS count, precision and sweep count,
`autotune` times candidates on the GPU with CUDA events over replays of the
step the library captures in a CUDA graph (factor + solve + sweeps), and
returns the fastest among those whose result stays accurate: the options
change only rounding, but with FP32 factors a different amalgamation can
leave the sweeps short of the FP64 result, so every candidate's x is compared
entry by entry with an FP64-factor solve with FP64 residual sweeps (default
options) of the same inputs and rejected beyond `tol` (max |x - ref| / max
|ref| per instance and right-hand side).  The sweeps matter for the
reference too: a pivot-free FP64 solve alone can be 2e-10 away from the
definition on an ill-conditioned instance of a batch.  With refine_tol > 0
the candidates and the reference run the adaptive sweeps of
pisp_set_refinement.  The default search is staged: first the solve tiling
with the default amalgamation and factor policy, then the amalgamation and
factor policy with the best tiling.  Results are cached in a JSON file (path
from $PISP_TUNE_CACHE, or the `cache` argument) keyed by a hash of the
pattern and the call shape.
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
# persistent solve tiling: (resident CTAs per SM, shifts per narrow task, widest warp front)
TILINGS = [(c, kf, wm) for c in (2, 3, 4) for kf, wm in ((1, 32), (1, 64), (2, 64), (2, 32))]
DEFAULT = dict(relax_small=8, relax_zeros=0.05, factor_policy=0, solve_schedule=0)


def candidates():
    """The full grid (amalgamation x factor policy x schedule), default tiling."""
    for (rs, rz), fp, sch in itertools.product(RELAX, POLICIES, SCHEDULES):
        yield dict(relax_small=rs, relax_zeros=rz, factor_policy=fp, solve_schedule=sch)


def _tiling(c, kf, wm):
    return dict(solve_ctas_per_sm=c, solve_kfuse=kf, solve_warp_maxF=wm)


def staged_candidates():
    """Stage 1: every solve tiling with the default analysis; stage 2 is built
    from stage 1's winner by `autotune`."""
    return [dict(DEFAULT, **_tiling(*t)) for t in TILINGS]


def _stage2(best: dict):
    """Amalgamation x factor policy (per-level owners, tile DAG, one launch),
    plus the one launch at 3 resident CTAs per SM with shared-memory fronts up
    to 128 wide (so that three CTAs fit)."""
    out = []
    for (rs, rz), fp in itertools.product(RELAX, (0, 2, 4)):
        o = dict(best, relax_small=rs, relax_zeros=rz, factor_policy=fp)
        if o != best:
            out.append(o)
    for rs, rz in RELAX:
        o = dict(best, relax_small=rs, relax_zeros=rz, factor_policy=4, factor_ctas_per_sm=3, factor_smem_maxF=128)
        if o != best:
            out.append(o)
    return out


def _key(sizes, row_ptr, col, K, R, precision, sweeps, refine_tol=0.0) -> str:
    h = hashlib.sha256()
    for a in (np.asarray(sizes, np.int64), np.asarray(row_ptr, np.int64), np.asarray(col, np.int32)):
        h.update(np.ascontiguousarray(a).tobytes())
    return f"{h.hexdigest()[:24]}-K{K}-R{R}-{precision}-s{sweeps}-a{refine_tol:g}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _entrywise(x, ref, inst) -> float:
    """max over instances g and right-hand sides r of max_{i in g} |x_ir - ref_ir| /
    max_{i in g} |ref_ir| (on the device; inst = the instance of each row)."""
    import torch
    G = int(inst[-1]) + 1 if inst.numel() else 0
    idx = inst[:, None].expand_as(ref)
    z = torch.zeros(G, ref.shape[1], dtype=ref.dtype, device=ref.device)
    scale = z.scatter_reduce(0, idx, ref.abs(), "amax").clamp_min(torch.finfo(ref.dtype).tiny)
    diff = z.scatter_reduce(0, idx, (x - ref).abs(), "amax")
    err = (diff / scale).max()
    return float(err) if torch.isfinite(err) else float("inf")


def _time(Solver, sizes, row_ptr, col, values, D, t, b, x, precision, sweeps, reps, opts, ref=None, inst=None,
          refine_tol=0.0):
    import torch
    s = Solver(sizes, row_ptr, col, **opts)
    try:
        s.set_refinement(refine_tol)
        s.graph_capture(values, D, t, b, x, precision=precision, sweeps=sweeps)
        for _ in range(2):
            s.graph_launch()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(reps):
            s.graph_launch()
        ev[1].record()
        ev[1].synchronize()
        err = _entrywise(x, ref, inst) if ref is not None else None
        return ev[0].elapsed_time(ev[1]) / reps, err
    finally:
        s.close()


def autotune(sizes, row_ptr, col, values, D, t, b, precision="fp32", sweeps=2, reps=5,
             cache: str | None = None, options=None, tol: float = 5e-11, refine_tol: float = 0.0) -> dict:
    """Fastest options for this pattern / call shape: {"options": {...}, "ms": ..., "all": [...]}.

    options: an explicit candidate list (timed as given); default: the staged
    search over the solve tiling, then the amalgamation and factor policy.
    refine_tol > 0: the candidates run adaptive sweeps (pisp_set_refinement)
    with at most `sweeps` sweeps.  tol bounds the entry-wise difference, per
    instance, from the reference."""
    import torch

    from .solver import Solver

    cache = cache or os.environ.get("PISP_TUNE_CACHE")
    R = b.shape[1] if b.dim() == 2 else 1
    key = _key(sizes, row_ptr, col, len(t), R, precision, sweeps, refine_tol)
    if cache:
        hit = _load(cache).get(key)
        if hit:
            return hit
    b2 = b.reshape(b.shape[0], -1).contiguous()
    x = torch.empty_like(b2)
    inst = torch.repeat_interleave(torch.arange(len(sizes), device=b2.device),
                                   torch.as_tensor(np.asarray(sizes, np.int64), device=b2.device))
    # the accuracy reference: FP64 factors, default options, FP64 sweeps (two
    # fixed, or adaptive up to four and to a tolerance no looser than 1e-12,
    # so that the reference sits at the FP64 floor whatever the candidates'
    # stopping tolerance)
    sref = Solver(sizes, row_ptr, col)
    try:
        sref.set_refinement(min(refine_tol, 1e-12) if refine_tol > 0 else 0.0)
        sref.factor(values, D, t, "fp64")
        ref = sref.solve(b2, sweeps=4 if refine_tol > 0 else 2).clone()
    finally:
        sref.close()
    results = []

    def run(cands):
        for opts in cands:
            ms, err = _time(Solver, sizes, row_ptr, col, values, D, t, b2, x, precision, sweeps, reps, opts, ref,
                            inst, refine_tol)
            results.append({"options": opts, "ms": ms, "err": err, "ok": bool(err <= tol)})

    def fastest():
        ok = [r for r in results if r["ok"]]
        return min(ok or results, key=lambda r: (r["ms"] if r["ok"] else float("inf"), r["err"]))

    if options is not None:
        run(options)
    else:
        run(staged_candidates())
        run(_stage2(fastest()["options"]))
    best = fastest()
    out = {"options": best["options"], "ms": best["ms"], "err": best["err"], "tol": tol,
           "rejected": sum(1 for r in results if not r["ok"]), "all": results}
    if cache:
        data = _load(cache)
        data[key] = out
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1)
        os.replace(tmp, cache)
    return out
