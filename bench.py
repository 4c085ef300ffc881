#!/usr/bin/env python
"""Throughput benchmark: combined solves/s of perturbation-induced static pivoting.

A step is one pass of the whole hot path over one batch of synthetic
power-flow Jacobians already resident in HBM: perturb + pivot-free factor of
all K shifted matrices, forward/backward solves of R right-hand sides, FP64
residual sweeps (FP32 factors) and the expansion-weighted FP64 combine, as
one replay of the CUDA graph the library captured (pisp_graph_capture).  The
metric counts combined solutions x_hat (instances x RHS) per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...    # the CPU oracle on bounded samples
  python bench.py --study dense|newton    # timing tables of next rows f4 / f2

Workloads (pfgen.CONFIGS): batching (default: 256 grids of 118-3000 buses,
K = 4, R = 8, FP32 factors + FP64 sweeps/combine), plain, precision,
differentiation, scale.  Under torchrun every rank solves its own independent
replica of the workload (weak scaling, no collective on the data path); rank
0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import pfgen  # noqa: E402

METRIC = "combined solves/s (K perturbed LUs + expansion) vs plain GPU path at rel err <=1e-10"
UNIT = "solves/s"
TOL = 1e-10
L2_BYTES = 129 * 1024 * 1024
# dram__bytes_read.sum + dram__bytes_write.sum per launch of a kernel family
# on a workload, from an ncu capture of that kernel on that workload (scaled
# to the full workload where the capture ran a reduced batch); an entry is
# removed when its kernel changes.
# Keys: (workload, family, instances, library options as sorted (name, value) pairs).
BATCH_TUNED = (("factor_ctas_per_sm", 3), ("factor_policy", 4), ("factor_smem_maxF", 128), ("relax_small", 16),
               ("relax_zeros", 0.1), ("solve_ctas_per_sm", 4), ("solve_kfuse", 1), ("solve_schedule", 0),
               ("solve_warp_maxF", 64))
TRAFFIC_PER_LAUNCH = {
    ("batching", "backward", 256, BATCH_TUNED): 670.31e6,            # 586.72 MB read + 83.59 MB written
    ("batching", "factor_persistent", 256, BATCH_TUNED): 1378.02e6,  # 619.55 MB read + 758.47 MB written
}

# factor precision and FP64 residual sweeps per workload; refine_tol > 0:
# adaptive sweeps (pisp_set_refinement), `sweeps` is then the maximum
BENCH = {
    "plain": dict(precision="fp64", sweeps=0, refine_tol=0.0),
    "precision": dict(precision="fp32", sweeps=8, refine_tol=1e-12),
    "batching": dict(precision="fp32", sweeps=8, refine_tol=1e-12),
    "differentiation": dict(precision="fp64", sweeps=0, refine_tol=0.0),
    "scale": dict(precision="fp32", sweeps=8, refine_tol=1e-12),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="pisp", choices=["pisp", "reference"])
    ap.add_argument("--workload", default="batching", choices=list(pfgen.CONFIGS))
    ap.add_argument("--instances", type=int, default=None,
                    help="batching only: the first G grids of the 256 (reduced batches for profiler captures)")
    ap.add_argument("--study", default=None, choices=["dense", "newton"],
                    help="timing study of next row f4 (dense batches vs n and G) or f2 (Newton loop)")
    ap.add_argument("--precision", default=None, choices=["fp32", "fp64"])
    ap.add_argument("--sweeps", type=int, default=None,
                    help="FP64 residual sweeps (with adaptive sweeps: the maximum)")
    ap.add_argument("--refine-tol", type=float, default=None,
                    help="stopping tolerance of the adaptive sweeps (0: fixed sweeps; default per workload)")
    ap.add_argument("--eps", type=float, default=1e-2)
    ap.add_argument("--no-graph", action="store_true", help="launch eagerly instead of a CUDA graph")
    ap.add_argument("--factor-policy", type=int, default=0, choices=[0, 1, 2, 3, 4],
                    help="fronts wider than 64: 0 single CTA / column-block owners (default), "
                         "1 CTA clusters, 2 single CTA / tile DAG, 3 single CTA / per-panel launches, "
                         "4 one persistent launch for the whole factorisation")
    ap.add_argument("--schedule", type=int, default=0, choices=[0, 1],
                    help="solve schedule: 0 persistent (default), 1 one launch per level")
    ap.add_argument("--kfuse", type=int, default=0, help="persistent solve: shifts per narrow-front task")
    ap.add_argument("--warp-maxf", type=int, default=0,
                    help="persistent solve: widest front with <= 32 pivots solved by one warp")
    ap.add_argument("--ctas", type=int, default=0, help="persistent solve: resident CTAs per SM (2, 3, 4)")
    ap.add_argument("--relax-small", type=int, default=-1, help="supernode amalgamation: pivot block size")
    ap.add_argument("--relax-zeros", type=float, default=-1.0, help="supernode amalgamation: zero fraction")
    ap.add_argument("--factor-tc", type=int, default=0, help="1: FP32 owner-tile updates on the tensor cores")
    ap.add_argument("--factor-ctas", type=int, default=0, help="one-launch factorisation: resident CTAs per SM")
    ap.add_argument("--factor-smem-maxf", type=int, default=0,
                    help="one-launch factorisation: widest front kept in one CTA's shared memory")
    ap.add_argument("--autotune", default="auto", choices=["auto", "on", "off"],
                    help="time candidate library options on this workload first and use the fastest "
                         "(auto: on for the batching workload)")
    ap.add_argument("--quick", action="store_true",
                    help="timed arm only (no plain-FP64 arm, e2e, CPU baseline or oracle check)")
    return ap.parse_args()


# ----------------------------------------------------------------- inputs --
def workload_instances(name: str, rank: int, G: int | None = None):
    c = pfgen.CONFIGS[name]
    if name == "batching":
        sizes = pfgen.batch_sizes(c["G"])
        G = c["G"] if G is None else max(1, min(int(G), c["G"]))
        insts = [pfgen.grid_jacobian(int(sizes[g]), None, 1000 * c["index"] + g + 100_000 * rank)
                 for g in range(G)]
    else:
        insts = [pfgen.grid_jacobian(c["N"], c.get("n_pv"), 1000 * c["index"] + 100_000 * rank)]
    return insts


def concat(insts):
    rp, cols, vals, off = [0], [], [], 0
    for I in insts:
        rp.extend((I.row_ptr[1:] + rp[-1]).tolist())
        cols.append(I.col + off)
        vals.append(I.val)
        off += I.n
    return ([I.n for I in insts], np.array(rp, np.int64), np.concatenate(cols).astype(np.int32),
            np.concatenate(vals), np.concatenate([I.D for I in insts]))


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------- clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if "Active" in v and "Not" not in v:
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- GPU arms --
class Arm:
    """One configured solver with device-resident inputs and a step function."""

    def __init__(self, pisp, torch, insts, K, R, eps, precision, sweeps, workload, dev, schedule=0,
                 factor_policy=0, options=None, extra=None, refine_tol=0.0):
        self.torch = torch
        self.insts = insts
        sizes, rp, col, val, D = concat(insts)
        t0 = time.perf_counter()
        opts = options or dict(solve_schedule=schedule, factor_policy=factor_policy)
        opts = dict(opts, **(extra or {}))
        self.options = opts
        self.s = pisp.Solver(sizes, rp, col, device=dev.index, **opts)
        self.analyze_ms = (time.perf_counter() - t0) * 1e3
        self.refine_tol = refine_tol
        self.s.set_refinement(refine_tol)
        self.N = sum(sizes)
        self.K, self.R, self.precision, self.sweeps = K, R, precision, sweeps
        self.t = pfgen.symmetric_shifts(K, eps)
        self.vals = torch.tensor(val, device=dev)
        self.D = torch.tensor(D, device=dev)
        self.b_host = pfgen.rhs(self.N, R, 1)
        self.b = torch.tensor(self.b_host, device=dev)
        self.x = torch.empty_like(self.b)
        self.adjoint = workload == "differentiation"
        if self.adjoint:
            self.g = torch.tensor(pfgen.rhs(self.N, R, 2), device=dev)
            self.gb = torch.empty_like(self.b)
            self.gv = torch.empty_like(self.vals)
        self.graph = False

    def step(self):
        s = self.s
        s.factor(self.vals, self.D, self.t, self.precision)
        s.solve(self.b, sweeps=self.sweeps, out=self.x)
        if self.adjoint:
            s.adjoint(self.g, out_b=self.gb, out_values=self.gv, sweeps=self.sweeps)

    def capture(self, profile: bool):
        """The whole step captured by the library (pisp_graph_capture); with
        profile, the per-family event brackets are recorded into the graph."""
        if profile:
            self.s.profile(True)
        kw = dict(g=self.g, out_b=self.gb, out_values=self.gv, adjoint_sweeps=self.sweeps) if self.adjoint else {}
        self.s.graph_capture(self.vals, self.D, self.t, self.b, self.x, precision=self.precision,
                             sweeps=self.sweeps, **kw)
        if profile:
            self.s.profile(False)
        self.torch.cuda.synchronize()
        self.graph = True

    def run(self):
        if self.graph:
            self.s.graph_launch()
        else:
            self.step()


def _entrywise(x, ref):
    """Per right-hand side: max_i |x_ir - ref_ir| / max_i |ref_ir|."""
    scale = np.abs(ref).max(axis=0)
    scale = np.where(scale > 0, scale, 1.0)
    return np.max(np.abs(x - ref), axis=0) / scale


THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _oracle_job(job):
    """One instance's x_hat by the CPU oracle (also run in spawned workers)."""
    import oracle
    inst, t, b = job
    return oracle.x_hat(oracle.to_scipy(inst), inst.D, t, b)


def oracle_refs(insts, t, b_host):
    """The oracle's x_hat of every instance: in this process for a single
    instance (BLAS threads = host cores), else in a pool of spawned processes
    with one BLAS thread each, largest instances first."""
    offs = np.concatenate([[0], np.cumsum([I.n for I in insts])])
    jobs = [(I, t, b_host[offs[g]:offs[g + 1]]) for g, I in enumerate(insts)]
    if len(jobs) == 1:
        return [_oracle_job(jobs[0])]
    import multiprocessing as mp
    order = sorted(range(len(jobs)), key=lambda g: -insts[g].n)
    saved = {k: os.environ.get(k) for k in THREAD_VARS}
    os.environ.update({k: "1" for k in THREAD_VARS})
    try:
        with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
            res = pool.map(_oracle_job, [jobs[g] for g in order], chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    out = [None] * len(jobs)
    for g, r in zip(order, res):
        out[g] = r
    return out


def oracle_check(arm, refs, xs=None, detail=12):
    """Error of x against the CPU oracle for every right-hand side of EVERY
    instance: entry-wise (max |x - ref| / max |ref| per instance and RHS) and
    normwise.  refs: oracle_refs of the arm's inputs; xs: the solution to
    check ([N][R], default arm.x).  Per-instance figures are listed for at
    most `detail` instances (else the five worst)."""
    import oracle
    x = arm.x.cpu().numpy() if xs is None else xs
    offs = np.concatenate([[0], np.cumsum([I.n for I in arm.insts])])
    per = []
    for g, I in enumerate(arm.insts):
        sl = slice(offs[g], offs[g + 1])
        ew = _entrywise(x[sl], refs[g])
        nw = oracle.rel_err(x[sl], refs[g])
        per.append({"instance": g, "n": I.n, "entrywise": [float(f"{v:.3e}") for v in ew],
                    "normwise": [float(f"{v:.3e}") for v in nw]})
    mx = max(max(p["entrywise"]) for p in per)
    out = {"tol": TOL, "instances": len(per), "results": sum(len(p["entrywise"]) for p in per),
           "max_entrywise": mx, "max_normwise": max(max(p["normwise"]) for p in per),
           "all_within_tol": bool(mx <= TOL)}
    if len(per) <= detail:
        out["per_instance"] = per
    else:
        worst = sorted(per, key=lambda p: -max(p["entrywise"]))[:5]
        out["worst_instances"] = [{"instance": p["instance"], "n": p["n"], "entrywise": max(p["entrywise"])}
                                  for p in worst]
    return out


def cpu_baseline(insts, K, R, eps, budget_s=12.0):
    """The oracle, as it stands, on a bounded sample of the workload (about budget_s of CPU work)."""
    import oracle
    t = pfgen.symmetric_shifts(K, eps)
    done_units, elapsed, calls = 0.0, 0.0, 0
    g = 0
    t0 = time.perf_counter()
    while elapsed < budget_s:
        I = insts[g % len(insts)]
        A = oracle.to_scipy(I)
        b = pfgen.rhs(I.n, R, 1)
        oracle.x_hat(A, I.D, t, b)
        done_units += R
        calls += K
        g += 1
        elapsed = time.perf_counter() - t0
    return {"value": done_units / elapsed, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{g} combined solve(s) of {R} RHS (K = {K} perturbed GEPP solves + combine each), "
                      f"{elapsed:.1f} s of CPU work (numpy/LAPACK, BLAS threads = host cores)"}


def min_bytes_per_launch(fam, st, K, R, p):
    """Minimum data one launch of a kernel family must move (the algorithmic
    bytes of the roofline): factor entries of the triangle it uses for all K
    shifts, their int32 indices read ONCE for all K, the vectors in and out.
    nnzU = (nnzF + N) / 2 entries of U (diagonal included), nnzL = (nnzF - N) / 2
    entries strictly below it.  The one-launch factorisation moves at least
    A's values, D, the factor pattern (once for all K) and the K factors; the
    Schur complements a multifrontal factorisation writes and reads back are
    not counted.  None for the per-level factor families (several launches
    per step, each over part of the fronts: the library's per-launch count is
    used there)."""
    N, nnzA, nnzF = float(st["N"]), float(st["nnzA"]), float(st["nnzF_stored"])
    nnzU, nnzL = (nnzF + N) / 2, (nnzF - N) / 2
    if fam == "factor_persistent":
        return 8 * nnzA + 8 * N + 4 * (nnzF + N) + K * p * nnzF
    if fam == "backward":       # U factors, indices, y in (factor precision), x out (FP64)
        return K * p * nnzU + 4 * nnzU + K * p * N * R + 8 * N * R
    if fam == "forward":        # L factors, indices, b in (FP64), y out (factor precision)
        return K * p * nnzL + 4 * nnzL + 8 * N * R + K * p * N * R
    if fam == "residual":       # A values + columns, b, the K solutions in, K residuals out
        return 12 * nnzA + 8 * N * R + 16 * N * K * R
    if fam == "combine":        # K solutions in, x out
        return 8 * N * K * R + 8 * N * R
    return None


def run_pisp(args, rank, world, local_rank):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2311_11833_gb300 as pisp

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    c = pfgen.CONFIGS[args.workload]
    bcfg = BENCH[args.workload]
    precision = args.precision or bcfg["precision"]
    sweeps = bcfg["sweeps"] if args.sweeps is None else args.sweeps
    refine_tol = bcfg["refine_tol"] if args.refine_tol is None else args.refine_tol
    if precision == "fp64" and args.sweeps is None:
        sweeps = 0
    K, R = c["K"], c["R"]
    insts = workload_instances(args.workload, rank, args.instances)
    tuned = None
    if args.autotune == "on" or (args.autotune == "auto" and args.workload == "batching"):
        from paper_2311_11833_gb300 import tune
        sizes, rp, col, val, D = concat(insts)
        tuned = tune.autotune(sizes, rp, col, torch.tensor(val, device=dev), torch.tensor(D, device=dev),
                              pfgen.symmetric_shifts(K, args.eps),
                              torch.tensor(pfgen.rhs(sum(sizes), R, 1), device=dev), precision, sweeps,
                              refine_tol=refine_tol)
    extra = {k: v for k, v in (("solve_kfuse", args.kfuse), ("solve_warp_maxF", args.warp_maxf),
                               ("solve_ctas_per_sm", args.ctas), ("factor_tc", args.factor_tc),
                               ("factor_ctas_per_sm", args.factor_ctas),
                               ("factor_smem_maxF", args.factor_smem_maxf)) if v}
    if args.relax_small >= 0:
        extra["relax_small"] = args.relax_small
    if args.relax_zeros >= 0:
        extra["relax_zeros"] = args.relax_zeros
    arm = Arm(pisp, torch, insts, K, R, args.eps, precision, sweeps, args.workload, dev, args.schedule,
              args.factor_policy, options=tuned["options"] if tuned else None, extra=extra, refine_tol=refine_tol)
    G = len(insts)
    units = G * R
    use_graph = not args.no_graph
    for _ in range(args.warmup):
        arm.step()
    torch.cuda.synchronize()
    if use_graph:
        arm.capture(profile=True)
        for _ in range(max(3, args.warmup)):
            arm.run()
    torch.cuda.synchronize()
    arm.s.profile_reset()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank) if rank == 0 else None
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))                      # evict L2 between steps (outside the events)
        if not use_graph:
            arm.s.profile(True)                    # fresh bracket list for this eager step
        ev[i][0].record()
        arm.run()
        ev[i][1].record()
        ev[i][1].synchronize()
        arm.s.profile_collect()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk = clocks.stop() if clocks else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if dist:
        tt = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
        total_ms = float(tt.item())
        tdist.barrier()
    value = units * world * args.steps / (total_ms / 1e3)
    prof = arm.s.profile_read()
    stats = arm.s.stats()
    # adaptive sweeps run as one device-side loop (family sweep_loop, not a
    # kernel); forward and backward then hold the first solve only, whose
    # launches cover every instance
    nsw, _ = arm.s.refinement_stats(sweeps)

    def full_launches_per_step(f):
        return prof[f]["launches"] / args.steps
    if not use_graph:
        arm.s.profile(False)
    if rank != 0:
        return None
    # roofline of the dominant kernel family: minimum bytes per launch over the
    # family's average launch time (CUDA events on the library's stream)
    peak, peak_kind = load_peaks()
    fam = max((f for f in prof if f != "sweep_loop"), key=lambda f: prof[f]["ms"])  # a kernel, not the loop
    pf = prof[fam]
    p = 4 if precision == "fp32" else 8
    fl = full_launches_per_step(fam) * args.steps
    launch_ms = pf["ms"] / max(1e-9, fl)
    lib_bytes = pf["bytes"] / max(1e-9, fl)
    mb = min_bytes_per_launch(fam, stats, K, R, p)
    alg = mb if mb is not None else lib_bytes
    achieved = alg / (launch_ms / 1e3) / 1e9 if launch_ms > 0 else 0.0
    opts_key = tuple(sorted(arm.options.items()))
    traffic = TRAFFIC_PER_LAUNCH.get((args.workload, fam, G, opts_key))
    roofline = {"bound": "hbm", "kernel": fam, "achieved": round(achieved, 2), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 5), "peak_source": peak_kind,
                "traffic": traffic, "algorithmic_bytes_per_launch": alg,
                "algorithmic_bytes_rule": "minimum (indices once for all K)" if mb is not None
                else "library count",
                "library_bytes_per_launch": lib_bytes,
                "avg_launch_us": round(1e3 * launch_ms, 3),
                "share_of_step": round(pf["ms"] / total_ms, 4) if world == 1 else None}

    def fam_roofline(f):
        v = prof[f]
        if v["launches"] == 0 or v["ms"] <= 0:
            return None
        lm = v["ms"] / (full_launches_per_step(f) * args.steps)
        mbf = min_bytes_per_launch(f, stats, K, R, p)
        by = mbf if mbf is not None else v["bytes"] / (full_launches_per_step(f) * args.steps)
        ach = by / (lm / 1e3) / 1e9
        return {"kernel": f, "achieved": round(ach, 2), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 5),
                "algorithmic_bytes_per_launch": by, "avg_launch_us": round(1e3 * lm, 3),
                "traffic": TRAFFIC_PER_LAUNCH.get((args.workload, f, G, opts_key))}

    def fam_summary(f, v):
        fl = full_launches_per_step(f)
        mbf = min_bytes_per_launch(f, stats, K, R, p)
        return {"ms_per_step": round(v["ms"] / args.steps, 4),
                "launches_per_step": v["launches"] / args.steps,
                "min_GBps": (round(mbf * fl / (v["ms"] / args.steps / 1e3) / 1e9, 2)
                             if v["ms"] > 0 and mbf is not None else None),
                "library_GBps": round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 2) if v["ms"] > 0 else 0.0}
    families = {f: fam_summary(f, v) for f, v in prof.items() if v["launches"] > 0}
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if precision == "fp32" else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "instances": G, "N": arm.N, "nnzA": int(stats["nnzA"]),
                   "K": K, "R": R, "shifts": "symmetric +-eps*alpha", "eps": args.eps,
                   "factor_precision": precision, "combine_precision": "fp64", "sweeps": sweeps,
                   "sweeps_mode": (f"adaptive per instance, at most {sweeps}, stop tol {refine_tol:g}"
                                   if refine_tol > 0 and sweeps else "fixed"),
                   "graph": "library (pisp_graph_capture)" if use_graph else None,
                   "solve_schedule": ["persistent", "per-level"][args.schedule],
                   "factor_policy": ["single-CTA/column-block-owners", "clusters", "single-CTA/tile-DAG",
                                     "single-CTA/per-panel", "one-launch-persistent"][
                       (tuned["options"].get("factor_policy", 0) if tuned else args.factor_policy)], "l2": "flushed between steps (256 MB write outside the events)",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "roofline_backward": fam_roofline("backward"),
        "families": families,
        "gpu_launches": int(stats["gpu_launches"]) * args.steps,
        "analyze_ms": round(arm.analyze_ms, 2),
        "autotune": ({"options": tuned["options"], "candidates": len(tuned["all"]),
                      "rejected_for_accuracy": tuned.get("rejected"), "tol": tuned.get("tol"),
                      "best_err_vs_fp64_factor_solve": tuned.get("err"),
                      "best_ms": round(tuned["ms"], 4),
                      "default_ms": round(next((r["ms"] for r in tuned["all"] if r["options"] == dict(
                          relax_small=8, relax_zeros=0.05, factor_policy=0, solve_schedule=0,
                          solve_ctas_per_sm=3 if precision == "fp32" else 2, solve_kfuse=1, solve_warp_maxF=32)),
                                            float("nan")), 4),
                      "search": "staged: solve tiling (CTAs/SM x shifts per task x widest warp front), "
                                "then amalgamation x factor policy; graph replays, CUDA events"}
                     if tuned else None),
        "sweeps_per_instance": {str(k): int(v) for k, v in zip(*np.unique(nsw, return_counts=True))},
        "wall_s_timed_region": round(wall, 3),
        "structure": {k: stats[k] for k in ("nnzL", "nnzF_stored", "n_supernodes", "n_levels",
                                            "max_front", "etree_height")},
    }
    if clk:
        out["clocks"] = clk
    if not args.quick:
        t_or = time.perf_counter()
        refs = oracle_refs(insts, arm.t, arm.b_host)
        chk = oracle_check(arm, refs)
        chk["oracle_wall_s"] = round(time.perf_counter() - t_or, 2)
        out["oracle_check"] = chk
        out["max_rel_err_vs_oracle"] = chk["max_entrywise"]
        # plain FP64 single-instance path: FP64 factors, no sweeps, instances
        # one after another, eager launches, no graph
        plain_ms = []
        arms = [Arm(pisp, torch, [I], K, R, args.eps, "fp64", 0, args.workload, dev) for I in insts]
        offs = np.concatenate([[0], np.cumsum([I.n for I in insts])])
        for g, a in enumerate(arms):  # the same right-hand sides as the batched arm
            a.b_host = arm.b_host[offs[g]:offs[g + 1]].copy()
            a.b = torch.tensor(a.b_host, device=dev)
            a.x = torch.empty_like(a.b)
        n_plain_steps = 5 if G > 1 else min(args.steps, 20)
        for a in arms:
            a.step()
        torch.cuda.synchronize()
        for i in range(n_plain_steps):
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for a in arms:
                a.step()
            e1.record()
            e1.synchronize()
            plain_ms.append(e0.elapsed_time(e1))
        # the plain path's x on every instance
        xp = np.zeros_like(arm.b_host)
        for g in range(G):
            xp[offs[g]:offs[g + 1]] = arms[g].x.cpu().numpy()
        plain_chk = oracle_check(arm, refs, xs=xp)
        plain_err = plain_chk["max_entrywise"]
        pv = units / (statistics.mean(plain_ms) / 1e3)
        out["plain_fp64_path"] = {"value": round(pv, 2), "ms_per_step": round(statistics.mean(plain_ms), 4),
                                  "steps": n_plain_steps, "max_rel_err_vs_oracle": plain_err,
                                  "results_checked": plain_chk["results"],
                                  "within_tol": plain_chk["all_within_tol"],
                                  "speedup_of_value": round(value / world / pv, 3)}
        del arms
        # end to end through the public API with host buffers (pinned): the
        # host-to-device copies of values, D and b, the factorisation, the
        # solve and the device-to-host copy of x, L2 flushed before each step
        sizes, rp, col, val, D = concat(insts)
        hv = torch.tensor(val).pin_memory().numpy()
        hD = torch.tensor(D).pin_memory().numpy()
        hb = torch.tensor(arm.b_host).pin_memory().numpy()
        hx = torch.empty(arm.b_host.shape, dtype=torch.float64).pin_memory().numpy()
        e2e_steps = min(args.steps, 20)
        arm.s.solve_host(hv, hD, arm.t, hb, precision, sweeps, out=hx)
        e2e_total = 0.0
        for i in range(e2e_steps):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            arm.s.solve_host(hv, hD, arm.t, hb, precision, sweeps, out=hx)
            e2e_total += time.perf_counter() - t0
        e2e_s = e2e_total / e2e_steps
        out["e2e"] = {"value": round(units * world / e2e_s, 2), "unit": UNIT,
                      "h2d_bytes_per_step": int(hv.nbytes + hD.nbytes + hb.nbytes),
                      "d2h_bytes_per_step": int(hx.nbytes), "ms_per_step": round(e2e_s * 1e3, 4),
                      "path": "pisp_solve_host: pinned host buffers, H2D + factor + solve + D2H, eager, "
                              "L2 flushed before each step"}
        out["cpu_baseline"] = cpu_baseline(insts, K, R, args.eps)
    return out


# ----------------------------------------------------------------- studies --
def _dense_instance(n, seed):
    return pfgen.random_sparse(n, 1.0, seed=seed, diag_boost=2.0 * math.sqrt(n))


def study_dense(args):
    """Next row f4: dense batches of G systems of size n, K = 10 shifts, one RHS,
    FP64: time of one captured factor + solve step against n and G (the
    flatness in the batch size the paper reports for its batched LU, Sec. IV)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2311_11833_gb300 as pisp
    dev = torch.device("cuda", 0)
    K, R = 10, 1
    rows = []
    clocks = ClockSampler(0)
    variants = [("fp64", 0, {}), ("fp32", 2, dict(factor_policy=4)),
                ("fp32", 2, dict(factor_policy=4, factor_tc=1))]
    for (prec, sw, extra), n, G in ((v, n, G) for v in variants for n in (64, 150, 300, 531)
                                    for G in (1, 2, 4, 8, 16)):
        if True:
            insts = [_dense_instance(n, 1000 * n + g) for g in range(G)]
            arm = Arm(pisp, torch, insts, K, R, args.eps, prec, sw, "dense", dev, extra=extra)
            arm.capture(profile=True)
            for _ in range(3):
                arm.run()
            torch.cuda.synchronize()
            arm.s.profile_reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 20
            e0.record()
            for _ in range(reps):
                arm.run()
                arm.s.profile_collect()
            e1.record()
            e1.synchronize()
            prof = arm.s.profile_read()
            fac = (prof["factor_small"]["ms"] + prof["factor_big"]["ms"] + prof["factor_persistent"]["ms"]) / reps
            sol = (prof["forward"]["ms"] + prof["backward"]["ms"]) / reps
            rows.append({"precision": prec, "sweeps": sw, "options": extra, "n": n, "G": G,
                         "ms_step": round(e0.elapsed_time(e1) / reps, 4),
                         "ms_factor": round(fac, 4), "ms_solve": round(sol, 4)})
            arm.s.close()
    clk = clocks.stop()
    return {"study": "dense batches (next row f4)", "K": K, "R": R,
            "shifts": "symmetric +-eps*alpha", "eps": args.eps,
            "family": "Gaussian, diagonal +-2 sqrt(n) (dense)", "timing": "CUDA events over 20 graph replays",
            "table": rows, "clocks": clk}


def study_newton(args):
    """Next row f2: the Newton-Raphson power-flow loop, analysed once and
    refactored every iteration: per-iteration host Jacobian time, device
    factor + solve time (CUDA events) and wall time, to max |F| <= 1e-10."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2311_11833_gb300 as pisp
    dev = torch.device("cuda", 0)
    cases = [("300-bus", 300, 60, 7, 1.0, 1e-3), ("2000-bus", 2000, 400, 2001, 1.0, 1e-3)]
    out = []
    clocks = ClockSampler(0)
    for name, N, npv, seed, ang, eps in cases:
        c = pfgen.power_flow_case(N, npv, seed=seed, angle_scale=ang)
        for precision, sweeps in (("fp64", 0), ("fp32", 2)):
            s = pisp.Solver(c.n, c.row_ptr, c.col, device=0)
            t = pfgen.symmetric_shifts(4, eps)
            x = c.flat_start()
            its = []
            for it in range(25):
                w0 = time.perf_counter()
                F = c.mismatch(x)
                r = float(np.max(np.abs(F)))
                if r <= 1e-10:
                    break
                h0 = time.perf_counter()
                vals = c.jacobian(x)
                D = pfgen.diag_rule(c.n, c.row_ptr, c.col, vals)
                h1 = time.perf_counter()
                vt, Dt, Ft = (torch.tensor(a, device=dev) for a in (vals, D, F))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                s.factor(vt, Dt, t, precision)
                dx = s.solve(Ft, sweeps=sweeps)
                e1.record()
                dxh = dx.cpu().numpy()
                x = x - dxh
                its.append({"max_F": float(f"{r:.3e}"), "host_jacobian_ms": round(1e3 * (h1 - h0), 3),
                            "device_factor_solve_ms": round(e0.elapsed_time(e1), 4),
                            "wall_ms": round(1e3 * (time.perf_counter() - w0), 3)})
            out.append({"case": name, "n": c.n, "nnz": c.nnz, "precision": precision, "sweeps": sweeps,
                        "eps": eps, "K": 4, "iterations": len(its),
                        "converged": bool(np.max(np.abs(c.mismatch(x))) <= 1e-10), "per_iteration": its})
            s.close()
    return {"study": "Newton-Raphson loop (next row f2)", "tol": 1e-10, "cases": out, "clocks": clocks.stop()}


def run_reference(args, rank, world):
    """The CPU oracle timed on the host cores: each step one perturbed GEPP solve."""
    if rank != 0:
        return None
    import oracle
    c = pfgen.CONFIGS[args.workload]
    K, R = c["K"], c["R"]
    insts = workload_instances(args.workload, 0, args.instances)
    t = pfgen.symmetric_shifts(K, args.eps)
    beta = oracle.weights_float(list(t))
    G = len(insts)
    mats = {}

    def one(i):
        # step i: perturbed solve k = i % K of instance (i // K) % G, folded into x_hat
        g, k = (i // K) % G, i % K
        if g not in mats:
            mats[g] = (oracle.to_scipy(insts[g]), pfgen.rhs(insts[g].n, R, 1))
        A, b = mats[g]
        xk = oracle.perturbed_solutions(A, insts[g].D, [t[k]], b)[0]
        return beta[k] * xk

    for i in range(args.warmup):
        one(i)
    times = []
    for i in range(args.steps):
        t0 = time.perf_counter()
        one(args.warmup + i)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps * R / K / total      # K perturbed solves make R combined solves
    return {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "instances": G, "K": K, "R": R, "eps": args.eps},
        "impl": "reference",
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "each step one perturbed partial-pivoting solve (1/K of a combined "
                                   "solve of R RHS) of the workload's instances, numpy/scipy FP64"},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.study:
        out = (study_dense if args.study == "dense" else study_newton)(args) if rank == 0 else None
    elif args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            import torch.distributed as tdist
            torch.cuda.set_device(local_rank)
            tdist.init_process_group("nccl")
        out = run_pisp(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as tdist
            tdist.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
