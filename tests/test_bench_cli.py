"""bench.py contract checks that need no GPU (the oracle reference arm)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "plain",
                        "--steps", "2", "--warmup", "1"], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
                "cpu_baseline", "e2e"):
        assert key in d
    assert d["impl"] == "reference" and d["steps"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["config"]["workload"] == "plain"


def test_product_arm_fails_loudly_without_a_gpu():
    """No CPU fallback: without a CUDA device the product arm exits non-zero and
    prints no result line."""
    import pytest
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    r = subprocess.run([sys.executable, "bench.py", "--steps", "1", "--warmup", "1"], cwd=ROOT,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode != 0
    assert not any(l.strip().startswith("{") for l in r.stdout.splitlines())


def test_minimum_bytes_count_indices_once_for_all_shifts():
    """The roofline's algorithmic bytes of a solve launch: K copies of the
    triangle's factor entries, ONE copy of their int32 indices, the vectors."""
    sys.path.insert(0, ROOT)
    import bench
    st = {"N": 10, "nnzA": 30, "nnzF_stored": 50}
    K, R, p = 4, 2, 4
    nnzU, nnzL = 30, 20                       # (nnzF + N) / 2, (nnzF - N) / 2
    assert bench.min_bytes_per_launch("backward", st, K, R, p) == K * p * nnzU + 4 * nnzU + K * p * 10 * R + 8 * 10 * R
    assert bench.min_bytes_per_launch("forward", st, K, R, p) == K * p * nnzL + 4 * nnzL + 8 * 10 * R + K * p * 10 * R
    assert bench.min_bytes_per_launch("factor_small", st, K, R, p) is None
    # the whole factorisation: A's values, D, the pattern once, K factors
    assert bench.min_bytes_per_launch("factor_persistent", st, K, R, p) == 8 * 30 + 8 * 10 + 4 * (50 + 10) + K * p * 50


def test_oracle_pool_matches_the_oracle_and_checks_every_instance():
    """The bench's oracle references come from spawned worker processes (one
    BLAS thread each): they equal the oracle run in this process up to the
    rounding order of the BLAS threads (3e-12 entry-wise on the worst of these
    instances, relative to each column's largest entry), and the check reports
    every instance of the batch."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import pfgen

    insts = bench.workload_instances("batching", 0, 3)
    t = pfgen.symmetric_shifts(4, 0.01)
    sizes = [I.n for I in insts]
    b = pfgen.rhs(sum(sizes), 2, 1)
    refs = bench.oracle_refs(insts, t, b)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    for g, I in enumerate(insts):
        direct = oracle.x_hat(oracle.to_scipy(I), I.D, t, b[offs[g]:offs[g + 1]])
        assert np.max(np.abs(refs[g] - direct).max(axis=0) / np.abs(direct).max(axis=0)) <= 1e-11

    class Arm:  # the fields oracle_check reads
        pass

    arm = Arm()
    arm.insts = insts
    x = np.concatenate(refs).copy()
    x[offs[1] + 3, 1] += 1e-6 * np.abs(refs[1][:, 1]).max()   # one wrong entry in instance 1
    chk = bench.oracle_check(arm, refs, xs=x)
    assert chk["instances"] == 3 and chk["results"] == 6
    assert not chk["all_within_tol"]
    bad = [p for p in chk["per_instance"] if max(p["entrywise"]) > bench.TOL]
    assert [p["instance"] for p in bad] == [1]
