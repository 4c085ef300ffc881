"""Host side of the autotuner: the candidate set, the cache key and the cache file.
(Timing the candidates needs a GPU and is covered by the GPU tests.)"""
import json

import numpy as np
import pytest
import torch

import pfgen
from paper_2311_11833_gb300 import tune


def test_candidates_cover_every_option_once():
    c = list(tune.candidates())
    assert len(c) == len(tune.RELAX) * len(tune.POLICIES) * len(tune.SCHEDULES) == 32
    assert len({tuple(sorted(d.items())) for d in c}) == 32
    assert {d["factor_policy"] for d in c} == {0, 1, 2, 3} and {d["solve_schedule"] for d in c} == {0, 1}


def test_key_depends_on_pattern_and_call_shape():
    inst = pfgen.make_instance("plain")
    k = tune._key([inst.n], inst.row_ptr, inst.col, 4, 2, "fp32", 2)
    assert k == tune._key([inst.n], inst.row_ptr.copy(), inst.col.copy(), 4, 2, "fp32", 2)
    col = inst.col.copy()
    col[[0, 1]] = col[[1, 0]]
    others = {tune._key([inst.n], inst.row_ptr, col, 4, 2, "fp32", 2),
              tune._key([inst.n], inst.row_ptr, inst.col, 6, 2, "fp32", 2),
              tune._key([inst.n], inst.row_ptr, inst.col, 4, 3, "fp32", 2),
              tune._key([inst.n], inst.row_ptr, inst.col, 4, 2, "fp64", 2),
              tune._key([inst.n], inst.row_ptr, inst.col, 4, 2, "fp32", 1)}
    assert k not in others and len(others) == 5


def test_key_depends_on_adaptive_sweeps():
    inst = pfgen.make_instance("plain")
    a = tune._key([inst.n], inst.row_ptr, inst.col, 4, 2, "fp32", 8)
    b = tune._key([inst.n], inst.row_ptr, inst.col, 4, 2, "fp32", 8, 1e-12)
    c = tune._key([inst.n], inst.row_ptr, inst.col, 4, 2, "fp32", 8, 1e-11)
    assert len({a, b, c}) == 3


def test_accuracy_guard_is_per_instance():
    """An error small against the batch's largest entry but large against its
    own instance's entries is caught."""
    ref = torch.tensor([[1000.0, 1.0], [-1000.0, 2.0], [1e-3, 1.0], [-2e-3, 4.0]], dtype=torch.float64)
    x = ref.clone()
    x[2, 0] += 1e-6
    inst = torch.tensor([0, 0, 1, 1])
    assert tune._entrywise(x, ref, inst) == pytest.approx(5e-4, rel=1e-9)
    assert tune._entrywise(ref, ref, inst) == 0.0
    x[3, 1] = float("nan")
    assert tune._entrywise(x, ref, inst) == float("inf")


def test_cache_hit_returns_without_timing(tmp_path):
    inst = pfgen.make_instance("plain")
    t = pfgen.symmetric_shifts(4)
    b = torch.zeros(inst.n, 2, dtype=torch.float64)
    key = tune._key([inst.n], inst.row_ptr, inst.col, len(t), 2, "fp32", 2)
    hit = {"options": {"relax_small": 16, "relax_zeros": 0.1, "factor_policy": 0, "solve_schedule": 0},
           "ms": 0.5, "all": []}
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({key: hit}))
    # values and D are not touched on a hit (no device needed)
    got = tune.autotune([inst.n], inst.row_ptr, inst.col, None, None, t, b, "fp32", 2, cache=str(path))
    assert got == hit


def test_unreadable_cache_is_empty(tmp_path):
    assert tune._load(str(tmp_path / "missing.json")) == {}
    bad = tmp_path / "bad.json"
    bad.write_text("{not json")
    assert tune._load(str(bad)) == {}


def test_staged_search_covers_the_solve_tiling_then_the_analysis():
    s1 = tune.staged_candidates()
    tilings = {(d["solve_ctas_per_sm"], d["solve_kfuse"], d["solve_warp_maxF"]) for d in s1}
    assert tilings == set(tune.TILINGS) and len(s1) == len(tune.TILINGS)
    assert all({k: d[k] for k in tune.DEFAULT} == tune.DEFAULT for d in s1)
    best = s1[5]
    s2 = tune._stage2(best)
    # stage 2 keeps stage 1's tiling and varies amalgamation and factor policy only
    assert all(d["solve_ctas_per_sm"] == best["solve_ctas_per_sm"] and d["solve_kfuse"] == best["solve_kfuse"]
               for d in s2)
    assert best not in s2 and len(s2) == len(tune.RELAX) * 4 - 1
    assert sum(1 for d in s2 if d.get("factor_ctas_per_sm") == 3) == len(tune.RELAX)
