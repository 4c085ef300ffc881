"""Splitting the perturbed solves over ranks (one process per GPU).

Two partitions of the same work exist:

* **instances** (a batch of independent grids): each rank analyses, factors
  and solves its own subset; no data crosses ranks.  `partition_instances`
  balances the subsets by a cost per instance (greedy longest-processing-time
  bin packing, deterministic).
* **shifts** (one large system): rank r factors and solves only its shifts
  t[r::world] and forms the partial combination sum_{k in r} beta_k x_k with
  the weights of the *full* shift set; one sum all-reduce of the n x R FP64
  partials then gives x_hat = sum_k beta_k x_k (Eq. x_star), because the
  combination is linear in the per-shift solutions.

The collective runs through torch.distributed (NCCL between GPUs, gloo on
CPU).  The per-rank partial solve is passed in as a callable so that the
reduction logic is the same whatever computes the partials.
"""
from __future__ import annotations

from typing import Callable, Sequence

import numpy as np


def partition_instances(costs: Sequence[float], world: int) -> list[list[int]]:
    """Instance indices per rank, balancing the summed cost (LPT greedy)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def shift_subset(K: int, rank: int, world: int) -> list[int]:
    """Shift indices handled by `rank` when the K shifts are split over `world` ranks."""
    return list(range(rank, K, world))


def split_weights(beta: Sequence[float], rank: int, world: int) -> np.ndarray:
    """The full-set weights restricted to this rank's shifts (others contribute elsewhere)."""
    beta = np.asarray(beta, dtype=np.float64)
    return beta[shift_subset(len(beta), rank, world)]


def solve_shift_split(partial: Callable[[np.ndarray, np.ndarray], "object"], t: Sequence[float],
                      beta: Sequence[float], group=None):
    """x_hat over all shifts from per-rank partial combinations.

    partial(t_sub, w_sub) must return this rank's sum_k w_sub[k] x_k (a torch
    tensor on the collective's device) for the shifts t_sub; ranks without
    shifts pass empty arrays and must return zeros of the same shape.  The
    partials are summed with one all-reduce.
    """
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    idx = shift_subset(len(t), rank, world)
    t_sub = np.asarray(t, dtype=np.float64)[idx]
    w_sub = np.asarray(beta, dtype=np.float64)[idx]
    x = partial(t_sub, w_sub)
    dist.all_reduce(x, op=dist.ReduceOp.SUM, group=group)
    return x


def gpu_partial(solver, values, D, b, precision: str = "fp32", sweeps: int = 2):
    """The CUDA partial for `solve_shift_split`: factor this rank's shifts, combine with w_sub."""
    import torch

    def run(t_sub, w_sub):
        if len(t_sub) == 0:
            return torch.zeros_like(b)
        solver.factor(values, D, t_sub, precision)
        return solver.solve(b, weights=w_sub, sweeps=sweeps)

    return run
