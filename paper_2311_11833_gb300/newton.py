"""Newton-Raphson over one analysed pattern, with the perturbed solve as its step.

Sec. IV takes its systems from Newton-Raphson on a distributed-slack AC power
flow: every iteration solves J(x_i) dx = F(x_i) with the same sparsity
pattern, so the symbolic analysis (ordering, supernodes, levels) is done once
and every iteration only refactors.  This loop does exactly that through an
analysed `Solver`: per iteration it uploads the Jacobian values and the
perturbation diagonal, runs pisp_factor_perturbed for the shifts t, and takes
dx = sum_k beta_k (J + t_k D)^{-1} F from pisp_solve (with `sweeps` FP64
residual corrections when the factors are FP32).

The mismatch and Jacobian are the caller's (host callables returning float64
arrays or tensors); the factorisation and the solve run in libpisp.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Sequence

import numpy as np
import torch

from ._lib import PispError


@dataclasses.dataclass
class NewtonResult:
    x: np.ndarray            # last iterate
    iterations: int          # Newton steps taken
    converged: bool          # max |F(x)| <= tol
    mismatch: list           # max |F(x_i)| for i = 0..iterations
    status: list             # worst factorisation status of each step (0 = ok)


def _device(solver) -> torch.device:
    d = solver.device
    return d if isinstance(d, torch.device) else torch.device("cuda", int(d))


def _to(v, dev) -> torch.Tensor:
    if isinstance(v, torch.Tensor):
        return v.to(device=dev, dtype=torch.float64).contiguous()
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).to(dev)


def newton(solver, mismatch: Callable, jacobian: Callable, x0, t: Sequence[float],
           diag: Callable, precision: str = "fp64", sweeps: int = 0, tol: float = 1e-10,
           max_iter: int = 20) -> NewtonResult:
    """x_{i+1} = x_i - sum_k beta_k (J(x_i) + t_k D_i)^{-1} F(x_i) until max |F| <= tol.

    solver   : a `Solver` analysed on the Jacobian's pattern (row_ptr, col)
    mismatch : x (float64 [n]) -> F(x) [n]
    jacobian : x -> the Jacobian's values on the solver's pattern [nnz]
    diag     : Jacobian values -> the perturbation diagonal D [n]
    Raises PispError if a perturbed factorisation reports a zero or
    non-finite pivot (its step would be NaN).
    """
    dev = _device(solver)
    x = np.array(x0, dtype=np.float64)
    hist, status = [], []
    for it in range(max_iter + 1):
        F = np.asarray(mismatch(x), dtype=np.float64)
        r = float(np.max(np.abs(F))) if F.size else 0.0
        hist.append(r)
        if r <= tol:
            return NewtonResult(x, it, True, hist, status)
        if it == max_iter or not np.isfinite(r):
            break
        vals = jacobian(x)
        vals_h = vals.detach().cpu().numpy() if isinstance(vals, torch.Tensor) else np.asarray(vals)
        D = diag(vals_h)
        solver.factor(_to(vals, dev), _to(D, dev), t, precision)
        worst = int(solver.status()[0])
        status.append(worst)
        if worst != 0:
            raise PispError(worst, f"Newton step {it}: perturbed factorisation status {worst}")
        dx = solver.solve(_to(F, dev), sweeps=sweeps)
        x = x - dx.detach().cpu().numpy().astype(np.float64)
    return NewtonResult(x, len(hist) - 1, False, hist, status)
