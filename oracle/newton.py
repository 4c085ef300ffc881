"""Newton-Raphson power flow with the perturbed solve as its linear step.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Sec. IV draws its
systems from Newton-Raphson on a distributed-slack AC power flow: every
iteration solves J(x_i) dx = F(x_i) and sets x_{i+1} = x_i - dx, with the same
sparsity pattern throughout.  Here the linear step is either the true solution
J^{-1} F (partial pivoting) or the method's combination
sum_k beta_k (J + t_k D)^{-1} F (Eq. x_star with Eq. avg_hats), optionally
followed by residual corrections (the optional error check of Alg. 1 turned
into a correction), so the two iteration counts can be compared.

The mismatch F and Jacobian J come from the input generator.  Pins: J
against central differences of F, F(x_star) = 0 at the planted solution, the
quadratic convergence of the exact loop and its limit x_star.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .core import refine, x_hat, x_star


def newton(case, x0, step: str = "exact", diag=None, t=None, refine_iters: int = 0,
           tol: float = 1e-10, max_iter: int = 30):
    """Returns (x, iterations or None if not converged, [max |F(x_i)|]).

    case  : object with mismatch(x), jacobian(x), row_ptr, col, n
    step  : "exact" (J^{-1} F) or "perturbed" (x_hat with shifts t, D = diag(J))
    diag  : callable J (scipy CSR) -> D, used by the perturbed step
    """
    x = np.array(x0, dtype=np.float64)
    hist = []
    for it in range(max_iter + 1):
        F = case.mismatch(x)
        hist.append(float(np.max(np.abs(F))))
        if hist[-1] <= tol:
            return x, it, hist
        if it == max_iter or not np.isfinite(hist[-1]):
            break
        J = sp.csr_matrix((case.jacobian(x), case.col, case.row_ptr), shape=(case.n, case.n))
        if step == "exact":
            dx = x_star(J, F)
        elif step == "perturbed":
            D = diag(J)
            dx = x_hat(J, D, t, F)
            if refine_iters:
                dx = refine(J, D, t, F, dx, iters=refine_iters)
        else:
            raise ValueError(step)
        x = x - dx
    return x, None, hist
