"""Rational brute force for tiny systems (test infrastructure only).

Everything here is exact: A, D, b, shifts and weights are Fractions, and the
solves are Gaussian elimination over the rationals.  Used to pin the floating
point oracle and, through it, the GPU path (Eq. x_star with Eq. xap / xam).
"""
from __future__ import annotations

from fractions import Fraction

from .core import weights


def solve(A, b):
    """Exact solution of A x = b (lists of Fractions), any nonzero pivot."""
    n = len(b)
    a = [[Fraction(v) for v in row] + [Fraction(b[i])] for i, row in enumerate(A)]
    for c in range(n):
        p = next(r for r in range(c, n) if a[r][c] != 0)
        a[c], a[p] = a[p], a[c]
        for r in range(c + 1, n):
            if a[r][c] != 0:
                f = a[r][c] / a[c][c]
                a[r] = [vr - f * vc for vr, vc in zip(a[r], a[c])]
    x = [Fraction(0)] * n
    for i in range(n - 1, -1, -1):
        s = a[i][n] - sum(a[i][j] * x[j] for j in range(i + 1, n))
        x[i] = s / a[i][i]
    return x


def x_hat(A, D, t, b):
    """sum_k beta_k (A + t_k D)^{-1} b exactly, with beta from the exact weights."""
    n = len(b)
    beta = weights(t)
    acc = [Fraction(0)] * n
    for bk, tk in zip(beta, t):
        M = [[Fraction(A[i][j]) + (Fraction(tk) * Fraction(D[i]) if i == j else 0)
              for j in range(n)] for i in range(n)]
        xk = solve(M, b)
        acc = [a + bk * v for a, v in zip(acc, xk)]
    return acc
