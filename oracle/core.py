"""Plain FP64 oracle of the perturb / solve / combine method (test infrastructure).

Section / equation references are to arXiv 2311.11833.  All floating point is
IEEE double; the combination weights are computed in exact rationals first.
"""
from __future__ import annotations

from fractions import Fraction
from typing import Sequence

import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg as spla

DENSE_MAX = 4096          # above this the perturbed solves use sparse GEPP


# ---------------------------------------------------------------- matrices --
def to_scipy(inst) -> sp.csr_matrix:
    """CSR matrix of an input instance (pfgen.Instance or (n, row_ptr, col, val))."""
    n, rp, ci, v = _parts(inst)
    return sp.csr_matrix((v, ci, rp), shape=(n, n))


def to_dense(inst) -> np.ndarray:
    return to_scipy(inst).toarray()


def _parts(inst):
    if hasattr(inst, "row_ptr"):
        return inst.n, inst.row_ptr, inst.col, inst.val
    return inst


# ----------------------------------------------------------------- weights --
def weights_gamma(m: int) -> list[Fraction]:
    """beta = (Gamma_m^T)^{-1} e_1 with Gamma_{alpha, j} = alpha^{2j} (Remark 2, Eq. gam).

    Exact Gauss-Jordan in rationals.  beta_alpha multiplies the averaged
    solution x_hat_alpha = (x_alpha^+ + x_alpha^-)/2 (Eq. avg_hats).
    """
    G = [[Fraction(a) ** (2 * j) for j in range(m)] for a in range(1, m + 1)]
    GT = [[G[c][r] for c in range(m)] for r in range(m)]
    rhs = [Fraction(1)] + [Fraction(0)] * (m - 1)
    return _solve_rational(GT, rhs)


def weights(t: Sequence) -> list[Fraction]:
    """Per-solve weights beta_k for an arbitrary list of distinct signed shifts t_k.

    By Eq. neumann_2, (A + t D)^{-1} = sum_j (-t)^j (A^{-1} D)^j A^{-1}, so
    sum_k beta_k x_k has coefficient sum_k beta_k (-t_k)^j on the j-th Neumann
    term.  Asking for (1, 0, ..., 0) over j = 0..K-1 is the K x K transposed
    Vandermonde system of Eq. gam written for the shifts themselves; the
    sign (-1)^j does not change its solution.  Floats are converted to
    rationals exactly, so the result is the exact solution for the given
    binary shifts.
    """
    tf = [x if isinstance(x, Fraction) else Fraction(x) for x in t]
    K = len(tf)
    if len(set(tf)) != K:
        raise ValueError("shifts must be distinct")
    VT = [[tf[k] ** j for k in range(K)] for j in range(K)]
    rhs = [Fraction(1)] + [Fraction(0)] * (K - 1)
    return _solve_rational(VT, rhs)


def weights_float(t: Sequence) -> np.ndarray:
    return np.array([float(b) for b in weights(t)], dtype=np.float64)


def _solve_rational(M, rhs):
    """Gauss-Jordan elimination in exact rationals (any nonzero pivot)."""
    n = len(rhs)
    a = [list(row) + [rhs[i]] for i, row in enumerate(M)]
    for c in range(n):
        p = next(r for r in range(c, n) if a[r][c] != 0)
        a[c], a[p] = a[p], a[c]
        piv = a[c][c]
        a[c] = [v / piv for v in a[c]]
        for r in range(n):
            if r != c and a[r][c] != 0:
                f = a[r][c]
                a[r] = [vr - f * vc for vr, vc in zip(a[r], a[c])]
    return [a[i][n] for i in range(n)]


# ------------------------------------------------------------------ solves --
def _gepp_solve(M, B):
    """Solve M X = B with partial pivoting (dense LAPACK or sparse SuperLU)."""
    if sp.issparse(M):
        if M.shape[0] <= DENSE_MAX:
            return np.linalg.solve(M.toarray(), B)
        lu = spla.splu(M.tocsc(), permc_spec="COLAMD", diag_pivot_thresh=1.0)
        return lu.solve(np.ascontiguousarray(B))
    return np.linalg.solve(M, B)


def _shifted(A, D, t):
    if sp.issparse(A):
        return (A + t * sp.diags(D)).tocsr()
    return A + t * np.diag(D)


def perturbed_solutions(A, D, t, B, transpose=False) -> np.ndarray:
    """x_k = (A + t_k D)^{-1} B for every shift (Eq. xap / xam); [K, n, R].

    With transpose=True solves (A + t_k D)^T y = B instead.
    """
    B2 = np.asarray(B, dtype=np.float64)
    vec = B2.ndim == 1
    if vec:
        B2 = B2[:, None]
    out = []
    for tk in t:
        M = _shifted(A, D, float(tk))
        if transpose:
            M = M.T.tocsr() if sp.issparse(M) else M.T
        out.append(_gepp_solve(M, B2))
    X = np.stack(out)
    return X[:, :, 0] if vec else X


def combine(X, beta) -> np.ndarray:
    """sum_k beta_k X_k accumulated in k order (Eq. x_star)."""
    acc = np.zeros_like(X[0])
    for bk, xk in zip(beta, X):
        acc = acc + float(bk) * xk
    return acc


def x_hat(A, D, t, B, beta=None) -> np.ndarray:
    """The combined solution sum_k beta_k (A + t_k D)^{-1} B (Eq. x_star with Eq. avg_hats)."""
    if beta is None:
        beta = weights_float(t)
    return combine(perturbed_solutions(A, D, t, B), beta)


def pistol(A, D, eps: float, m: int, B) -> np.ndarray:
    """Algorithm 1, symmetric scheme, in the paper's order.

    1. perturb A by +alpha*eps*D and -alpha*eps*D, alpha = 1..m;
    2. solve each perturbed system (partial pivoting here);
    3. form the averages x_hat_alpha (Eq. avg_hats);
    4. combine them with beta = (Gamma_m^T)^{-1} e_1 (Eq. x_star_vand).
    """
    beta = weights_gamma(m)
    xh = []
    for a in range(1, m + 1):
        xp = perturbed_solutions(A, D, [a * eps], B)[0]
        xm = perturbed_solutions(A, D, [-a * eps], B)[0]
        xh.append(0.5 * (xp + xm))
    return combine(np.stack(xh), beta)


def x_star(A, B) -> np.ndarray:
    """The true solution A^{-1} B, by partial-pivoting LU."""
    B2 = np.asarray(B, dtype=np.float64)
    return _gepp_solve(A, B2)


def refine(A, D, t, B, x, iters: int = 1, beta=None) -> np.ndarray:
    """x <- x + sum_k beta_k (A + t_k D)^{-1} (B - A x), `iters` times (FP64).

    The residual is the optional error check of Alg. 1; using the same
    combined perturbed operator on it gives one correction step.
    """
    if beta is None:
        beta = weights_float(t)
    x = np.array(x, dtype=np.float64, copy=True)
    for _ in range(iters):
        r = np.asarray(B, dtype=np.float64) - A @ x
        x = x + x_hat(A, D, t, r, beta)
    return x


def adjoint(A, D, t, B, W, beta=None):
    """Reverse-mode derivative of L = sum(W * x_hat) with x_hat = sum_k beta_k x_k.

    dL/db = sum_k beta_k (A + t_k D)^{-T} W;
    dL/dA_ij = -sum_k beta_k sum_r lambda_k[i, r] x_k[j, r], on A's pattern
    (D held fixed).  Returns (grad_b, grad_vals in A's CSR order).
    """
    if beta is None:
        beta = weights_float(t)
    As = A if sp.issparse(A) else sp.csr_matrix(A)
    As = As.tocsr()
    As.sort_indices()
    W2 = np.asarray(W, dtype=np.float64)
    B2 = np.asarray(B, dtype=np.float64)
    if W2.ndim == 1:
        W2, B2 = W2[:, None], B2[:, None]
    X = perturbed_solutions(As, D, t, B2)
    Lam = perturbed_solutions(As, D, t, W2, transpose=True)
    grad_b = combine(Lam, beta)
    rows = np.repeat(np.arange(As.shape[0]), np.diff(As.indptr))
    cols = As.indices
    g = np.zeros(len(cols))
    for bk, lk, xk in zip(beta, Lam, X):
        g -= float(bk) * np.einsum("er,er->e", lk[rows], xk[cols])
    if np.asarray(W).ndim == 1:
        grad_b = grad_b[:, 0]
    return grad_b, g


def true_gradient(A, B, W):
    """dL/db and dL/dA of L = sum(W * A^{-1} B) (the unperturbed derivative)."""
    As = (A if sp.issparse(A) else sp.csr_matrix(A)).tocsr()
    As.sort_indices()
    W2 = np.asarray(W, dtype=np.float64)
    B2 = np.asarray(B, dtype=np.float64)
    if W2.ndim == 1:
        W2, B2 = W2[:, None], B2[:, None]
    x = _gepp_solve(As, B2)
    lam = _gepp_solve(As.T.tocsr(), W2)
    rows = np.repeat(np.arange(As.shape[0]), np.diff(As.indptr))
    g = -np.einsum("er,er->e", lam[rows], x[As.indices])
    gb = lam[:, 0] if np.asarray(W).ndim == 1 else lam
    return gb, g


# ------------------------------------------------------------ diagnostics --
def residual_norm(A, x, B) -> np.ndarray:
    """Relative residual ||A x - b|| / ||b|| per RHS (the metric of Fig. 1)."""
    r = A @ x - B
    return np.linalg.norm(np.atleast_2d(r.T), axis=-1) / np.linalg.norm(np.atleast_2d(np.asarray(B).T), axis=-1)


def rel_err(x, ref) -> np.ndarray:
    """Relative forward error ||x - ref|| / ||ref|| per RHS (columns)."""
    x = np.atleast_2d(np.asarray(x).T)
    ref = np.atleast_2d(np.asarray(ref).T)
    return np.linalg.norm(x - ref, axis=-1) / np.linalg.norm(ref, axis=-1)


def spectral_radius(A, D) -> float:
    """rho(A^{-1} D), the convergence radius quantity of Sec. II-B.

    Up to n = 1500: every eigenvalue of the dense A^{-1} D (LAPACK).  Above:
    the largest-magnitude eigenvalues of the operator v -> A^{-1} (D v) by
    implicitly restarted Arnoldi (ARPACK), which, unlike a plain power
    iteration, also converges when the dominant eigenvalues are a complex
    pair (power-flow Jacobians are unsymmetric).
    """
    Ad = A.toarray() if sp.issparse(A) else np.asarray(A, dtype=np.float64)
    n = Ad.shape[0]
    Dv = np.asarray(D, dtype=np.float64)
    if n <= 1500:
        M = np.linalg.solve(Ad, np.diag(Dv))
        return float(np.max(np.abs(np.linalg.eigvals(M))))
    lu = scipy.linalg.lu_factor(Ad)
    op = spla.LinearOperator((n, n), matvec=lambda v: scipy.linalg.lu_solve(lu, Dv * np.ravel(v)),
                             dtype=np.float64)
    vals = spla.eigs(op, k=6, which="LM", tol=1e-10, maxiter=20 * n,
                     v0=np.random.default_rng(0).standard_normal(n), return_eigenvectors=False)
    return float(np.max(np.abs(vals)))


def cond1(A) -> float:
    """kappa_1(A) = ||A||_1 ||A^{-1}||_1, by the dense inverse (diagnostic of the
    conditioning that static pivoting leaves unguarded, Sec. I)."""
    Ad = A.toarray() if sp.issparse(A) else np.asarray(A, dtype=np.float64)
    Ainv = np.linalg.solve(Ad, np.eye(Ad.shape[0]))
    return float(np.abs(Ad).sum(axis=0).max() * np.abs(Ainv).sum(axis=0).max())


def pivot_stats(A, D, t: float, perm=None):
    """Growth and pivot spread of the pivot-free LU of P (A + t D) P^T.

    Returns (growth, pivot_ratio): growth = max|U_ij| / max|(A + t D)_ij| and
    pivot_ratio = min|u_jj| / max|u_jj|.  A static pivot order controls
    neither (Sec. I); these are the quantities to watch.
    """
    _, U = pivot_free_lu(A, D, t, perm)
    Ad = A.toarray() if sp.issparse(A) else np.asarray(A, dtype=np.float64)
    M = Ad + float(t) * np.diag(np.asarray(D, dtype=np.float64))
    d = np.abs(np.diag(U))
    return float(np.abs(U).max() / np.abs(M).max()), float(d.min() / d.max())


def error_identity(A, D, t, B, beta=None) -> np.ndarray:
    """Closed form of x_hat - x* from the Neumann series (Sec. II-B).

    With M = A^{-1} D and the weights above, the scalar identity
    sum_k beta_k / (1 + t_k r) - 1 = -r^K prod(t) / prod(1 + t_k r) gives
    x_hat - x* = -(prod_k t_k) M^K prod_k (I + t_k M)^{-1} x*.
    Evaluated here by explicit dense matrix products (an independent route
    from the perturbed solves): returns that vector.
    """
    Ad = A.toarray() if sp.issparse(A) else np.asarray(A, dtype=np.float64)
    n = Ad.shape[0]
    M = np.linalg.solve(Ad, np.diag(D))
    xs = np.linalg.solve(Ad, np.asarray(B, dtype=np.float64))
    v = xs
    for tk in t:
        v = np.linalg.solve(np.eye(n) + float(tk) * M, v)
    for _ in range(len(t)):
        v = M @ v
    return -float(np.prod(np.asarray(t, dtype=np.float64))) * v


def pivot_free_lu(A, D, t: float, perm=None):
    """Dense Doolittle LU of P (A + t D) P^T without pivoting.

    perm[i] = original index placed at position i.  Returns (L, U) with unit
    lower L; raises ZeroDivisionError on an exact zero pivot.  This is the
    factor the pivot-free route must produce: it is unique when it exists.
    """
    Ad = A.toarray() if sp.issparse(A) else np.array(A, dtype=np.float64)
    M = Ad + t * np.diag(D)
    if perm is not None:
        p = np.asarray(perm)
        M = M[np.ix_(p, p)]
    n = M.shape[0]
    U = M.copy()
    L = np.eye(n)
    for c in range(n):
        piv = U[c, c]
        if piv == 0.0:
            raise ZeroDivisionError(f"zero pivot at position {c}")
        L[c + 1:, c] = U[c + 1:, c] / piv
        U[c + 1:, c:] -= np.outer(L[c + 1:, c], U[c, c:])
        U[c + 1:, c] = 0.0
    return L, np.triu(U)
