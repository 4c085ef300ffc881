"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, a transposed operand, a wrong weight) fails at least one of them.
"""
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse as sp

import oracle
import pfgen
from oracle import exact

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rationals(name):
    vals, extra = [], {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            if line.startswith("series"):
                extra["series"] = [Fraction(v) for v in line.split()[1:]]
            else:
                vals.append([Fraction(v) for v in line.split()])
    return vals, extra


# ------------------------------------------------------------ weights pins --
def test_example3_weights():
    """Example 3: (Gamma_2^T)^{-1} e_1 = (4/3, -1/3) exactly."""
    gold, _ = _rationals("example3_weights.txt")
    assert oracle.weights_gamma(2) == [row[0] for row in gold]


def test_example2_weights_corrected():
    """Example 2 (m = 3), read with the missing -5/4 normalisation."""
    gold, extra = _rationals("example2_weights.txt")
    beta = oracle.weights_gamma(3)
    assert beta == [row[0] for row in gold]
    # the printed combination x31* - 9/4 x21* equals -5/4 times ours
    # x21* = (x2 - 4 x1)/(-3), x31* = (x3 - 9 x1)/(-8) -> weights on (x1, x2, x3)
    x21 = [Fraction(4, 3), Fraction(-1, 3), Fraction(0)]
    x31 = [Fraction(9, 8), Fraction(0), Fraction(-1, 8)]
    printed = [a - Fraction(9, 4) * b for a, b in zip(x31, x21)]
    assert [p / Fraction(-5, 4) for p in printed] == beta
    # series coefficients of the normalised combination: sum_a beta_a a^{2j}
    series = [sum(b * Fraction(a) ** (2 * j) for a, b in zip((1, 2, 3), beta)) for j in range(4)]
    assert series == extra["series"]


def test_example1_series():
    """Example 1: coefficients 1, 0, -4, -20 on (A^-1 eps D)^{2j} A^-1 b."""
    gold, _ = _rationals("example1_series.txt")
    beta = oracle.weights_gamma(2)
    series = [sum(b * Fraction(a) ** (2 * j) for a, b in zip((1, 2), beta)) for j in range(4)]
    assert series == [row[0] for row in gold]
    # Eq. lin_comb1 as printed: (x2 - 4 x1) / (-3)
    assert beta == [Fraction(-4, -3), Fraction(1, -3)]


def test_gamma_rows():
    """Eq. avg_hats: the averaged solution alpha carries alpha^{2j} on term j.

    On the 1x1 system a = d = 1 the oracle's averaged solution is a power
    series in eps whose coefficients must be the rows of Gamma.
    """
    gold, _ = _rationals("avg_hats_gamma.txt")
    eps = 1e-2
    for a, row in zip((1, 2, 3), gold):
        X = oracle.perturbed_solutions(np.eye(1), np.ones(1), [a * eps, -a * eps], np.ones(1))
        xh = 0.5 * (X[0, 0] + X[1, 0])
        series = sum(float(c) * eps ** (2 * j) for j, c in enumerate(row))
        # next term is a^8 eps^8 <= 6561e-16
        assert abs(xh - series) <= 1.0001 * float(a) ** 8 * eps ** 8 / (1 - (a * eps) ** 2) + 1e-15


@pytest.mark.parametrize("K", [2, 4, 6, 8])
def test_weights_symmetric_match_gamma(K):
    """Per-solve weights of the symmetric set are half the paper's beta per +- pair."""
    eps = Fraction(1, 100)
    t = []
    for a in range(1, K // 2 + 1):
        t += [a * eps, -a * eps]
    w = oracle.weights(t)
    g = oracle.weights_gamma(K // 2)
    for a in range(K // 2):
        assert w[2 * a] == w[2 * a + 1] == g[a] / 2


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5, 8])
def test_weights_one_sided_binomial(K):
    """Shifts t_k = k*eps: weights are (-1)^{k+1} C(K, k), e.g. (4, -6, 4, -1)."""
    from math import comb
    t = [Fraction(k, 100) for k in range(1, K + 1)]
    assert oracle.weights(t) == [Fraction((-1) ** (k + 1) * comb(K, k)) for k in range(1, K + 1)]


def test_weights_moment_conditions_float_shifts():
    """sum_k beta_k t_k^j = delta_j0 for j < K, for the binary doubles in use."""
    t = pfgen.symmetric_shifts(6)
    w = oracle.weights(list(t))
    tf = [Fraction(x) for x in t]
    for j in range(6):
        assert sum(b * x ** j for b, x in zip(w, tf)) == (1 if j == 0 else 0)


# ------------------------------------------------------------ closed forms --
def test_two_by_two_cramer():
    A = np.array([[2.0, -1.0], [0.5, 3.0]])
    D = np.array([2.0, 3.0])
    b = np.array([1.0, -2.0])
    t = pfgen.symmetric_shifts(4)
    beta = oracle.weights_float(t)
    xh = np.zeros(2)
    for bk, tk in zip(beta, t):
        a, bb, c, d = A[0, 0] + tk * D[0], A[0, 1], A[1, 0], A[1, 1] + tk * D[1]
        det = a * d - bb * c
        xh += bk * np.array([(b[0] * d - bb * b[1]) / det, (a * b[1] - c * b[0]) / det])
    np.testing.assert_allclose(oracle.x_hat(A, D, t, b), xh, rtol=1e-14, atol=0)


def test_diagonal_closed_form_and_identity():
    """Diagonal A, D: x_hat_i = (b_i/a_i) sum_k beta_k / (1 + t_k d_i / a_i)."""
    rng = np.random.default_rng(1)
    n = 9
    a = rng.uniform(0.5, 2.0, n) * np.sign(rng.standard_normal(n))
    d = rng.uniform(0.1, 3.0, n)
    b = rng.standard_normal(n)
    for t in (pfgen.symmetric_shifts(4, 0.05), pfgen.one_sided_shifts(4, 0.03)):
        beta = oracle.weights_float(t)
        ref = (b / a) * sum(bk / (1 + tk * d / a) for bk, tk in zip(beta, t))
        got = oracle.x_hat(np.diag(a), d, t, b)
        np.testing.assert_allclose(got, ref, rtol=1e-13)
        # exact error: x_hat - x* = -(prod t) r^K / prod(1 + t r) x*, r = d/a
        r = d / a
        err = -np.prod(t) * r ** len(t) / np.prod([1 + tk * r for tk in t], axis=0) * (b / a)
        np.testing.assert_allclose(got - b / a, err, rtol=1e-6, atol=1e-17)


@pytest.mark.parametrize("K,one_sided", [(4, False), (6, False), (4, True), (2, False)])
def test_error_identity_general(K, one_sided):
    """x_hat - x* = -(prod t) M^K prod (I + t_k M)^{-1} x* on a random 7x7 (Sec. II-B)."""
    rng = np.random.default_rng(7 + K)
    n = 7
    A = rng.standard_normal((n, n)) + 3 * np.eye(n)
    D = np.abs(np.diag(A))
    B = rng.standard_normal((n, 2))
    t = pfgen.one_sided_shifts(K, 0.05) if one_sided else pfgen.symmetric_shifts(K, 0.05)
    xh = oracle.x_hat(A, D, t, B)
    xs = oracle.x_star(A, B)
    ident = oracle.error_identity(A, D, t, B)
    scale = np.abs(xs).max()
    assert np.abs((xh - xs) - ident).max() <= 1e-12 * scale
    # the error itself is far above rounding, so the identity is not vacuous
    assert np.abs(xh - xs).max() > 1e3 * 1e-16 * scale


def test_pistol_matches_general_weights():
    """Alg. 1 with averages + (Gamma_m^T)^{-1} e_1 equals the per-solve weighted sum."""
    inst = pfgen.random_sparse(12, 0.3, seed=3)
    A = oracle.to_dense(inst)
    B = np.random.default_rng(0).standard_normal((12, 3))
    for m in (1, 2, 3):
        np.testing.assert_allclose(oracle.pistol(A, inst.D, 0.02, m, B),
                                   oracle.x_hat(A, inst.D, pfgen.symmetric_shifts(2 * m, 0.02), B),
                                   rtol=1e-12, atol=1e-14)


# --------------------------------------------------------- rational brute --
@pytest.mark.parametrize("seed", range(4))
def test_exact_rational_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 7))
    A = rng.integers(-5, 6, size=(n, n)).astype(float)
    A += np.diag(rng.choice([-9.0, 9.0], size=n))
    D = rng.integers(1, 4, size=n).astype(float)
    b = rng.integers(-4, 5, size=n).astype(float)
    t = [Fraction(1, 16), Fraction(-1, 16), Fraction(1, 8), Fraction(-1, 8)]
    ex = exact.x_hat(A.tolist(), D.tolist(), t, b.tolist())
    got = oracle.x_hat(A, D, [float(x) for x in t], b)
    np.testing.assert_allclose(got, [float(v) for v in ex], rtol=1e-13, atol=1e-15)


# -------------------------------------------------------- order invariants --
def _well_posed(n=20, seed=5):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) / np.sqrt(n) + 2.0 * np.eye(n)
    D = np.abs(np.diag(A))
    b = rng.standard_normal(n)
    return A, D, b


def test_remark1_pair_average_is_second_order():
    """Remark 1: (x+ + x-)/2 - x* = O(eps^2); x+ alone is O(eps)."""
    A, D, b = _well_posed()
    xs = oracle.x_star(A, b)
    e1, e2 = [], []
    for eps in (1e-2, 5e-3):
        X = oracle.perturbed_solutions(A, D, [eps, -eps], b)
        e1.append(np.linalg.norm(X[0] - xs))
        e2.append(np.linalg.norm(0.5 * (X[0] + X[1]) - xs))
    assert np.log2(e1[0] / e1[1]) == pytest.approx(1.0, abs=0.05)
    assert np.log2(e2[0] / e2[1]) == pytest.approx(2.0, abs=0.05)


@pytest.mark.parametrize("m", [1, 2, 3])
def test_theorem1_error_order(m):
    """Theorem 1: with m averaged pairs the error is O(eps^{2m})."""
    A, D, b = _well_posed()
    rho = oracle.spectral_radius(A, D)
    xs = oracle.x_star(A, b)
    eps = [0.04 / rho, 0.02 / rho]
    err = [np.linalg.norm(oracle.pistol(A, D, e, m, b) - xs) for e in eps]
    assert err[0] > 1e-13 and err[1] > 1e-14
    assert np.log2(err[0] / err[1]) == pytest.approx(2 * m, abs=0.15)


# ------------------------------------------------ spectral radius pins --
# rho(A^{-1} D) decides where Theorem 1 applies (Sec. II-B) and gates
# assertions elsewhere, so both of its branches (dense eigenvalues up to
# n = 1500, Arnoldi above) are pinned to values fixed independently of it.
@pytest.mark.parametrize("n", [7, 1600])
def test_spectral_radius_diagonal_closed_form(n):
    """Diagonal A and D: A^{-1} D = diag(d_i / a_i), so rho = max |d_i / a_i|."""
    rng = np.random.default_rng(n)
    a = rng.uniform(0.5, 2.0, n) * rng.choice([-1.0, 1.0], n)
    d = rng.uniform(0.1, 1.0, n)
    d[n // 3] = 3.0                        # one clearly dominant ratio
    A = sp.diags(a).tocsr()
    assert oracle.spectral_radius(A, d) == pytest.approx(float(np.max(np.abs(d / a))), rel=1e-9)


def _complex_pair_system(n):
    """A, D with A^{-1} D = blockdiag(C, 0.5 I), C = [[1, 4], [-1, 1]] placed on
    rows/columns (p, q): C has the eigenvalues 1 +- 2i, so rho = sqrt(5), and
    C is not normal, so a power iteration's norm ratio oscillates."""
    C_inv = np.linalg.inv(np.array([[1.0, 4.0], [-1.0, 1.0]]))
    A = np.eye(n) * 2.0                   # A^{-1} D = 0.5 I off the block (D = 1)
    p, q = (n - 1) // 2, (n - 1) // 2 + 1
    A[np.ix_([p, q], [p, q])] = C_inv
    return A, np.ones(n)


@pytest.mark.parametrize("n", [2, 1600])
def test_spectral_radius_complex_dominant_pair(n):
    A, D = _complex_pair_system(n)
    assert oracle.spectral_radius(A, D) == pytest.approx(np.sqrt(5.0), rel=1e-9)


def test_spectral_radius_arnoldi_branch_matches_dense_eigenvalues():
    """Just above the branch point, the Arnoldi estimate equals the largest
    |eigenvalue| of the dense A^{-1} D computed by LAPACK."""
    inst = pfgen.random_sparse(1550, 0.004, seed=77, diag_boost=1.0)
    A = oracle.to_dense(inst)
    rng = np.random.default_rng(5)
    D = rng.uniform(0.2, 2.0, inst.n)
    ref = float(np.max(np.abs(np.linalg.eigvals(np.linalg.solve(A, np.diag(D))))))
    assert oracle.spectral_radius(sp.csr_matrix(A), D) == pytest.approx(ref, rel=1e-8)


def test_error_falls_with_order_inside_convergence_region():
    A, D, b = _well_posed()
    rho = oracle.spectral_radius(A, D)
    eps = 0.05 / rho
    xs = oracle.x_star(A, b)
    errs = [np.linalg.norm(oracle.pistol(A, D, eps, m, b) - xs) for m in (1, 2, 3, 4)]
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))


# ------------------------------------------------------------- refinement --
def test_refine_diagonal_closed_form():
    """One correction squares the per-component relative error on diagonal systems."""
    rng = np.random.default_rng(11)
    n = 8
    a = rng.uniform(0.5, 2.0, n)
    d = rng.uniform(0.5, 2.0, n)
    b = rng.standard_normal(n)
    t = pfgen.symmetric_shifts(2, 0.05)
    A = np.diag(a)
    xh = oracle.x_hat(A, d, t, b)
    x1 = oracle.refine(A, d, t, b, xh, iters=1)
    beta = oracle.weights_float(t)
    s = sum(bk * a / (a + tk * d) for bk, tk in zip(beta, t))      # M A = diag(s)
    xs = b / a
    np.testing.assert_allclose(x1 - xs, (1 - s) ** 2 * (-xs), rtol=1e-6, atol=1e-16)


# ---------------------------------------------------------------- adjoint --
def test_adjoint_matches_central_differences():
    inst = pfgen.random_sparse(10, 0.35, seed=21)
    A = oracle.to_scipy(inst)
    D = inst.D
    t = pfgen.symmetric_shifts(4)
    rng = np.random.default_rng(2)
    B = rng.standard_normal((10, 2))
    W = rng.standard_normal((10, 2))
    gb, gv = oracle.adjoint(A, D, t, B, W)
    L = lambda vals, BB: float(np.sum(W * oracle.x_hat(oracle.to_scipy((10, inst.row_ptr, inst.col, vals)), D, t, BB)))
    h = 1e-6
    for e in (0, 5, len(inst.val) // 2, len(inst.val) - 1):
        vp, vm = inst.val.copy(), inst.val.copy()
        step = h * max(1.0, abs(inst.val[e]))
        vp[e] += step
        vm[e] -= step
        fd = (L(vp, B) - L(vm, B)) / (2 * step)
        assert fd == pytest.approx(gv[e], rel=1e-6, abs=1e-9)
    for i, r in ((0, 0), (7, 1)):
        Bp, Bm = B.copy(), B.copy()
        Bp[i, r] += h
        Bm[i, r] -= h
        fd = (L(inst.val, Bp) - L(inst.val, Bm)) / (2 * h)
        assert fd == pytest.approx(gb[i, r], rel=1e-6, abs=1e-9)


def test_adjoint_close_to_true_gradient():
    """The combined derivative differs from -lambda* x*^T only by the expansion error."""
    inst = pfgen.random_sparse(10, 0.35, seed=22)
    A = oracle.to_scipy(inst)
    t = pfgen.symmetric_shifts(4, 1e-3)
    rng = np.random.default_rng(3)
    B, W = rng.standard_normal(10), rng.standard_normal(10)
    gb, gv = oracle.adjoint(A, inst.D, t, B, W)
    tb, tv = oracle.true_gradient(A, B, W)
    np.testing.assert_allclose(gb, tb, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(gv, tv, rtol=1e-8, atol=1e-10)


# ------------------------------------------------------------ pivot-free --
def test_pivot_free_lu_matches_lapack_when_no_swaps():
    """On a column diagonally dominant matrix GEPP swaps nothing, so its L, U are ours."""
    rng = np.random.default_rng(4)
    n = 15
    A = rng.standard_normal((n, n))
    A += np.diag(np.abs(A).sum(axis=0) + 1.0)
    D = np.abs(np.diag(A))
    P, L, U = scipy.linalg.lu(A + 0.01 * np.diag(D))
    assert np.array_equal(P, np.eye(n))
    L2, U2 = oracle.pivot_free_lu(A, D, 0.01)
    np.testing.assert_allclose(L2, L, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(U2, U, rtol=1e-12, atol=1e-13)


def test_pivot_free_lu_permuted_reconstructs():
    inst = pfgen.random_sparse(11, 0.3, seed=5)
    A = oracle.to_dense(inst)
    perm = np.random.default_rng(6).permutation(11)
    L, U = oracle.pivot_free_lu(A, inst.D, -0.02, perm)
    M = (A - 0.02 * np.diag(inst.D))[np.ix_(perm, perm)]
    np.testing.assert_allclose(L @ U, M, rtol=1e-12, atol=1e-12)
    assert np.allclose(np.tril(L, -1) + np.eye(11), L) and np.allclose(np.triu(U), U)


@pytest.mark.parametrize("delta", [0.3, 1e-2, 1e-5])
def test_cond1_and_pivot_stats_closed_forms(delta):
    """A = [[d, 1], [1, 1]]: kappa_1 = 4 / (1 - d); unpivoted U = [[d, 1], [0, 1 - 1/d]],
    so growth = max(d, 1, 1/d - 1) and pivot ratio = min(d, 1/d - 1) / max(d, 1/d - 1);
    in the swapped order U = [[1, 1], [0, d - 1]]: growth 1, ratio 1 - d."""
    A = np.array([[delta, 1.0], [1.0, 1.0]])
    assert oracle.cond1(A) == pytest.approx(4.0 / (1.0 - delta), rel=1e-12)
    u22 = 1.0 / delta - 1.0
    g, r = oracle.pivot_stats(A, np.zeros(2), 0.0)
    assert g == pytest.approx(max(1.0, u22), rel=1e-12)
    assert r == pytest.approx(min(delta, u22) / max(delta, u22), rel=1e-12)
    g, r = oracle.pivot_stats(A, np.zeros(2), 0.0, perm=[1, 0])
    assert g == pytest.approx(1.0, rel=1e-12) and r == pytest.approx(1.0 - delta, rel=1e-12)
    # a shift on the diagonal: A + t I = [[d + t, 1], [1, 1 + t]]
    t = 0.25
    u22 = (1.0 + t) - 1.0 / (delta + t)
    g, r = oracle.pivot_stats(A, np.ones(2), t)
    assert g == pytest.approx(max(delta + t, 1.0, abs(u22)) / (1.0 + t), rel=1e-12)
    assert r == pytest.approx(min(delta + t, abs(u22)) / max(delta + t, abs(u22)), rel=1e-12)


def test_cond1_and_pivot_stats_of_a_diagonal_matrix():
    d = np.array([3.0, -0.5, 8.0, 2.0])
    assert oracle.cond1(np.diag(d)) == pytest.approx(16.0, rel=1e-14)
    g, r = oracle.pivot_stats(np.diag(d), np.ones(4), 0.25)
    assert g == pytest.approx(1.0) and r == pytest.approx(0.25 / 8.25, rel=1e-14)   # |d + 0.25|


def test_pivot_free_zero_pivot_raises():
    A = np.array([[0.0, 1.0], [1.0, 0.0]])
    with pytest.raises(ZeroDivisionError):
        oracle.pivot_free_lu(A, np.ones(2), 0.0)


# ------------------------------------------------------- sparse vs dense --
def test_sparse_gepp_matches_dense():
    inst = pfgen.make_instance("plain")
    A = oracle.to_scipy(inst)
    b = pfgen.rhs(inst.n, 2, 1)
    t = pfgen.symmetric_shifts(4)
    old = oracle.core.DENSE_MAX
    try:
        dense = oracle.x_hat(A, inst.D, t, b)
        oracle.core.DENSE_MAX = 16
        sparse = oracle.x_hat(A, inst.D, t, b)
    finally:
        oracle.core.DENSE_MAX = old
    np.testing.assert_allclose(sparse, dense, rtol=1e-10, atol=1e-12 * np.abs(dense).max())


def test_generator_shapes():
    inst = pfgen.make_instance("plain")
    assert inst.n == 300 + inst.meta["n_pq"] and inst.meta["n_pq"] == 239
    assert 3000 < inst.nnz < 5000
    A = oracle.to_scipy(inst)
    assert np.all(A.diagonal() != 0)
    assert np.all(inst.D > 0)
    # deterministic
    inst2 = pfgen.make_instance("plain")
    assert np.array_equal(inst.val, inst2.val) and np.array_equal(inst.col, inst2.col)
