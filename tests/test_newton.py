"""Next row f2: Newton-Raphson distributed-slack power flow (Sec. IV's use case).

One pattern is analysed once and refactored every iteration.  The power-flow
case has a planted solution x_star (the specified injections are those of a
random operating point), so convergence is checked against a known answer.

CPU tests pin the mismatch F and Jacobian J (central differences, F(x_star) = 0),
the exact Newton loop of the oracle (quadratic convergence to x_star), the
iteration counts with the perturbed step, and the library's Newton loop with a
stand-in solver; the GPU test runs that loop on libpisp and compares it with
the oracle's loop.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
import pfgen
from oracle.newton import newton as oracle_newton

CASES = {"light": (300, 60, 7, 1.0), "heavy": (300, 60, 12, 1.5)}    # (N, PV buses, seed, angle scale)


def _case(name):
    N, npv, seed, a = CASES[name]
    return pfgen.power_flow_case(N, npv, seed=seed, angle_scale=a)


def _jac(c, x):
    return sp.csr_matrix((c.jacobian(x), c.col, c.row_ptr), shape=(c.n, c.n))


def _drule(J):
    return pfgen.diag_rule(J.shape[0], J.indptr, J.indices, J.data)


def test_mismatch_vanishes_at_the_planted_solution():
    for name in CASES:
        c = _case(name)
        assert np.max(np.abs(c.mismatch(c.x_star))) < 1e-13
        assert np.max(np.abs(c.mismatch(c.flat_start()))) > 1.0


def test_jacobian_matches_central_differences():
    c = _case("light")
    rng = np.random.default_rng(0)
    x = c.flat_start() + 0.05 * rng.standard_normal(c.n)
    J = _jac(c, x).toarray()
    h = 1e-6
    Jfd = np.empty_like(J)
    for j in range(c.n):
        e = np.zeros(c.n)
        e[j] = h
        Jfd[:, j] = (c.mismatch(x + e) - c.mismatch(x - e)) / (2 * h)
    assert np.max(np.abs(J - Jfd)) <= 1e-8 * np.max(np.abs(J))
    assert np.all(Jfd[J == 0] == 0)               # the fixed pattern covers every dependence


def test_pattern_is_the_grid_jacobians():
    """Same draws as the benchmark generator: at the planted point the Jacobian is
    the one `grid_jacobian` builds for the same seed (angle scale 1)."""
    c = pfgen.power_flow_case(300, 60, seed=1000)
    inst = pfgen.make_instance("plain")
    assert np.array_equal(c.row_ptr, inst.row_ptr) and np.array_equal(c.col, inst.col)
    np.testing.assert_array_equal(c.jacobian(c.x_star), inst.val)


@pytest.mark.parametrize("name,its", [("light", 7), ("heavy", 9)])
def test_exact_newton_converges_quadratically(name, its):
    c = _case(name)
    x, it, h = oracle_newton(c, c.flat_start(), "exact")
    assert it == its
    assert np.max(np.abs(x - c.x_star)) < 1e-10
    tail = [v for v in h if v < 1e-3]
    assert len(tail) >= 3
    for a, b in zip(tail[:-1], tail[1:]):
        assert b <= 100 * a * a + 1e-13          # F_{i+1} <= C F_i^2 (C is about 50 here)


@pytest.mark.parametrize("D,eps,K", [("diag", 1e-3, 4), ("gauss", 2e-3, 4), ("gauss", 2e-3, 2)])
def test_perturbed_newton_takes_the_exact_iteration_count(D, eps, K):
    """With alpha_max * eps * rho(J^{-1} D) well inside 1 (Theorem 1) the perturbed
    step is accurate to far below the Newton error, so the iteration count is the
    exact loop's and the limit is x_star."""
    c = _case("light")
    g = np.random.default_rng(5).standard_normal(c.n)
    fn = _drule if D == "diag" else (lambda J: g)
    x, it, _ = oracle_newton(c, c.flat_start(), "perturbed", fn, pfgen.symmetric_shifts(K, eps))
    assert it == 7
    assert np.max(np.abs(x - c.x_star)) < 1e-10


def test_perturbed_newton_stalls_at_the_edge_of_the_region():
    """diag|J_ii| with eps = 1e-2: rho(J^{-1} D) grows from 29 at the flat start to 45
    at the solution, so alpha_max * eps * rho reaches 0.9 and the K = 4 combination
    no longer contracts the slowest mode: the mismatch stalls near 1e-3."""
    c = _case("light")
    assert oracle.spectral_radius(_jac(c, c.x_star), _drule(_jac(c, c.x_star))) > 40
    x, it, h = oracle_newton(c, c.flat_start(), "perturbed", _drule, pfgen.symmetric_shifts(4, 1e-2),
                             max_iter=15)
    assert it is None
    assert 1e-4 < h[-1] < 1e-2 and h[-1] > 0.5 * h[-5]
    # at the heavier load the same step diverges
    c = _case("heavy")
    x, it, h = oracle_newton(c, c.flat_start(), "perturbed", _drule, pfgen.symmetric_shifts(4, 1e-2),
                             max_iter=15)
    assert it is None and h[-1] > 100 * h[0]


class _OracleSolver:
    """Stand-in with the Solver's calls, computing with the oracle on the CPU, to
    test the Newton loop's host logic without a GPU."""

    device = torch.device("cpu")

    def __init__(self, c):
        self.c = c

    def factor(self, values, D, t, precision):
        self.J = sp.csr_matrix((values.numpy(), self.c.col, self.c.row_ptr), shape=(self.c.n, self.c.n))
        self.D, self.t = D.numpy(), list(t)
        self.calls = getattr(self, "calls", 0) + 1
        return self

    def status(self):
        return 0, None, None

    def solve(self, b, sweeps=0):
        return torch.from_numpy(oracle.x_hat(self.J, self.D, self.t, b.numpy()))


def test_library_loop_follows_the_oracle_loop_on_the_cpu():
    import paper_2311_11833_gb300 as pisp
    c = _case("heavy")
    t = pfgen.symmetric_shifts(4, 1e-3)
    fn = lambda v: pfgen.diag_rule(c.n, c.row_ptr, c.col, v)     # noqa: E731
    s = _OracleSolver(c)
    res = pisp.newton(s, c.mismatch, c.jacobian, c.flat_start(), t, fn)
    x, it, h = oracle_newton(c, c.flat_start(), "perturbed", _drule, t)
    assert res.converged and res.iterations == it == s.calls
    np.testing.assert_allclose(res.mismatch, h, rtol=1e-6, atol=1e-12)
    assert np.max(np.abs(res.x - c.x_star)) < 1e-10
    # not converged within the limit: reported, not raised
    res = pisp.newton(s, c.mismatch, c.jacobian, c.flat_start(), t, fn, max_iter=2)
    assert not res.converged and res.iterations == 2 and len(res.mismatch) == 3


def test_library_loop_raises_on_a_failed_factorisation():
    import paper_2311_11833_gb300 as pisp
    c = _case("light")

    class Bad(_OracleSolver):
        def status(self):
            return 4, None, None

    with pytest.raises(pisp.PispError):
        pisp.newton(Bad(c), c.mismatch, c.jacobian, c.flat_start(), [1e-3, -1e-3],
                    lambda v: np.ones(c.n))


@pytest.mark.gpu
@pytest.mark.parametrize("name,precision,sweeps", [("light", "fp64", 0), ("heavy", "fp64", 0),
                                                    ("heavy", "fp32", 2)])
def test_newton_on_the_gpu(name, precision, sweeps):
    """The Newton loop on libpisp: one analysis, a refactorisation per iteration; the
    iteration count is the oracle loop's (within one step: the two solves differ
    by rounding) and the limit is the planted solution."""
    import paper_2311_11833_gb300 as pisp
    c = _case(name)
    t = pfgen.symmetric_shifts(4, 1e-3)
    fn = lambda v: pfgen.diag_rule(c.n, c.row_ptr, c.col, v)     # noqa: E731
    _, it, _ = oracle_newton(c, c.flat_start(), "perturbed", _drule, t)
    s = pisp.Solver(c.n, c.row_ptr, c.col)
    try:
        res = pisp.newton(s, c.mismatch, c.jacobian, c.flat_start(), t, fn,
                          precision=precision, sweeps=sweeps)
    finally:
        s.close()
    assert res.converged and all(v == 0 for v in res.status)
    assert abs(res.iterations - it) <= 1
    assert np.max(np.abs(res.x - c.x_star)) < 1e-9
