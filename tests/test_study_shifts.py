"""Perturbation-strategy study (next row f1): choice of the diagonal D and of the
shift set, and stopping the expansion order m on the residual (the optional residual
check of Alg. 1), on the 300-bus grid.

The CPU tests run the oracle and check what the method itself predicts: the
error falls with m only while the largest shift stays inside the Neumann region,
alpha_max * eps * rho(A^{-1} D) < 1 (Sec. II-B, Theorem 1); with a Gaussian diagonal
and eps = 2e-3 (the paper's perturbation, Sec. IV) rho is small and the error falls
as eps^{2m} to the rounding floor; the symmetric +-alpha*eps set beats the one-sided
set at equal K; stopping m where the residual stops falling picks the m with the
smallest forward error.  The GPU test checks that the library's x_hat equals the
oracle's for the same D choices (including a diagonal with negative entries).
"""
import numpy as np
import pytest

import oracle
import pfgen
from _parity import entrywise_err


def _setup():
    inst = pfgen.make_instance("plain")
    A = oracle.to_scipy(inst)
    b = pfgen.rhs(inst.n, 1, 7)
    diag = np.abs(A.diagonal())
    rng = np.random.default_rng(5)
    strategies = {
        "diag": (inst.D, 1e-2),                               # D = diag|A_ii|
        "identity": (np.full(inst.n, diag.mean()), 1e-2),     # scaled identity
        "gaussian": (rng.standard_normal(inst.n), 2e-3),      # normal diagonal, paper's eps
    }
    return inst, A, b, strategies


def _one_sided(K, eps):
    return np.array([eps * (k + 1) for k in range(K)])


def _errors(A, D, b, xs, shift_sets):
    out = []
    for t in shift_sets:
        xh = oracle.x_hat(A, D, t, b)
        out.append((float(oracle.rel_err(xh, xs)[0]), float(oracle.residual_norm(A, xh, b)[0])))
    return out


def _adaptive_m(residuals):
    """Index of the last order whose residual was still falling (stop at the first rise)."""
    best = 0
    for i in range(1, len(residuals)):
        if residuals[i] >= residuals[i - 1]:
            break
        best = i
    return best


def test_order_helps_only_inside_the_neumann_region():
    inst, A, b, S = _setup()
    xs = oracle.x_star(A, b)
    ms = (1, 2, 3, 4)
    # D = diag|A_ii|: rho = 27, so alpha * eps * rho = 0.27 alpha; m = 4 puts the largest
    # shift outside the region and the error rises again after m = 2
    D, eps = S["diag"]
    rho = oracle.spectral_radius(A, D)
    assert 20 < rho < 35
    e = _errors(A, D, b, xs, [pfgen.symmetric_shifts(2 * m, eps) for m in ms])
    err = [x[0] for x in e]
    assert 4 * eps * rho > 1
    assert err[1] < 0.5 * err[0]
    assert int(np.argmin(err)) == 1 and err[3] > err[1]
    # scaled identity: rho * eps > 1 already for m = 1, no order gives a usable solution
    D, eps = S["identity"]
    assert oracle.spectral_radius(A, D) * eps > 1
    e = _errors(A, D, b, xs, [pfgen.symmetric_shifts(2 * m, eps) for m in ms])
    assert min(x[0] for x in e) > 0.5


def test_gaussian_diagonal_error_falls_as_eps_to_the_2m():
    inst, A, b, S = _setup()
    xs = oracle.x_star(A, b)
    D, eps = S["gaussian"]
    rho = oracle.spectral_radius(A, D)
    assert rho * eps < 0.01
    e = _errors(A, D, b, xs, [pfgen.symmetric_shifts(2 * m, eps) for m in (1, 2, 3)])
    err = [x[0] for x in e]
    # each extra pair of solves gains about (eps * rho)^2 until the rounding floor
    assert err[1] < 1e-3 * err[0]
    assert err[2] < 1e-12


@pytest.mark.parametrize("name", ["diag", "gaussian"])
def test_symmetric_shifts_beat_one_sided(name):
    inst, A, b, S = _setup()
    xs = oracle.x_star(A, b)
    D, eps = S[name]
    for K in (2, 4):
        sym = _errors(A, D, b, xs, [pfgen.symmetric_shifts(K, eps)])[0][0]
        one = _errors(A, D, b, xs, [_one_sided(K, eps)])[0][0]
        assert sym < one


@pytest.mark.parametrize("name", ["diag", "gaussian"])
def test_residual_stop_picks_the_best_order(name):
    inst, A, b, S = _setup()
    xs = oracle.x_star(A, b)
    D, eps = S[name]
    e = _errors(A, D, b, xs, [pfgen.symmetric_shifts(2 * m, eps) for m in (1, 2, 3, 4)])
    err, res = [x[0] for x in e], [x[1] for x in e]
    m_star = _adaptive_m(res)
    assert err[m_star] <= 1.5 * min(err)


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["diag", "identity", "gaussian"])
def test_library_matches_oracle_for_each_strategy(name):
    import torch
    import paper_2311_11833_gb300 as pisp
    inst, A, b, S = _setup()
    D, eps = S[name]
    s = pisp.Solver(inst.n, inst.row_ptr, inst.col)
    dev = "cuda"
    for K in (2, 4, 6):
        t = pfgen.symmetric_shifts(K, eps)
        s.factor(torch.tensor(inst.val, device=dev), torch.tensor(D, device=dev), t, "fp64")
        x = s.solve(torch.tensor(b, device=dev)).cpu().numpy()
        ref = oracle.x_hat(A, D, t, b)
        assert entrywise_err(x, ref) <= 1e-10
    s.close()
