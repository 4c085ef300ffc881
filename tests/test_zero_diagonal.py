"""Next row f3: a zero diagonal (Sec. IV: the pivot-free solve of the unperturbed
Jacobian returned NaN/Inf because a zero was met on the diagonal; a Hopcroft-Karp row
permutation was tried as a comparison).

Two zero-diagonal cases are built from the 300-bus Jacobian:

* swapped: the P equations of two non-adjacent buses trade places, so exactly two
  diagonal entries are structurally zero.  In the solver's fill-reducing order one of
  them reaches its pivot untouched (an exact zero pivot); the perturbed systems are
  pivot-free factorable with element growth O(1/eps), and their combination converges
  to A^{-1} b as eps^K (the product of the shifts in the error identity).
* lambda-first: the slack-participation unknown lambda is ordered first, which moves
  every diagonal entry but a few off the diagonal.  Perturbation does not rescue this
  one (the perturbed pivot-free factors grow past 1e12); the row matching does.

CPU tests pin the row matching (pisp_match_rows) against scipy's maximum bipartite
matching and the matrix-level facts with the oracle, in the order the solver's own
analysis picks; the GPU test checks on the swapped case that (a) the unperturbed
pivot-free factorisation reports a zero pivot and NaN, (b) the perturbed method gives
the oracle's x_hat and A^{-1} b, and (c) after the row matching the unperturbed
pivot-free solve gives A^{-1} b.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import maximum_bipartite_matching

import oracle
import pfgen
from _parity import entrywise_err
from test_abi import HostSymbolic

SWAP = (342, 456)     # P-equation rows of two non-adjacent buses of the 300-bus case


def _swapped():
    A = oracle.to_scipy(pfgen.make_instance("plain")).tocsr()
    p = np.arange(A.shape[0])
    p[SWAP[0]], p[SWAP[1]] = SWAP[1], SWAP[0]
    M = A[p, :].tocsr()
    M.sort_indices()
    return M


def _lambda_first():
    inst = pfgen.make_instance("plain")
    A = oracle.to_scipy(inst).tocsc()
    n = inst.n
    colperm = np.concatenate([[n - 1], np.arange(n - 1)])
    Ap = A[:, colperm].tocsr()
    Ap.sort_indices()
    return Ap


def _zero_diag_rule(M):
    """D: |A_ii| where the diagonal is nonzero, else the largest magnitude of row i
    (the generator's rule, applied to a sorted CSR matrix)."""
    return pfgen.diag_rule(M.shape[0], M.indptr, M.indices, M.data)


def _solver_order(lib, M):
    hs = HostSymbolic(lib, [M.shape[0]], M.indptr.astype(np.int64), M.indices.astype(np.int32))
    try:
        assert hs.rc == 0
        return hs.perm.copy()
    finally:
        hs.close()


@pytest.fixture(scope="module")
def pisp():
    import paper_2311_11833_gb300 as p
    p.load()
    return p


@pytest.fixture(scope="module")
def lib(pisp):
    import paper_2311_11833_gb300._lib as L
    return L.load()


def test_swapped_rows_meet_a_zero_pivot_in_the_solver_order(lib):
    M = _swapped()
    A = oracle.to_scipy(pfgen.make_instance("plain"))
    a, b = SWAP
    assert A[a, b] == 0 and A[b, a] == 0                      # the buses are not adjacent
    assert np.flatnonzero(M.diagonal() == 0).tolist() == [a, b]
    with pytest.raises(ZeroDivisionError):
        oracle.pivot_free_lu(M, np.zeros(M.shape[0]), 0.0, _solver_order(lib, M))


def test_perturbation_rescues_the_swapped_rows(lib):
    """Each perturbed system is pivot-free factorable in the solver order with growth
    O(1/eps), and x_hat approaches A^{-1} b as eps^K, K = 4 (the error identity of
    the Neumann expansion carries the product of the shifts)."""
    M = _swapped()
    n = M.shape[0]
    perm = _solver_order(lib, M)
    D = _zero_diag_rule(M)
    b = pfgen.rhs(n, 1, 7)
    xs = oracle.x_star(M, b)
    err = {}
    for eps in (1e-2, 1e-4):
        t = pfgen.symmetric_shifts(4, eps)
        for tk in t:
            _, U = oracle.pivot_free_lu(M, D, tk, perm)
            growth = np.abs(U).max() / abs(M).max()
            assert growth < 0.2 / eps
        err[eps] = float(np.max(oracle.rel_err(oracle.x_hat(M, D, t, b), xs)))
    assert 1e-3 < err[1e-2] < 5e-2
    assert err[1e-4] < 1e-9


def test_lambda_first_has_zero_diagonal_and_fails_pivot_free(lib):
    Ap = _lambda_first()
    assert Ap[0, 0] == 0 and np.count_nonzero(Ap.diagonal()) < 10
    with pytest.raises(ZeroDivisionError):
        oracle.pivot_free_lu(Ap, np.zeros(Ap.shape[0]), 0.0)
    # the perturbation leaves pivots of size eps, but with nearly every diagonal
    # entry zero their reciprocals compound: the factor is useless
    _, U = oracle.pivot_free_lu(Ap, _zero_diag_rule(Ap), 1e-2, _solver_order(lib, Ap))
    assert np.abs(U).max() / abs(Ap).max() > 1e12


@pytest.mark.parametrize("case", ["swapped", "lambda_first"])
def test_match_rows_gives_a_pivot_free_factorable_matrix(pisp, lib, case):
    Ap = _swapped() if case == "swapped" else _lambda_first()
    n = Ap.shape[0]
    rp = pisp.match_rows(n, Ap.indptr, Ap.indices)
    assert sorted(rp.tolist()) == list(range(n))
    M = Ap[rp, :]
    assert np.count_nonzero(M.diagonal()) == n
    # the CSR helper builds the same matrix
    ptr, col, val = pisp.permute_rows(Ap.indptr, Ap.indices, Ap.data, rp)
    M2 = sp.csr_matrix((val, col, ptr), shape=(n, n))
    assert (M2 != M).nnz == 0
    # and the matched matrix is pivot-free factorable in the solver order
    M2.sort_indices()
    L, U = oracle.pivot_free_lu(M2, np.zeros(n), 0.0, _solver_order(lib, M2))
    assert np.all(np.isfinite(U)) and np.min(np.abs(np.diag(U))) > 1e-3


@pytest.mark.parametrize("seed", range(6))
def test_match_rows_size_matches_scipy(pisp, seed):
    rng = np.random.default_rng(seed)
    n = 40
    M = sp.random(n, n, density=0.06, random_state=rng, format="csr")
    M.sort_indices()
    ref = maximum_bipartite_matching(M, perm_type="row")   # row matched to each column, -1 if none
    full = bool(np.all(ref >= 0))
    if full:
        rp = pisp.match_rows(n, M.indptr, M.indices)
        assert sorted(rp.tolist()) == list(range(n))
        assert all(M[rp[c], c] != 0 for c in range(n))
    else:
        with pytest.raises(pisp.PispError):
            pisp.match_rows(n, M.indptr, M.indices)


@pytest.mark.parametrize("seed", range(8))
def test_match_rows_on_planted_matchings(pisp, seed):
    """Larger patterns: a random permutation (a perfect matching that the diagonal
    does not show) plus random entries, and the same with one column emptied
    (structurally singular); the result is checked against scipy's matching size."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(200, 3000))
    perm = rng.permutation(n)
    extra = sp.random(n, n, density=3.0 / n, random_state=rng, format="csr")
    M = (sp.csr_matrix((np.ones(n), (perm, np.arange(n))), shape=(n, n)) + extra).tocsr()
    M.sort_indices()
    rp = pisp.match_rows(n, M.indptr, M.indices)
    assert sorted(rp.tolist()) == list(range(n))
    assert np.all(np.asarray(M[rp, :].todense()).diagonal() != 0)
    M = M.tolil()
    M[:, int(rng.integers(n))] = 0
    M = M.tocsr()
    M.eliminate_zeros()
    M.sort_indices()
    assert np.any(maximum_bipartite_matching(M, perm_type="row") < 0)
    with pytest.raises(pisp.PispError):
        pisp.match_rows(n, M.indptr, M.indices)


def test_match_rows_rejects_bad_patterns(pisp):
    with pytest.raises(pisp.PispError):
        pisp.match_rows(2, [0, 1, 1], [0])            # empty row: no full matching
    with pytest.raises(pisp.PispError):
        pisp.match_rows(2, [0, 1, 2], [0, 5])         # column out of range
    assert len(pisp.match_rows(0, [0], [])) == 0
    with pytest.raises(ValueError):
        pisp.match_rows(3, [0, 1, 2], [0, 1])         # row_ptr too short for n
    with pytest.raises(ValueError):
        pisp.match_rows(2, [0, 1, 3], [0, 1])         # col shorter than row_ptr[n]


@pytest.mark.gpu
def test_zero_diagonal_on_the_gpu(pisp):
    import torch
    M = _swapped()
    n = M.shape[0]
    b = pfgen.rhs(n, 1, 7)
    xs = oracle.x_star(M, b)
    dev = "cuda"
    vals = torch.tensor(M.data, device=dev)
    # (a) unperturbed pivot-free: a zero pivot is reported and x is NaN
    s = pisp.Solver(n, M.indptr, M.indices)
    s.factor(vals, torch.zeros(n, dtype=torch.float64, device=dev), [0.0], "fp64")
    worst, codes, _ = s.status()
    assert worst in (4, 5)
    assert np.all(np.isnan(s.solve(torch.tensor(b, device=dev)).cpu().numpy()))
    # (b) perturbed (zero diagonal entries of D take the row's largest entry): every
    # perturbed factorisation is pivot-free, x is the oracle's x_hat, and at
    # eps = 1e-4 that is A^{-1} b.  A pivot-free solve in this order differs from the
    # oracle's x_hat by 5e-14 in fp64 (growth 1.2e3, cond 2.6e3).
    D = _zero_diag_rule(M)
    t = pfgen.symmetric_shifts(4, 1e-4)
    s.factor(vals, torch.tensor(D, device=dev), t, "fp64")
    assert s.status()[0] == 0
    x = s.solve(torch.tensor(b, device=dev)).cpu().numpy()
    assert entrywise_err(x, oracle.x_hat(M, D, t, b)) <= 1e-10
    assert entrywise_err(x, xs) <= 1e-9
    s.close()
    # (c) rows matched: the unperturbed pivot-free solve gives A^{-1} b
    rp = pisp.match_rows(n, M.indptr, M.indices)
    ptr, col, val = pisp.permute_rows(M.indptr, M.indices, M.data, rp)
    s = pisp.Solver(n, ptr, col)
    s.factor(torch.tensor(val, device=dev), torch.zeros(n, dtype=torch.float64, device=dev), [0.0], "fp64")
    assert s.status()[0] == 0
    x = s.solve(torch.tensor(b[rp], device=dev)).cpu().numpy()
    assert entrywise_err(x, xs) <= 1e-10
    s.close()
