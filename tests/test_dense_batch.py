"""Next row f4: dense batched systems (the paper's own measurement, Sec. IV and
Fig. 2, uses dense batched LU and triangular solves).

The library needs no separate dense path: a dense instance analyses to a single
root front of size n with no update rows, so G dense instances of any sizes are G
fronts of one level, factored for all K shifts in the same launches (shared-memory
fronts up to 160 columns in FP64 and 224 in FP32, column-block owner tiles above)
and solved by the same persistent solve.  The test family is Gaussian with a
diagonal of +-2 sqrt(n): diagonally dominant enough that the pivot-free LU has
growth near 1 (kappa_1 <= 93, rho(A^{-1} D) about 1.5 for n <= 300).
"""
import numpy as np
import pytest

import oracle
import pfgen
from _parity import entrywise_err
from test_abi import HostSymbolic

SIZES = (1, 7, 64, 150, 300)


def _dense(n):
    return pfgen.random_sparse(n, 1.0, seed=n, diag_boost=2.0 * np.sqrt(n))


def _concat(insts):
    rp, cols, off = [0], [], 0
    for I in insts:
        rp.extend((I.row_ptr[1:] + rp[-1]).tolist())
        cols.append(I.col + off)
        off += I.n
    return ([I.n for I in insts], np.array(rp, np.int64), np.concatenate(cols).astype(np.int32),
            np.concatenate([I.val for I in insts]), np.concatenate([I.D for I in insts]))


@pytest.fixture(scope="module")
def lib():
    import paper_2311_11833_gb300._lib as L
    return L.load()


def test_dense_instances_are_one_front_each(lib):
    insts = [_dense(n) for n in SIZES]
    assert all(I.nnz == I.n * I.n for I in insts)
    sizes, rp, col, _, _ = _concat(insts)
    hs = HostSymbolic(lib, sizes, rp, col)
    try:
        assert hs.rc == 0
        assert hs.stats["n_supernodes"] == len(SIZES) and hs.stats["n_levels"] == 1
        assert list(hs.c1 - hs.c0) == list(SIZES) and np.all(hs.ms == 0)
        assert hs.stats["max_front"] == max(SIZES)
    finally:
        hs.close()


def test_dense_family_is_safe_without_pivoting():
    t = pfgen.symmetric_shifts(4)
    for n in SIZES:
        I = _dense(n)
        A = oracle.to_dense(I)
        assert oracle.cond1(A) < 100
        assert max(oracle.pivot_stats(A, I.D, tk)[0] for tk in t) < 1.1
        assert oracle.spectral_radius(A, I.D) < 2.0


@pytest.mark.gpu
@pytest.mark.parametrize("precision,sweeps,opts,extra", [
    ("fp64", 0, {}, ()), ("fp32", 2, {}, ()),
    # one launch, owner-tile updates on the tensor cores, with the paper's n = 531
    ("fp32", 2, dict(factor_policy=4, factor_tc=1), (531,))])
def test_dense_batch_on_the_gpu(precision, sweeps, opts, extra):
    import torch
    import paper_2311_11833_gb300 as pisp
    insts = [_dense(n) for n in SIZES + extra]
    sizes, rp, col, val, D = _concat(insts)
    t = pfgen.symmetric_shifts(4)
    R = 3
    N = sum(sizes)
    b = pfgen.rhs(N, R, 5)
    s = pisp.Solver(sizes, rp, col, **opts)
    try:
        s.factor(torch.tensor(val, device="cuda"), torch.tensor(D, device="cuda"), t, precision)
        assert s.status()[0] == 0
        x = s.solve(torch.tensor(b, device="cuda"), sweeps=sweeps).cpu().numpy()
    finally:
        s.close()
    off = 0
    for I in insts:
        ref = oracle.x_hat(oracle.to_scipy(I), I.D, t, b[off:off + I.n])
        assert entrywise_err(x[off:off + I.n], ref) <= 1e-10
        off += I.n
