"""The symbolic structure passes its index checks on every pattern the library is run on.

pisp_analyze ends with a check of every index array the kernels follow (assembly
and extend-add maps inside their fronts, offsets equal to prefix sums of the front
sizes, children before parents on lower levels); a failure returns
PISP_ERR_BOUNDS instead of handing the kernels a bad map.  These tests run the
analysis on host-only handles for the benchmark workloads, the patterns of the GPU
tests and random patterns, under every amalgamation setting the autotuner tries and
both orderings, and require every one to pass.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import pfgen
from test_abi import HostSymbolic

RELAX = [(8, 0.05), (4, 0.0), (16, 0.10), (32, 0.20)]


@pytest.fixture(scope="module")
def lib():
    import paper_2311_11833_gb300._lib as L
    return L.load()


def _concat(insts):
    sizes = [I.n for I in insts]
    rps, cols, off, nz = [np.zeros(1, np.int64)], [], 0, 0
    for I in insts:
        rps.append(I.row_ptr[1:] + nz)
        cols.append(I.col + off)
        off += I.n
        nz += I.nnz
    return sizes, np.concatenate(rps), np.concatenate(cols).astype(np.int32)


def _check(lib, insts, **opt):
    sizes, rp, col = _concat(insts)
    hs = HostSymbolic(lib, sizes, rp, col, **opt)
    try:
        assert hs.rc == 0, lib.pisp_last_error(hs.h)
    finally:
        hs.close()


def _csr(M):
    M = M.tocsr()
    M.sort_indices()
    return pfgen.Instance(n=M.shape[0], row_ptr=M.indptr.astype(np.int64), col=M.indices.astype(np.int32),
                          val=M.data.astype(np.float64), D=np.ones(M.shape[0]), meta={})


@pytest.mark.parametrize("rs,rz", RELAX)
@pytest.mark.parametrize("wl", ["plain", "precision", "differentiation", "scale"])
def test_workloads(lib, wl, rs, rz):
    _check(lib, [pfgen.make_instance(wl)], relax_small=rs, relax_zeros=rz)


@pytest.fixture(scope="module")
def batch():
    return [pfgen.make_instance("batching", g) for g in range(pfgen.CONFIGS["batching"]["G"])]


@pytest.mark.parametrize("rs,rz", RELAX)
def test_full_batch(lib, batch, rs, rz):
    _check(lib, batch, relax_small=rs, relax_zeros=rz)


GPU_TEST_PATTERNS = [(1, 1.0, 11), (2, 1.0, 12), (7, 0.4, 17), (33, 0.15, 43), (100, 0.05, 110),
                     (257, 0.02, 267), (64, 0.1, 74), (220, 0.03, 220), (300, 0.03, 300),
                     (700, 0.012, 700), (420, 0.02, 420), (1200, 0.006, 1200), (1200, 0.012, 1200),
                     (2200, 0.008, 2200), (40, 0.1, 8), (30, 0.15, 12), (9, 0.3, 4), (12, 0.3, 5),
                     (5, 0.5, 1), (96, 0.08, 11), (128, 0.08, 12)]


@pytest.mark.parametrize("ordering", [0, 1])
@pytest.mark.parametrize("rs,rz", RELAX)
def test_random_patterns(lib, ordering, rs, rz):
    for n, d, seed in GPU_TEST_PATTERNS:
        _check(lib, [pfgen.random_sparse(n, d, seed=seed)], ordering=ordering, relax_small=rs, relax_zeros=rz)
    rng = np.random.default_rng(rs)
    for _ in range(20):
        n = int(rng.integers(1, 400))
        _check(lib, [pfgen.random_sparse(n, float(rng.uniform(0.0, 0.2)), seed=int(rng.integers(1 << 30)))],
               ordering=ordering, relax_small=rs, relax_zeros=rz)


def test_uneven_batches_and_a_diagonal_instance(lib):
    n = 6
    diag = pfgen.Instance(n=n, row_ptr=np.arange(n + 1, dtype=np.int64), col=np.arange(n, dtype=np.int32),
                          val=np.ones(n), D=np.ones(n), meta={})
    _check(lib, [diag, pfgen.random_sparse(9, 0.3, seed=4)])
    insts = [pfgen.make_instance("batching", g) for g in (1, 3, 5, 9, 13)]
    _check(lib, insts + [pfgen.random_sparse(5, 0.5, seed=3)])


def test_zero_diagonal_and_power_flow_patterns(lib):
    import test_zero_diagonal as zd
    import paper_2311_11833_gb300 as pisp
    for M in (zd._swapped(), zd._lambda_first()):
        _check(lib, [_csr(M)])
        rp = pisp.match_rows(M.shape[0], M.indptr, M.indices)
        _check(lib, [_csr(M[rp, :])])
    for N, npv, seed, a in [(300, 60, 7, 1.0), (300, 60, 12, 1.5)]:
        c = pfgen.power_flow_case(N, npv, seed=seed, angle_scale=a)
        _check(lib, [_csr(sp.csr_matrix((c.jacobian(c.x_star), c.col, c.row_ptr), shape=(c.n, c.n)))])


@pytest.mark.parametrize("wl,fronts,blocks", [("plain", 7, 8), ("precision", 8, 17),
                                               ("differentiation", 8, 15), ("scale", 11, 60)])
def test_critical_chain_of_the_solve(lib, wl, fronts, blocks):
    """Longest leaf-to-root chain of the assembly tree, in fronts and in 32-pivot
    diagonal blocks: the dependency bound of a solve pass."""
    inst = pfgen.make_instance(wl)
    hs = HostSymbolic(lib, [inst.n], inst.row_ptr, inst.col)
    try:
        c0, c1, ms, rows = hs.c0, hs.c1, hs.ms, hs.rows
    finally:
        hs.close()
    S = len(c0)
    owner = np.zeros(inst.n, np.int64)
    for s in range(S):
        owner[c0[s]:c1[s]] = s
    roff = np.concatenate([[0], np.cumsum(ms)])
    depth_f, depth_b = np.zeros(S, np.int64), np.zeros(S, np.int64)
    for s in range(S):                       # children before parents
        depth_f[s] += 1
        depth_b[s] += (c1[s] - c0[s] + 31) // 32
        if ms[s] > 0:
            p = owner[rows[roff[s]]]         # the parent owns the first update row
            depth_f[p] = max(depth_f[p], depth_f[s])
            depth_b[p] = max(depth_b[p], depth_b[s])
    assert (int(depth_f.max()), int(depth_b.max())) == (fronts, blocks)


def test_batch_analysis_equals_instance_by_instance(lib, batch):
    """A batch is analysed on several host threads and merged in instance order:
    every instance's permutation block and supernodes equal those of the same
    instance analysed alone (shifted by its offsets)."""
    insts = batch[:40]
    sizes, rp, col = _concat(insts)
    hb = HostSymbolic(lib, sizes, rp, col)
    try:
        assert hb.rc == 0
        perm, c0, c1, ms, rows = hb.perm, hb.c0, hb.c1, hb.ms, hb.rows
    finally:
        hb.close()
    roff = np.concatenate([[0], np.cumsum(ms)])
    off, s0 = 0, 0
    for inst in insts:
        h1 = HostSymbolic(lib, [inst.n], inst.row_ptr, inst.col)
        try:
            S1 = len(h1.c0)
            np.testing.assert_array_equal(perm[off:off + inst.n], h1.perm + off)
            np.testing.assert_array_equal(c0[s0:s0 + S1], h1.c0 + off)
            np.testing.assert_array_equal(c1[s0:s0 + S1], h1.c1 + off)
            np.testing.assert_array_equal(ms[s0:s0 + S1], h1.ms)
            np.testing.assert_array_equal(rows[roff[s0]:roff[s0 + S1]], h1.rows + off)
        finally:
            h1.close()
        off += inst.n
        s0 += S1
    assert s0 == len(c0)
