"""CPU checks of the C ABI library: symbols, host helpers, symbolic structure.

No GPU compute happens here; the symbolic phase runs on a host-only handle
(device -1).
"""
import ctypes

import numpy as np
import pytest

import oracle
import pfgen


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2311_11833_gb300 as pisp
    return pisp.load()


def test_exports_every_header_symbol(lib):
    import paper_2311_11833_gb300 as pisp
    names = pisp.header_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []


@pytest.mark.parametrize("t", [pfgen.symmetric_shifts(4), pfgen.symmetric_shifts(6),
                               pfgen.one_sided_shifts(4), pfgen.symmetric_shifts(8, 3e-3),
                               np.array([0.5]), np.array([-0.01, 0.03, 0.07])])
def test_weights_match_oracle(lib, t):
    import paper_2311_11833_gb300 as pisp
    got = pisp.weights(t)
    ref = oracle.weights_float(list(t))
    np.testing.assert_allclose(got, ref, rtol=1e-14, atol=1e-15)


def test_weights_reject_bad_shifts(lib):
    import paper_2311_11833_gb300 as pisp
    with pytest.raises(pisp.PispError):
        pisp.weights([0.01, 0.01])
    with pytest.raises(pisp.PispError):
        pisp.weights([])


class HostSymbolic:
    """A host-only handle (device -1) for structure checks."""

    def __init__(self, lib, sizes, row_ptr, col, **opt):
        from paper_2311_11833_gb300._lib import PispOptions, PispStats
        self.lib = lib
        self.h = ctypes.c_void_p()
        assert lib.pisp_create(ctypes.byref(self.h), -1, None) == 0
        sizes = np.asarray(sizes, np.int32)
        rp = np.ascontiguousarray(row_ptr, np.int64)
        cl = np.ascontiguousarray(col, np.int32)
        o = PispOptions(opt.get("ordering", 0), opt.get("relax_small", -1), opt.get("relax_zeros", -1.0), 0, 0,
                        0, 0, 0, 0, 0, 0, opt.get("analyze_threads", 0))
        self.rc = lib.pisp_analyze(self.h, len(sizes), sizes.ctypes.data_as(ctypes.c_void_p),
                                   rp.ctypes.data_as(ctypes.c_void_p), cl.ctypes.data_as(ctypes.c_void_p),
                                   ctypes.byref(o))
        self.N = int(sizes.sum())
        if self.rc == 0:
            st = PispStats()
            assert lib.pisp_get_stats(self.h, ctypes.byref(st)) == 0
            self.stats = st.as_dict()
            self.perm = np.zeros(self.N, np.int32)
            assert lib.pisp_get_perm(self.h, self.perm.ctypes.data_as(ctypes.c_void_p)) == 0
            S = self.stats["n_supernodes"]
            self.c0, self.c1, self.ms = (np.zeros(S, np.int32) for _ in range(3))
            assert lib.pisp_get_supernodes(self.h, self.c0.ctypes.data_as(ctypes.c_void_p),
                                           self.c1.ctypes.data_as(ctypes.c_void_p),
                                           self.ms.ctypes.data_as(ctypes.c_void_p), None) == 0
            self.rows = np.zeros(int(self.ms.sum()), np.int32)
            assert lib.pisp_get_supernodes(self.h, None, None, None,
                                           self.rows.ctypes.data_as(ctypes.c_void_p)) == 0

    def close(self):
        self.lib.pisp_destroy(self.h)

    def pattern(self):
        """Dense boolean pattern of L + U implied by the supernodes (permuted)."""
        P = np.zeros((self.N, self.N), bool)
        off = 0
        for a, b, m in zip(self.c0, self.c1, self.ms):
            idx = np.concatenate([np.arange(a, b), self.rows[off:off + m]])
            off += m
            for c in range(a, b):
                below = idx[idx >= c]
                P[below, c] = True
                P[c, below] = True
        return P


def _concat(insts):
    rp, cols, off = [0], [], 0
    for I in insts:
        rp.extend((I.row_ptr[1:] + rp[-1]).tolist())
        cols.append(I.col + off)
        off += I.n
    return [I.n for I in insts], np.array(rp, np.int64), np.concatenate(cols).astype(np.int32)


@pytest.mark.parametrize("case", ["plain", "random12", "random40", "batch3"])
def test_symbolic_covers_pivot_free_fill(lib, case):
    """Every nonzero of the pivot-free L and U lies inside the supernodal pattern."""
    if case == "plain":
        insts = [pfgen.make_instance("plain")]
    elif case == "batch3":
        insts = [pfgen.random_sparse(n, 0.2, seed=n) for n in (7, 1, 23)]
    else:
        n = int(case[6:])
        insts = [pfgen.random_sparse(n, 0.15, seed=n)]
    sizes, rp, col = _concat(insts)
    hs = HostSymbolic(lib, sizes, rp, col)
    assert hs.rc == 0
    try:
        N = hs.N
        perm = hs.perm
        assert sorted(perm.tolist()) == list(range(N))
        # permutation stays inside each instance block
        off = 0
        for n in sizes:
            assert set(perm[off:off + n].tolist()) == set(range(off, off + n))
            off += n
        # supernodes tile the columns, rows sorted and below the pivot block
        assert hs.c0[0] == 0 and hs.c1[-1] == N
        assert np.all(hs.c1[:-1] == hs.c0[1:]) and np.all(hs.c1 > hs.c0)
        off = 0
        for a, b, m in zip(hs.c0, hs.c1, hs.ms):
            r = hs.rows[off:off + m]
            off += m
            assert np.all(np.diff(r) > 0) and (m == 0 or r[0] >= b)
        pattern = hs.pattern()
        from scipy.sparse import block_diag
        A = block_diag([oracle.to_scipy(I) for I in insts]).toarray()
        D = np.concatenate([I.D for I in insts])
        L, U = oracle.pivot_free_lu(A, D, 0.01, perm)
        nz = (np.abs(np.tril(L, -1)) > 0) | (np.abs(np.triu(U)) > 0)
        assert not np.any(nz & ~pattern)
        assert hs.stats["nnzL"] >= np.count_nonzero(np.tril(L, -1))
    finally:
        hs.close()


def test_symbolic_natural_ordering_and_relaxation(lib):
    inst = pfgen.make_instance("plain")
    hs = HostSymbolic(lib, [inst.n], inst.row_ptr, inst.col, ordering=1)
    # the given order is only postordered on its elimination tree: same fill
    A = oracle.to_dense(inst)
    L, _ = oracle.pivot_free_lu(A, inst.D, 0.01)
    nzl = np.count_nonzero(np.tril(L, -1))
    assert hs.rc == 0 and nzl <= hs.stats["nnzL"] <= 1.01 * nzl   # symmetrised structure
    md = HostSymbolic(lib, [inst.n], inst.row_ptr, inst.col)
    assert md.stats["nnzL"] < 0.2 * hs.stats["nnzL"]                # the ordering matters
    md.close()
    hs.close()
    a = HostSymbolic(lib, [inst.n], inst.row_ptr, inst.col, relax_small=1, relax_zeros=0.0)
    b = HostSymbolic(lib, [inst.n], inst.row_ptr, inst.col, relax_small=16, relax_zeros=0.3)
    # relaxed amalgamation: fewer, larger supernodes, same exact fill
    assert b.stats["n_supernodes"] < a.stats["n_supernodes"]
    assert a.stats["nnzL"] == b.stats["nnzL"]
    assert b.stats["nnzF_stored"] >= a.stats["nnzF_stored"]
    a.close()
    b.close()


def test_symbolic_fill_is_reasonable(lib):
    """The minimum-degree ordering keeps fill near that of a library ordering."""
    import scipy.sparse.linalg as sla
    inst = pfgen.make_instance("precision")
    hs = HostSymbolic(lib, [inst.n], inst.row_ptr, inst.col)
    A = oracle.to_scipy(inst).tocsc()
    lu = sla.splu(A, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                  options=dict(SymmetricMode=True))
    assert hs.stats["nnzL"] <= 1.3 * (lu.L.nnz - inst.n)
    assert hs.stats["n_levels"] <= 20
    hs.close()


def test_analyze_rejects_bad_patterns(lib):
    h = ctypes.c_void_p()
    assert lib.pisp_create(ctypes.byref(h), -1, None) == 0
    n = np.array([2, 2], np.int32)
    rp = np.array([0, 1, 2, 3, 4], np.int64)
    col = np.array([0, 3, 2, 3], np.int32)      # row 1 points into instance 1
    rc = lib.pisp_analyze(h, 2, n.ctypes.data_as(ctypes.c_void_p), rp.ctypes.data_as(ctypes.c_void_p),
                          col.ctypes.data_as(ctypes.c_void_p), None)
    assert rc == 1 and b"outside" in lib.pisp_last_error(h)
    rp_bad = np.array([0, 2, 1, 3, 4], np.int64)
    rc = lib.pisp_analyze(h, 2, n.ctypes.data_as(ctypes.c_void_p), rp_bad.ctypes.data_as(ctypes.c_void_p),
                          col.ctypes.data_as(ctypes.c_void_p), None)
    assert rc == 1
    # numeric calls on a host-only handle fail cleanly
    t = np.array([0.01])
    assert lib.pisp_factor_perturbed(h, None, None, t.ctypes.data_as(ctypes.c_void_p), 1, 64) != 0
    lo, hi = np.zeros(2), np.zeros(2)
    assert lib.pisp_get_pivot_range(h, lo.ctypes.data_as(ctypes.c_void_p),
                                    hi.ctypes.data_as(ctypes.c_void_p)) == 3      # NOT_FACTORED
    assert lib.pisp_get_pivot_range(None, None, None) == 1
    lib.pisp_destroy(h)


def test_empty_instances_analyze(lib):
    sizes = [0, 3, 0]
    rp = np.array([0, 1, 2, 3], np.int64)
    col = np.array([0, 1, 2], np.int32)
    hs = HostSymbolic(lib, sizes, rp, col)
    assert hs.rc == 0 and hs.stats["N"] == 3 and hs.stats["n_supernodes"] >= 1
    hs.close()


@pytest.mark.parametrize("wl,n,S,levels,max_front,n_wide", [
    ("plain", 539, 114, 7, 50, 0),
    ("precision", 3599, 802, 8, 307, 2),
    ("differentiation", 2436, 564, 8, 225, 1),
    ("scale", 17999, 4033, 11, 1594, 23),
])
def test_workload_structures_are_stable(lib, wl, n, S, levels, max_front, n_wide):
    """The symbolic phase is deterministic on the benchmark patterns: supernodes, levels,
    widest front and the number of fronts wider than the shared-memory path (which decide
    the kernels the factorisation uses) are reproduced exactly, and a second analysis gives
    the same permutation."""
    inst = pfgen.make_instance(wl)
    assert inst.n == n
    a = HostSymbolic(lib, [inst.n], inst.row_ptr, inst.col)
    b = HostSymbolic(lib, [inst.n], inst.row_ptr, inst.col)
    try:
        assert a.rc == 0 and b.rc == 0
        F = (a.c1 - a.c0) + a.ms
        assert len(F) == S == a.stats["n_supernodes"]
        assert a.stats["n_levels"] == levels
        assert a.stats["max_front"] == max_front == F.max()
        assert int((F > 224).sum()) == n_wide
        assert np.array_equal(a.perm, b.perm)
        assert np.array_equal(a.ms, b.ms) and np.array_equal(a.rows, b.rows)
    finally:
        a.close()
        b.close()


def test_analyze_thread_cap_gives_the_same_structure(lib):
    """pisp_options.analyze_threads only changes how many host threads share the
    instances of a batch: 1 thread and the default give the same structure."""
    insts = [pfgen.make_instance("batching", g) for g in range(12)]
    rp, cols, off = [0], [], 0
    for I in insts:
        rp.extend((I.row_ptr[1:] + rp[-1]).tolist())
        cols.append(I.col + off)
        off += I.n
    sizes = [I.n for I in insts]
    rp = np.array(rp, np.int64)
    col = np.concatenate(cols).astype(np.int32)
    a = HostSymbolic(lib, sizes, rp, col)
    b = HostSymbolic(lib, sizes, rp, col, analyze_threads=1)
    assert a.rc == 0 and b.rc == 0
    assert np.array_equal(a.perm, b.perm) and np.array_equal(a.c0, b.c0)
    assert np.array_equal(a.ms, b.ms) and np.array_equal(a.rows, b.rows)
    c = HostSymbolic(lib, sizes, rp, col, analyze_threads=-1)
    assert c.rc == 1                                   # PISP_ERR_INVALID_ARG
    for h in (a, b, c):
        h.close()


def test_refinement_calls_check_their_arguments(lib):
    """pisp_set_refinement takes a finite tol >= 0 (no device needed);
    pisp_refinement_stats reports NOT_FACTORED before any solve."""
    h = ctypes.c_void_p()
    assert lib.pisp_create(ctypes.byref(h), -1, None) == 0
    for bad in (-1e-12, float("nan"), float("inf")):
        assert lib.pisp_set_refinement(h, bad) == 1                     # INVALID_ARG
    assert lib.pisp_set_refinement(h, 0.0) == 0
    assert lib.pisp_set_refinement(h, 1e-12) == 0
    assert lib.pisp_set_refinement(None, 1e-12) == 1
    n = np.array([2], np.int32)
    rp = np.array([0, 1, 2], np.int64)
    col = np.array([0, 1], np.int32)
    assert lib.pisp_analyze(h, 1, n.ctypes.data_as(ctypes.c_void_p), rp.ctypes.data_as(ctypes.c_void_p),
                            col.ctypes.data_as(ctypes.c_void_p), None) == 0
    nsw = np.zeros(1, np.int32)
    work = np.zeros(4)
    assert lib.pisp_refinement_stats(h, nsw.ctypes.data_as(ctypes.c_void_p), work.ctypes.data_as(ctypes.c_void_p),
                                     None, 4) == 3                            # NOT_FACTORED: no solve yet
    assert lib.pisp_refinement_stats(h, None, None, None, -1) == 1
    lib.pisp_destroy(h)
