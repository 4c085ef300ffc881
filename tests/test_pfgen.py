"""The seeded input generator follows its stated recipe.

Both the CUDA path's tests and the oracle draw their inputs from `pfgen`, so its
recipe (a random recursive spanning tree plus uniform extra lines to mean degree
2.7; r ~ U[0.005, 0.05], x ~ U[0.02, 0.3] pu; |V| ~ U[0.95, 1.05], theta ~ N(0, 0.1)
with theta_slack = 0; one slack, round(0.2 N) PV buses; participation U[0.5, 1.5]
over slack and PV buses, normalised; n = N + N_PQ with every diagonal entry
structurally nonzero) is checked here, with the sizes the workloads are quoted at.
"""
import numpy as np
import pytest

import pfgen


def _connected(N, fr, to):
    root = list(range(N))

    def find(a):
        while root[a] != a:
            root[a] = root[root[a]]
            a = root[a]
        return a

    for a, b in zip(fr.tolist(), to.tolist()):
        root[find(a)] = find(b)
    return len({find(i) for i in range(N)}) == 1


@pytest.mark.parametrize("N,seed", [(30, 1), (300, 1001), (2000, 2001)])
def test_grid_recipe(N, seed):
    n_pv = int(round(0.2 * N))
    fr, to, y, Vm, Va, pv, part = pfgen._grid(np.random.default_rng(seed), N, n_pv)
    assert len(fr) == int(round(1.35 * N))                       # mean degree 2.7
    assert np.all(fr < to)                                        # no self loops, one orientation
    assert len(set(zip(fr.tolist(), to.tolist()))) == len(fr)     # no duplicate lines
    assert _connected(N, fr, to)                                  # the spanning tree is inside
    z = 1.0 / y
    assert np.all((z.real >= 0.005) & (z.real <= 0.05) & (z.imag >= 0.02) & (z.imag <= 0.3))
    assert np.all((Vm >= 0.95) & (Vm <= 1.05)) and Va[0] == 0.0
    assert abs(np.std(Va[1:]) - 0.1) < 0.05
    assert len(pv) == n_pv and 0 not in pv and len(set(pv.tolist())) == n_pv
    on = np.zeros(N, bool)
    on[0] = True
    on[pv] = True
    assert np.all(part[on] > 0) and np.all(part[~on] == 0)
    assert part.sum() == pytest.approx(1.0, rel=1e-14)
    assert part[on].max() / part[on].min() <= 3.0                 # raw draws in [0.5, 1.5]


@pytest.mark.parametrize("wl,n", [("plain", 539), ("precision", 3599), ("differentiation", 2436),
                                   ("scale", 17999)])
def test_workload_sizes_and_diagonal(wl, n):
    inst = pfgen.make_instance(wl)
    N = pfgen.CONFIGS[wl]["N"]
    assert inst.n == n == N + inst.meta["n_pq"]
    assert inst.meta["n_pq"] == N - 1 - int(round(0.2 * N))
    rows = np.repeat(np.arange(inst.n), np.diff(inst.row_ptr))
    diag = inst.col == rows
    assert diag.sum() == inst.n                                   # every diagonal entry present
    assert np.all(inst.val[diag] != 0)
    assert np.all(np.diff(inst.col)[np.diff(rows) == 0] > 0)      # sorted, no duplicates


def test_batch_sizes_and_totals():
    N = pfgen.batch_sizes(pfgen.CONFIGS["batching"]["G"])
    assert len(N) == 256 and N.min() >= 118 and N.max() <= 3000
    n = N + (N - 1 - np.rint(0.2 * N).astype(np.int64))           # N + N_PQ per grid
    assert int(n.sum()) == 400191
    logs = np.log(N)
    assert abs(np.median(logs) - 0.5 * (np.log(118) + np.log(3000))) < 0.3   # log-uniform


def test_perturbation_diagonal_rule():
    inst = pfgen.random_sparse(30, 0.2, seed=3, zero_diag=True)
    A = inst.dense()
    D = pfgen.perturbation_diag(inst)
    d = np.abs(np.diag(A))
    weak = d <= 1e-12 * np.abs(A).max()
    assert np.all(D[~weak] == d[~weak])
    assert np.all(D[weak] == np.where(np.abs(A[weak]).max(axis=1) > 0, np.abs(A[weak]).max(axis=1), 1.0))
    np.testing.assert_array_equal(pfgen.diag_rule(inst.n, inst.row_ptr, inst.col, inst.val), D)


def test_shifts_and_right_hand_sides():
    np.testing.assert_array_equal(pfgen.symmetric_shifts(6, 0.01), [0.01, -0.01, 0.02, -0.02, 0.03, -0.03])
    np.testing.assert_array_equal(pfgen.one_sided_shifts(3, 0.5), [0.5, 1.0, 1.5])
    with pytest.raises(ValueError):
        pfgen.symmetric_shifts(3)
    b = pfgen.rhs(4000, 5, 1)
    assert b.shape == (4000, 5) and abs(b.mean()) < 0.03 and abs(b.std() - 1.0) < 0.03
    np.testing.assert_array_equal(b, pfgen.rhs(4000, 5, 1))      # seeded


def test_instances_are_reproducible():
    a, b = pfgen.make_instance("plain"), pfgen.make_instance("plain")
    for f in ("row_ptr", "col", "val", "D"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    c = pfgen.make_instance("plain", 1)
    assert not (c.nnz == a.nnz and np.array_equal(c.val, a.val))
