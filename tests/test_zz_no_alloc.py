"""The allocation-free entry point against the oracle and the regular path.

pisp_dense_solve_static serves callers that may not allocate device memory
when they call (a budget fixed at start-up, host callbacks or real-time loops
that cannot take cudaMalloc's implicit synchronisation, frameworks that pass
only their own input and output buffers).  It keeps its per-perturbation
solutions in a static device array instead of allocated workspace, so its
answer must equal the oracle's x_hat and that of pisp_factor_perturbed +
pisp_solve on the same system, and it must stay right when the array is
reused by the next call -- also when that call is smaller than the one
before, so that stale entries of the larger call sit beyond the part it
writes.
"""
import ctypes

import numpy as np
import pytest

import oracle
import pfgen
from _parity import entrywise_err

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2311_11833_gb300 as pisp
    return torch, pisp, pisp.load()


def _static_solve(torch, lib, A, D, t, b):
    n, R = b.shape
    At = torch.tensor(A, dtype=torch.float64, device="cuda")
    Dt = torch.tensor(D, dtype=torch.float64, device="cuda")
    bt = torch.tensor(b, dtype=torch.float64, device="cuda")
    x = torch.full((n, R), float("nan"), dtype=torch.float64, device="cuda")
    th = np.ascontiguousarray(t, dtype=np.float64)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.pisp_dense_solve_static(stream, n, ctypes.c_void_p(At.data_ptr()),
                                     ctypes.c_void_p(Dt.data_ptr()), th.ctypes.data_as(ctypes.c_void_p),
                                     len(th), ctypes.c_void_p(bt.data_ptr()), R, ctypes.c_void_p(x.data_ptr()))
    torch.cuda.synchronize()
    return rc, x.cpu().numpy()


def test_static_entry_matches_oracle_and_regular_path_on_consecutive_calls(env):
    torch, pisp, lib = env
    # small, then the largest size the entry point takes, then small again:
    # the third call runs over the larger leftovers of the second
    cases = [(96, 4, 3, 11), (128, 16, 64, 12), (96, 4, 3, 11), (37, 2, 1, 13)]
    for n, K, R, seed in cases:
        inst = pfgen.random_sparse(n, 0.08, seed=seed)
        A = oracle.to_dense(inst)
        t = pfgen.symmetric_shifts(K)
        b = pfgen.rhs(n, R, seed)
        ref = oracle.x_hat(A, inst.D, t, b)
        rc, x = _static_solve(torch, lib, A, inst.D, t, b)
        assert rc == 0
        assert entrywise_err(x, ref) <= TOL64
        # the regular (allocating) entry points on the same system
        s = pisp.Solver(n, inst.row_ptr, inst.col)
        s.factor(torch.tensor(inst.val, device="cuda"), torch.tensor(inst.D, device="cuda"), t, "fp64")
        x_reg = s.solve(torch.tensor(b, device="cuda")).cpu().numpy()
        s.close()
        assert entrywise_err(x, x_reg) <= TOL64


def test_static_entry_rejects_sizes_beyond_its_limits(env):
    torch, pisp, lib = env
    t = pfgen.symmetric_shifts(2)
    n = 129                                   # PISP_STATIC_MAX_N + 1
    rc, _ = _static_solve(torch, lib, np.eye(n), np.ones(n), t, np.ones((n, 1)))
    assert rc == 10                           # PISP_ERR_UNSUPPORTED
    rc, _ = _static_solve(torch, lib, np.eye(4), np.ones(4), t, np.ones((4, 65)))
    assert rc == 10
    rc, _ = _static_solve(torch, lib, np.eye(4), np.ones(4), np.linspace(0.01, 0.17, 17), np.ones((4, 1)))
    assert rc == 10                           # K = 17 > PISP_K_MAX
