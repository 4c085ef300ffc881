"""The Python binding rejects buffers that do not match the analysed pattern before
any call into libpisp: every pointer the library reads or writes is sized from the
pattern (N unknowns, nnz entries, R right-hand sides of the last solve), so a short
buffer would otherwise be read or written past its end."""
import numpy as np
import pytest
import torch

import pfgen


def _shell(N=5, nnz=13, R=2):
    """A Solver object with the sizes of an analysed pattern but no handle (enough
    for the argument checks, which run before any library call)."""
    from paper_2311_11833_gb300.solver import Solver
    s = Solver.__new__(Solver)
    s.device, s.N, s.nnz, s.R, s.G, s.K = 0, N, nnz, R, 1, 0
    s._h = None
    return s


def test_solve_host_checks_host_buffers():
    s = _shell()
    t = [0.01, -0.01]
    with pytest.raises(ValueError):
        s.solve_host(np.zeros(12), np.zeros(5), t, np.zeros(5))         # values short
    with pytest.raises(ValueError):
        s.solve_host(np.zeros(13), np.zeros(4), t, np.zeros(5))         # D short
    with pytest.raises(ValueError):
        s.solve_host(np.zeros(13), np.zeros(5), t, np.zeros((5, 2)), out=np.zeros(5))
    with pytest.raises(TypeError):
        s.solve_host(np.zeros(13), np.zeros(5), t, np.zeros(5), out=np.zeros(5, np.float32))
    with pytest.raises(TypeError):
        s.solve_host(np.zeros(13), np.zeros(5), t, np.zeros((5, 2)), out=np.zeros((2, 5)).T)


def test_device_buffers_must_be_cuda_float64():
    s = _shell()
    with pytest.raises(TypeError):
        s.solve(torch.zeros(5, dtype=torch.float64))                     # host tensor
    with pytest.raises(TypeError):
        s._dev_out(torch.zeros(10, dtype=torch.float64), "out", 10)


def test_solver_rejects_a_short_column_array():
    from paper_2311_11833_gb300.solver import Solver
    if not torch.cuda.is_available():
        with pytest.raises(RuntimeError):                               # no CPU fallback
            Solver(2, [0, 1, 2], [0, 1])
    else:
        with pytest.raises(ValueError):
            Solver(2, [0, 1, 2], [0])


@pytest.mark.gpu
def test_device_buffers_are_sized_from_the_pattern():
    import paper_2311_11833_gb300 as pisp
    inst = pfgen.random_sparse(9, 0.3, seed=4)
    s = pisp.Solver(inst.n, inst.row_ptr, inst.col)
    dev = "cuda"
    s.factor(torch.tensor(inst.val, device=dev), torch.tensor(inst.D, device=dev),
             pfgen.symmetric_shifts(2), "fp64")
    b = torch.tensor(pfgen.rhs(9, 2, 1), device=dev)
    with pytest.raises(ValueError):
        s.solve(b, out=torch.empty(17, dtype=torch.float64, device=dev))   # 9 x 2 needed
    with pytest.raises(ValueError):
        s.solve(b, out=torch.empty((2, 9), dtype=torch.float64, device=dev).t())  # not contiguous
    x = s.solve(b)
    with pytest.raises(ValueError):
        s.refine(b, x[:, :1].contiguous())
    with pytest.raises(ValueError):
        s.adjoint(torch.zeros((9, 3), dtype=torch.float64, device=dev))    # last solve had R = 2
    with pytest.raises(ValueError):
        s.combine(out=torch.empty(9, dtype=torch.float64, device=dev))
    gb, gv = s.adjoint(torch.zeros((9, 2), dtype=torch.float64, device=dev))
    assert gb.shape == (9, 2) and gv.shape == (inst.nnz,)
    # a refine with more right-hand sides than the last solve may reallocate the
    # kept per-perturbation solutions: combine then refuses instead of reading them
    b3 = torch.tensor(pfgen.rhs(9, 3, 2), device=dev)
    s.refine(b3, torch.zeros((9, 3), dtype=torch.float64, device=dev))
    with pytest.raises(pisp.PispError):
        s.combine()
    s.close()
