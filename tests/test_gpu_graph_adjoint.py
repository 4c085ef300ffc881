"""GPU tests of the library-owned CUDA graph, the bounded waits and the
FP32 adjoint.

* The graph: the timed path of the benchmark is a replay of the step that
  pisp_graph_capture recorded (factor, solve, sweeps, combine).  A replay
  reads the current contents of the captured buffers, so new values, D and
  b copied into them must give the oracle's x_hat for the NEW inputs (Sec. I
  batch solving; Alg. 1 run again on new values, as in Newton-Raphson).
* The waits: a dependency that can never be met must end in
  PISP_ERR_TIMEOUT from pisp_get_status, with the launch returning.
* The adjoint: with FP32 factors and FP64 sweeps on the transposed systems,
  dL/db and dL/dA reach the FP64 definition (derivative of Eq. x_star), and
  they match central differences of the FP64 forward on the 1354-bus case.
"""
import numpy as np
import pytest

import oracle
import pfgen
from _parity import entrywise_err, grad_entrywise_err

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module")
def pisp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2311_11833_gb300 as p
    return p


def _dev(a):
    import torch
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def _concat(insts):
    rp, cols, vals, off = [0], [], [], 0
    for I in insts:
        rp.extend((I.row_ptr[1:] + rp[-1]).tolist())
        cols.append(I.col + off)
        vals.append(I.val)
        off += I.n
    return ([I.n for I in insts], np.array(rp, np.int64), np.concatenate(cols).astype(np.int32),
            np.concatenate(vals), np.concatenate([I.D for I in insts]))


def _with_values(I, val):
    return pfgen.Instance(n=I.n, row_ptr=I.row_ptr, col=I.col, val=val, D=None, meta={})


# ------------------------------------------------------------------ graph --
def test_graph_replay_with_new_inputs_matches_oracle_batching_config(pisp):
    """All 256 grids, FP32 factors + 3 sweeps, captured once; the replay runs on
    new values (a 1 % perturbation of every entry), a new D from them and a new
    b, copied into the captured buffers; sampled instances against the oracle."""
    import torch
    c = pfgen.CONFIGS["batching"]
    insts = [pfgen.make_instance("batching", g) for g in range(c["G"])]
    t = pfgen.symmetric_shifts(c["K"])
    sizes, rp, col, val, D = _concat(insts)
    N = sum(sizes)
    s = pisp.Solver(sizes, rp, col)
    vals_d, D_d = _dev(val), _dev(D)
    b0 = pfgen.rhs(N, c["R"], 3)
    b_d = _dev(b0)
    x_d = torch.empty_like(b_d)
    s.graph_capture(vals_d, D_d, t, b_d, x_d, precision="fp32", sweeps=3)
    # new inputs, in place
    rng = np.random.default_rng(17)
    val2 = val * (1.0 + 0.01 * rng.standard_normal(val.size))
    offs = np.concatenate([[0], np.cumsum(sizes)])
    noff = np.concatenate([[0], np.cumsum([I.nnz for I in insts])])
    new_insts = []
    for g, I in enumerate(insts):
        J = _with_values(I, val2[noff[g]:noff[g + 1]])
        J.D = pfgen.perturbation_diag(J)
        new_insts.append(J)
    D2 = np.concatenate([J.D for J in new_insts])
    b2 = pfgen.rhs(N, c["R"], 4)
    vals_d.copy_(_dev(val2))
    D_d.copy_(_dev(D2))
    b_d.copy_(_dev(b2))
    x_d.fill_(float("nan"))
    for _ in range(2):                       # two replays in a row
        s.graph_launch()
    torch.cuda.synchronize()
    assert s.status()[0] == 0
    x = x_d.cpu().numpy()
    assert np.all(np.isfinite(x))
    for g in (0, 31, 128, 200, 255):
        J = new_insts[g]
        sl = slice(offs[g], offs[g + 1])
        ref = oracle.x_hat(oracle.to_scipy(J), J.D, t, b2[sl])
        assert entrywise_err(x[sl], ref) <= TOL64, g
    # an eager call invalidates the graph (it may rebuild what the graph uses)
    s.factor(vals_d, D_d, t, "fp32")
    with pytest.raises(pisp.PispError):
        s.graph_launch()
    s.close()


def test_graph_replay_with_adjoint_matches_oracle(pisp):
    """A captured step with the adjoint (FP64): replays on new b and g."""
    import torch
    inst = pfgen.make_instance("plain")
    t = pfgen.symmetric_shifts(4)
    R = 3
    s = pisp.Solver(inst.n, inst.row_ptr, inst.col)
    vals_d, D_d = _dev(inst.val), _dev(inst.D)
    b_d, g_d = _dev(pfgen.rhs(inst.n, R, 1)), _dev(pfgen.rhs(inst.n, R, 2))
    x_d, gb_d = torch.empty_like(b_d), torch.empty_like(b_d)
    gv_d = torch.empty_like(vals_d)
    s.graph_capture(vals_d, D_d, t, b_d, x_d, precision="fp64", g=g_d, out_b=gb_d, out_values=gv_d)
    b2, W2 = pfgen.rhs(inst.n, R, 5), pfgen.rhs(inst.n, R, 6)
    b_d.copy_(_dev(b2))
    g_d.copy_(_dev(W2))
    s.graph_launch()
    torch.cuda.synchronize()
    A = oracle.to_scipy(inst)
    assert entrywise_err(x_d.cpu().numpy(), oracle.x_hat(A, inst.D, t, b2)) <= TOL64
    rb, rv = oracle.adjoint(A, inst.D, t, b2, W2)
    assert entrywise_err(gb_d.cpu().numpy(), rb) <= TOL64
    assert grad_entrywise_err(gv_d.cpu().numpy(), rv) <= TOL64
    s.close()


# ------------------------------------------------------------------ waits --
def test_wait_that_cannot_be_met_reports_timeout(pisp):
    """A completion target raised beyond reach: the waits on it give up after
    the poll limit, the launch returns and pisp_get_status says TIMEOUT; with
    the true targets back, the next factorisation and solve are correct."""
    import time
    import torch
    inst = pfgen.make_instance("precision")
    t = pfgen.symmetric_shifts(4)
    b = pfgen.rhs(inst.n, 2, 3)
    s = pisp.Solver(inst.n, inst.row_ptr, inst.col)
    vals_d, D_d, b_d = _dev(inst.val), _dev(inst.D), _dev(b)
    s.factor(vals_d, D_d, t, "fp64")
    s.set_wait_limit(polls=2000, unreachable=True)
    t0 = time.perf_counter()
    s.solve(b_d)
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 30.0       # every wait ended
    worst, _, _ = s.status()
    assert worst == 6                            # PISP_ERR_TIMEOUT
    s.set_wait_limit(0, False)
    s.factor(vals_d, D_d, t, "fp64")             # clears the record
    x = s.solve(b_d).cpu().numpy()
    assert s.status()[0] == 0
    assert entrywise_err(x, oracle.x_hat(oracle.to_scipy(inst), inst.D, t, b)) <= TOL64
    s.close()


# ---------------------------------------------------------------- adjoint --
def test_fp32_adjoint_with_sweeps_reaches_fp64_differentiation_config(pisp):
    """The 1354-bus workload (K = 4, R = 64) with FP32 factors: forward and
    adjoint sweeps bring x_hat, dL/db and dL/dvalues to the oracle's FP64
    values; without adjoint sweeps the gradients are only FP32-accurate."""
    c = pfgen.CONFIGS["differentiation"]
    inst = pfgen.make_instance("differentiation")
    t = pfgen.symmetric_shifts(c["K"])
    b = pfgen.rhs(inst.n, c["R"], 1)
    W = pfgen.rhs(inst.n, c["R"], 2)
    s = pisp.Solver(inst.n, inst.row_ptr, inst.col)
    s.factor(_dev(inst.val), _dev(inst.D), t, "fp32")
    x = s.solve(_dev(b), sweeps=3).cpu().numpy()
    A = oracle.to_scipy(inst)
    assert entrywise_err(x, oracle.x_hat(A, inst.D, t, b)) <= TOL64
    rb, rv = oracle.adjoint(A, inst.D, t, b, W)
    gb0, gv0 = s.adjoint(_dev(W), sweeps=0)
    e0 = entrywise_err(gb0.cpu().numpy(), rb)
    gb, gv = s.adjoint(_dev(W), sweeps=3)
    assert entrywise_err(gb.cpu().numpy(), rb) <= TOL64
    assert grad_entrywise_err(gv.cpu().numpy(), rv) <= TOL64
    assert e0 > 1e3 * TOL64                      # the sweeps are what closes the gap
    s.close()


def test_autograd_fp32_passes_sweeps_to_the_adjoint(pisp):
    inst = pfgen.make_instance("plain")
    t = pfgen.symmetric_shifts(4)
    R = 2
    s = pisp.Solver(inst.n, inst.row_ptr, inst.col)
    vals = _dev(inst.val).requires_grad_(True)
    b = _dev(pfgen.rhs(inst.n, R, 7)).requires_grad_(True)
    W = pfgen.rhs(inst.n, R, 8)
    x = pisp.solve(s, vals, b, _dev(inst.D), t, "fp32", sweeps=3)
    (x * _dev(W)).sum().backward()
    rb, rv = oracle.adjoint(oracle.to_scipy(inst), inst.D, t, b.detach().cpu().numpy(), W)
    assert entrywise_err(b.grad.cpu().numpy(), rb) <= TOL64
    assert grad_entrywise_err(vals.grad.cpu().numpy(), rv) <= TOL64
    s.close()


def test_central_differences_differentiation_config(pisp):
    """dL/dvalues and dL/db of L = sum(w * x_hat) on the 1354-bus workload
    (K = 4, R = 64, FP64) against central differences of the GPU forward with
    the relative step h = 1e-6 max(1, |a_e|): a random direction over all of
    A's pattern and one over all of b (relative tolerance 1e-5), and 64 sampled
    entries of A and 8 of b.

    A central difference cannot be more accurate than the rounding noise of
    the two losses it subtracts: on this system (rho(A^{-1} D) = 666) that is
    a few 1e-13 of |L| = 1e4 even for the oracle's partial-pivoting LU, which
    is 1e-3 absolute per entry at h = 1e-6.  That noise, delta, is measured as
    the difference between the GPU loss and the oracle's loss at the base
    point, and a sampled entry passes if |fd - g| <= 1e-5 |g| + 10 delta / step."""
    import torch
    c = pfgen.CONFIGS["differentiation"]
    inst = pfgen.make_instance("differentiation")
    t = pfgen.symmetric_shifts(c["K"])
    s = pisp.Solver(inst.n, inst.row_ptr, inst.col)
    vals = _dev(inst.val)
    Dt = _dev(inst.D)
    b_h, w_h = pfgen.rhs(inst.n, c["R"], 1), pfgen.rhs(inst.n, c["R"], 2)
    b, w = _dev(b_h), _dev(w_h)
    s.factor(vals, Dt, t, "fp64")
    x0 = s.solve(b)
    L0 = float((x0 * w).sum())
    gb, gv = s.adjoint(w)
    gb, gv = gb.cpu().numpy(), gv.cpu().numpy()
    L_oracle = float((oracle.x_hat(oracle.to_scipy(inst), inst.D, t, b_h) * w_h).sum())
    delta = max(abs(L0 - L_oracle), 1e-13 * abs(L0))

    def L(v, bb):
        s.factor(v, Dt, t, "fp64")
        return float((s.solve(bb) * w).sum())

    h = 1e-6
    rng = np.random.default_rng(1354)
    # directional derivatives over the whole pattern and the whole of b
    scale = np.maximum(1.0, np.abs(inst.val))
    d = rng.choice([-1.0, 1.0], inst.nnz) * scale
    dd = _dev(d)
    fd = (L(vals + h * dd, b) - L(vals - h * dd, b)) / (2 * h)
    assert abs(fd - gv @ d) <= 1e-5 * abs(gv @ d) + 10 * delta / h
    db = rng.choice([-1.0, 1.0], (inst.n, c["R"]))
    dbt = _dev(db)
    fd = (L(vals, b + h * dbt) - L(vals, b - h * dbt)) / (2 * h)
    assert abs(fd - np.sum(gb * db)) <= 1e-5 * abs(np.sum(gb * db)) + 10 * delta / h
    # sampled entries
    bad = []
    for e in rng.choice(inst.nnz, 64, replace=False):
        step = h * scale[e]
        vp, vm = vals.clone(), vals.clone()
        vp[e] += step
        vm[e] -= step
        fd = (L(vp, b) - L(vm, b)) / (2 * step)
        if abs(fd - gv[e]) > 1e-5 * abs(gv[e]) + 10 * delta / step:
            bad.append((int(e), fd, gv[e]))
    assert not bad, (delta, bad)
    for i, r in rng.integers(0, [inst.n, c["R"]], size=(8, 2)):
        bp, bm = b.clone(), b.clone()
        bp[i, r] += h
        bm[i, r] -= h
        fd = (L(vals, bp) - L(vals, bm)) / (2 * h)
        assert abs(fd - gb[i, r]) <= 1e-5 * abs(gb[i, r]) + 10 * delta / h
    s.close()
    torch.cuda.synchronize()
