"""Seeded synthetic inputs: distributed-slack AC power-flow Jacobians.

This module is the one piece shared by the CUDA path's tests/benchmarks and
the CPU oracle.  It builds *inputs only* (a sparse matrix A in CSR form, the
perturbation diagonal D, right-hand sides and the signed shift list); it holds
none of the perturb / factor / combine arithmetic of the solver.

The workload stands in for the paper's PGLib 300-bus Newton-Raphson Jacobian
(Sec. IV): a reduced distributed-slack power-flow Jacobian J evaluated at a
random (V, theta) point, so that many different Jacobians of one sparsity
pattern can be drawn, as the paper does with "many different V, theta
initializations".  The PGLib data is not available, so the grid itself is
synthetic:

* bus graph: a random recursive spanning tree (bus i attaches to a uniformly
  drawn earlier bus, after a random relabelling) plus uniformly drawn extra
  non-duplicate edges until the mean degree is 2.7 (E = round(1.35 N));
* lines: r ~ U[0.005, 0.05], x ~ U[0.02, 0.3] pu, series admittance 1/(r+jx),
  no line charging and no shunts;
* buses: bus 0 is the slack, round(0.2 N) PV buses, the rest PQ;
  |V| ~ U[0.95, 1.05], theta ~ N(0, 0.1) rad, theta_slack = 0;
* distributed slack: participation factors p_i ~ U[0.5, 1.5] on slack + PV
  buses, normalised to sum 1; the slack mismatch P_i - P_i^spec - p_i*lambda.

Unknowns are ordered [theta_i (i != slack); |V|_i (PQ); lambda] and equations
[P_i (i != slack); Q_i (PQ); P_slack], so every diagonal entry is structurally
nonzero (d P_slack / d lambda = -p_slack).  n = N + N_PQ.

The perturbation matrix is D = diag(|A_ii|); where |A_ii| is negligible
(<= 1e-12 max|A|) the row's largest magnitude is used instead.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Instance", "grid_jacobian", "perturbation_diag", "symmetric_shifts",
    "one_sided_shifts", "rhs", "CONFIGS", "make_instance", "batch_sizes",
    "random_sparse", "csr_to_dense", "PowerFlowCase", "power_flow_case", "diag_rule",
]


@dataclasses.dataclass
class Instance:
    """One sparse system: CSR (row_ptr int64, col int32, val float64), D, meta."""
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    D: np.ndarray
    meta: dict

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def dense(self) -> np.ndarray:
        return csr_to_dense(self.n, self.row_ptr, self.col, self.val)


def csr_to_dense(n, row_ptr, col, val):
    A = np.zeros((n, n), dtype=np.float64)
    for i in range(n):
        s, e = int(row_ptr[i]), int(row_ptr[i + 1])
        A[i, col[s:e]] += val[s:e]
    return A


def _grid(rng: np.random.Generator, N: int, n_pv: int):
    """Random bus graph, line admittances and bus data (see module doc)."""
    relabel = rng.permutation(N)
    # random recursive tree on labels 0..N-1, then relabel
    parents = np.array([rng.integers(0, i) for i in range(1, N)], dtype=np.int64) if N > 1 else np.zeros(0, np.int64)
    edges = set()
    for i in range(1, N):
        a, b = int(relabel[i]), int(relabel[parents[i - 1]])
        edges.add((min(a, b), max(a, b)))
    E_target = int(round(1.35 * N))
    max_edges = N * (N - 1) // 2
    E_target = min(E_target, max_edges)
    while len(edges) < E_target:
        a, b = (int(v) for v in rng.integers(0, N, size=2))
        if a == b:
            continue
        edges.add((min(a, b), max(a, b)))
    edges = sorted(edges)
    fr = np.array([e[0] for e in edges], dtype=np.int64)
    to = np.array([e[1] for e in edges], dtype=np.int64)
    r = rng.uniform(0.005, 0.05, size=len(edges))
    x = rng.uniform(0.02, 0.3, size=len(edges))
    y = 1.0 / (r + 1j * x)
    Vm = rng.uniform(0.95, 1.05, size=N)
    Va = rng.normal(0.0, 0.1, size=N)
    Va[0] = 0.0
    # bus types: 0 = slack, PV drawn among 1..N-1
    pv = np.sort(rng.choice(np.arange(1, N), size=n_pv, replace=False)) if n_pv > 0 else np.zeros(0, np.int64)
    part = np.zeros(N)
    part_buses = np.concatenate([[0], pv]).astype(np.int64)
    part[part_buses] = rng.uniform(0.5, 1.5, size=len(part_buses))
    part /= part.sum()
    return fr, to, y, Vm, Va, pv, part


class _Layout:
    """Unknown and equation indices of the reduced distributed-slack formulation.

    Unknowns [theta_i (i != slack); |V|_i (PQ); lambda], equations
    [P_i (i != slack); Q_i (PQ); P_slack]; -1 marks an entry that does not exist.
    """

    def __init__(self, N: int, pv: np.ndarray):
        is_pv = np.zeros(N, dtype=bool)
        is_pv[pv] = True
        self.N = N
        self.pq = np.array([i for i in range(1, N) if not is_pv[i]], dtype=np.int64)
        self.th_idx = -np.ones(N, dtype=np.int64)
        self.th_idx[1:] = np.arange(N - 1)
        self.vm_idx = -np.ones(N, dtype=np.int64)
        self.vm_idx[self.pq] = (N - 1) + np.arange(len(self.pq))
        self.lam_idx = N - 1 + len(self.pq)
        self.n = self.lam_idx + 1
        self.p_row = -np.ones(N, dtype=np.int64)
        self.p_row[1:] = np.arange(N - 1)
        self.p_row[0] = self.n - 1
        self.q_row = -np.ones(N, dtype=np.int64)
        self.q_row[self.pq] = (N - 1) + np.arange(len(self.pq))


def _admittance(N: int, fr, to, y):
    """Diagonal of the bus admittance matrix and the off-diagonal entries per bus."""
    Ydiag = np.zeros(N, dtype=np.complex128)
    np.add.at(Ydiag, fr, y)
    np.add.at(Ydiag, to, y)
    nbr = [[] for _ in range(N)]          # (j, Y_ij)
    for a, b, yy in zip(fr.tolist(), to.tolist(), y.tolist()):
        nbr[a].append((b, -yy))
        nbr[b].append((a, -yy))
    return Ydiag, nbr


def _injections(Ydiag, nbr, Vm, Va):
    """Complex power injections S_i = V_i * conj(sum_j Y_ij V_j); returns (P, Q)."""
    V = Vm * np.exp(1j * Va)
    I = Ydiag * V
    for i in range(len(Vm)):
        for j, yij in nbr[i]:
            I[i] += yij * V[j]
    S = V * np.conj(I)
    return S.real, S.imag


def _jacobian_csr(lay: _Layout, Ydiag, nbr, part, Vm, Va):
    """Polar power-flow Jacobian at (Vm, Va) as CSR (row_ptr, col, val).

    The pattern depends on the topology only, never on the values.
    """
    N, n = lay.N, lay.n
    P, Q = _injections(Ydiag, nbr, Vm, Va)
    p_row, q_row, th_idx, vm_idx = lay.p_row, lay.q_row, lay.th_idx, lay.vm_idx
    rows = [dict() for _ in range(n)]

    def put(r, c, v):
        if r >= 0 and c >= 0:
            rows[r][c] = rows[r].get(c, 0.0) + v

    for i in range(N):
        Gii, Bii = Ydiag[i].real, Ydiag[i].imag
        # diagonal blocks
        put(p_row[i], th_idx[i], -Q[i] - Bii * Vm[i] ** 2)
        put(p_row[i], vm_idx[i], P[i] / Vm[i] + Gii * Vm[i])
        put(q_row[i], th_idx[i], P[i] - Gii * Vm[i] ** 2)
        put(q_row[i], vm_idx[i], Q[i] / Vm[i] - Bii * Vm[i])
        for j, yij in nbr[i]:
            th = Va[i] - Va[j]
            c, s = math.cos(th), math.sin(th)
            g, b = yij.real, yij.imag
            t1 = g * s - b * c
            t2 = g * c + b * s
            put(p_row[i], th_idx[j], Vm[i] * Vm[j] * t1)
            put(p_row[i], vm_idx[j], Vm[i] * t2)
            put(q_row[i], th_idx[j], -Vm[i] * Vm[j] * t2)
            put(q_row[i], vm_idx[j], Vm[i] * t1)
        if part[i] != 0.0:
            put(p_row[i], lay.lam_idx, -part[i])
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    cols, vals = [], []
    for r in range(n):
        items = sorted(rows[r].items())
        row_ptr[r + 1] = row_ptr[r] + len(items)
        cols.extend(c for c, _ in items)
        vals.extend(v for _, v in items)
    return row_ptr, np.asarray(cols, dtype=np.int32), np.asarray(vals, dtype=np.float64)


def grid_jacobian(N: int, n_pv: int | None = None, seed: int = 0) -> Instance:
    """Reduced distributed-slack polar power-flow Jacobian at a random point."""
    if n_pv is None:
        n_pv = int(round(0.2 * N))
    rng = np.random.default_rng(seed)
    fr, to, y, Vm, Va, pv, part = _grid(rng, N, n_pv)
    lay = _Layout(N, pv)
    Ydiag, nbr = _admittance(N, fr, to, y)
    row_ptr, col, val = _jacobian_csr(lay, Ydiag, nbr, part, Vm, Va)
    inst = Instance(n=lay.n, row_ptr=row_ptr, col=col, val=val, D=None,
                    meta=dict(N=N, n_pv=n_pv, n_pq=len(lay.pq), seed=seed, n_lines=len(fr)))
    inst.D = perturbation_diag(inst)
    return inst


@dataclasses.dataclass
class PowerFlowCase:
    """A solvable distributed-slack power flow with a planted solution.

    The specified injections are those of a random operating point (Vm*, Va*)
    with slack share lambda*: P_spec_i = P_i(V*) - p_i lambda*, Q_spec_i =
    Q_i(V*), so F(x_star) = 0.  The unknowns and equations are ordered as in
    `grid_jacobian`; the Jacobian pattern (row_ptr, col) is fixed by the
    topology, so one symbolic analysis serves every Newton iteration.
    """
    N: int
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    x_star: np.ndarray
    P_spec: np.ndarray
    Q_spec: np.ndarray
    Vm_fixed: np.ndarray      # |V| of the slack and PV buses (PQ entries unused)
    part: np.ndarray
    meta: dict
    _lay: _Layout = dataclasses.field(repr=False)
    _Ydiag: np.ndarray = dataclasses.field(repr=False)
    _nbr: list = dataclasses.field(repr=False)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def state(self, x):
        """(Vm, Va, lambda) of the unknown vector x."""
        lay = self._lay
        Va = np.zeros(self.N)
        Va[1:] = x[lay.th_idx[1:]]
        Vm = self.Vm_fixed.copy()
        Vm[lay.pq] = x[lay.vm_idx[lay.pq]]
        return Vm, Va, float(x[lay.lam_idx])

    def mismatch(self, x) -> np.ndarray:
        """F(x): P_i - P_spec_i - p_i lambda (every bus), Q_i - Q_spec_i (PQ buses)."""
        lay = self._lay
        Vm, Va, lam = self.state(np.asarray(x, dtype=np.float64))
        P, Q = _injections(self._Ydiag, self._nbr, Vm, Va)
        F = np.zeros(self.n)
        F[lay.p_row] = P - self.P_spec - self.part * lam
        F[lay.q_row[lay.pq]] = Q[lay.pq] - self.Q_spec[lay.pq]
        return F

    def jacobian(self, x) -> np.ndarray:
        """dF/dx at x: the values on the fixed pattern (row_ptr, col)."""
        Vm, Va, _ = self.state(np.asarray(x, dtype=np.float64))
        rp, col, val = _jacobian_csr(self._lay, self._Ydiag, self._nbr, self.part, Vm, Va)
        assert np.array_equal(rp, self.row_ptr) and np.array_equal(col, self.col)
        return val

    def flat_start(self) -> np.ndarray:
        """theta = 0, |V| = 1 on PQ buses, lambda = 0."""
        x = np.zeros(self.n)
        x[self._lay.vm_idx[self._lay.pq]] = 1.0
        return x


def power_flow_case(N: int, n_pv: int | None = None, seed: int = 0,
                    angle_scale: float = 1.0) -> PowerFlowCase:
    """Grid as in `grid_jacobian` (same draws); the drawn point, with its angles
    scaled by `angle_scale` (heavier loading for larger values) and lambda* ~
    U[-1, 1] pu, is the planted solution."""
    if n_pv is None:
        n_pv = int(round(0.2 * N))
    rng = np.random.default_rng(seed)
    fr, to, y, Vm, Va, pv, part = _grid(rng, N, n_pv)
    lam = float(rng.uniform(-1.0, 1.0))
    Va = Va * angle_scale
    lay = _Layout(N, pv)
    Ydiag, nbr = _admittance(N, fr, to, y)
    P, Q = _injections(Ydiag, nbr, Vm, Va)
    x_star = np.zeros(lay.n)
    x_star[lay.th_idx[1:]] = Va[1:]
    x_star[lay.vm_idx[lay.pq]] = Vm[lay.pq]
    x_star[lay.lam_idx] = lam
    row_ptr, col, _ = _jacobian_csr(lay, Ydiag, nbr, part, Vm, Va)
    return PowerFlowCase(N=N, n=lay.n, row_ptr=row_ptr, col=col, x_star=x_star,
                         P_spec=P - part * lam, Q_spec=Q, Vm_fixed=Vm.copy(), part=part,
                         meta=dict(N=N, n_pv=n_pv, n_pq=len(lay.pq), seed=seed,
                                   angle_scale=angle_scale, n_lines=len(fr)),
                         _lay=lay, _Ydiag=Ydiag, _nbr=nbr)


def diag_rule(n: int, row_ptr, col, val) -> np.ndarray:
    """The perturbation diagonal of `perturbation_diag` for raw CSR arrays."""
    return perturbation_diag(Instance(n=n, row_ptr=np.asarray(row_ptr), col=np.asarray(col),
                                      val=np.asarray(val, dtype=np.float64), D=None, meta={}))


def perturbation_diag(inst: Instance) -> np.ndarray:
    """D = diag(|A_ii|), falling back to the row's max |A_ij| where negligible."""
    n = inst.n
    D = np.zeros(n)
    rowmax = np.zeros(n)
    amax = np.max(np.abs(inst.val)) if inst.nnz else 0.0
    for i in range(n):
        s, e = int(inst.row_ptr[i]), int(inst.row_ptr[i + 1])
        c = inst.col[s:e]
        v = inst.val[s:e]
        if e > s:
            rowmax[i] = np.max(np.abs(v))
        hit = np.nonzero(c == i)[0]
        if hit.size:
            D[i] = abs(v[hit[0]])
    weak = D <= 1e-12 * amax
    D[weak] = np.where(rowmax[weak] > 0, rowmax[weak], 1.0)
    return D


def symmetric_shifts(K: int, eps: float = 1e-2) -> np.ndarray:
    """Signed shifts t = (+eps, -eps, +2eps, -2eps, ...): the +-alpha*eps scheme, alpha = 1..K/2."""
    if K % 2:
        raise ValueError("symmetric shift sets need even K")
    t = []
    for a in range(1, K // 2 + 1):
        t += [a * eps, -a * eps]
    return np.asarray(t, dtype=np.float64)


def one_sided_shifts(K: int, eps: float = 1e-2) -> np.ndarray:
    """Shifts t_k = eps*k, k = 1..K (the one-sided variant)."""
    return eps * np.arange(1, K + 1, dtype=np.float64)


def rhs(n: int, R: int, seed: int) -> np.ndarray:
    """b ~ N(0, 1), row-major [n][R]."""
    return np.random.default_rng(seed + 7_000_000).standard_normal((n, R))


def batch_sizes(G: int, lo: int = 118, hi: int = 3000, seed: int = 3000) -> np.ndarray:
    """Bus counts drawn log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=G))).astype(np.int64)


# Named workloads: bus count(s), K, R, factor precision.
CONFIGS = {
    "plain": dict(index=1, N=300, n_pv=60, K=4, R=1, precision="fp64"),
    "precision": dict(index=2, N=2000, n_pv=400, K=6, R=16, precision="fp32"),
    "batching": dict(index=3, G=256, K=4, R=8, precision="fp32"),
    "differentiation": dict(index=4, N=1354, K=4, R=64, precision="fp64"),
    "scale": dict(index=5, N=10000, K=8, R=32, precision="fp32"),
}


def make_instance(config: str, instance: int = 0) -> Instance:
    """Instance `instance` of a named workload, seed = 1000*index + instance."""
    c = CONFIGS[config]
    seed = 1000 * c["index"] + instance
    if config == "batching":
        N = int(batch_sizes(c["G"])[instance])
        return grid_jacobian(N, None, seed)
    return grid_jacobian(c["N"], c.get("n_pv"), seed)


def random_sparse(n: int, density: float, seed: int, diag_boost: float = 4.0,
                  zero_diag: bool = False) -> Instance:
    """Small random unsymmetric sparse matrix with a structurally full diagonal.

    Used for edge-case tests (tiny n, ragged sizes); values ~ N(0,1) with the
    diagonal boosted so that the perturbed systems stay nonsingular.
    """
    rng = np.random.default_rng(seed)
    mask = rng.random((n, n)) < density
    np.fill_diagonal(mask, True)
    A = np.where(mask, rng.standard_normal((n, n)), 0.0)
    if not zero_diag:
        A[np.arange(n), np.arange(n)] += diag_boost * np.sign(rng.standard_normal(n) + 1e-300)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    cols, vals = [], []
    for i in range(n):
        nz = np.nonzero(mask[i])[0]
        cols.extend(nz.tolist())
        vals.extend(A[i, nz].tolist())
        row_ptr[i + 1] = row_ptr[i] + len(nz)
    inst = Instance(n=n, row_ptr=row_ptr, col=np.asarray(cols, np.int32),
                    val=np.asarray(vals, np.float64), D=None,
                    meta=dict(kind="random", density=density, seed=seed))
    inst.D = perturbation_diag(inst)
    return inst
