"""Python front end of libpisp: the same calls as include/pisp.h.

PyTorch provides device memory, the stream and autograd; every arithmetic
step runs in the CUDA library.  There is no CPU fallback: without libpisp.so
or without a CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np
import torch

from . import _lib
from ._lib import FP32, FP64, PispOptions, PispStats, check

_PREC = {"fp32": FP32, "fp64": FP64, FP32: FP32, FP64: FP64, torch.float32: FP32, torch.float64: FP64}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _host_f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _dev_f64(t: torch.Tensor, name: str, shape=None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.contiguous()


def _host_out(a, name: str, size: int) -> np.ndarray:
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous:
        raise TypeError(f"{name} must be a C-contiguous float64 numpy array")
    if a.size != size:
        raise ValueError(f"{name} has {a.size} entries, expected {size}")
    return a


def weights(t: Sequence[float]) -> np.ndarray:
    """pisp_weights: per-solve weights prod_{l != k} t_l / (t_l - t_k)."""
    lib = _lib.load()
    tt = _host_f64(t)
    out = np.zeros(len(tt))
    check(lib.pisp_weights(tt.ctypes.data_as(ctypes.c_void_p), len(tt), out.ctypes.data_as(ctypes.c_void_p)))
    return out


def match_rows(n: int, row_ptr, col) -> np.ndarray:
    """pisp_match_rows: row_perm with row_perm[c] the row matched to column c."""
    lib = _lib.load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    if int(n) < 0 or rp.shape != (int(n) + 1,):
        raise ValueError("row_ptr must have n + 1 entries")
    if cl.size < (int(rp[-1]) if rp.size else 0):
        raise ValueError("col is shorter than row_ptr[n]")
    out = np.zeros(int(n), dtype=np.int32)
    check(lib.pisp_match_rows(int(n), rp.ctypes.data_as(ctypes.c_void_p), cl.ctypes.data_as(ctypes.c_void_p),
                              out.ctypes.data_as(ctypes.c_void_p)))
    return out


def permute_rows(row_ptr, col, val, row_perm):
    """CSR of the matrix whose row c is row row_perm[c] of (row_ptr, col, val)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    lens = np.diff(row_ptr)[row_perm]
    new_ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    idx = np.concatenate([np.arange(row_ptr[r], row_ptr[r + 1]) for r in row_perm]) if len(row_perm) else \
        np.zeros(0, dtype=np.int64)
    return new_ptr, np.asarray(col)[idx], np.asarray(val)[idx]


class Solver:
    """One analysed sparsity pattern (G instances, block diagonal) on one device.

    row_ptr / col describe the concatenated CSR pattern (global indices);
    `n` is the list of instance sizes (an int for a single instance).
    """

    def __init__(self, n, row_ptr, col, device: int | None = None, ordering: int = 0,
                 relax_small: int = -1, relax_zeros: float = -1.0, solve_schedule: int = 0,
                 factor_policy: int = 0, solve_kfuse: int = 0, solve_warp_maxF: int = 0,
                 solve_ctas_per_sm: int = 0, factor_smem_maxF: int = 0, factor_tc: int = 0,
                 factor_ctas_per_sm: int = 0, analyze_threads: int = 0):
        self._lib = _lib.load()
        if not torch.cuda.is_available():
            raise RuntimeError("libpisp needs a CUDA device")
        self.device = torch.cuda.current_device() if device is None else int(device)
        sizes = np.atleast_1d(np.asarray(n, dtype=np.int32))
        self.G = len(sizes)
        self.sizes = sizes
        self.N = int(sizes.sum())
        rp = np.ascontiguousarray(np.asarray(row_ptr, dtype=np.int64))
        cl = np.ascontiguousarray(np.asarray(col, dtype=np.int32))
        if rp.shape != (self.N + 1,):
            raise ValueError("row_ptr must have N + 1 entries")
        if cl.size < int(rp[-1]):
            raise ValueError("col is shorter than row_ptr[N]")
        self.nnz = int(rp[-1])
        self._row_ptr, self._col = rp, cl
        h = ctypes.c_void_p()
        check(self._lib.pisp_create(ctypes.byref(h), self.device, None))
        self._h = h
        opt = PispOptions(ordering, relax_small, relax_zeros, solve_schedule, factor_policy, solve_kfuse,
                          solve_warp_maxF, solve_ctas_per_sm, factor_smem_maxF, factor_tc, factor_ctas_per_sm,
                          analyze_threads)
        check(self._lib.pisp_analyze(self._h, self.G, sizes.ctypes.data_as(ctypes.c_void_p),
                                     rp.ctypes.data_as(ctypes.c_void_p),
                                     cl.ctypes.data_as(ctypes.c_void_p), ctypes.byref(opt)), self._h)
        self.K = 0
        self.t = None
        self.precision = None
        self.R = 0

    # ------------------------------------------------------------- plumbing --
    def _dev(self, t, name: str, shape=None) -> torch.Tensor:
        """A float64 CUDA tensor on this solver's device (every pointer the
        library reads or writes is sized from the analysed pattern)."""
        t = _dev_f64(t, name, shape)
        if t.device.index != self.device:
            raise ValueError(f"{name} is on {t.device}, the solver on cuda:{self.device}")
        return t

    def _dev_out(self, t, name: str, numel: int) -> torch.Tensor:
        t2 = self._dev(t, name)
        if t2.data_ptr() != t.data_ptr() or t.numel() != numel:
            raise ValueError(f"{name} must be contiguous with {numel} entries")
        return t

    def _sync_stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        check(self._lib.pisp_set_stream(self._h, ctypes.c_void_p(s)), self._h)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pisp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ ABI --
    def factor(self, values: torch.Tensor, D: torch.Tensor, t: Sequence[float], precision="fp64"):
        """pisp_factor_perturbed: pivot-free LU of P (A + t_k D) P^T for all k."""
        values = self._dev(values, "values", (self.nnz,))
        D = self._dev(D, "D", (self.N,))
        tt = _host_f64(t)
        prec = _PREC[precision]
        self._sync_stream()
        check(self._lib.pisp_factor_perturbed(self._h, _ptr(values), _ptr(D),
                                              tt.ctypes.data_as(ctypes.c_void_p), len(tt), prec), self._h)
        self.K, self.t, self.precision = len(tt), tt, prec
        return self

    def solve(self, b: torch.Tensor, weights=None, sweeps: int = 0, out: torch.Tensor | None = None):
        """pisp_solve: x = sum_k w_k (A + t_k D)^{-1} b; b is [N] or [N, R]."""
        vec = b.dim() == 1
        b2 = self._dev(b, "b").reshape(self.N, -1)
        R = b2.shape[1]
        x = self._dev_out(out, "out", self.N * R) if out is not None else torch.empty_like(b2)
        w = None if weights is None else _host_f64(weights)
        self._sync_stream()
        check(self._lib.pisp_solve(self._h, _ptr(b2), R,
                                   None if w is None else w.ctypes.data_as(ctypes.c_void_p),
                                   _ptr(x), int(sweeps)), self._h)
        self.R = R
        return x.reshape(-1) if vec else x

    def combine(self, weights=None, out: torch.Tensor | None = None):
        """pisp_combine: re-weights the kept per-perturbation solutions."""
        x = self._dev_out(out, "out", self.N * self.R) if out is not None else \
            torch.empty((self.N, self.R), dtype=torch.float64, device=f"cuda:{self.device}")
        w = None if weights is None else _host_f64(weights)
        self._sync_stream()
        check(self._lib.pisp_combine(self._h, None if w is None else w.ctypes.data_as(ctypes.c_void_p),
                                     _ptr(x)), self._h)
        return x

    def refine(self, b: torch.Tensor, x: torch.Tensor, iters: int = 1, sweeps: int = 0):
        """pisp_refine: x += sum_k beta_k (A + t_k D)^{-1} (b - A x), in place."""
        vec = b.dim() == 1
        b2 = self._dev(b, "b").reshape(self.N, -1)
        x2 = self._dev_out(x, "x", b2.numel()).reshape(self.N, -1)
        self._sync_stream()
        check(self._lib.pisp_refine(self._h, _ptr(b2), _ptr(x2), b2.shape[1], int(iters), int(sweeps)),
              self._h)
        return x.reshape(-1) if vec else x

    def adjoint(self, g: torch.Tensor, weights=None, need_b=True, need_values=True,
                out_b: torch.Tensor | None = None, out_values: torch.Tensor | None = None,
                sweeps: int = 0):
        """pisp_adjoint: (dL/db, dL/dvalues) for dL/dx = g of the last solve.

        out_b / out_values: preallocated outputs (e.g. inside a CUDA graph);
        without them the outputs that are needed are allocated.  sweeps: FP64
        residual corrections of the transposed solves (use the forward
        solve's count with FP32 factors)."""
        g2 = self._dev(g, "g").reshape(self.N, -1)
        if g2.shape[1] != self.R:
            raise ValueError(f"g has {g2.shape[1]} columns, the last solve had R = {self.R}")
        if out_b is not None:
            gb = self._dev_out(out_b, "out_b", g2.numel())
        else:
            gb = torch.empty_like(g2) if need_b else None
        if out_values is not None:
            gv = self._dev_out(out_values, "out_values", self.nnz)
        else:
            gv = torch.empty(self.nnz, dtype=torch.float64, device=g2.device) if need_values else None
        w = None if weights is None else _host_f64(weights)
        self._sync_stream()
        check(self._lib.pisp_adjoint(self._h, _ptr(g2), None if w is None else w.ctypes.data_as(ctypes.c_void_p),
                                     _ptr(gb), _ptr(gv), int(sweeps)), self._h)
        if gb is not None and out_b is None and g.dim() == 1:
            gb = gb.reshape(-1)
        return gb, gv

    def graph_capture(self, values: torch.Tensor, D: torch.Tensor, t, b: torch.Tensor, x: torch.Tensor,
                      precision="fp64", sweeps: int = 0, weights=None, g: torch.Tensor | None = None,
                      out_b: torch.Tensor | None = None, out_values: torch.Tensor | None = None,
                      adjoint_sweeps: int = 0):
        """pisp_graph_capture: one factor + solve (+ adjoint) step captured into a
        library-owned CUDA graph; graph_launch() replays it on the current
        stream, reading the current contents of these same tensors."""
        values = self._dev(values, "values", (self.nnz,))
        D = self._dev(D, "D", (self.N,))
        b2 = self._dev(b, "b")
        if b2.data_ptr() != b.data_ptr() or b2.numel() % max(self.N, 1):
            raise ValueError("b must be a contiguous [N] or [N, R] tensor")
        R = b2.numel() // self.N if self.N else 1
        x = self._dev_out(x, "x", self.N * R)
        tt = _host_f64(t)
        w = None if weights is None else _host_f64(weights)
        gg = gb = gv = None
        if g is not None:
            gg = self._dev(g, "g")
            if gg.data_ptr() != g.data_ptr() or gg.numel() != self.N * R:
                raise ValueError("g must be contiguous with N * R entries")
            gb = self._dev_out(out_b, "out_b", self.N * R) if out_b is not None else None
            gv = self._dev_out(out_values, "out_values", self.nnz) if out_values is not None else None
        self._sync_stream()
        check(self._lib.pisp_graph_capture(
            self._h, _ptr(values), _ptr(D), tt.ctypes.data_as(ctypes.c_void_p), len(tt), _PREC[precision],
            _ptr(b2), R, None if w is None else w.ctypes.data_as(ctypes.c_void_p), _ptr(x), int(sweeps),
            _ptr(gg), _ptr(gb), _ptr(gv), int(adjoint_sweeps)), self._h)
        self.K, self.t, self.precision, self.R = len(tt), tt, _PREC[precision], R
        self._graph_refs = (values, D, b, x, g, out_b, out_values)   # keep the buffers alive
        return self

    def graph_launch(self):
        """pisp_graph_launch: replays the captured step on the current stream."""
        self._sync_stream()
        check(self._lib.pisp_graph_launch(self._h), self._h)

    def set_wait_limit(self, polls: int = 0, unreachable: bool = False):
        """pisp_set_wait_limit: poll limit of the solves' dependency waits (0 = default);
        unreachable=True makes one wait run out on purpose (test hook)."""
        check(self._lib.pisp_set_wait_limit(self._h, int(polls), 1 if unreachable else 0), self._h)

    def set_refinement(self, tol: float = 0.0):
        """pisp_set_refinement: tol > 0 makes `sweeps` a maximum and stops each
        instance's FP64 residual sweeps on its own (converged or stagnated);
        tol = 0 restores fixed sweeps."""
        check(self._lib.pisp_set_refinement(self._h, float(tol)), self._h)
        return self

    def refinement_stats(self, max_sweeps: int = 0, rows: bool = False):
        """pisp_refinement_stats: (sweeps each instance took in the last solve
        [G], fraction of the solve work each sweep 1..max_sweeps covered[,
        fraction of the rows]); rows=True adds the third array."""
        nsw = np.zeros(self.G, dtype=np.int32)
        work = np.zeros(max(int(max_sweeps), 0), dtype=np.float64)
        frow = np.zeros_like(work)
        self._sync_stream()
        check(self._lib.pisp_refinement_stats(self._h, nsw.ctypes.data_as(ctypes.c_void_p),
                                              work.ctypes.data_as(ctypes.c_void_p) if work.size else None,
                                              frow.ctypes.data_as(ctypes.c_void_p) if frow.size else None,
                                              int(max_sweeps)), self._h)
        return (nsw, work, frow) if rows else (nsw, work)

    def status(self):
        """pisp_get_status: (worst code, per-(instance, k) codes, first failing columns)."""
        st = np.zeros(self.G * self.K, dtype=np.int32)
        bc = np.zeros(self.G * self.K, dtype=np.int32)
        self._sync_stream()
        worst = self._lib.pisp_get_status(self._h, st.ctypes.data_as(ctypes.c_void_p),
                                          bc.ctypes.data_as(ctypes.c_void_p))
        if worst not in (0, 4, 5, 6):
            check(worst, self._h)
        return worst, st.reshape(self.G, self.K), bc.reshape(self.G, self.K)

    def stats(self) -> dict:
        s = PispStats()
        check(self._lib.pisp_get_stats(self._h, ctypes.byref(s)), self._h)
        return s.as_dict()

    def perm(self) -> np.ndarray:
        p = np.zeros(self.N, dtype=np.int32)
        check(self._lib.pisp_get_perm(self._h, p.ctypes.data_as(ctypes.c_void_p)), self._h)
        return p

    def supernodes(self):
        S = self.stats()["n_supernodes"]
        c0 = np.zeros(S, np.int32)
        c1 = np.zeros(S, np.int32)
        ms = np.zeros(S, np.int32)
        check(self._lib.pisp_get_supernodes(self._h, c0.ctypes.data_as(ctypes.c_void_p),
                                            c1.ctypes.data_as(ctypes.c_void_p),
                                            ms.ctypes.data_as(ctypes.c_void_p), None), self._h)
        rows = np.zeros(int(ms.sum()), np.int32)
        check(self._lib.pisp_get_supernodes(self._h, None, None, None,
                                            rows.ctypes.data_as(ctypes.c_void_p)), self._h)
        return c0, c1, ms, rows

    def front(self, s: int, k: int) -> np.ndarray:
        F = ctypes.c_int32()
        check(self._lib.pisp_get_front(self._h, s, k, None, ctypes.byref(F)), self._h)
        out = np.zeros(F.value * F.value)
        self._sync_stream()
        check(self._lib.pisp_get_front(self._h, s, k, out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(F)),
              self._h)
        return out.reshape(F.value, F.value, order="F")

    def pivot_range(self):
        """pisp_get_pivot_range: (min |u_jj|, max |u_jj|), each [G, K], of the last factorisation."""
        lo = np.zeros(self.G * self.K)
        hi = np.zeros(self.G * self.K)
        self._sync_stream()
        check(self._lib.pisp_get_pivot_range(self._h, lo.ctypes.data_as(ctypes.c_void_p),
                                             hi.ctypes.data_as(ctypes.c_void_p)), self._h)
        return lo.reshape(self.G, self.K), hi.reshape(self.G, self.K)

    def solve_host(self, values: np.ndarray, D: np.ndarray, t, b: np.ndarray, precision="fp64",
                   sweeps: int = 0, out: np.ndarray | None = None) -> np.ndarray:
        """pisp_solve_host: end to end from host buffers (copies included)."""
        vals = _host_f64(values)
        DD = _host_f64(D)
        tt = _host_f64(t)
        if vals.size != self.nnz or DD.size != self.N:
            raise ValueError(f"values needs {self.nnz} entries and D {self.N}")
        bb = _host_f64(b).reshape(self.N, -1)
        x = _host_out(out, "out", bb.size) if out is not None else np.empty_like(bb)
        self._sync_stream()
        check(self._lib.pisp_solve_host(self._h, vals.ctypes.data_as(ctypes.c_void_p),
                                        DD.ctypes.data_as(ctypes.c_void_p),
                                        tt.ctypes.data_as(ctypes.c_void_p), len(tt), _PREC[precision],
                                        bb.ctypes.data_as(ctypes.c_void_p), bb.shape[1],
                                        x.ctypes.data_as(ctypes.c_void_p), int(sweeps)), self._h)
        self.K, self.t, self.precision, self.R = len(tt), tt, _PREC[precision], bb.shape[1]
        return x


    # ------------------------------------------------------------ profiling --
    def profile(self, on: bool):
        """pisp_profile: start / stop recording CUDA-event brackets per kernel family."""
        check(self._lib.pisp_profile(self._h, 1 if on else 0), self._h)

    def profile_collect(self):
        self._sync_stream()
        check(self._lib.pisp_profile_collect(self._h), self._h)

    def profile_reset(self):
        check(self._lib.pisp_profile_reset(self._h), self._h)

    def profile_read(self) -> dict:
        """{family: {"ms", "bytes", "launches"}} accumulated since the last reset."""
        out = {}
        for f in range(_lib.PROF_FAMILIES):
            ms, by, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
            check(self._lib.pisp_profile_read(self._h, f, ctypes.byref(ms), ctypes.byref(by),
                                              ctypes.byref(n)), self._h)
            out[self._lib.pisp_profile_name(f).decode()] = {"ms": ms.value, "bytes": by.value,
                                                            "launches": n.value}
        return out


class _PerturbedSolve(torch.autograd.Function):
    """x = sum_k beta_k (A + t_k D)^{-1} b with gradients for values and b.

    The backward pass reuses the K factors of the forward pass transposed
    (pisp_adjoint) with as many FP64 residual sweeps as the forward solve
    used, so FP32 factors give gradients at the accuracy of the forward
    result; D and t are held fixed.
    """

    @staticmethod
    def forward(ctx, values, b, solver, D, t, precision, sweeps):
        solver.factor(values.detach(), D, t, precision)
        x = solver.solve(b.detach(), sweeps=sweeps)
        ctx.solver = solver
        ctx.sweeps = sweeps
        ctx.vec = b.dim() == 1
        return x

    @staticmethod
    def backward(ctx, gx):
        s = ctx.solver
        need_v, need_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        gb, gv = s.adjoint(gx.contiguous(), need_b=need_b, need_values=need_v, sweeps=ctx.sweeps)
        return gv, gb, None, None, None, None, None


def solve(solver: Solver, values: torch.Tensor, b: torch.Tensor, D: torch.Tensor, t, precision="fp64",
          sweeps: int = 0) -> torch.Tensor:
    """Differentiable perturbed solve + combine (autograd through pisp_adjoint)."""
    return _PerturbedSolve.apply(values, b, solver, D, t, precision, sweeps)
