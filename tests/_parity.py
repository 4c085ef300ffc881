"""Entry-wise parity measures shared by the GPU tests.

A normwise error ||x - ref|| / ||ref|| can hide a small component of x that
is wrong by far more than the tolerance.  These measures bound every entry:
an entry of right-hand side r counts against the largest magnitude of the
reference's column r, and an entry of a gradient on A's pattern against the
largest magnitude of the reference gradient.
"""
import numpy as np


def entrywise_err(x, ref) -> float:
    """max over columns r and rows i of |x[i, r] - ref[i, r]| / max_i |ref[i, r]|."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if x.shape != ref.shape:
        raise ValueError(f"shape {x.shape} != {ref.shape}")
    if x.ndim == 1:
        x, ref = x[:, None], ref[:, None]
    if x.size == 0:
        return 0.0
    if not np.all(np.isfinite(x)):
        return float("inf")
    scale = np.abs(ref).max(axis=0)
    scale = np.where(scale > 0, scale, 1.0)
    return float(np.max(np.abs(x - ref) / scale))


def per_rhs_entrywise_err(x, ref) -> np.ndarray:
    """The same measure for each column separately ([R])."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if x.ndim == 1:
        x, ref = x[:, None], ref[:, None]
    scale = np.abs(ref).max(axis=0)
    scale = np.where(scale > 0, scale, 1.0)
    return np.max(np.abs(x - ref), axis=0) / scale


def grad_entrywise_err(g, ref) -> float:
    """max_e |g_e - ref_e| / max_e |ref_e| for a gradient on A's pattern."""
    g = np.asarray(g, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    if not np.all(np.isfinite(g)):
        return float("inf")
    scale = float(np.abs(ref).max()) if ref.size else 1.0
    return float(np.max(np.abs(g - ref)) / (scale if scale > 0 else 1.0)) if ref.size else 0.0
