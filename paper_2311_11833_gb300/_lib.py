"""ctypes binding of libpisp.so (argument marshalling only).

Every computation happens in the CUDA library; this module only declares the
C signatures of include/pisp.h and raises if the library is missing.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpisp.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "pisp.h")

c_int32, c_int64, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
P = ctypes.POINTER

ERRORS = {
    0: "PISP_OK", 1: "PISP_ERR_INVALID_ARG", 2: "PISP_ERR_NOT_ANALYZED", 3: "PISP_ERR_NOT_FACTORED",
    4: "PISP_ERR_ZERO_PIVOT", 5: "PISP_ERR_NONFINITE", 6: "PISP_ERR_TIMEOUT", 7: "PISP_ERR_BOUNDS",
    8: "PISP_ERR_CUDA", 9: "PISP_ERR_OOM", 10: "PISP_ERR_UNSUPPORTED",
}
FP32, FP64 = 32, 64
K_MAX = 16


class PispOptions(ctypes.Structure):
    _fields_ = [("ordering", c_int32), ("relax_small", c_int32), ("relax_zeros", c_double),
                ("solve_schedule", c_int32), ("factor_policy", c_int32), ("solve_kfuse", c_int32),
                ("solve_warp_maxF", c_int32), ("solve_ctas_per_sm", c_int32),
                ("factor_smem_maxF", c_int32), ("factor_tc", c_int32), ("factor_ctas_per_sm", c_int32),
                ("analyze_threads", c_int32)]


class PispStats(ctypes.Structure):
    _fields_ = [
        ("N", c_int64), ("nnzA", c_int64), ("nnzL", c_int64), ("nnzF_stored", c_int64),
        ("front_elems", c_int64), ("G", c_int32), ("n_supernodes", c_int32), ("n_levels", c_int32),
        ("max_front", c_int32), ("etree_height", c_int32), ("K", c_int32), ("precision", c_int32),
        ("gpu_launches", c_int32), ("flops_factor", c_double), ("flops_solve", c_double),
        ("analyze_ms", c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_SIGS = {
    "pisp_create": (c_int32, [P(c_void_p), c_int32, c_void_p]),
    "pisp_destroy": (c_int32, [c_void_p]),
    "pisp_set_stream": (c_int32, [c_void_p, c_void_p]),
    "pisp_last_error": (ctypes.c_char_p, [c_void_p]),
    "pisp_analyze": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, P(PispOptions)]),
    "pisp_factor_perturbed": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32]),
    "pisp_solve": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_int32]),
    "pisp_combine": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "pisp_refine": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32]),
    "pisp_adjoint": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32]),
    "pisp_graph_capture": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p,
                                     c_int32, c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_void_p,
                                     c_int32]),
    "pisp_graph_launch": (c_int32, [c_void_p]),
    "pisp_set_wait_limit": (c_int32, [c_void_p, c_int64, c_int32]),
    "pisp_set_refinement": (c_int32, [c_void_p, c_double]),
    "pisp_refinement_stats": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32]),
    "pisp_weights": (c_int32, [c_void_p, c_int32, c_void_p]),
    "pisp_match_rows": (c_int32, [c_int32, c_void_p, c_void_p, c_void_p]),
    "pisp_get_status": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "pisp_get_stats": (c_int32, [c_void_p, P(PispStats)]),
    "pisp_get_perm": (c_int32, [c_void_p, c_void_p]),
    "pisp_get_supernodes": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "pisp_get_front": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, P(c_int32)]),
    "pisp_get_pivot_range": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "pisp_solve_host": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32,
                                  c_void_p, c_int32, c_void_p, c_int32]),
    "pisp_dense_solve_static": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_int32,
                                          c_void_p, c_int32, c_void_p]),
    "pisp_profile": (c_int32, [c_void_p, c_int32]),
    "pisp_profile_collect": (c_int32, [c_void_p]),
    "pisp_profile_read": (c_int32, [c_void_p, c_int32, P(c_double), P(c_double), P(c_int64)]),
    "pisp_profile_reset": (c_int32, [c_void_p]),
    "pisp_profile_name": (ctypes.c_char_p, [c_int32]),
}
PROF_FAMILIES = 8

_lib = None


def header_functions() -> list[str]:
    """Names of every function declared in include/pisp.h."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(pisp_\w+)\s*\(", text, re.M)))


def load():
    """Loads libpisp.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libpisp.so not built ({LIB_PATH}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class PispError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def check(code, handle=None):
    if code != 0:
        lib = load()
        msg = lib.pisp_last_error(handle)
        raise PispError(code, msg.decode() if msg else "")
    return code
