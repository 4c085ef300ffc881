"""GB300-native perturbation-induced static pivoting (arXiv 2311.11833).

K diagonally perturbed systems (A + t_k D) x_k = b are factored pivot-free
in the same launches on the GPU and combined with the paper's expansion
weights to recover A^{-1} b.  The arithmetic lives in libpisp.so (CUDA,
sm_103a); this package is its thin Python binding.
"""
from ._lib import FP32, FP64, K_MAX, PispError, header_functions, load  # noqa: F401
from .solver import Solver, match_rows, permute_rows, solve, weights  # noqa: F401
from .newton import NewtonResult, newton  # noqa: F401

__all__ = ["Solver", "solve", "weights", "match_rows", "permute_rows", "newton", "NewtonResult", "load", "PispError", "FP32",
           "FP64", "K_MAX", "header_functions"]
