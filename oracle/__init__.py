"""CPU FP64 oracle for perturbation-induced static pivoting (arXiv 2311.11833).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this package: only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path; the only common dependency is the seeded input
generator ``pfgen`` (inputs only, none of the method's arithmetic).

What it computes, by the plain definitions of the paper:

* ``weights_gamma(m)`` - the combination coefficients beta = (Gamma_m^T)^{-1} e_1
  of Remark 2 (Eq. x_star_vand, Eq. gam), in exact rationals.
* ``weights(t)`` - the same construction for an arbitrary signed shift list t
  (one coefficient per perturbed solve): the coefficients of the Neumann terms
  (A^{-1} D)^j A^{-1} b, j = 0..K-1, are sum_k beta_k (-t_k)^j (Eq. neumann_2),
  and requiring them to be e_1 gives the transposed Vandermonde system in t.
  Solved exactly in rationals (floats are converted exactly).
* ``pistol`` - Algorithm 1 for the symmetric +-alpha*eps scheme: perturbed
  solves x_alpha^{+-} (Eq. xap, xam), averages x_hat_alpha (Eq. avg_hats),
  combination by Remark 2.
* ``x_hat`` - sum_k beta_k (A + t_k D)^{-1} B for any shift list; every
  perturbed solve is done with partial pivoting (the pivot-free LU is only
  the fast route to the same vectors).
* ``refine`` - the FP64 residual r = B - A x and one correction
  x + sum_k beta_k (A + t_k D)^{-1} r (the optional residual check of
  Alg. 1 turned into a correction).
* ``adjoint`` - lambda_k = (A + t_k D)^{-T} W, dL/db = sum_k beta_k lambda_k,
  dL/dA_ij = -sum_k beta_k sum_r lambda_k[i,r] x_k[j,r] on A's pattern.
* ``pivot_free_lu`` - dense Doolittle LU without pivoting of a given
  symmetric permutation of A + t D (unique when it exists), for factor-level
  comparisons on small systems.
* diagnostics: ``spectral_radius`` rho(A^{-1} D), ``cond1`` kappa_1(A),
  ``pivot_stats`` (growth factor and pivot spread of the pivot-free LU),
  ``rel_err`` and ``residual_norm`` (the forward error and the residual of Fig. 1).
* ``exact`` - brute force in rational arithmetic for tiny systems.

Every function cites the passage of the paper it follows.  Parity of each
function is pinned by the ``-m "not gpu"`` tests against values printed in the
paper (Examples 1-3), closed forms (2x2, diagonal systems), the exact error
identity derived from the Neumann series, finite differences and rational
brute force.
"""
from .core import (  # noqa: F401
    weights_gamma, weights, weights_float, pistol, perturbed_solutions, combine,
    x_hat, x_star, refine, adjoint, true_gradient, residual_norm, rel_err,
    pivot_free_lu, spectral_radius, to_dense, to_scipy, error_identity, cond1, pivot_stats,
)
from . import exact, newton  # noqa: F401
