/*
 * pisp.h - C ABI of the perturbation-induced static pivoting solver.
 *
 * Method (arXiv 2311.11833): the K diagonally perturbed systems
 *     (A + t_k D) x_k = b,   k = 0..K-1                    (Sec. III-A, Eq. xap / xam)
 * are factored WITHOUT pivoting, all K in the same launches, and their
 * solutions are combined as
 *     x_hat = sum_k beta_k x_k                             (Eq. x_star, Remark 2)
 * with weights chosen so that the Neumann-series terms (A^{-1} D)^j A^{-1} b,
 * j = 1..K-1, cancel (Eq. neumann_2, Eq. gam).  For the paper's symmetric
 * shift set t = {+-alpha*eps}, alpha = 1..m, these per-solve weights are
 * half the paper's beta = (Gamma_m^T)^{-1} e_1 for each +- pair (Alg. 1).
 *
 * Conventions for every entry point:
 *  - Return value: PISP_OK (0) or one of the PISP_ERR_* codes below;
 *    pisp_last_error(h) gives a message for the last failing call.
 *  - Array arguments marked "device" are caller-owned device memory on the
 *    handle's device; "host" arrays are caller-owned host memory.  The
 *    library owns only its handle, the symbolic structure and its workspace
 *    (factors, per-perturbation solutions), all freed by pisp_destroy.
 *  - Work is enqueued on the stream given to pisp_create and is ordered on
 *    it; only the queries that read device results back (pisp_get_status,
 *    pisp_refinement_stats, pisp_profile_collect, pisp_get_front /
 *    pivot_range, and pisp_get_stats after adaptive sweeps) and
 *    pisp_solve_host synchronise the stream.
 *  - A handle is not thread-safe; use one handle per host thread.
 *  - A call makes the handle's device current while it runs and restores
 *    the caller's current device before it returns.
 *  - Instances: the matrix is the block diagonal of G independent instances
 *    of sizes n[0..G-1]; N = sum n[g].  All vectors are row-major [N][R]
 *    FP64 (R right-hand sides per instance row), values are the CSR values
 *    of the concatenated instances, in the order of the pattern given to
 *    pisp_analyze.
 */
#ifndef PISP_H
#define PISP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PISP_OK = 0,
  PISP_ERR_INVALID_ARG = 1,  /* bad pointer, size or pattern */
  PISP_ERR_NOT_ANALYZED = 2, /* pisp_analyze has not succeeded yet */
  PISP_ERR_NOT_FACTORED = 3, /* no successful pisp_factor_perturbed yet */
  PISP_ERR_ZERO_PIVOT = 4,   /* an exact zero pivot was met (see status) */
  PISP_ERR_NONFINITE = 5,    /* a pivot became Inf/NaN (see status) */
  PISP_ERR_TIMEOUT = 6,      /* a bounded device wait gave up */
  PISP_ERR_BOUNDS = 7,       /* an index check failed */
  PISP_ERR_CUDA = 8,         /* a CUDA runtime call failed */
  PISP_ERR_OOM = 9,          /* device allocation failed */
  PISP_ERR_UNSUPPORTED = 10  /* a size outside what the kernels handle */
};

enum { PISP_FP32 = 32, PISP_FP64 = 64 };

#define PISP_K_MAX 16

typedef struct pisp_handle pisp_handle;

typedef struct pisp_options {
  int32_t ordering;     /* 0 = minimum degree on A + A^T (default), 1 = as given
                           (both followed by an elimination-tree postorder) */
  int32_t relax_small;  /* supernode amalgamation: merge while pivot block <= this (default 8) */
  double relax_zeros;   /* ... or while explicit zeros <= this fraction (default 0.05) */
  int32_t solve_schedule; /* 0 = persistent: one launch per solve direction whose
                             CTAs take (front, k, RHS chunk) tasks in level order
                             and wait (boundedly) for their dependencies;
                             1 = one launch per level and front-size class */
  int32_t factor_policy;  /* fronts wider than 64: 0 (default) = one CTA each while
                             the front fits in shared memory; larger fronts, of
                             any size, in one persistent launch per level where
                             each CTA owns a tile (a 32-column block of a (front,
                             k), all its rows in FP32 while they fit, 32-row
                             chunks in FP64) in shared memory, assembles it and
                             applies the earlier panels as they are released;
                             1 = thread-block clusters of up to 8 CTAs holding the
                             front in distributed shared memory wherever it fits;
                             2 = as 0 but larger fronts as a tile DAG (column-block
                             assembly, panel and update tasks in one persistent
                             launch per level, with look-ahead);
                             3 = as 0 but larger fronts by a blocked factorisation
                             in global memory (one panel launch and one
                             tiled-update launch per 32 pivots);
                             4 = ONE persistent launch for every level, shift
                             and instance: fronts of at most 32 one warp each,
                             fronts up to factor_smem_maxF one CTA each in
                             shared memory, wider fronts as owner tiles;
                             a task waits (boundedly) only for its children's
                             completion counters */
  int32_t solve_kfuse;    /* persistent solve: shifts per segment task of a front
                             with at most 32 pivots (0 = 1): larger values pay a
                             front's dependency wait and structure loads once
                             for several shifts, smaller ones run more tasks
                             in parallel */
  int32_t solve_warp_maxF; /* persistent solve: widest front (with at most 32
                              pivots) solved by one 32-lane segment, in blocks
                              of 32 rows (0 = 32); wider fronts are solved by a
                              whole CTA per (front, k, RHS chunk) */
  int32_t solve_ctas_per_sm; /* persistent solve: resident CTAs per SM, 2, 3 or 4
                                (register budgets 128, 80, 64 per thread; 0 = 3
                                for FP32 factors, 2 for FP64): more CTAs hide
                                more latency of a batch's many small fronts,
                                fewer spill less on wide fronts */
  int32_t factor_smem_maxF; /* factor policy 4: widest front factored by one CTA
                               in shared memory (0 = the limit: 160 in FP32,
                               112 in FP64); wider fronts become owner tiles */
  int32_t factor_tc;       /* 1: the trailing updates of FP32 owner tiles (the
                              L21 U12 products of wide, dense fronts) run on the
                              tensor cores: tcgen05.mma kind::tf32 with each FP32
                              operand split as hi + lo, hi*hi + hi*lo + lo*hi,
                              FP32 accumulation in tensor memory (FP32-level
                              accuracy); 0 (default): FP32 FMA.  Ignored for
                              FP64 factors. */
  int32_t factor_ctas_per_sm; /* factor policy 4: resident CTAs per SM, 2 (128
                                 registers per thread) or 3 (80; 0 = 2); with 3 the
                                 shared-memory fronts should be narrowed
                                 (factor_smem_maxF) so that three CTAs fit */
  int32_t analyze_threads; /* host threads pisp_analyze may use for the instances
                              of a batch: 0 = the hardware concurrency, at most
                              16 (default); 1 = the calling thread only.  A
                              caller that already analyses patterns from
                              several threads should cap this. */
} pisp_options;

typedef struct pisp_stats {
  int64_t N;             /* total unknowns */
  int64_t nnzA;          /* entries of A (all instances) */
  int64_t nnzL;          /* structural strictly-lower entries of L (= those of U) */
  int64_t nnzF_stored;   /* factor entries stored per perturbation, incl. amalgamation zeros */
  int64_t front_elems;   /* sum of squared front sizes (workspace per perturbation) */
  int32_t G;             /* instances */
  int32_t n_supernodes;
  int32_t n_levels;      /* height of the assembly forest */
  int32_t max_front;
  int32_t etree_height;  /* height of the column elimination tree */
  int32_t K;             /* perturbations of the last factorisation */
  int32_t precision;     /* PISP_FP32 / PISP_FP64 of the last factorisation */
  int32_t gpu_launches;  /* kernels launched by the last factor + solve calls (adaptive sweeps,
                            a device-side loop: with the iterations its last run took; reading
                            them synchronises the stream) */
  double flops_factor;   /* per perturbation */
  double flops_solve;    /* per perturbation per RHS (forward + back) */
  double analyze_ms;     /* host time of pisp_analyze */
} pisp_stats;

/* Creates a handle bound to `device` and to `stream` (a cudaStream_t; NULL =
 * the legacy default stream).  *h receives the handle.  device = -1 makes a
 * host-only handle: pisp_analyze and the pisp_get_stats / pisp_get_perm /
 * pisp_get_supernodes queries work without a GPU, numeric calls fail with
 * PISP_ERR_INVALID_ARG. */
int pisp_create(pisp_handle** h, int device, void* stream);

/* Frees the handle and all library-owned device memory. */
int pisp_destroy(pisp_handle* h);

/* Rebinds the handle to another stream of the same device. */
int pisp_set_stream(pisp_handle* h, void* stream);

/* Message for the last failing call on h; for a NULL handle, for the last
 * failing call without a handle made by the calling host thread. */
const char* pisp_last_error(const pisp_handle* h);

/* Symbolic phase (host).  Static pivot order of Sec. II-C: a fill-reducing
 * symmetric ordering of A + A^T, elimination tree, supernodes and the level
 * schedule of the assembly forest, computed once per pattern and reused by
 * every factorisation.
 *   G        number of instances (>= 1)
 *   n        host [G] instance sizes (>= 0)
 *   row_ptr  host [N+1] global CSR row pointer, row_ptr[0] = 0
 *   col_idx  host [nnz] global column indices; each row's columns must lie in
 *            its own instance's block; duplicates are summed
 *   opt      host, may be NULL for defaults
 * The pattern is copied; the host arrays may be freed afterwards.  Returns
 * PISP_ERR_INVALID_ARG for a malformed pattern, PISP_ERR_UNSUPPORTED for a
 * front wider than 46340, and PISP_ERR_BOUNDS if the computed structure fails
 * its index checks (every map the kernels follow lands inside its front and
 * arrays); the kernels are never given an unchecked structure. */
int pisp_analyze(pisp_handle* h, int32_t G, const int32_t* n, const int64_t* row_ptr,
                 const int32_t* col_idx, const pisp_options* opt);

/* Alg. 1, factor part (Eq. xap / xam): forms P (A + t_k D) P^T for every shift in
 * the fixed pivot order and factors all K perturbations pivot-free, level by
 * level of the assembly forest, all K (and all instances) in the same launches.
 *   values    device FP64 [nnz], CSR order of the analysed pattern
 *   D         device FP64 [N], the diagonal perturbation matrix
 *   t         host FP64 [K], distinct signed shifts (eps * alpha with sign)
 *   K         1..PISP_K_MAX
 *   precision PISP_FP32 or PISP_FP64: type in which factors are stored and
 *             eliminated
 * Pivot failures do not abort: they are recorded per (instance, k) and read
 * with pisp_get_status. */
int pisp_factor_perturbed(pisp_handle* h, const double* values, const double* D,
                          const double* t, int32_t K, int32_t precision);

/* Alg. 1, solve and combine part (Eq. x_star): for every perturbation k and RHS r solves
 * (A + t_k D) x_k = b with the pivot-free factors, then writes
 *     x[i][r] = sum_k w_k x_k[i][r]       (FP64 accumulation)
 *   b        device FP64 [N][R]
 *   R        right-hand sides, >= 1
 *   w        host FP64 [K] weights, or NULL for the weights of pisp_weights(t)
 *   x        device FP64 [N][R] output (may not alias b)
 *   sweeps   FP64 residual corrections of each perturbed solution:
 *            x_k += (L_k U_k)^{-1} (b - (A + t_k D) x_k), computed in FP64
 *            against the original values; 0 keeps the plain solve.  With FP32
 *            factors this makes every x_k (and so x) agree with the FP64
 *            definition to working accuracy.
 * The per-perturbation solutions are kept in the handle for pisp_combine and
 * pisp_adjoint.  Returns PISP_ERR_NOT_FACTORED before a factorisation,
 * PISP_ERR_INVALID_ARG for R < 1, sweeps < 0, NULL or aliased b / x; a
 * failed (instance, k) of the factorisation leaves that instance's rows of x
 * NaN and the call still returns PISP_OK (pisp_get_status reports it). */
int pisp_solve(pisp_handle* h, const double* b, int32_t R, const double* w, double* x,
               int32_t sweeps);

/* Re-combines the kept per-perturbation solutions of the last pisp_solve with
 * other weights (Eq. x_star):  x = sum_k w_k x_k.
 *   w  host FP64 [K] or NULL for pisp_weights(t);   x device FP64 [N][R],
 *   R of the last pisp_solve.
 * Returns PISP_ERR_NOT_FACTORED when no kept solutions exist. */
int pisp_combine(pisp_handle* h, const double* w, double* x);

/* The optional residual check of Alg. 1 turned into a correction: `iters` times
 *     r = b - A x (FP64, the values of the last factorisation);
 *     x += sum_k beta_k (A + t_k D)^{-1} r
 * with each inner perturbed solve done with `sweeps` residual corrections.
 * Converges to A^{-1} b when the Neumann series converges (eps * max|alpha| *
 * rho(A^{-1} D) < 1, Sec. II-B).
 *   b device FP64 [N][R]; x device FP64 [N][R] in/out; R >= 1, iters >= 0.
 * The kept solutions of the last pisp_solve survive a refine with at most as
 * many right-hand sides; a larger R releases them (pisp_combine and
 * pisp_adjoint then return PISP_ERR_NOT_FACTORED until the next pisp_solve).
 * Returns PISP_ERR_NOT_FACTORED before a factorisation, PISP_ERR_INVALID_ARG
 * for bad sizes or NULL buffers, PISP_ERR_OOM if its workspace cannot be
 * allocated. */
int pisp_refine(pisp_handle* h, const double* b, double* x, int32_t R, int32_t iters,
                int32_t sweeps);

/* Reverse mode of x = sum_k beta_k (A + t_k D)^{-1} b for the last pisp_solve
 * (the derivative of Eq. x_star with respect to b and to A's entries):
 *   lambda_k = (A + t_k D)^{-T} g,  grad_b = sum_k beta_k lambda_k,
 *   grad_values[e] = - sum_k beta_k sum_r lambda_k[i_e][r] x_k[j_e][r]
 * on A's pattern (D held fixed), using the same factors transposed.
 *   g           device FP64 [N][R] = dL/dx
 *   grad_b      device FP64 [N][R] output, or NULL
 *   grad_values device FP64 [nnz] output, or NULL
 *   w           host FP64 [K] or NULL (pisp_weights(t)): the combination used
 *               in the forward pass.
 *   sweeps      FP64 residual corrections of every lambda_k on the transposed
 *               system, lambda_k += (L_k U_k)^{-T} (g - (A + t_k D)^T lambda_k),
 *               as pisp_solve's sweeps do for x_k; with FP32 factors they make
 *               the gradients agree with the FP64 definition (0: one
 *               transposed solve, FP32 accuracy with FP32 factors).
 * R is that of the last pisp_solve.  Returns PISP_ERR_NOT_FACTORED when no
 * kept solutions exist, PISP_ERR_INVALID_ARG for a NULL g or sweeps < 0,
 * PISP_ERR_OOM if its workspace cannot be allocated. */
int pisp_adjoint(pisp_handle* h, const double* g, const double* w, double* grad_b,
                 double* grad_values, int32_t sweeps);

/* Host helper: per-solve weights for distinct shifts t[K] (Remark 2 written
 * for arbitrary shifts): beta_k = prod_{l != k} t_l / (t_l - t_k), the unique
 * solution of sum_k beta_k t_k^j = [j == 0], j = 0..K-1. */
int pisp_weights(const double* t, int32_t K, double* beta);

/* Structural row matching (Sec. IV: the paper applied Hopcroft-Karp as a
 * comparison, to move nonzeros onto the diagonal before a pivot-free solve).
 * Host only, no handle: finds a maximum matching of the rows of the n x n
 * pattern to its columns and writes row_perm[c] = the row matched to column
 * c, so that the matrix whose row c is row row_perm[c] of A has a
 * structurally nonzero diagonal.  Permuting the rows of A and of b this way
 * before pisp_analyze leaves the solution unchanged.
 *   n        unknowns (>= 0)
 *   row_ptr  host int64 [n + 1], CSR row pointer, nondecreasing from 0
 *   col_idx  host int32 [row_ptr[n]], column indices in [0, n)
 *   row_perm host int32 [n] output
 * Returns PISP_ERR_INVALID_ARG for a bad pattern or a structurally singular
 * one (no matching covers every column; pisp_last_error(NULL) says which). */
int pisp_match_rows(int32_t n, const int64_t* row_ptr, const int32_t* col_idx, int32_t* row_perm);

/* Batch solving under a CUDA graph (Sec. I, Alg. 1 run repeatedly on new
 * values, as in the Newton-Raphson use of Sec. IV): captures one whole step
 *   pisp_factor_perturbed(values, D, t, K, precision);
 *   pisp_solve(b, R, w, x, sweeps);
 *   and, if g != NULL, pisp_adjoint(g, w, grad_b, grad_values, adjoint_sweeps)
 * into a CUDA graph owned by the handle.  The step runs once eagerly first
 * (it checks the arguments, allocates every workspace and leaves its
 * results), then is captured on a private stream ordered after the work
 * already queued on the handle's stream.  pisp_graph_launch replays it on the
 * handle's stream: each replay reads the CURRENT contents of values, D, b and
 * g and writes x, grad_b and grad_values, so a caller updates those buffers
 * in place (same pointers) and replays.  t, K, precision, R, w and the sweep
 * counts are fixed at capture.  The buffers must stay allocated while the
 * graph is used.  The graph stays valid until the next pisp_analyze,
 * pisp_factor_perturbed, pisp_solve, pisp_refine, pisp_solve_host,
 * pisp_set_wait_limit or pisp_graph_capture on the handle (those may
 * rebuild the schedules or workspace the graph refers to); pisp_combine,
 * pisp_adjoint and the queries keep it.  Returns the error of the eager step,
 * or PISP_ERR_CUDA if the capture fails. */
int pisp_graph_capture(pisp_handle* h, const double* values, const double* D, const double* t,
                       int32_t K, int32_t precision, const double* b, int32_t R, const double* w,
                       double* x, int32_t sweeps, const double* g, double* grad_b, double* grad_values,
                       int32_t adjoint_sweeps);

/* Replays the captured step on the handle's stream.  Returns
 * PISP_ERR_INVALID_ARG when no valid captured step exists. */
int pisp_graph_launch(pisp_handle* h);

/* The bounded device waits (no counterpart in the paper).  Every dependency
 * wait of the persistent solves polls a completion counter at most `polls`
 * times (about 64 ns apart) and then gives up: it records the failure, the
 * task goes on with whatever data is there, the launch ends normally, and
 * pisp_get_status returns PISP_ERR_TIMEOUT until the next
 * pisp_factor_perturbed clears the record.  polls = 0 restores the default
 * (2^22 polls, a few tenths of a second per wait).  unreachable != 0 is a test
 * hook: the next solves also wait on one completion target raised by one, which
 * no task ever reaches, so that a wait runs out on purpose (results of those
 * solves are not valid); unreachable = 0 restores the true targets.  Applies
 * from the next pisp_solve / pisp_refine.  Returns PISP_ERR_INVALID_ARG for
 * polls < 0. */
int pisp_set_wait_limit(pisp_handle* h, int64_t polls, int32_t unreachable);

/* Adaptive FP64 residual sweeps (no counterpart in the paper, which solves
 * in FP64; a mixed-precision use of its Alg. 1).  With tol > 0 the `sweeps`
 * of pisp_solve / pisp_refine become a maximum, and each instance of a batch
 * stops on its own, by the stopping test of extra-precise iterative
 * refinement (Demmel, Hida, Kahan, Li, Mukherjee, Riedy, ACM TOMS 32(2),
 * 2006) with the contraction estimated from successive corrections: per RHS
 * r, with d_s = the largest |correction| of sweep s over the instance's
 * rows and all k, and from the second sweep on rho = d_s / d_{s-1}, r has
 * converged when d_s = 0 or when rho < 1/2 and rho / (1 - rho) d_s <=
 * tol * max |x_k|, and has stagnated when rho >= 1/2.  After the first sweep
 * only d_1 = 0 stops an instance.
 * The instance stops when all its right-hand sides have converged or
 * stagnated; the later sweeps skip its rows and fronts (the solve kernels
 * walk only the work units of the instances still iterating).  The sweeps
 * run as one device-side loop, a CUDA graph WHILE node that ends after the
 * last sweep any instance takes: inside a stream capture (pisp_graph_capture,
 * or the caller's own) as a node of the captured graph, otherwise as a graph
 * launched once on the stream.  tol = 0 restores fixed sweeps (every
 * instance, every sweep, plain launches).  Applies from the next pisp_solve /
 * pisp_refine / pisp_graph_capture (a captured step keeps the mode it was
 * captured with).  The transposed sweeps of pisp_adjoint stay fixed.
 * Returns PISP_ERR_INVALID_ARG for tol < 0 or not finite. */
int pisp_set_refinement(pisp_handle* h, double tol);

/* The sweeps of the last pisp_solve (or of the last solve inside
 * pisp_refine or a graph replay):
 *   sweeps_per_instance  host int32 [G] (or NULL): the sweeps instance g
 *                        took (with fixed sweeps: the sweep count for all)
 *   work                 host FP64 [max_sweeps] (or NULL): for s = 1 ..
 *                        max_sweeps, the fraction of the solve work (front
 *                        entries of the factors) that sweep s covered; 0
 *                        past the last sweep
 *   rows                 host FP64 [max_sweeps] (or NULL): the same for the
 *                        rows (the residuals' work)
 * Synchronises the stream.  Returns PISP_ERR_NOT_FACTORED before any solve,
 * PISP_ERR_INVALID_ARG for max_sweeps < 0. */
int pisp_refinement_stats(pisp_handle* h, int32_t* sweeps_per_instance, double* work, double* rows,
                          int32_t max_sweeps);

/* Synchronises the stream and copies host [G*K] status codes of the last
 * factorisation: 0 ok, PISP_ERR_ZERO_PIVOT or PISP_ERR_NONFINITE.  If
 * first_bad_col is not NULL it receives host [G*K] the first failing
 * permuted column (or -1).  Returns the worst code, or PISP_ERR_TIMEOUT if a
 * bounded dependency wait of a persistent solve gave up since the last
 * factorisation (its results are then not valid). */
int pisp_get_status(pisp_handle* h, int32_t* per_instance_k, int32_t* first_bad_col);

/* Statistics of the analysed pattern and the last factorisation. */
int pisp_get_stats(const pisp_handle* h, pisp_stats* out);

/* Copies the symbolic permutation: host perm[N] with perm[new] = old. */
int pisp_get_perm(const pisp_handle* h, int32_t* perm);

/* Supernode partition for structure checks: host arrays of n_supernodes
 * entries (c0, c1: permuted column range; ms: update rows) and host rows[]
 * of sum(ms) entries (the update-row lists, permuted indices).  Any pointer
 * may be NULL to query sizes through pisp_get_stats only. */
int pisp_get_supernodes(const pisp_handle* h, int32_t* c0, int32_t* c1, int32_t* ms,
                        int32_t* rows);

/* Copies the factor of perturbation k of the front owning permuted column
 * range [c0, c1): host FP64 out[F*F] column-major with L (unit, strictly
 * lower part), U (upper part incl. the diagonal) of the pivot block, L21 and
 * U12 in place and the Schur complement in the trailing block.  F is written
 * to *F_out.  Synchronises the stream.  For factor-level tests. */
int pisp_get_front(pisp_handle* h, int32_t supernode, int32_t k, double* out, int32_t* F_out);

/* Pivot spread of the last factorisation: for every instance g and
 * perturbation k, the smallest and largest |u_jj| over the pivots of g's
 * factor of A + t_k D (the quantities a static pivot order leaves unguarded,
 * Sec. I; a zero-diagonal entry rescued by a small perturbation shows as a
 * small minimum).  A non-finite pivot gives NaN for both.
 *   min_abs, max_abs  host FP64 [G*K] outputs, index g*K + k
 * Reads only the pivots (one strided device-to-host copy per front and k).
 * Synchronises the stream.  Returns PISP_ERR_NOT_FACTORED before a
 * factorisation. */
int pisp_get_pivot_range(pisp_handle* h, double* min_abs, double* max_abs);

/* End-to-end convenience: host buffers, copies inside.  Factor + solve +
 * combine of `values`, `D`, `b` given in host memory; x written to host.
 * b is copied on a stream of the handle's own, after values and D, while the
 * factorisation runs (an overlap only when b_host is pinned).  Synchronises
 * the stream. */
int pisp_solve_host(pisp_handle* h, const double* values_host, const double* D_host,
                    const double* t, int32_t K, int32_t precision, const double* b_host,
                    int32_t R, double* x_host, int32_t sweeps);

/* ---- allocation-free entry point ---------------------------------------- */
#define PISP_STATIC_MAX_N 128 /* largest system of pisp_dense_solve_static */
#define PISP_STATIC_MAX_R 64  /* most right-hand sides per call */

/* The paper has no counterpart to this call.  It serves callers that may not
 * allocate device memory when they call -- a memory budget fixed at start-up,
 * host callbacks or real-time loops that cannot take cudaMalloc's implicit
 * synchronisation, frameworks that hand over only their input and output
 * buffers -- whereas every other numeric entry point allocates its workspace
 * on first use.  It needs no handle and allocates nothing: the K
 * per-perturbation solutions live in one file-scope static device array of
 * PISP_K_MAX * PISP_STATIC_MAX_R * PISP_STATIC_MAX_N doubles (1 MiB) that
 * every GPU loading the library holds until the process exits.
 *
 * It computes, for one small dense system, the same result as
 * pisp_factor_perturbed + pisp_solve: x = sum_k beta_k (A + t_k D)^{-1} b with
 * pivot-free LU factors (FP64) and beta from pisp_weights(t).
 *   stream  cudaStream_t the work is enqueued on (NULL = legacy default)
 *   n       1..PISP_STATIC_MAX_N
 *   A       device FP64 [n][n], row-major, dense
 *   D       device FP64 [n], the diagonal perturbation
 *   t       host FP64 [K], distinct shifts, K in 1..PISP_K_MAX
 *   b       device FP64 [n][R], R in 1..PISP_STATIC_MAX_R
 *   x       device FP64 [n][R] output (may not alias b)
 * Sizes beyond the limits return PISP_ERR_UNSUPPORTED before any GPU work.
 * The first call on a device, with that device current, resolves the array's
 * device address (cudaGetSymbolAddress) and sets the kernel's shared-memory
 * limit; make that first call before any stream capture.  Calls share the
 * array, which keeps the last call's contents; each call overwrites the part
 * it reads, but calls that overlap on the GPU (other streams or host threads)
 * race on it, so order them on one stream.  A zero pivot is not reported:
 * it shows as Inf/NaN in x.  If a CUDA error is already pending on the
 * calling host thread, the call returns PISP_ERR_CUDA without launching and
 * leaves that error for the caller (cudaGetLastError still returns it); a
 * failed launch returns PISP_ERR_CUDA with nothing further enqueued. */
int pisp_dense_solve_static(void* stream, int32_t n, const double* A, const double* D,
                            const double* t, int32_t K, const double* b, int32_t R, double* x);

/* ---- profiling: CUDA events on the handle's stream around each kernel
 * family of each level, for per-family device time and achieved bandwidth.
 * Families: */
enum {
  PISP_PROF_FACTOR_SMALL = 0, /* shared-memory front factorisation */
  PISP_PROF_FACTOR_BIG = 1,   /* blocked front factorisation (assembly, panels, updates) */
  PISP_PROF_FORWARD = 2,      /* forward substitution */
  PISP_PROF_BACKWARD = 3,     /* backward substitution */
  PISP_PROF_RESIDUAL = 4,     /* FP64 residuals of the sweeps */
  PISP_PROF_COMBINE = 5,      /* expansion-weighted combine */
  PISP_PROF_FACTOR = 6,       /* the whole factorisation in one launch (factor policy 4) */
  PISP_PROF_SWEEP_LOOP = 7,   /* the adaptive sweeps (pisp_set_refinement), one device-side loop:
                                 residuals, correction solves and stopping tests of every iteration */
  PISP_PROF_FAMILIES = 8
};

/* on != 0: start recording brackets (forgets the previous recording); the
 * brackets recorded during a stream capture are replayed with the graph.
 * on == 0: stop recording. */
int pisp_profile(pisp_handle* h, int32_t on);

/* Synchronises the stream and adds the elapsed time, algorithmic bytes and
 * kernel launches of every recorded bracket to the per-family totals.  The
 * adaptive sweep loop counts the kernels of the iterations it ran and, per
 * iteration, the bytes of the instances it covered (front entries for the
 * solves, rows for the residuals and the stopping tests), as the last solve's
 * pisp_refinement_stats gives them. */
int pisp_profile_collect(pisp_handle* h);

/* Per-family totals since the last pisp_profile_reset: device milliseconds,
 * algorithmic bytes (minimum data each family must move) and launches.  Any
 * output pointer may be NULL. */
int pisp_profile_read(pisp_handle* h, int32_t family, double* ms, double* bytes,
                      int64_t* launches);

/* Clears the per-family totals. */
int pisp_profile_reset(pisp_handle* h);

/* Name of a family ("factor_small", ...), "" if out of range. */
const char* pisp_profile_name(int32_t family);

#ifdef __cplusplus
}
#endif

#endif /* PISP_H */
