// Internal declarations shared by the CUDA translation units of libpisp.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/pisp.h"

namespace pisp {

// Launchers set kernel attributes (shared-memory limits) and read the SM
// count once per device: these are per-device properties, so the flags are
// indexed by the current device.
constexpr int kMaxDevices = 64;
inline int current_device() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return 0;
  return d;
}

// Device view of the symbolic structure (all arrays live on the device).
struct SymDev {
  const int32_t* c0;         // [S] first permuted column of each supernode
  const int32_t* ns;         // [S] pivots
  const int32_t* ms;         // [S] update rows
  const int32_t* inst;       // [S] instance of each supernode
  const int64_t* front_off;  // [S+1] prefix of F^2
  const int64_t* vec_off;    // [S+1] prefix of F
  const int64_t* row_off;    // [S] offset into rows/emap
  const int32_t* child_off;  // [S+1]
  const int32_t* child;      // children, ascending
  const int64_t* amap_off;   // [S+1]
  const int32_t* amap_src;   // A value index
  const int32_t* amap_dst;   // position i + j*F in the front
  const int64_t* amap_coff;  // [sum F + 1] first entry of column j of front s at vec_off[s] + j
  const int32_t* rows;       // update rows (permuted global index)
  const int32_t* emap;       // position of each update row in the parent front
  const int32_t* parent;     // [S] parent supernode or -1
  const int64_t* inv_off;    // [sum F + 1] contributions to position vec_off[s] + j
  const int32_t* inv_child;  //   contributing child
  const int32_t* inv_a;      //   its update-row index
  const int64_t* inv_vbase;  //   the child's vec_off
  const int32_t* inv_cF;     //   the child's front size
  const int32_t* inv_col;    //   position in the child's front
  const int32_t* perm;       // [N] perm[new] = old
  const int32_t* iperm;      // [N] iperm[old] = new
  const int32_t* row_inst;   // [N] instance of each original row
  const int64_t* row_ptr;    // [N+1] CSR of A (original order)
  const int32_t* col;        // [nnz]
  const int64_t* at_ptr;     // [N+1] CSC of A: entries of column j at at_ptr[j]..at_ptr[j+1]
  const int32_t* at_row;     //   their rows
  const int32_t* at_src;     //   their CSR entry indices
  int64_t N;
  int32_t S;
};

// Shifts and combination weights, passed by value to kernels.
struct Shifts {
  double t[PISP_K_MAX];
  double w[PISP_K_MAX];
  int32_t K;
};

// One level of the assembly forest, split by front size.
struct LevelPlan {
  // small fronts (factored in shared memory), grouped by size class
  struct Group {
    int64_t off;      // offset into the device list of small fronts
    int32_t count;    // fronts in the group
    int32_t maxF;     // largest front in the group
    int32_t cluster;  // 0: one CTA per (front, k); C > 0: clusters of C CTAs
  };
  Group groups[8];
  int32_t n_groups = 0;
  // big fronts (blocked factorisation in global memory)
  int64_t big_off = 0;
  int32_t big_count = 0;
  int32_t big_maxF = 0;
  int32_t big_maxns = 0;
  // tile-DAG schedule of the big fronts (see launch_factor_big_dag)
  int64_t dag_task_off = 0;   // offset into the device task list
  int32_t dag_tasks = 0;
  int64_t dag_flag_off = 0;   // offset into the device flag area (per level)
  int32_t dag_flags = 0;
  int32_t dag_owner = 0;      // 1: the tasks are owner tiles
  int32_t own_ch = 0;         //    rows per owner tile (a multiple of 32)
  // every front of the level for the solves, grouped by size class
  Group sgroups[8];
  int32_t n_sgroups = 0;
  // algorithmic bytes per perturbation (a + b * R) of each kernel family,
  // used for the achieved-bandwidth figures of the profiling interface
  double bytes_fsmall = 0, bytes_fbig = 0;
  double bytes_fwd_a = 0, bytes_fwd_b = 0, bytes_bwd_a = 0, bytes_bwd_b = 0;
};

// Host copies needed to size the launches of the big-front path.
struct BigFrontHost {
  int32_t F, ns;
};

// One task of the tile-DAG factorisation of a level's big fronts.  Column
// blocks are 32 wide; kind 0 assembles block j, kind 1 factors the panel of
// pivots [32p, 32p+32), kind 2 applies panel p to block j (triangular solve
// of its U rows, then the trailing update of the rows below).  flags points
// at the (front, k) pair's counters: J "updates applied" per column block,
// then P "panel done" flags.
//
// The owner schedule (kind 3) uses the same record: one task per (front b,
// perturbation k, 32-column block j, row chunk q in p), flags pointing at the
// pair's P x Q "rows released" and P x J "U rows released" flags.
enum DagKind { kDagAsm = 0, kDagPanel = 1, kDagUpdate = 2, kDagOwner = 3 };
struct DagTask {
  int32_t kind, b, k, p, j, flags;
};

// Tasks of the one-launch factorisation (factor policy 4), all levels:
//   kFacWarp : s = offset of a group in the warp-front list, q = first task,
//              j = tasks in the group; task i is (front list[s + i / K],
//              k = i % K), 8 tasks (one per warp) per record;
//   kFacCta  : front s, perturbation k, factored in shared memory;
//   kFacOwner: owner tile (column block j, row chunk q) of front s,
//              perturbation k; flags = offset of the (front, k) pair's
//              release flags.
enum FactorKind { kFacWarp = 0, kFacCta = 1, kFacOwner = 2 };
struct FactorTask {
  int32_t kind, s, k, q, j, flags;
};

// Builds the task list of one level (b indexes the level's big-front list).
void build_dag_tasks(const BigFrontHost* big, int32_t nbig, int32_t K, std::vector<DagTask>& out,
                     int32_t& nflags);
// Owner tiles (32-column block j, chunk q of CH rows) of one level, sorted by
// (j, q) so that a tile only waits on tiles with smaller tickets; the record
// carries q in its p field.
void build_owner_tasks(const BigFrontHost* big, int32_t nbig, int32_t K, int32_t CH,
                       std::vector<DagTask>& out, int32_t& nflags);

// ---- factor (factor.cu) ----
// Each launcher returns the number of kernels launched (>= 0) or -1 on a
// launch error.  Small fronts of one level (shared-memory path):
int launch_factor_small(int precision, const SymDev& sd, const LevelPlan& lp,
                        const int32_t* d_small, const double* vals, const double* D,
                        const Shifts& sh, void* fronts, int32_t* status, int32_t* badcol,
                        cudaStream_t st);
// One size-class group of a level (the groups of a level are independent):
int launch_factor_small_group(int precision, const SymDev& sd, const LevelPlan& lp, int g,
                              const int32_t* d_small, const double* vals, const double* D,
                              const Shifts& sh, void* fronts, int32_t* status, int32_t* badcol,
                              cudaStream_t st);
// Big fronts of one level (blocked path):
int launch_factor_big(int precision, const SymDev& sd, const LevelPlan& lp, const int32_t* d_big,
                      const BigFrontHost* big_host, const double* vals, const double* D,
                      const Shifts& sh, void* fronts, int32_t* status, int32_t* badcol,
                      cudaStream_t st);
// Big fronts of one level as one persistent launch over the level's task
// list (tile DAG, or owner tiles when lp.dag_owner); ticket (1 int)
// and flags (lp.dag_flags ints) must be zero; err is set if a bounded
// dependency wait gave up.  tc != 0: FP32 owner-tile updates on the tensor
// cores (3xTF32, tcgen05).
int launch_factor_big_dag(int precision, const SymDev& sd, const LevelPlan& lp, const int32_t* d_big,
                          const DagTask* tasks, int* ticket, int* flags, int* err,
                          const double* vals, const double* D, const Shifts& sh, void* fronts,
                          int32_t* status, int32_t* badcol, int tc, cudaStream_t st);
// The whole factorisation in one persistent launch (factor policy 4): ticket
// (1 int), fdone (S*K ints) and flags must be zero; need[s] = 1 for warp and
// shared-memory fronts, tiles per (front, k) for owner fronts.
int launch_factor_persistent(int precision, const SymDev& sd, const FactorTask* tasks, int ntasks, int* ticket,
                             int* fdone, const int* need, int* flags, int* err, const int32_t* wlist,
                             const double* vals, const double* D, const Shifts& sh, void* fronts,
                             int32_t* status, int32_t* badcol, int CH, size_t smem, int64_t polls, int tc,
                             int ctas, cudaStream_t st);
// widest front the one-launch factorisation keeps in shared memory (wider:
// owner tiles), and its dynamic shared memory per CTA
int persistent_cta_front_limit(int precision);
size_t factor_persistent_smem(int precision, int CH, bool has_owner, int maxCtaF);
// largest front the tile-DAG path takes (its panel must fit in shared memory)
int max_dag_front(int precision);
// rows per owner tile for a level whose widest front is maxF (tc != 0: leave
// room for the tensor-core staging)
int owner_chunk_rows(int precision, int maxF, int tc);
// largest front (in elements of the given precision) the shared-memory path takes
int small_front_limit(int precision);
// CTAs per cluster for a front of size F factored in distributed shared
// memory: 0 for F <= 64 (single-CTA kernel), -1 if the front does not fit
// (blocked path in global memory)
int front_cluster_size(int F, int precision);
// largest front the blocked path can take (its panel must fit in shared memory)
int max_big_front(int precision);
// largest front the solve kernels can take
int max_solve_front(int precision);

// ---- solve (solve.cu) ----
enum RhsMode { RHS_BROADCAST = 0, RHS_PER_K = 1 };

// Work unit of the persistent solve schedule.  Segment units cover 256/SEG
// consecutive segment tasks of one group (a task = one front, a group of d
// consecutive shifts, one RHS chunk of 8): a = offset of the group in the
// schedule's front list, b = first task, c = tasks in the group, d = shifts
// per task.  Block units are one (front a, perturbation b, RHS chunk c of d
// right-hand sides), solved by a whole CTA.
enum UnitKind { kUnitSeg8 = 0, kUnitSeg16 = 1, kUnitSeg32 = 2, kUnitBlk = 3 };
struct SolveUnit {
  int32_t kind, a, b, c, d;
};
constexpr int kSolveChunk = 8;  // largest RHS chunk of a task (segment tasks use exactly 8)

// One launch solving every level of the forest (forward = L, bottom-up, or
// backward = U, top-down).  ticket (1 int) and done (S*K ints) must be zero;
// nch[s] is the number of RHS chunks (tasks) per (front s, k); err is set to 1
// if a bounded dependency wait gave up after `polls` polls (<= 0: the default
// limit of 2^22 polls); ctas = resident CTAs per SM the kernel is compiled
// for (2, 3 or 4; <= 0: 3 for FP32, 2 for FP64).  Adaptive sweeps: ucount
// (device, or nullptr) holds the length of a compacted list (nunits is then
// its capacity), act[g] (device, or nullptr) = 0 skips instance g's fronts.
int launch_solve_persistent(int precision, bool forward, const SymDev& sd, const SolveUnit* units,
                            int nunits, const int* ucount, const uint8_t* act, int* ticket, int* done,
                            int* err, const int* nch, const int32_t* d_all, const void* fronts,
                            const double* rhs, int rhs_mode, void* V, double* out, double* acc, int32_t R,
                            int32_t K, int32_t max_blk_F, int32_t ctas, int64_t polls, cudaStream_t st);
// RHS chunk for the CTAs solving one big front at a time (persistent schedule)
int pick_chunk(int fronts_in_level, int K, int R);
int launch_forward_level(int precision, bool trans, const SymDev& sd, const LevelPlan& lp,
                         const int32_t* d_all, const void* fronts, const double* rhs,
                         int rhs_mode, void* V, int32_t R, int32_t K, cudaStream_t st);
int launch_backward_level(int precision, bool trans, const SymDev& sd, const LevelPlan& lp,
                          const int32_t* d_all, const void* fronts, const void* V, double* out,
                          double* acc, int32_t R, int32_t K, cudaStream_t st);
int launch_combine(const SymDev& sd, const double* X, const Shifts& sh, int32_t R, double* x,
                   cudaStream_t st);
// The instances still iterating in the adaptive sweeps (device arrays
// written by the stopping test): act[g] flags, their number *nact, their ids
// ai[0..nact) in increasing order, and arow[q] = the rows of ai[0..q)
// (arow[nact] = all their rows).  Active row a belongs to instance ai[q] for
// the largest q with arow[q] <= a, at original row inst_off[ai[q]] + a - arow[q].
struct ActiveSet {
  const uint8_t* act;
  const int32_t* nact;
  const int32_t* ai;
  const int64_t* arow;
  const int64_t* inst_off;  // [G+1] first original row of each instance
};
// Rows a residual launch covers: every row; every row with Rk = 0 on the rows
// of instances that have stopped (whose correction is then exactly 0, for a
// solve that is not gated); only the rows of the active set.
enum ResidualMode { kResAll = 0, kResZeroStopped = 1, kResActive = 2 };
int launch_residual_per_k(const SymDev& sd, const double* vals, const double* D,
                          const Shifts& sh, const double* b, const double* X, int32_t R,
                          double* Rk, const ActiveSet& as, int mode, cudaStream_t st);
// Per instance g of the active set: X += Y on its rows, then per RHS r the
// largest |Y| and |X| over its rows and all k, atomically maxed into
// dmax/xmax [G][R] (zero on entry) as bit patterns.
int launch_refine_stats(const SymDev& sd, const ActiveSet& as, double* X, const double* Y, int32_t K, int32_t R,
                        unsigned long long* dmax, unsigned long long* xmax, cudaStream_t st);
// One CTA: the stopping test after sweep s = *sweep + 1 (s >= S: every
// instance stops), *sweep = s, nsw[g] = the sweeps instance g took, dmax /
// xmax zeroed again, then the active set: pre[g] = the active instances
// before g (G+1 ints), *nact, ai [G], arow [G+1].  has_cond: sets the
// conditional `cond` of a device-side sweep loop to continue while an
// instance is active and s < S.
int launch_refine_decide(int32_t G, int32_t R, double tol, int32_t S, int32_t* sweep,
                         cudaGraphConditionalHandle cond, int has_cond, uint8_t* act, unsigned long long* dmax,
                         unsigned long long* xmax, double* prevd, int32_t* nsw, int32_t* pre, int32_t* nact,
                         int32_t* ai, int64_t* arow, const int64_t* inst_off, cudaStream_t st);
// Every instance active, no sweep done: act, pre, *nact, ai, arow, *sweep.
int launch_refine_init(int32_t G, uint8_t* act, int32_t* pre, int32_t* nact, int32_t* ai, int64_t* arow,
                       const int64_t* inst_off, int32_t* sweep, cudaStream_t st);
// In-order compaction of the forward and backward unit lists to the units
// whose instance range [lo, hi] (rf, rb: int32 pairs) holds an active
// instance, into cf / cb with lengths in ucount[0..1]; cnt holds
// compact_scratch(nf, nb) ints of scratch.  Returns the kernels launched.
int compact_scratch(int32_t nf, int32_t nb);
int launch_compact_units(const SolveUnit* uf, const int32_t* rf, int32_t nf, SolveUnit* cf, const SolveUnit* ub,
                         const int32_t* rb, int32_t nb, SolveUnit* cb, const int32_t* pre, int32_t* cnt,
                         int32_t* ucount, cudaStream_t st);
// FP64 residuals of the transposed perturbed systems (adjoint sweeps)
int launch_residual_T_per_k(const SymDev& sd, const double* vals, const double* D,
                            const Shifts& sh, const double* g, const double* Lam, int32_t R,
                            double* Rk, cudaStream_t st);
int launch_residual(const SymDev& sd, const double* vals, const double* b, const double* x,
                    int32_t R, double* r, cudaStream_t st);
int launch_axpy(int64_t n, const double* y, double* x, cudaStream_t st);
int launch_grad_values(const SymDev& sd, const double* Lam, const double* X, const Shifts& sh,
                       int32_t R, double* grad, cudaStream_t st);
int launch_fill_nan_failed(const SymDev& sd, const int32_t* status, int32_t K, int32_t R,
                           double* x, cudaStream_t st);

}  // namespace pisp
