// C ABI of libpisp: handle, symbolic upload, level plans and the host-side
// orchestration of the level-scheduled factor / solve launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pisp.h"
#include "pisp_internal.h"
#include "symbolic.h"

namespace {

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
  ~Buf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  // grow-only device buffer; returns false on allocation failure
  bool ensure(size_t want) {
    want = std::max<size_t>(want, 256);
    if (want <= bytes) return true;
    release();
    if (cudaMalloc(&p, want) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return false;
    }
    bytes = want;
    return true;
  }
  template <typename T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

thread_local std::string g_last_error;  // for calls without a valid handle, per host thread

}  // namespace

struct pisp_handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  bool analyzed = false, factored = false, solved = false;
  pisp::Symbolic sym;
  double analyze_ms = 0.0;
  // device symbolic
  Buf c0, ns, ms, inst, front_off, vec_off, row_off, child_off, child, amap_off, amap_src,
      amap_dst, amap_coff, rows, emap, perm, iperm, row_inst, row_ptr, col, parent, inv_off, inv_child, inv_a, inv_vbase,
      inv_cF, inv_col, at_ptr, at_row, at_src;
  // persistent solve schedule (depends on K and R)
  int32_t schedule = 0;
  int32_t factor_policy = 0;
  int32_t units_K = 0, units_R = 0;
  int32_t n_units_f = 0, n_units_b = 0, units_maxF = 0;
  Buf units_f, units_b, ticket, done, serr, nch, d_wl;
  // adaptive FP64 residual sweeps (pisp_set_refinement): stopping tolerance
  // (0 = every sweep for every instance), the instance range [lo, hi] of
  // each persistent solve unit, the compacted unit lists and their lengths,
  // per-instance flags / sweep counts / correction sizes, instance offsets
  double sweep_tol = 0.0;
  int32_t last_sweeps = 0;
  bool last_adaptive = false, any_solve = false;
  bool last_loop = false;       // the last solve's sweeps ran as a device-side loop
  int32_t loop_kernels = 0;     // kernels per iteration of that loop
  cudaStream_t body_stream = nullptr;  // captures the loop's body
  std::vector<double> inst_w;  // solve work of each instance (front entries)
  Buf rng_f, rng_b, units_fc, units_bc, ucount, r_act, r_pre, r_dmax, r_xmax, r_prevd, r_nsw, d_inst_off;
  Buf r_nact, r_ai, r_arow, r_ccnt, r_sweep;
  // bounded waits of the persistent solves: polls before giving up (0 = the
  // default), and the test hook that makes one dependency unreachable
  int64_t wait_polls = 0;
  int32_t wait_unreachable = 0;
  // persistent solve tiling (pisp_options.solve_kfuse / solve_warp_maxF)
  int32_t kfuse = 1, warp_maxF = 32, solve_ctas = 0;
  int32_t factor_smem_maxF = 0;  // one-launch factorisation: widest shared-memory front (0 = limit)
  int32_t factor_tc = 0;         // FP32 owner-tile updates on the tensor cores
  int32_t factor_ctas = 0;       // one-launch factorisation: resident CTAs per SM (2 or 3; 0 = 2)
  pisp::SymDev sd{};
  // level plans (depend on the factor precision)
  int plan_precision = 0;
  std::vector<pisp::LevelPlan> plans;
  std::vector<int32_t> h_small, h_big, h_all;
  std::vector<pisp::BigFrontHost> h_bigF;
  std::vector<pisp::DagTask> h_dag;
  int32_t dag_max_flags = 0;
  Buf d_small, d_big, d_all, d_dag, dag_ticket, dag_flags;
  // one-launch factorisation (factor policy 4): all-level task list, the
  // warp-front list, completion targets, counters and owner release flags
  int32_t n_ftasks = 0, fac_CH = 32, fac_nflags = 0;
  size_t fac_smem = 0;
  double fac_bytes = 0;
  Buf d_ftasks, d_fwl, d_fneed, fdone, fflags, fticket;
  // numeric state
  int32_t K = 0, precision = 0, K_hint = 1, plan_K = 0;
  double t[PISP_K_MAX] = {}, beta[PISP_K_MAX] = {}, w_last[PISP_K_MAX] = {};
  Buf fronts, vals, D, status, badcol;
  // solve state
  int32_t R = 0;
  Buf V, X, Y, Rk, Lam, X2, rtmp, dtmp;
  // host-buffer entry point staging; b is copied on its own stream, after
  // the values and D and during the factorisation
  Buf in_vals, in_D, in_b, out_x;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copy_ev[2] = {};
  int launches = 0;
  // library-owned CUDA graph of one factor + solve step (pisp_graph_capture)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t cap_ev = nullptr;
  bool graph_valid = false;
  bool capturing = false;  // inside pisp_graph_capture's own factor + solve calls
  void drop_graph() {
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    if (graph) cudaGraphDestroy(graph);
    graph_exec = nullptr;
    graph = nullptr;
    graph_valid = false;
  }
  // profiling: CUDA events bracketing each kernel family per level
  // sweep = -1: a whole device-side sweep loop (launches per iteration, and
  // the bytes of one sweep over every instance split into rows and solve
  // work, scaled at collection per iteration by the share it covered)
  struct Bracket {
    int fam, e0, e1, launches;
    double bytes;
    int sweep;
    double bytes_rows, bytes_work;
  };
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;
  int prof_next = 0;
  std::vector<Bracket> prof_br;
  double prof_ms[PISP_PROF_FAMILIES] = {}, prof_bytes[PISP_PROF_FAMILIES] = {};
  int64_t prof_launches[PISP_PROF_FAMILIES] = {};
  // side streams for the independent size classes of a level, forked from
  // and joined back into `stream` with events (parallel branches when the
  // caller captures the work into a CUDA graph)
  static constexpr int kSide = 3;
  cudaStream_t side[kSide] = {}, big_side = nullptr;  // big_side: the level's wide fronts
  cudaEvent_t fork_ev = nullptr, join_ev[kSide] = {}, big_join = nullptr;
  ~pisp_handle() {
    drop_graph();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (copy_stream) cudaStreamDestroy(copy_stream);
    for (cudaEvent_t e : copy_ev)
      if (e) cudaEventDestroy(e);
    if (body_stream) cudaStreamDestroy(body_stream);
    if (cap_ev) cudaEventDestroy(cap_ev);
    for (cudaEvent_t e : prof_ev) cudaEventDestroy(e);
    for (int i = 0; i < kSide; ++i) {
      if (side[i]) cudaStreamDestroy(side[i]);
      if (join_ev[i]) cudaEventDestroy(join_ev[i]);
    }
    if (big_side) cudaStreamDestroy(big_side);
    if (big_join) cudaEventDestroy(big_join);
    if (fork_ev) cudaEventDestroy(fork_ev);
  }
};

namespace {

size_t esize(int precision) { return precision == PISP_FP32 ? 4 : 8; }

// NVTX range over one ABI call, so that profilers can scope a capture to a
// phase (factor, solve, ...); without an attached tool it costs a pointer test.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

int fail(pisp_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg; else g_last_error = msg;
  return code;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(h, PISP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// The handle's device is made current for one ABI call and the caller's
// current device is restored when the call returns, so the library never
// leaves a different device current behind (streams and buffers stay bound to
// the handle's device).
struct DeviceScope {
  int prev = -1;
  DeviceScope() = default;
  DeviceScope(const DeviceScope&) = delete;
  DeviceScope& operator=(const DeviceScope&) = delete;
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int set_device(pisp_handle* h, DeviceScope& scope) {
  if (h->device < 0)
    return fail(h, PISP_ERR_INVALID_ARG, "host-only handle (device -1): numeric calls need a device");
  int cur = -1;
  CK(cudaGetDevice(&cur));
  if (cur != h->device) {
    CK(cudaSetDevice(h->device));
    if (scope.prev < 0) scope.prev = cur;
  }
  return PISP_OK;
}

template <typename T>
int upload(pisp_handle* h, Buf& b, const std::vector<T>& v) {
  if (!b.ensure(v.size() * sizeof(T))) return fail(h, PISP_ERR_OOM, "device allocation failed");
  if (!v.empty()) CK(cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return PISP_OK;
}

#define TRY(x)            \
  do {                    \
    int rc_ = (x);        \
    if (rc_) return rc_;  \
  } while (0)

// Factor path of a front of size F > 64: 0 = one CTA with the front in shared
// memory, C >= 1 = a cluster of C CTAs (distributed shared memory), -1 = the
// blocked global-memory path.  Policy 0 (default): one CTA while the front
// fits, else the global path.  Policy 1: clusters wherever the front fits in
// at most 8 CTAs' shared memory.
int factor_path(const pisp_handle* h, int F, int precision) {
  if (h->factor_policy == 1) return pisp::front_cluster_size(F, precision);
  return F <= pisp::small_front_limit(precision) ? 0 : -1;
}

// Task list of the one-launch factorisation (factor policy 4): per level,
// bottom-up, the owner tiles of the fronts wider than the shared-memory
// limit (in (block, chunk) order, every tile after the ones it waits for),
// then one task per (front, k) for the shared-memory fronts, then groups of
// 8 (front, k) warp tasks for the fronts of at most 32.
int build_persistent_factor(pisp_handle* h, int precision, int32_t K) {
  const pisp::Symbolic& S = h->sym;
  const int Fc = h->factor_smem_maxF > 0 ? std::min(h->factor_smem_maxF, pisp::persistent_cta_front_limit(precision))
                                         : pisp::persistent_cta_front_limit(precision);
  int maxBig = 0, maxCta = 0;
  for (const auto& sn : S.sn) {
    if (sn.F() > Fc) maxBig = std::max(maxBig, sn.F());
    else if (sn.F() > 32) maxCta = std::max(maxCta, sn.F());
  }
  const int CH = maxBig > 0 ? pisp::owner_chunk_rows(precision, maxBig, h->factor_tc) : 32;
  std::vector<pisp::FactorTask> ft;
  std::vector<int32_t> wl, need(S.sn.size(), 1);
  int64_t nflags = 0;
  for (int l = 0; l < S.n_levels; ++l) {
    std::vector<int32_t> lst(S.level_sn.begin() + S.level_off[l], S.level_sn.begin() + S.level_off[l + 1]);
    std::sort(lst.begin(), lst.end(), [&](int32_t a, int32_t b) {
      const int fa = S.sn[a].F(), fb = S.sn[b].F();
      return fa != fb ? fa > fb : a < b;
    });
    std::vector<int32_t> big, cta, warp;
    for (int32_t sn : lst) {
      const int F = S.sn[sn].F();
      (F > Fc ? big : (F > 32 ? cta : warp)).push_back(sn);
    }
    if (!big.empty()) {
      std::vector<pisp::BigFrontHost> bh;
      for (int32_t sn : big) bh.push_back({S.sn[sn].F(), S.sn[sn].ns()});
      std::vector<pisp::DagTask> tk;
      int32_t nfl = 0;
      pisp::build_owner_tasks(bh.data(), (int32_t)bh.size(), K, CH, tk, nfl);
      for (const auto& t : tk)
        ft.push_back({pisp::kFacOwner, big[t.b], t.k, t.p, t.j, (int32_t)(nflags + t.flags)});
      for (size_t b = 0; b < big.size(); ++b)
        need[big[b]] = ((bh[b].F + 31) / 32) * ((bh[b].F + CH - 1) / CH);
      nflags += nfl;
      if (nflags >= INT32_MAX) return fail(h, PISP_ERR_UNSUPPORTED, "too many factor flags");
    }
    for (int32_t sn : cta)
      for (int k = 0; k < K; ++k) ft.push_back({pisp::kFacCta, sn, k, 0, 0, 0});
    if (!warp.empty()) {
      const int64_t off = (int64_t)wl.size(), tasks = (int64_t)warp.size() * K;
      if (off + (int64_t)warp.size() >= INT32_MAX || tasks >= INT32_MAX)
        return fail(h, PISP_ERR_UNSUPPORTED, "too many factor tasks");
      wl.insert(wl.end(), warp.begin(), warp.end());
      for (int64_t b = 0; b < tasks; b += 8)
        ft.push_back({pisp::kFacWarp, (int32_t)off, 0, (int32_t)b, (int32_t)tasks, 0});
    }
  }
  if ((int64_t)ft.size() >= INT32_MAX) return fail(h, PISP_ERR_UNSUPPORTED, "too many factor tasks");
  TRY(upload(h, h->d_ftasks, ft));
  TRY(upload(h, h->d_fwl, wl));
  TRY(upload(h, h->d_fneed, need));
  if (!h->fdone.ensure(S.sn.size() * (size_t)K * sizeof(int)) || !h->fflags.ensure((size_t)nflags * sizeof(int)) ||
      !h->fticket.ensure(sizeof(int)))
    return fail(h, PISP_ERR_OOM, "device allocation failed (factor schedule)");
  h->n_ftasks = (int32_t)ft.size();
  h->fac_CH = CH;
  h->fac_nflags = (int32_t)nflags;
  h->fac_smem = pisp::factor_persistent_smem(precision, CH, maxBig > 0, maxCta);
  return PISP_OK;
}

// Groups the supernodes of every level by front size: small fronts into
// shared-memory classes, big fronts into the blocked path, and all fronts into
// solve classes.
int build_plans(pisp_handle* h, int precision) {
  const pisp::Symbolic& S = h->sym;
  const int scls[6] = {8, 16, 32, 128, 512, INT_MAX};
  h->plans.assign(S.n_levels, pisp::LevelPlan());
  h->h_small.clear();
  h->h_big.clear();
  h->h_all.clear();
  h->h_bigF.clear();
  h->h_dag.clear();
  h->dag_max_flags = 0;
  for (int l = 0; l < S.n_levels; ++l) {
    pisp::LevelPlan& lp = h->plans[l];
    std::vector<int32_t> lst(S.level_sn.begin() + S.level_off[l],
                             S.level_sn.begin() + S.level_off[l + 1]);
    std::sort(lst.begin(), lst.end(), [&](int32_t a, int32_t b) {
      const int fa = S.sn[a].F(), fb = S.sn[b].F();
      return fa != fb ? fa < fb : a < b;
    });
    // on-chip fronts: single-CTA classes up to 64, then clusters of 1..8 CTAs
    const int fcls[3] = {16, 32, 64};
    int lo = 0;
    for (int c = 0; c < 3; ++c) {
      pisp::LevelPlan::Group G{(int64_t)h->h_small.size(), 0, 0, 0};
      for (int32_t s : lst) {
        const int F = S.sn[s].F();
        if (F > lo && F <= fcls[c]) {
          h->h_small.push_back(s);
          ++G.count;
          G.maxF = std::max(G.maxF, F);
        }
      }
      if (G.count) lp.groups[lp.n_groups++] = G;
      lo = fcls[c];
    }
    // fronts above 64: the factor path of each front (single CTA in shared
    // memory, a cluster of C CTAs in distributed shared memory, or the blocked
    // global-memory path) comes from the handle's factor policy
    auto path = [&](int F) { return factor_path(h, F, precision); };
    for (int C = 1; C <= 8; C *= 2) {
      pisp::LevelPlan::Group G{(int64_t)h->h_small.size(), 0, 0, C};
      for (int32_t s : lst) {
        const int F = S.sn[s].F();
        if (F > 64 && path(F) == C) {
          h->h_small.push_back(s);
          ++G.count;
          G.maxF = std::max(G.maxF, F);
        }
      }
      if (G.count) lp.groups[lp.n_groups++] = G;
    }
    {
      pisp::LevelPlan::Group G{(int64_t)h->h_small.size(), 0, 0, 0};
      for (int32_t s : lst) {
        const int F = S.sn[s].F();
        if (F > 64 && path(F) == 0) {
          h->h_small.push_back(s);
          ++G.count;
          G.maxF = std::max(G.maxF, F);
        }
      }
      if (G.count) lp.groups[lp.n_groups++] = G;
    }
    lp.big_off = (int64_t)h->h_big.size();
    for (int32_t s : lst) {
      const int F = S.sn[s].F();
      if (F > 64 && path(F) < 0) {
        h->h_big.push_back(s);
        h->h_bigF.push_back({F, S.sn[s].ns()});
        ++lp.big_count;
        lp.big_maxF = std::max(lp.big_maxF, F);
        lp.big_maxns = std::max(lp.big_maxns, S.sn[s].ns());
      }
    }
    // big fronts as one persistent launch per level: owner tiles (policy 0,
    // any front size) or the tile DAG (policy 2, while a panel fits in shared
    // memory); else (and under policies 1 and 3) one panel launch and one
    // update launch per 32 pivots
    const bool owner = h->factor_policy == 0;
    const bool dag = h->factor_policy == 2 && lp.big_maxF <= pisp::max_dag_front(precision);
    if (lp.big_count > 0 && (owner || dag)) {
      std::vector<pisp::DagTask> tk;
      int32_t nfl = 0;
      if (owner) {
        lp.own_ch = pisp::owner_chunk_rows(precision, lp.big_maxF, h->factor_tc);
        pisp::build_owner_tasks(h->h_bigF.data() + lp.big_off, lp.big_count, h->K_hint, lp.own_ch, tk, nfl);
      }
      else
        pisp::build_dag_tasks(h->h_bigF.data() + lp.big_off, lp.big_count, h->K_hint, tk, nfl);
      lp.dag_owner = owner ? 1 : 0;
      lp.dag_task_off = (int64_t)h->h_dag.size();
      lp.dag_tasks = (int32_t)tk.size();
      lp.dag_flags = nfl;
      h->h_dag.insert(h->h_dag.end(), tk.begin(), tk.end());
      h->dag_max_flags = std::max(h->dag_max_flags, nfl);
    }
    lo = 0;
    for (int c = 0; c < 6; ++c) {
      pisp::LevelPlan::Group G{(int64_t)h->h_all.size(), 0, 0, 0};
      for (int32_t s : lst) {
        const int F = S.sn[s].F();
        if (F > lo && F <= scls[c]) {
          h->h_all.push_back(s);
          ++G.count;
          G.maxF = std::max(G.maxF, F);
        }
      }
      if (G.count) lp.sgroups[lp.n_sgroups++] = G;
      lo = scls[c];
    }
    // algorithmic bytes per perturbation: what each kernel family must read
    // and write at least (values, indices, factor entries, vectors)
    const double p = (double)esize(precision);
    for (int32_t s : lst) {
      const pisp::Supernode& sn = S.sn[s];
      const double F = sn.F(), ns = sn.ns(), ms = sn.ms;
      double child = 0, childv = 0;
      for (int64_t q = S.child_off[s]; q < S.child_off[s + 1]; ++q) {
        const double cms = S.sn[S.child[q]].ms;
        child += cms * cms * p + cms * 4;
        childv += cms;
      }
      const double amap = (double)(S.amap_off[s + 1] - S.amap_off[s]);
      const double fac = amap * 16 + ns * 12 + child + F * F * p;
      if (sn.F() > 64 && path(sn.F()) < 0) lp.bytes_fbig += fac + 2 * F * F * p;
      else lp.bytes_fsmall += fac;
      lp.bytes_fwd_a += ns * 4 + childv * 4 + (ns * F - ns * (ns + 1) / 2) * p;
      lp.bytes_fwd_b += ns * 8 + childv * p + F * p;
      lp.bytes_bwd_a += ms * 4 + (ns * (ns + 1) / 2 + ns * ms) * p;
      lp.bytes_bwd_b += ms * 8 + ns * p + ns * 8;
    }
  }
  TRY(upload(h, h->d_small, h->h_small));
  TRY(upload(h, h->d_big, h->h_big));
  TRY(upload(h, h->d_all, h->h_all));
  TRY(upload(h, h->d_dag, h->h_dag));
  if (!h->dag_ticket.ensure(sizeof(int)) || !h->dag_flags.ensure((size_t)h->dag_max_flags * sizeof(int)))
    return fail(h, PISP_ERR_OOM, "device allocation failed (factor schedule)");
  if (h->factor_policy == 4) {
    TRY(build_persistent_factor(h, precision, h->K_hint));
    h->fac_bytes = 0;
    for (const auto& lp : h->plans) h->fac_bytes += lp.bytes_fsmall + lp.bytes_fbig;
  }
  h->plan_precision = precision;
  h->units_K = h->units_R = 0;
  return PISP_OK;
}

// Work units of the persistent solve, per level: fronts with more than 32
// pivots, or wider than h->warp_maxF, get one unit per (front, k, RHS chunk),
// solved by a whole CTA; every other front is split into segment tasks of 8,
// 16 or 32 lanes by its size (32 lanes, in blocks of 32 rows, for fronts
// wider than 32 with at most 32 pivots), one task per (front, group of
// h->kfuse consecutive shifts, RHS chunk of 8), 256/SEG tasks per unit.
// Within a level the CTA units come first, then the segment groups from the
// widest down; the forward order is levels bottom-up, the backward order
// top-down.  The fronts of the segment groups are listed in h->h_wl.
int build_units(pisp_handle* h, int32_t K, int32_t R) {
  const pisp::Symbolic& S = h->sym;
  const int segch = (R + pisp::kSolveChunk - 1) / pisp::kSolveChunk;
  std::vector<std::vector<pisp::SolveUnit>> per_level(S.n_levels);
  std::vector<int32_t> nch(S.sn.size(), segch);
  std::vector<std::vector<int32_t>> per_level_rng(S.n_levels);  // [lo, hi] instance range per unit
  std::vector<int32_t> wl;
  int maxF = 0;
  for (int l = 0; l < S.n_levels; ++l) {
    auto& U = per_level[l];
    auto& UR = per_level_rng[l];
    std::vector<int32_t> lst(S.level_sn.begin() + S.level_off[l], S.level_sn.begin() + S.level_off[l + 1]);
    std::sort(lst.begin(), lst.end(), [&](int32_t a, int32_t b) {
      const int fa = S.sn[a].F(), fb = S.sn[b].F();
      return fa != fb ? fa > fb : a < b;  // widest first
    });
    std::vector<int32_t> blk, g32w, g32, g16, g8;
    for (int32_t sn : lst) {
      const int F = S.sn[sn].F(), ns = S.sn[sn].ns();
      if (ns > 32 || F > std::max(32, h->warp_maxF)) blk.push_back(sn);
      else if (F > 32) g32w.push_back(sn);
      else if (F > 16) g32.push_back(sn);
      else if (F > 8) g16.push_back(sn);
      else g8.push_back(sn);
    }
    const int rc = pisp::pick_chunk(std::max<int>(1, (int)blk.size()), K, R);
    const int bch = (R + rc - 1) / rc;
    for (int32_t sn : blk) {
      maxF = std::max(maxF, S.sn[sn].F());
      nch[sn] = bch;
      for (int k = 0; k < K; ++k)
        for (int c = 0; c < bch; ++c) {
          U.push_back({pisp::kUnitBlk, sn, k, c, rc});
          UR.push_back(S.sn[sn].instance);
          UR.push_back(S.sn[sn].instance);
        }
    }
    auto seg_group = [&](const std::vector<int32_t>& g, int seg) -> int {
      if (g.empty()) return PISP_OK;
      const int kind = seg == 8 ? pisp::kUnitSeg8 : (seg == 16 ? pisp::kUnitSeg16 : pisp::kUnitSeg32);
      const int64_t off = (int64_t)wl.size();
      const int kf = std::max(1, std::min(h->kfuse, (int)K));
      const int64_t tasks = (int64_t)g.size() * ((K + kf - 1) / kf) * segch;
      if (tasks >= INT32_MAX || off >= INT32_MAX) return fail(h, PISP_ERR_UNSUPPORTED, "too many solve tasks");
      wl.insert(wl.end(), g.begin(), g.end());
      const int64_t per_front = (int64_t)((K + kf - 1) / kf) * segch;
      for (int64_t b = 0; b < tasks; b += 256 / seg) {
        U.push_back({kind, (int32_t)off, (int32_t)b, (int32_t)tasks, kf});
        int32_t lo = INT32_MAX, hi = -1;
        for (int64_t q = b; q < std::min(tasks, b + 256 / seg); q += 1) {
          const int32_t in = S.sn[g[q / per_front]].instance;
          lo = std::min(lo, in);
          hi = std::max(hi, in);
        }
        UR.push_back(lo);
        UR.push_back(hi);
      }
      return PISP_OK;
    };
    TRY(seg_group(g32w, 32));
    TRY(seg_group(g32, 32));
    TRY(seg_group(g16, 16));
    TRY(seg_group(g8, 8));
  }
  if (h->wait_unreachable) {
    // test hook: one front's completion target can never be reached, so the
    // waits on it (its parent's in the forward pass, its children's in the
    // backward pass) run out of polls
    for (size_t q = 0; q < S.sn.size(); ++q)
      if (S.sn[q].parent >= 0) {
        nch[q] += 1;
        break;
      }
  }
  std::vector<pisp::SolveUnit> f, b;
  std::vector<int32_t> rf, rb;
  for (int l = 0; l < S.n_levels; ++l) {
    f.insert(f.end(), per_level[l].begin(), per_level[l].end());
    rf.insert(rf.end(), per_level_rng[l].begin(), per_level_rng[l].end());
  }
  for (int l = S.n_levels - 1; l >= 0; --l) {
    b.insert(b.end(), per_level[l].begin(), per_level[l].end());
    rb.insert(rb.end(), per_level_rng[l].begin(), per_level_rng[l].end());
  }
  TRY(upload(h, h->units_f, f));
  TRY(upload(h, h->units_b, b));
  TRY(upload(h, h->rng_f, rf));
  TRY(upload(h, h->rng_b, rb));
  if (!h->units_fc.ensure(f.size() * sizeof(pisp::SolveUnit)) ||
      !h->units_bc.ensure(b.size() * sizeof(pisp::SolveUnit)) || !h->ucount.ensure(2 * sizeof(int32_t)))
    return fail(h, PISP_ERR_OOM, "device allocation failed (solve schedule)");
  TRY(upload(h, h->nch, nch));
  TRY(upload(h, h->d_wl, wl));
  if (!h->ticket.ensure(2 * sizeof(int)) || !h->serr.ensure(sizeof(int)) ||
      !h->done.ensure((size_t)S.sn.size() * K * sizeof(int)))
    return fail(h, PISP_ERR_OOM, "device allocation failed (solve schedule)");
  h->n_units_f = (int32_t)f.size();
  h->n_units_b = (int32_t)b.size();
  h->units_maxF = maxF;
  h->units_K = K;
  h->units_R = R;
  return PISP_OK;
}

int set_weights(pisp_handle* h, const double* w, double* out) {
  if (w) {
    for (int k = 0; k < h->K; ++k) {
      if (!std::isfinite(w[k])) return fail(h, PISP_ERR_INVALID_ARG, "non-finite weight");
      out[k] = w[k];
    }
  } else {
    for (int k = 0; k < h->K; ++k) out[k] = h->beta[k];
  }
  return PISP_OK;
}

pisp::Shifts make_shifts(const pisp_handle* h, const double* w) {
  pisp::Shifts sh{};
  sh.K = h->K;
  for (int k = 0; k < h->K; ++k) {
    sh.t[k] = h->t[k];
    sh.w[k] = w[k];
  }
  return sh;
}

const char* kFamilyNames[PISP_PROF_FAMILIES] = {"factor_small", "factor_big", "forward",
                                                "backward",     "residual",   "combine",
                                                "factor_persistent", "sweep_loop"};

// Event record that also works inside a stream capture: there it must become
// an event-record node of the graph (external record) to be timed on replay.
void record_event(pisp_handle* h, cudaEvent_t e, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  cudaEventRecordWithFlags(e, st,
                           cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                               : cudaEventRecordDefault);
}

// Records a start event of a profiling bracket; returns its index or -1.
int prof_begin(pisp_handle* h, cudaStream_t st = nullptr) {
  if (!h->prof_on) return -1;
  if (h->prof_next + 2 > (int)h->prof_ev.size()) {
    for (int q = 0; q < 64; ++q) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      h->prof_ev.push_back(e);
    }
  }
  const int i = h->prof_next;
  h->prof_next += 2;
  record_event(h, h->prof_ev[i], st ? st : h->stream);
  return i;
}

// Closes the bracket on the stream it was opened on (default: the handle's).
void prof_end(pisp_handle* h, int i, int fam, double bytes, int launches, cudaStream_t st = nullptr) {
  if (i < 0 || launches <= 0) return;
  record_event(h, h->prof_ev[i + 1], st ? st : h->stream);
  h->prof_br.push_back({fam, i, i + 1, launches, bytes, 0, 0.0, 0.0});
}

int count(pisp_handle* h, int n) {
  if (n < 0) {
    cudaError_t e = cudaGetLastError();
    return fail(h, PISP_ERR_CUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
  }
  h->launches += n;
  return PISP_OK;
}

// forward + backward over all levels; `rhs` broadcast [N][R] (original order)
// or per-perturbation [N][K][R] (permuted order); results to `out`
// (and added to `acc` when given).  Adaptive sweeps (persistent schedule):
// act skips the fronts of instances that have stopped and the compacted unit
// lists are walked.
int solve_pass(pisp_handle* h, bool trans, const double* rhs, int rhs_mode, double* out,
               double* acc, int32_t R, const uint8_t* act = nullptr) {
  const int L = h->sym.n_levels;
  if (!trans && h->schedule == 0) {
    if (h->units_K != h->K || h->units_R != R) TRY(build_units(h, h->K, R));
    const size_t nd = (size_t)h->sym.sn.size() * h->K * sizeof(int);
    double bf = 0, bb = 0;
    for (int l = 0; l < L; ++l) {
      bf += h->K * (h->plans[l].bytes_fwd_a + h->plans[l].bytes_fwd_b * R);
      bb += h->K * (h->plans[l].bytes_bwd_a + h->plans[l].bytes_bwd_b * R);
    }
    if (acc) bb += 16.0 * h->sym.N * h->K * R;
    CK(cudaMemsetAsync(h->ticket.p, 0, 2 * sizeof(int), h->stream));
    CK(cudaMemsetAsync(h->done.p, 0, nd, h->stream));
    const bool cmp = act != nullptr;  // gated: the compacted lists (whole lists before the first test)
    const int* ucf = cmp ? h->ucount.as<int>() : nullptr;
    const int* ucb = cmp ? h->ucount.as<int>() + 1 : nullptr;
    int pb = prof_begin(h);
    int n = pisp::launch_solve_persistent(
        h->precision, true, h->sd, (cmp ? h->units_fc : h->units_f).as<pisp::SolveUnit>(), h->n_units_f, ucf, act,
        h->ticket.as<int>(), h->done.as<int>(), h->serr.as<int>(), h->nch.as<int>(), h->d_wl.as<int32_t>(),
        h->fronts.p, rhs, rhs_mode, h->V.p, out, acc, R, h->K, h->units_maxF, h->solve_ctas, h->wait_polls,
        h->stream);
    TRY(count(h, n));
    prof_end(h, pb, PISP_PROF_FORWARD, bf, n);
    CK(cudaMemsetAsync(h->done.p, 0, nd, h->stream));
    pb = prof_begin(h);
    n = pisp::launch_solve_persistent(
        h->precision, false, h->sd, (cmp ? h->units_bc : h->units_b).as<pisp::SolveUnit>(), h->n_units_b, ucb, act,
        h->ticket.as<int>() + 1, h->done.as<int>(), h->serr.as<int>(), h->nch.as<int>(), h->d_wl.as<int32_t>(),
        h->fronts.p, rhs, rhs_mode, h->V.p, out, acc, R, h->K, h->units_maxF, h->solve_ctas, h->wait_polls,
        h->stream);
    TRY(count(h, n));
    prof_end(h, pb, PISP_PROF_BACKWARD, bb, n);
    return PISP_OK;
  }
  for (int l = 0; l < L; ++l) {
    const pisp::LevelPlan& lp = h->plans[l];
    const int pb = prof_begin(h);
    const int n = pisp::launch_forward_level(h->precision, trans, h->sd, lp, h->d_all.as<int32_t>(),
                                             h->fronts.p, rhs, rhs_mode, h->V.p, R, h->K, h->stream);
    TRY(count(h, n));
    prof_end(h, pb, PISP_PROF_FORWARD, h->K * (lp.bytes_fwd_a + lp.bytes_fwd_b * R), n);
  }
  for (int l = L - 1; l >= 0; --l) {
    const pisp::LevelPlan& lp = h->plans[l];
    const int pb = prof_begin(h);
    const int n = pisp::launch_backward_level(h->precision, trans, h->sd, lp, h->d_all.as<int32_t>(),
                                              h->fronts.p, h->V.p, out, acc, R, h->K, h->stream);
    TRY(count(h, n));
    prof_end(h, pb, PISP_PROF_BACKWARD,
             h->K * (lp.bytes_bwd_a + lp.bytes_bwd_b * R) + (acc ? 16.0 * h->sym.N * h->K * R / L : 0.0), n);
  }
  return PISP_OK;
}

// Sweeps per instance of the last solve, and for s = 1 .. max_sweeps the
// fraction of the solve work (front entries, fs[s]) and of the rows (fr[s])
// that sweep s covered (index 0 unused).  Synchronises the stream.
int sweep_fractions(pisp_handle* h, int max_sweeps, std::vector<int32_t>& nsw, std::vector<double>& fs,
                    std::vector<double>& fr) {
  const int32_t G = h->sym.G;
  nsw.assign(G, h->last_sweeps);
  if (h->last_adaptive) {
    CK(cudaMemcpyAsync(nsw.data(), h->r_nsw.p, (size_t)G * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  fs.assign(max_sweeps + 1, 0.0);
  fr.assign(max_sweeps + 1, 0.0);
  double ws = 0.0, wr = 0.0;
  for (int g = 0; g < G; ++g) {
    const double rows = (double)(h->sym.inst_off[g + 1] - h->sym.inst_off[g]);
    ws += h->inst_w[g];
    wr += rows;
    for (int s = 1; s <= std::min(max_sweeps, nsw[g]); ++s) {
      fs[s] += h->inst_w[g];
      fr[s] += rows;
    }
  }
  for (int s = 1; s <= max_sweeps; ++s) {
    fs[s] = ws > 0 ? fs[s] / ws : 0.0;
    fr[s] = wr > 0 ? fr[s] / wr : 0.0;
  }
  return PISP_OK;
}

// Algorithmic bytes of one forward + backward pass (all instances), as the
// brackets count them.
double solve_bytes(const pisp_handle* h, int32_t R) {
  double b = 0.0;
  for (int l = 0; l < h->sym.n_levels; ++l)
    b += h->K * (h->plans[l].bytes_fwd_a + h->plans[l].bytes_fwd_b * R + h->plans[l].bytes_bwd_a +
                 h->plans[l].bytes_bwd_b * R);
  return b;
}

// One adaptive sweep for the instances still iterating, the body of the
// device-side sweep loop: the FP64 residuals of their rows, the gated solves
// of their corrections (compacted unit lists of the persistent schedule; the
// per-level schedule solves every row, with zero residuals outside the active
// set), the corrections added to their solutions with the correction and
// solution sizes, the stopping test (which drives the loop's conditional
// `cond`) and the active set and unit lists of the next sweep.  No profiling
// brackets: a conditional body holds no events.
int sweep_body(pisp_handle* h, const double* rhs, double* X_out, int32_t R, int32_t S, const pisp::Shifts& sh,
               cudaGraphConditionalHandle cond) {
  const bool persistent = h->schedule == 0;
  const int32_t G = h->sym.G;
  uint8_t* act = h->r_act.as<uint8_t>();
  const pisp::ActiveSet as{act, h->r_nact.as<int32_t>(), h->r_ai.as<int32_t>(), h->r_arow.as<int64_t>(),
                           h->d_inst_off.as<int64_t>()};
  TRY(count(h, pisp::launch_residual_per_k(h->sd, h->vals.as<double>(), h->D.as<double>(), sh, rhs, X_out, R,
                                           h->Rk.as<double>(), as,
                                           persistent ? pisp::kResActive : pisp::kResZeroStopped, h->stream)));
  // the corrections go to Y only: the stats launch below adds them to X
  const bool prof_was = h->prof_on;
  h->prof_on = false;
  const int rc = solve_pass(h, false, h->Rk.as<double>(), pisp::RHS_PER_K, h->Y.as<double>(), nullptr, R,
                            persistent ? act : nullptr);
  h->prof_on = prof_was;
  TRY(rc);
  TRY(count(h, pisp::launch_refine_stats(h->sd, as, X_out, h->Y.as<double>(), h->K, R,
                                         h->r_dmax.as<unsigned long long>(), h->r_xmax.as<unsigned long long>(),
                                         h->stream)));
  TRY(count(h, pisp::launch_refine_decide(G, R, h->sweep_tol, S, h->r_sweep.as<int32_t>(), cond, 1, act,
                                          h->r_dmax.as<unsigned long long>(), h->r_xmax.as<unsigned long long>(),
                                          h->r_prevd.as<double>(), h->r_nsw.as<int32_t>(), h->r_pre.as<int32_t>(),
                                          h->r_nact.as<int32_t>(), h->r_ai.as<int32_t>(), h->r_arow.as<int64_t>(),
                                          h->d_inst_off.as<int64_t>(), h->stream)));
  if (persistent)
    TRY(count(h, pisp::launch_compact_units(
                     h->units_f.as<pisp::SolveUnit>(), h->rng_f.as<int32_t>(), h->n_units_f,
                     h->units_fc.as<pisp::SolveUnit>(), h->units_b.as<pisp::SolveUnit>(), h->rng_b.as<int32_t>(),
                     h->n_units_b, h->units_bc.as<pisp::SolveUnit>(), h->r_pre.as<int32_t>(),
                     h->r_ccnt.as<int32_t>(), h->ucount.as<int32_t>(), h->stream)));
  return PISP_OK;
}

// The adaptive sweeps as a device-side loop: a WHILE conditional node added
// to graph g after deps (its body one sweep_body, captured on a side stream
// into the node's body graph) that runs while the stopping test leaves an
// instance active, at most S times.
int add_sweep_loop(pisp_handle* h, cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                   cudaGraphNode_t* node_out, const double* rhs, double* X_out, int32_t R, int32_t S,
                   const pisp::Shifts& sh) {
  cudaGraphConditionalHandle cond = 0;
  CK(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  std::vector<cudaGraphNode_t> dv(deps, deps + ndeps);
  CK(cudaGraphAddNode(node_out, g, dv.data(), nullptr, dv.size(), &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  if (!h->body_stream) CK(cudaStreamCreateWithFlags(&h->body_stream, cudaStreamNonBlocking));
  CK(cudaStreamBeginCaptureToGraph(h->body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  const cudaStream_t outer = h->stream;
  h->stream = h->body_stream;
  const int launches0 = h->launches;
  const int rc = sweep_body(h, rhs, X_out, R, S, sh, cond);
  h->loop_kernels = h->launches - launches0;
  h->stream = outer;
  cudaGraph_t body_out = nullptr;
  const cudaError_t e = cudaStreamEndCapture(h->body_stream, &body_out);
  TRY(rc);
  if (e != cudaSuccess) return fail(h, PISP_ERR_CUDA, std::string("sweep loop capture: ") + cudaGetErrorString(e));
  return PISP_OK;
}

// The sweep loop on h->stream: inside a stream capture in progress, as a node
// of the graph being captured; otherwise as a graph of its own, built,
// launched once and destroyed (an executable graph destroyed in flight is
// freed when it completes), its host-side construction overlapping the work
// already queued.
int run_sweep_loop(pisp_handle* h, const double* rhs, double* X_out, int32_t R, int32_t S, const pisp::Shifts& sh) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  CK(cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, &g, &deps, nullptr, &ndeps));
  cudaGraphNode_t node = nullptr;
  if (cs == cudaStreamCaptureStatusActive) {
    if (!g) return fail(h, PISP_ERR_CUDA, "stream capture without a graph");
    TRY(add_sweep_loop(h, g, deps, ndeps, &node, rhs, X_out, R, S, sh));
    CK(cudaStreamUpdateCaptureDependencies(h->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return PISP_OK;
  }
  CK(cudaGraphCreate(&g, 0));
  int rc = add_sweep_loop(h, g, nullptr, 0, &node, rhs, X_out, R, S, sh);
  cudaGraphExec_t ge = nullptr;
  if (rc == PISP_OK && cudaGraphInstantiate(&ge, g, 0) != cudaSuccess)
    rc = fail(h, PISP_ERR_CUDA, std::string("sweep loop instantiate: ") + cudaGetErrorString(cudaGetLastError()));
  cudaGraphDestroy(g);
  TRY(rc);
  const cudaError_t e = cudaGraphLaunch(ge, h->stream);
  cudaGraphExecDestroy(ge);
  if (e != cudaSuccess) return fail(h, PISP_ERR_CUDA, std::string("sweep loop launch: ") + cudaGetErrorString(e));
  return PISP_OK;
}

// Per-perturbation solves of `rhs` (broadcast, original order) into X_out,
// followed by at most `sweeps` FP64 residual corrections of every x_k: all of
// them for every instance, or (pisp_set_refinement) per instance until its
// stopping test holds, as a device-side loop.
int solve_core(pisp_handle* h, const double* rhs, double* X_out, int32_t R, int32_t sweeps,
               const pisp::Shifts& sh) {
  TRY(solve_pass(h, false, rhs, pisp::RHS_BROADCAST, X_out, nullptr, R));
  const double N = (double)h->sym.N, KR = (double)h->K * R;
  const bool adapt = h->sweep_tol > 0.0 && sweeps > 0;
  const int32_t G = h->sym.G;
  h->last_sweeps = sweeps;
  h->last_adaptive = adapt;
  h->last_loop = false;
  h->any_solve = true;
  if (!adapt) {
    const pisp::ActiveSet none{};
    for (int it = 0; it < sweeps; ++it) {
      const int pb = prof_begin(h);
      const int n = pisp::launch_residual_per_k(h->sd, h->vals.as<double>(), h->D.as<double>(), sh, rhs, X_out, R,
                                                h->Rk.as<double>(), none, pisp::kResAll, h->stream);
      TRY(count(h, n));
      prof_end(h, pb, PISP_PROF_RESIDUAL, h->sym.nnzA * 12.0 + N * 20.0 + N * R * 8.0 + 2.0 * N * KR * 8.0, n);
      TRY(solve_pass(h, false, h->Rk.as<double>(), pisp::RHS_PER_K, h->Y.as<double>(), X_out, R));
    }
    return PISP_OK;
  }
  const size_t gr = (size_t)G * R * sizeof(unsigned long long);
  if (!h->r_act.ensure((size_t)G) || !h->r_pre.ensure((size_t)(G + 1) * sizeof(int32_t)) ||
      !h->r_nsw.ensure((size_t)G * sizeof(int32_t)) || !h->r_dmax.ensure(gr) || !h->r_xmax.ensure(gr) ||
      !h->r_prevd.ensure((size_t)G * R * sizeof(double)) || !h->r_nact.ensure(sizeof(int32_t)) ||
      !h->r_ai.ensure((size_t)G * sizeof(int32_t)) || !h->r_arow.ensure((size_t)(G + 1) * sizeof(int64_t)) ||
      !h->r_sweep.ensure(sizeof(int32_t)) ||
      !h->r_ccnt.ensure((size_t)pisp::compact_scratch(h->n_units_f, h->n_units_b) * sizeof(int32_t)))
    return fail(h, PISP_ERR_OOM, "device allocation failed (adaptive sweeps)");
  // every instance active; the compacted unit lists are the whole lists
  CK(cudaMemsetAsync(h->r_dmax.p, 0, gr, h->stream));
  CK(cudaMemsetAsync(h->r_xmax.p, 0, gr, h->stream));
  TRY(count(h, pisp::launch_refine_init(G, h->r_act.as<uint8_t>(), h->r_pre.as<int32_t>(), h->r_nact.as<int32_t>(),
                                        h->r_ai.as<int32_t>(), h->r_arow.as<int64_t>(),
                                        h->d_inst_off.as<int64_t>(), h->r_sweep.as<int32_t>(), h->stream)));
  if (h->schedule == 0)
    TRY(count(h, pisp::launch_compact_units(
                     h->units_f.as<pisp::SolveUnit>(), h->rng_f.as<int32_t>(), h->n_units_f,
                     h->units_fc.as<pisp::SolveUnit>(), h->units_b.as<pisp::SolveUnit>(), h->rng_b.as<int32_t>(),
                     h->n_units_b, h->units_bc.as<pisp::SolveUnit>(), h->r_pre.as<int32_t>(),
                     h->r_ccnt.as<int32_t>(), h->ucount.as<int32_t>(), h->stream)));
  const int pb = prof_begin(h);
  TRY(run_sweep_loop(h, rhs, X_out, R, sweeps, sh));
  h->last_loop = true;
  if (pb >= 0) {  // the loop as one bracket; bytes and launches are scaled at collection
    record_event(h, h->prof_ev[pb + 1], h->stream);
    h->prof_br.push_back({PISP_PROF_SWEEP_LOOP, pb, pb + 1, h->loop_kernels, 0.0, -1,
                          h->sym.nnzA * 12.0 + N * 20.0 + N * R * 8.0 + 5.0 * N * KR * 8.0, solve_bytes(h, R)});
  }
  return PISP_OK;
}

int ensure_solve_buffers(pisp_handle* h, int32_t R) {
  const size_t nkr = (size_t)h->sym.N * h->K * R * sizeof(double);
  const size_t v = (size_t)h->K * R * h->sym.vec_off.back() * esize(h->precision);
  if (!h->V.ensure(v) || !h->X.ensure(nkr) || !h->Y.ensure(nkr) || !h->Rk.ensure(nkr))
    return fail(h, PISP_ERR_OOM, "device allocation failed (solve workspace)");
  return PISP_OK;
}

}  // namespace

extern "C" {

const char* pisp_last_error(const pisp_handle* h) {
  return h ? h->err.c_str() : g_last_error.c_str();
}

int pisp_create(pisp_handle** out, int device, void* stream) {
  if (!out) return fail(nullptr, PISP_ERR_INVALID_ARG, "null output pointer");
  *out = nullptr;
  if (device != -1) {
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev)
      return fail(nullptr, PISP_ERR_CUDA, "no such CUDA device");
  }
  pisp_handle* h = new pisp_handle();
  h->device = device;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  *out = h;
  return PISP_OK;
}

int pisp_destroy(pisp_handle* h) {
  if (!h) return PISP_OK;
  if (h->device < 0) {
    delete h;
    return PISP_OK;
  }
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != h->device) cudaSetDevice(h->device);
  delete h;
  if (cur >= 0) cudaSetDevice(cur);
  return PISP_OK;
}

int pisp_set_stream(pisp_handle* h, void* stream) {
  if (!h) return fail(h, PISP_ERR_INVALID_ARG, "null handle");
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  return PISP_OK;
}

}  // extern "C"

namespace {

int analyze_impl(pisp_handle* h, int32_t G, const int32_t* n, const int64_t* row_ptr,
                 const int32_t* col_idx, const pisp_options* opt) {
  NvtxRange nvtx_("pisp_analyze");
  h->drop_graph();
  DeviceScope dev_scope_;
  if (G < 1 || !n || !row_ptr) return fail(h, PISP_ERR_INVALID_ARG, "bad instance description");
  int64_t N = 0;
  for (int g = 0; g < G; ++g) N += n[g] < 0 ? 0 : n[g];
  if (row_ptr[N] > 0 && !col_idx) return fail(h, PISP_ERR_INVALID_ARG, "null col_idx");
  if (h->device >= 0) {
    TRY(set_device(h, dev_scope_));
    if (!h->fork_ev) {  // side streams of the factorisation (created outside any capture)
      CK(cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
      for (int i = 0; i < pisp_handle::kSide; ++i) {
        CK(cudaStreamCreateWithFlags(&h->side[i], cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&h->join_ev[i], cudaEventDisableTiming));
      }
      CK(cudaStreamCreateWithFlags(&h->big_side, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&h->big_join, cudaEventDisableTiming));
    }
  }
  pisp::SymbolicOptions so;
  h->schedule = opt ? opt->solve_schedule : 0;
  h->factor_policy = opt ? opt->factor_policy : 0;
  h->kfuse = opt && opt->solve_kfuse > 0 ? opt->solve_kfuse : 1;
  h->warp_maxF = opt && opt->solve_warp_maxF > 0 ? opt->solve_warp_maxF : 32;
  h->solve_ctas = opt && opt->solve_ctas_per_sm > 0 ? std::min(4, std::max(2, opt->solve_ctas_per_sm)) : 0;
  h->factor_smem_maxF = opt && opt->factor_smem_maxF > 0 ? opt->factor_smem_maxF : 0;
  h->factor_tc = opt && opt->factor_tc ? 1 : 0;
  h->factor_ctas = opt && opt->factor_ctas_per_sm > 0 ? opt->factor_ctas_per_sm : 0;
  h->units_K = h->units_R = 0;
  if (opt) {
    so.ordering = opt->ordering;
    if (opt->relax_small >= 0) so.relax_small = opt->relax_small;
    if (opt->relax_zeros >= 0) so.relax_zeros = opt->relax_zeros;
    if (opt->analyze_threads < 0) return fail(h, PISP_ERR_INVALID_ARG, "analyze_threads must be >= 0");
    so.threads = opt->analyze_threads;
  }
  h->analyzed = h->factored = h->solved = false;
  h->any_solve = h->last_adaptive = false;
  h->plan_precision = 0;
  const auto t0 = std::chrono::steady_clock::now();
  std::string msg = pisp::analyze(G, n, row_ptr, col_idx, so, h->sym);
  h->analyze_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (!msg.empty()) return fail(h, PISP_ERR_INVALID_ARG, msg);
  msg = pisp::validate(h->sym);
  if (!msg.empty()) return fail(h, PISP_ERR_BOUNDS, msg);
  const pisp::Symbolic& S = h->sym;
  if (S.max_front > 46340) return fail(h, PISP_ERR_UNSUPPORTED, "front larger than 46340");
  if (h->device < 0) {  // host-only handle: symbolic structure for inspection only
    h->analyzed = true;
    return PISP_OK;
  }
  // upload the structure
  const int nS = (int)S.sn.size();
  std::vector<int32_t> c0(nS), ns(nS), ms(nS), inst(nS), child_off(nS + 1), par(nS);
  std::vector<int64_t> row_off(nS);
  for (int s = 0; s < nS; ++s) {
    c0[s] = S.sn[s].c0;
    ns[s] = S.sn[s].ns();
    ms[s] = S.sn[s].ms;
    inst[s] = S.sn[s].instance;
    par[s] = S.sn[s].parent;
    row_off[s] = S.sn[s].row_off;
  }
  for (int s = 0; s <= nS; ++s) child_off[s] = (int32_t)S.child_off[s];
  std::vector<int32_t> row_inst(S.N);
  for (int g = 0; g < G; ++g)
    for (int64_t i = S.inst_off[g]; i < S.inst_off[g + 1]; ++i) row_inst[i] = g;
  std::vector<int64_t> rp(row_ptr, row_ptr + S.N + 1);
  std::vector<int32_t> cl(col_idx ? col_idx : nullptr, col_idx ? col_idx + S.nnzA : nullptr);
  TRY(upload(h, h->c0, c0));
  TRY(upload(h, h->ns, ns));
  TRY(upload(h, h->ms, ms));
  TRY(upload(h, h->inst, inst));
  TRY(upload(h, h->front_off, S.front_off));
  TRY(upload(h, h->vec_off, S.vec_off));
  TRY(upload(h, h->row_off, row_off));
  TRY(upload(h, h->child_off, child_off));
  TRY(upload(h, h->child, S.child));
  TRY(upload(h, h->amap_off, S.amap_off));
  TRY(upload(h, h->amap_src, S.amap_src));
  TRY(upload(h, h->amap_dst, S.amap_dst));
  TRY(upload(h, h->amap_coff, S.amap_coff));
  TRY(upload(h, h->rows, S.rows));
  TRY(upload(h, h->emap, S.emap));
  TRY(upload(h, h->perm, S.perm));
  TRY(upload(h, h->iperm, S.iperm));
  TRY(upload(h, h->row_inst, row_inst));
  TRY(upload(h, h->d_inst_off, S.inst_off));
  h->inst_w.assign(G, 0.0);
  for (int s = 0; s < nS; ++s) h->inst_w[S.sn[s].instance] += (double)S.sn[s].F() * S.sn[s].F();
  TRY(upload(h, h->row_ptr, rp));
  TRY(upload(h, h->col, cl));
  TRY(upload(h, h->parent, par));
  TRY(upload(h, h->inv_off, S.inv_off));
  TRY(upload(h, h->inv_child, S.inv_child));
  TRY(upload(h, h->inv_a, S.inv_a));
  TRY(upload(h, h->inv_vbase, S.inv_vbase));
  TRY(upload(h, h->inv_cF, S.inv_cF));
  TRY(upload(h, h->inv_col, S.inv_col));
  {
    // columns of A (CSC by counting sort): row and CSR entry of every entry of
    // column j, for the transposed residuals of the adjoint sweeps
    std::vector<int64_t> atp(S.N + 1, 0);
    for (int64_t e = 0; e < S.nnzA; ++e) ++atp[cl[e] + 1];
    for (int64_t j = 0; j < S.N; ++j) atp[j + 1] += atp[j];
    std::vector<int32_t> atr(S.nnzA), ats(S.nnzA);
    std::vector<int64_t> fill(atp.begin(), atp.end() - 1);
    for (int64_t i = 0; i < S.N; ++i)
      for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
        const int64_t q = fill[cl[e]]++;
        atr[q] = (int32_t)i;
        ats[q] = (int32_t)e;
      }
    TRY(upload(h, h->at_ptr, atp));
    TRY(upload(h, h->at_row, atr));
    TRY(upload(h, h->at_src, ats));
  }
  pisp::SymDev& sd = h->sd;
  sd.c0 = h->c0.as<int32_t>();
  sd.ns = h->ns.as<int32_t>();
  sd.ms = h->ms.as<int32_t>();
  sd.inst = h->inst.as<int32_t>();
  sd.front_off = h->front_off.as<int64_t>();
  sd.vec_off = h->vec_off.as<int64_t>();
  sd.row_off = h->row_off.as<int64_t>();
  sd.child_off = h->child_off.as<int32_t>();
  sd.child = h->child.as<int32_t>();
  sd.amap_off = h->amap_off.as<int64_t>();
  sd.amap_src = h->amap_src.as<int32_t>();
  sd.amap_dst = h->amap_dst.as<int32_t>();
  sd.amap_coff = h->amap_coff.as<int64_t>();
  sd.rows = h->rows.as<int32_t>();
  sd.emap = h->emap.as<int32_t>();
  sd.perm = h->perm.as<int32_t>();
  sd.iperm = h->iperm.as<int32_t>();
  sd.row_inst = h->row_inst.as<int32_t>();
  sd.row_ptr = h->row_ptr.as<int64_t>();
  sd.col = h->col.as<int32_t>();
  sd.parent = h->parent.as<int32_t>();
  sd.inv_off = h->inv_off.as<int64_t>();
  sd.inv_child = h->inv_child.as<int32_t>();
  sd.inv_a = h->inv_a.as<int32_t>();
  sd.inv_vbase = h->inv_vbase.as<int64_t>();
  sd.inv_cF = h->inv_cF.as<int32_t>();
  sd.inv_col = h->inv_col.as<int32_t>();
  sd.at_ptr = h->at_ptr.as<int64_t>();
  sd.at_row = h->at_row.as<int32_t>();
  sd.at_src = h->at_src.as<int32_t>();
  sd.N = S.N;
  sd.S = nS;
  h->analyzed = true;
  return PISP_OK;
}

}  // namespace

extern "C" {

int pisp_analyze(pisp_handle* h, int32_t G, const int32_t* n, const int64_t* row_ptr,
                 const int32_t* col_idx, const pisp_options* opt) {
  if (!h) return fail(h, PISP_ERR_INVALID_ARG, "null handle");
  // no C++ exception may cross the C boundary: host allocation failures of
  // the analysis (or of its staging vectors) become error codes
  try {
    return analyze_impl(h, G, n, row_ptr, col_idx, opt);
  } catch (const std::bad_alloc&) {
    h->analyzed = false;
    return fail(h, PISP_ERR_OOM, "out of host memory in pisp_analyze");
  } catch (const std::exception& e) {
    h->analyzed = false;
    return fail(h, PISP_ERR_INVALID_ARG, std::string("pisp_analyze failed: ") + e.what());
  }
}

int pisp_match_rows(int32_t n, const int64_t* row_ptr, const int32_t* col_idx, int32_t* row_perm) {
  if (n < 0 || (n > 0 && (!row_ptr || !row_perm))) return fail(nullptr, PISP_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return PISP_OK;
  if (row_ptr[0] != 0) return fail(nullptr, PISP_ERR_INVALID_ARG, "row_ptr[0] must be 0");
  for (int32_t i = 0; i < n; ++i)
    if (row_ptr[i + 1] < row_ptr[i]) return fail(nullptr, PISP_ERR_INVALID_ARG, "row_ptr must be nondecreasing");
  if (row_ptr[n] > 0 && !col_idx) return fail(nullptr, PISP_ERR_INVALID_ARG, "null col_idx");
  for (int64_t e = 0; e < row_ptr[n]; ++e)
    if (col_idx[e] < 0 || col_idx[e] >= n) return fail(nullptr, PISP_ERR_INVALID_ARG, "column index out of range");
  std::vector<int32_t> row_of_col;
  const std::string err = pisp::match_rows(n, row_ptr, col_idx, row_of_col);
  if (!err.empty()) return fail(nullptr, PISP_ERR_INVALID_ARG, err);
  std::copy(row_of_col.begin(), row_of_col.end(), row_perm);
  return PISP_OK;
}

int pisp_weights(const double* t, int32_t K, double* beta) {
  if (!t || !beta || K < 1 || K > PISP_K_MAX)
    return fail(nullptr, PISP_ERR_INVALID_ARG, "pisp_weights: bad arguments");
  for (int k = 0; k < K; ++k) {
    if (!std::isfinite(t[k])) return fail(nullptr, PISP_ERR_INVALID_ARG, "non-finite shift");
    for (int l = 0; l < k; ++l)
      if (t[l] == t[k]) return fail(nullptr, PISP_ERR_INVALID_ARG, "shifts must be distinct");
  }
  // Lagrange basis polynomial of node t_k evaluated at 0: the unique weights
  // with sum_k beta_k t_k^j = [j == 0] for j < K.
  for (int k = 0; k < K; ++k) {
    long double p = 1.0L;
    for (int l = 0; l < K; ++l)
      if (l != k) p *= (long double)t[l] / ((long double)t[l] - (long double)t[k]);
    beta[k] = (double)p;
  }
  return PISP_OK;
}

int pisp_factor_perturbed(pisp_handle* h, const double* values, const double* D,
                          const double* t, int32_t K, int32_t precision) {
  if (!h) return fail(h, PISP_ERR_INVALID_ARG, "null handle");
  if (!h->capturing) h->graph_valid = false;
  NvtxRange nvtx_("pisp_factor_perturbed");
  if (!h->analyzed) return fail(h, PISP_ERR_NOT_ANALYZED, "pisp_analyze has not succeeded");
  if (K < 1 || K > PISP_K_MAX || !t) return fail(h, PISP_ERR_INVALID_ARG, "K must be in 1..16");
  if (precision != PISP_FP32 && precision != PISP_FP64)
    return fail(h, PISP_ERR_INVALID_ARG, "precision must be PISP_FP32 or PISP_FP64");
  const pisp::Symbolic& S = h->sym;
  if ((S.nnzA > 0 && !values) || (S.N > 0 && !D)) return fail(h, PISP_ERR_INVALID_ARG, "null values or D");
  // the owner tiles (policy 0) take fronts of any size; the per-panel path,
  // which the other policies fall back to, needs a panel in shared memory
  if (S.max_front > pisp::max_solve_front(precision) ||
      (h->factor_policy != 0 && h->factor_policy != 4 && S.max_front > pisp::max_big_front(precision)))
    return fail(h, PISP_ERR_UNSUPPORTED, "front too large for this precision");
  double beta[PISP_K_MAX];
  if (pisp_weights(t, K, beta) != PISP_OK) return fail(h, PISP_ERR_INVALID_ARG, g_last_error);
  DeviceScope dev_scope_;
  TRY(set_device(h, dev_scope_));
  h->factored = h->solved = false;
  h->K_hint = K;
  if (h->plan_precision != precision || h->plan_K != K) TRY(build_plans(h, precision));
  h->plan_K = K;
  h->K = K;
  h->precision = precision;
  for (int k = 0; k < K; ++k) {
    h->t[k] = t[k];
    h->beta[k] = beta[k];
  }
  if (!h->fronts.ensure((size_t)K * S.front_elems * esize(precision)) ||
      !h->vals.ensure(S.nnzA * sizeof(double)) || !h->D.ensure(S.N * sizeof(double)) ||
      !h->status.ensure((size_t)S.G * K * sizeof(int32_t)) ||
      !h->badcol.ensure((size_t)S.G * K * sizeof(int32_t)))
    return fail(h, PISP_ERR_OOM, "device allocation failed (factor workspace)");
  if (S.nnzA) CK(cudaMemcpyAsync(h->vals.p, values, S.nnzA * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  if (S.N) CK(cudaMemcpyAsync(h->D.p, D, S.N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemsetAsync(h->status.p, 0, (size_t)S.G * K * sizeof(int32_t), h->stream));
  CK(cudaMemsetAsync(h->badcol.p, 0x7f, (size_t)S.G * K * sizeof(int32_t), h->stream));
  if (!h->serr.ensure(sizeof(int))) return fail(h, PISP_ERR_OOM, "device allocation failed");
  CK(cudaMemsetAsync(h->serr.p, 0, sizeof(int), h->stream));
  h->launches = 0;
  const pisp::Shifts sh = make_shifts(h, h->beta);
  if (h->factor_policy == 4) {
    // every level, every shift and every instance in one persistent launch
    CK(cudaMemsetAsync(h->fticket.p, 0, sizeof(int), h->stream));
    CK(cudaMemsetAsync(h->fdone.p, 0, S.sn.size() * (size_t)K * sizeof(int), h->stream));
    if (h->fac_nflags) CK(cudaMemsetAsync(h->fflags.p, 0, (size_t)h->fac_nflags * sizeof(int), h->stream));
    const int pb = prof_begin(h);
    const int n = pisp::launch_factor_persistent(
        precision, h->sd, h->d_ftasks.as<pisp::FactorTask>(), h->n_ftasks, h->fticket.as<int>(), h->fdone.as<int>(),
        h->d_fneed.as<int>(), h->fflags.as<int>(), h->serr.as<int>(), h->d_fwl.as<int32_t>(), h->vals.as<double>(),
        h->D.as<double>(), sh, h->fronts.p, h->status.as<int32_t>(), h->badcol.as<int32_t>(), h->fac_CH,
        h->fac_smem, h->wait_polls, h->factor_tc, h->factor_ctas, h->stream);
    TRY(count(h, n));
    prof_end(h, pb, PISP_PROF_FACTOR, K * h->fac_bytes, n);
    h->factored = true;
    return PISP_OK;
  }
  for (int l = 0; l < S.n_levels; ++l) {
    // The fronts of a level are independent: its wide fronts (owner kernel)
    // and each size class of its narrow ones go to their own streams, forked
    // from the work queued so far and joined before the next level (parallel
    // branches when the caller captures the work into a CUDA graph).
    const pisp::LevelPlan& lp = h->plans[l];
    const bool mixed = lp.big_count > 0 && lp.n_groups > 0;
    const int used = lp.n_groups > 1 ? std::min(lp.n_groups - 1, pisp_handle::kSide) : 0;
    if (used > 0 || mixed) CK(cudaEventRecord(h->fork_ev, h->stream));
    for (int i = 0; i < used; ++i) CK(cudaStreamWaitEvent(h->side[i], h->fork_ev, 0));
    const cudaStream_t bst = mixed ? h->big_side : h->stream;
    if (mixed) CK(cudaStreamWaitEvent(bst, h->fork_ev, 0));
    if (lp.big_count > 0) {
      const int pb = prof_begin(h, bst);
      int n = 0;
      if (lp.dag_tasks > 0) {
        CK(cudaMemsetAsync(h->dag_ticket.p, 0, sizeof(int), bst));
        CK(cudaMemsetAsync(h->dag_flags.p, 0, (size_t)lp.dag_flags * sizeof(int), bst));
        n = pisp::launch_factor_big_dag(precision, h->sd, lp, h->d_big.as<int32_t>(),
                                        h->d_dag.as<pisp::DagTask>(), h->dag_ticket.as<int>(),
                                        h->dag_flags.as<int>(), h->serr.as<int>(), h->vals.as<double>(),
                                        h->D.as<double>(), sh, h->fronts.p, h->status.as<int32_t>(),
                                        h->badcol.as<int32_t>(), h->factor_tc, bst);
      } else {
        n = pisp::launch_factor_big(precision, h->sd, lp, h->d_big.as<int32_t>(), h->h_bigF.data(),
                                    h->vals.as<double>(), h->D.as<double>(), sh, h->fronts.p,
                                    h->status.as<int32_t>(), h->badcol.as<int32_t>(), bst);
      }
      TRY(count(h, n));
      prof_end(h, pb, PISP_PROF_FACTOR_BIG, K * lp.bytes_fbig, n, bst);
    }
    if (lp.n_groups > 0) {
      const int pb = prof_begin(h);
      int n = 0;
      for (int g = 0; g < lp.n_groups && n >= 0; ++g) {
        const cudaStream_t st = g == 0 ? h->stream : h->side[(g - 1) % pisp_handle::kSide];
        const int m = pisp::launch_factor_small_group(precision, h->sd, lp, g, h->d_small.as<int32_t>(),
                                                      h->vals.as<double>(), h->D.as<double>(), sh,
                                                      h->fronts.p, h->status.as<int32_t>(),
                                                      h->badcol.as<int32_t>(), st);
        n = m < 0 ? -1 : n + m;
      }
      for (int i = 0; i < used; ++i) {
        CK(cudaEventRecord(h->join_ev[i], h->side[i]));
        CK(cudaStreamWaitEvent(h->stream, h->join_ev[i], 0));
      }
      TRY(count(h, n));
      prof_end(h, pb, PISP_PROF_FACTOR_SMALL, K * lp.bytes_fsmall, n);
    }
    if (mixed) {
      CK(cudaEventRecord(h->big_join, bst));
      CK(cudaStreamWaitEvent(h->stream, h->big_join, 0));
    }
  }
  h->factored = true;
  return PISP_OK;
}

int pisp_solve(pisp_handle* h, const double* b, int32_t R, const double* w, double* x,
               int32_t sweeps) {
  if (!h) return fail(h, PISP_ERR_INVALID_ARG, "null handle");
  if (!h->capturing) h->graph_valid = false;
  NvtxRange nvtx_("pisp_solve");
  if (!h->factored) return fail(h, PISP_ERR_NOT_FACTORED, "no factorisation");
  if (R < 1 || sweeps < 0) return fail(h, PISP_ERR_INVALID_ARG, "R must be >= 1, sweeps >= 0");
  if (h->sym.N > 0 && (!b || !x)) return fail(h, PISP_ERR_INVALID_ARG, "null b or x");
  if (b == x && b) return fail(h, PISP_ERR_INVALID_ARG, "x may not alias b");
  DeviceScope dev_scope_;
  TRY(set_device(h, dev_scope_));
  TRY(set_weights(h, w, h->w_last));
  TRY(ensure_solve_buffers(h, R));
  const pisp::Shifts sh = make_shifts(h, h->w_last);
  TRY(solve_core(h, b, h->X.as<double>(), R, sweeps, sh));
  const int pb = prof_begin(h);
  const int n = pisp::launch_combine(h->sd, h->X.as<double>(), sh, R, x, h->stream);
  TRY(count(h, n));
  prof_end(h, pb, PISP_PROF_COMBINE, (double)h->sym.N * R * 8.0 * (h->K + 1) + h->sym.N * 4.0, n);
  TRY(count(h, pisp::launch_fill_nan_failed(h->sd, h->status.as<int32_t>(), h->K, R, x, h->stream)));
  h->R = R;
  h->solved = true;
  return PISP_OK;
}

int pisp_combine(pisp_handle* h, const double* w, double* x) {
  if (!h) return fail(h, PISP_ERR_INVALID_ARG, "null handle");
  NvtxRange nvtx_("pisp_combine");
  if (!h->solved) return fail(h, PISP_ERR_NOT_FACTORED, "pisp_solve has not run");
  if (h->sym.N > 0 && !x) return fail(h, PISP_ERR_INVALID_ARG, "null x");
  DeviceScope dev_scope_;
  TRY(set_device(h, dev_scope_));
  double ww[PISP_K_MAX];
  TRY(set_weights(h, w, ww));
  const pisp::Shifts sh = make_shifts(h, ww);
  TRY(count(h, pisp::launch_combine(h->sd, h->X.as<double>(), sh, h->R, x, h->stream)));
  TRY(count(h, pisp::launch_fill_nan_failed(h->sd, h->status.as<int32_t>(), h->K, h->R, x, h->stream)));
  return PISP_OK;
}

int pisp_refine(pisp_handle* h, const double* b, double* x, int32_t R, int32_t iters,
                int32_t sweeps) {
  if (!h) return fail(h, PISP_ERR_INVALID_ARG, "null handle");
  if (!h->capturing) h->graph_valid = false;
  NvtxRange nvtx_("pisp_refine");
  if (!h->factored) return fail(h, PISP_ERR_NOT_FACTORED, "no factorisation");
  if (R < 1 || iters < 0 || sweeps < 0) return fail(h, PISP_ERR_INVALID_ARG, "bad R/iters/sweeps");
  if (h->sym.N > 0 && (!b || !x)) return fail(h, PISP_ERR_INVALID_ARG, "null b or x");
  DeviceScope dev_scope_;
  TRY(set_device(h, dev_scope_));
  // more right-hand sides than the last solve may reallocate the store of the
  // kept per-perturbation solutions: they are then gone, and pisp_combine /
  // pisp_adjoint refuse until the next pisp_solve
  if (h->solved && R > h->R) h->solved = false;
  TRY(ensure_solve_buffers(h, R));
  const size_t nkr = (size_t)h->sym.N * h->K * R * sizeof(double);
  const size_t nr = (size_t)h->sym.N * R * sizeof(double);
  if (!h->X2.ensure(nkr) || !h->rtmp.ensure(nr) || !h->dtmp.ensure(nr))
    return fail(h, PISP_ERR_OOM, "device allocation failed (refine workspace)");
  const pisp::Shifts sh = make_shifts(h, h->beta);
  for (int it = 0; it < iters; ++it) {
    TRY(count(h, pisp::launch_residual(h->sd, h->vals.as<double>(), b, x, R, h->rtmp.as<double>(), h->stream)));
    TRY(solve_core(h, h->rtmp.as<double>(), h->X2.as<double>(), R, sweeps, sh));
    TRY(count(h, pisp::launch_combine(h->sd, h->X2.as<double>(), sh, R, h->dtmp.as<double>(), h->stream)));
    TRY(count(h, pisp::launch_axpy((int64_t)h->sym.N * R, h->dtmp.as<double>(), x, h->stream)));
  }
  TRY(count(h, pisp::launch_fill_nan_failed(h->sd, h->status.as<int32_t>(), h->K, R, x, h->stream)));
  return PISP_OK;
}

int pisp_adjoint(pisp_handle* h, const double* g, const double* w, double* grad_b,
                 double* grad_values, int32_t sweeps) {
  if (!h) return fail(h, PISP_ERR_INVALID_ARG, "null handle");
  NvtxRange nvtx_("pisp_adjoint");
  if (!h->solved) return fail(h, PISP_ERR_NOT_FACTORED, "pisp_solve has not run");
  if (h->sym.N > 0 && !g) return fail(h, PISP_ERR_INVALID_ARG, "null g");
  if (sweeps < 0) return fail(h, PISP_ERR_INVALID_ARG, "sweeps must be >= 0");
  DeviceScope dev_scope_;
  TRY(set_device(h, dev_scope_));
  double ww[PISP_K_MAX];
  TRY(set_weights(h, w, ww));
  const int32_t R = h->R;
  if (!h->Lam.ensure((size_t)h->sym.N * h->K * R * sizeof(double)))
    return fail(h, PISP_ERR_OOM, "device allocation failed (adjoint workspace)");
  const pisp::Shifts sh = make_shifts(h, ww);
  TRY(solve_pass(h, true, g, pisp::RHS_BROADCAST, h->Lam.as<double>(), nullptr, R));
  // FP64 residual sweeps of every lambda_k on the transposed systems, as the
  // forward sweeps do for x_k: with FP32 factors the adjoint then reaches the
  // FP64 definition too (Rk and Y are the solve's workspace, sized for R)
  for (int it = 0; it < sweeps; ++it) {
    TRY(count(h, pisp::launch_residual_T_per_k(h->sd, h->vals.as<double>(), h->D.as<double>(), sh, g,
                                               h->Lam.as<double>(), R, h->Rk.as<double>(), h->stream)));
    TRY(solve_pass(h, true, h->Rk.as<double>(), pisp::RHS_PER_K, h->Y.as<double>(), h->Lam.as<double>(), R));
  }
  if (grad_b) TRY(count(h, pisp::launch_combine(h->sd, h->Lam.as<double>(), sh, R, grad_b, h->stream)));
  if (grad_values)
    TRY(count(h, pisp::launch_grad_values(h->sd, h->Lam.as<double>(), h->X.as<double>(), sh, R,
                                          grad_values, h->stream)));
  return PISP_OK;
}

int pisp_graph_capture(pisp_handle* h, const double* values, const double* D, const double* t,
                       int32_t K, int32_t precision, const double* b, int32_t R, const double* w,
                       double* x, int32_t sweeps, const double* g, double* grad_b, double* grad_values,
                       int32_t adjoint_sweeps) {
  if (!h) return fail(h, PISP_ERR_INVALID_ARG, "null handle");
  NvtxRange nvtx_("pisp_graph_capture");
  if (!h->analyzed) return fail(h, PISP_ERR_NOT_ANALYZED, "pisp_analyze has not succeeded");
  DeviceScope dev_scope_;
  TRY(set_device(h, dev_scope_));
  h->drop_graph();
  // one eager step: checks the arguments, allocates every workspace the step
  // needs (nothing may be allocated during the capture) and leaves its results
  auto step = [&]() -> int {
    TRY(pisp_factor_perturbed(h, values, D, t, K, precision));
    TRY(pisp_solve(h, b, R, w, x, sweeps));
    if (g) TRY(pisp_adjoint(h, g, w, grad_b, grad_values, adjoint_sweeps));
    return PISP_OK;
  };
  TRY(step());
  if (h->prof_on) {  // only the brackets recorded into the graph are replayed
    h->prof_next = 0;
    h->prof_br.clear();
  }
  if (!h->cap_stream) {
    CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->cap_ev, cudaEventDisableTiming));
  }
  // capture on a private stream ordered after the work queued so far
  CK(cudaEventRecord(h->cap_ev, h->stream));
  CK(cudaStreamWaitEvent(h->cap_stream, h->cap_ev, 0));
  const cudaStream_t user = h->stream;
  h->stream = h->cap_stream;
  h->capturing = true;
  cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
  int rc = e == cudaSuccess ? step() : PISP_ERR_CUDA;
  cudaGraph_t gr = nullptr;
  const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(h->cap_stream, &gr) : e;
  h->capturing = false;
  h->stream = user;
  if (rc) {
    if (gr) cudaGraphDestroy(gr);
    return rc;
  }
  if (e2 != cudaSuccess || !gr)
    return fail(h, PISP_ERR_CUDA, std::string("stream capture failed: ") + cudaGetErrorString(e2));
  h->graph = gr;
  CK(cudaGraphInstantiate(&h->graph_exec, h->graph, 0));
  h->graph_valid = true;
  return PISP_OK;
}

int pisp_graph_launch(pisp_handle* h) {
  if (!h) return fail(h, PISP_ERR_INVALID_ARG, "null handle");
  if (!h->graph_valid || !h->graph_exec)
    return fail(h, PISP_ERR_INVALID_ARG, "no valid captured step (pisp_graph_capture)");
  DeviceScope dev_scope_;
  TRY(set_device(h, dev_scope_));
  CK(cudaGraphLaunch(h->graph_exec, h->stream));
  return PISP_OK;
}

int pisp_set_wait_limit(pisp_handle* h, int64_t polls, int32_t unreachable) {
  if (!h) return fail(h, PISP_ERR_INVALID_ARG, "null handle");
  if (polls < 0) return fail(h, PISP_ERR_INVALID_ARG, "polls must be >= 0");
  h->wait_polls = polls;
  h->wait_unreachable = unreachable ? 1 : 0;
  h->units_K = h->units_R = 0;  // the next persistent solve rebuilds its targets
  h->graph_valid = false;
  return PISP_OK;
}

int pisp_set_refinement(pisp_handle* h, double tol) {
  if (!h) return fail(h, PISP_ERR_INVALID_ARG, "null handle");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(h, PISP_ERR_INVALID_ARG, "tol must be finite and >= 0");
  h->sweep_tol = tol;
  return PISP_OK;
}

int pisp_refinement_stats(pisp_handle* h, int32_t* sweeps_per_instance, double* work, double* rows,
                          int32_t max_sweeps) {
  if (!h) return fail(h, PISP_ERR_INVALID_ARG, "null handle");
  if (max_sweeps < 0) return fail(h, PISP_ERR_INVALID_ARG, "max_sweeps must be >= 0");
  if (!h->any_solve) return fail(h, PISP_ERR_NOT_FACTORED, "no solve");
  DeviceScope dev_scope_;
  TRY(set_device(h, dev_scope_));
  std::vector<int32_t> nsw;
  std::vector<double> fs, fr;
  TRY(sweep_fractions(h, std::max(max_sweeps, 1), nsw, fs, fr));
  if (sweeps_per_instance) std::copy(nsw.begin(), nsw.end(), sweeps_per_instance);
  for (int q = 0; q < max_sweeps; ++q) {
    if (work) work[q] = fs[q + 1];
    if (rows) rows[q] = fr[q + 1];
  }
  return PISP_OK;
}

int pisp_get_status(pisp_handle* h, int32_t* per_instance_k, int32_t* first_bad_col) {
  if (!h) return fail(h, PISP_ERR_INVALID_ARG, "null handle");
  if (!h->factored) return fail(h, PISP_ERR_NOT_FACTORED, "no factorisation");
  DeviceScope dev_scope_;
  TRY(set_device(h, dev_scope_));
  const size_t n = (size_t)h->sym.G * h->K;
  std::vector<int32_t> st(n), bc(n);
  CK(cudaMemcpyAsync(st.data(), h->status.p, n * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(bc.data(), h->badcol.p, n * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  int serr = 0;
  CK(cudaMemcpyAsync(&serr, h->serr.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (serr) {
    h->err = "a bounded dependency wait of the persistent solve gave up";
    return PISP_ERR_TIMEOUT;
  }
  int worst = PISP_OK;
  for (size_t q = 0; q < n; ++q) {
    int code = PISP_OK;
    if (st[q] & 1) code = PISP_ERR_ZERO_PIVOT;
    else if (st[q] & 2) code = PISP_ERR_NONFINITE;
    if (per_instance_k) per_instance_k[q] = code;
    if (first_bad_col) first_bad_col[q] = code ? bc[q] : -1;
    if (code == PISP_ERR_ZERO_PIVOT || (code && worst == PISP_OK)) worst = code;
  }
  return worst;
}

int pisp_get_stats(const pisp_handle* h, pisp_stats* o) {
  if (!h || !o) return PISP_ERR_INVALID_ARG;
  if (!h->analyzed) return PISP_ERR_NOT_ANALYZED;
  const pisp::Symbolic& S = h->sym;
  std::memset(o, 0, sizeof(*o));
  o->N = S.N;
  o->nnzA = S.nnzA;
  o->nnzL = S.nnzL;
  o->nnzF_stored = S.nnzF_stored;
  o->front_elems = S.front_elems;
  o->G = S.G;
  o->n_supernodes = (int32_t)S.sn.size();
  o->n_levels = S.n_levels;
  o->max_front = S.max_front;
  o->etree_height = S.etree_height;
  o->K = h->K;
  o->precision = h->precision;
  o->gpu_launches = h->launches;
  if (h->last_loop && h->loop_kernels > 0 && h->r_sweep.p) {
    // a device-side sweep loop counted its body once: add its further iterations
    pisp_handle* hh = const_cast<pisp_handle*>(h);
    DeviceScope dev_scope_;
    if (set_device(hh, dev_scope_) == PISP_OK) {
      int32_t iters = 0;
      if (cudaMemcpyAsync(&iters, h->r_sweep.p, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream) == cudaSuccess &&
          cudaStreamSynchronize(h->stream) == cudaSuccess && iters > 1)
        o->gpu_launches += h->loop_kernels * (iters - 1);
    }
  }
  o->flops_factor = S.flops_factor;
  o->flops_solve = S.flops_solve;
  o->analyze_ms = h->analyze_ms;
  return PISP_OK;
}

int pisp_get_perm(const pisp_handle* h, int32_t* perm) {
  if (!h || !perm) return PISP_ERR_INVALID_ARG;
  if (!h->analyzed) return PISP_ERR_NOT_ANALYZED;
  std::copy(h->sym.perm.begin(), h->sym.perm.end(), perm);
  return PISP_OK;
}

int pisp_get_supernodes(const pisp_handle* h, int32_t* c0, int32_t* c1, int32_t* ms,
                        int32_t* rows) {
  if (!h) return PISP_ERR_INVALID_ARG;
  if (!h->analyzed) return PISP_ERR_NOT_ANALYZED;
  const auto& S = h->sym;
  for (size_t s = 0; s < S.sn.size(); ++s) {
    if (c0) c0[s] = S.sn[s].c0;
    if (c1) c1[s] = S.sn[s].c1;
    if (ms) ms[s] = S.sn[s].ms;
  }
  if (rows) std::copy(S.rows.begin(), S.rows.end(), rows);
  return PISP_OK;
}

int pisp_get_front(pisp_handle* h, int32_t s, int32_t k, double* out, int32_t* F_out) {
  if (!h) return fail(h, PISP_ERR_INVALID_ARG, "null handle");
  if (!h->factored) return fail(h, PISP_ERR_NOT_FACTORED, "no factorisation");
  if (s < 0 || s >= (int32_t)h->sym.sn.size() || k < 0 || k >= h->K)
    return fail(h, PISP_ERR_INVALID_ARG, "supernode or k out of range");
  DeviceScope dev_scope_;
  TRY(set_device(h, dev_scope_));
  const int64_t F = h->sym.sn[s].F();
  if (F_out) *F_out = (int32_t)F;
  if (!out) return PISP_OK;
  const size_t es = esize(h->precision);
  const size_t off = ((size_t)h->K * h->sym.front_off[s] + (size_t)k * F * F) * es;
  std::vector<unsigned char> buf(F * F * es);
  CK(cudaMemcpyAsync(buf.data(), (const char*)h->fronts.p + off, buf.size(), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int64_t q = 0; q < F * F; ++q)
    out[q] = es == 4 ? (double)reinterpret_cast<const float*>(buf.data())[q]
                     : reinterpret_cast<const double*>(buf.data())[q];
  return PISP_OK;
}

int pisp_get_pivot_range(pisp_handle* h, double* min_abs, double* max_abs) {
  if (!h) return fail(h, PISP_ERR_INVALID_ARG, "null handle");
  if (!h->factored) return fail(h, PISP_ERR_NOT_FACTORED, "no factorisation");
  if (!min_abs || !max_abs) return fail(h, PISP_ERR_INVALID_ARG, "null output");
  DeviceScope dev_scope_;
  TRY(set_device(h, dev_scope_));
  const pisp::Symbolic& S = h->sym;
  const int K = h->K;
  const size_t es = esize(h->precision);
  const size_t GK = (size_t)S.G * K;
  std::vector<double> lo(GK, HUGE_VAL), hi(GK, 0.0);
  std::vector<char> bad(GK, 0);
  // pivots of perturbation k, permuted column c, at buf[k * N + c]
  std::vector<unsigned char> buf((size_t)S.N * K * es);
  for (size_t s = 0; s < S.sn.size(); ++s) {
    const pisp::Supernode& sn = S.sn[s];
    const int64_t F = sn.F(), ns = sn.ns();
    for (int k = 0; k < K; ++k) {
      // u_jj of the front's pivot block sits at j + j*F of the column-major
      // F x F front of (s, k): every (F + 1)-th element, ns of them
      const char* src = (const char*)h->fronts.p + ((size_t)K * S.front_off[s] + (size_t)k * F * F) * es;
      CK(cudaMemcpy2DAsync(buf.data() + ((size_t)k * S.N + sn.c0) * es, es, src, (size_t)(F + 1) * es, es,
                           (size_t)ns, cudaMemcpyDeviceToHost, h->stream));
    }
  }
  CK(cudaStreamSynchronize(h->stream));
  for (size_t s = 0; s < S.sn.size(); ++s) {
    const pisp::Supernode& sn = S.sn[s];
    for (int k = 0; k < K; ++k) {
      const size_t q = (size_t)sn.instance * K + k;
      for (int32_t c = sn.c0; c < sn.c1; ++c) {
        const size_t e = (size_t)k * S.N + c;
        const double u = std::fabs(es == 4 ? (double)reinterpret_cast<const float*>(buf.data())[e]
                                           : reinterpret_cast<const double*>(buf.data())[e]);
        if (!std::isfinite(u)) bad[q] = 1;
        lo[q] = std::min(lo[q], u);
        hi[q] = std::max(hi[q], u);
      }
    }
  }
  for (size_t q = 0; q < GK; ++q) {
    const bool empty = lo[q] == HUGE_VAL;  // an instance with no unknowns
    min_abs[q] = bad[q] || empty ? NAN : lo[q];
    max_abs[q] = bad[q] || empty ? NAN : hi[q];
  }
  return PISP_OK;
}

int pisp_solve_host(pisp_handle* h, const double* values_host, const double* D_host,
                    const double* t, int32_t K, int32_t precision, const double* b_host,
                    int32_t R, double* x_host, int32_t sweeps) {
  if (!h) return fail(h, PISP_ERR_INVALID_ARG, "null handle");
  NvtxRange nvtx_("pisp_solve_host");
  h->graph_valid = false;
  if (!h->analyzed) return fail(h, PISP_ERR_NOT_ANALYZED, "pisp_analyze has not succeeded");
  if (R < 1) return fail(h, PISP_ERR_INVALID_ARG, "R must be >= 1");
  const pisp::Symbolic& S = h->sym;
  if ((S.nnzA && !values_host) || (S.N && (!D_host || !b_host || !x_host)))
    return fail(h, PISP_ERR_INVALID_ARG, "null host buffer");
  DeviceScope dev_scope_;
  TRY(set_device(h, dev_scope_));
  const size_t nv = S.nnzA * sizeof(double), nd = S.N * sizeof(double);
  const size_t nb = (size_t)S.N * R * sizeof(double);
  if (!h->in_vals.ensure(nv) || !h->in_D.ensure(nd) || !h->in_b.ensure(nb) || !h->out_x.ensure(nb))
    return fail(h, PISP_ERR_OOM, "device allocation failed (host staging)");
  if (!h->copy_stream) {
    CK(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    for (cudaEvent_t& e : h->copy_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  if (nv) CK(cudaMemcpyAsync(h->in_vals.p, values_host, nv, cudaMemcpyHostToDevice, h->stream));
  if (nd) CK(cudaMemcpyAsync(h->in_D.p, D_host, nd, cudaMemcpyHostToDevice, h->stream));
  // b after the values and D (the factorisation needs those first), copied
  // while the factorisation runs; the solve waits for it
  CK(cudaEventRecord(h->copy_ev[0], h->stream));
  CK(cudaStreamWaitEvent(h->copy_stream, h->copy_ev[0], 0));
  if (nb) CK(cudaMemcpyAsync(h->in_b.p, b_host, nb, cudaMemcpyHostToDevice, h->copy_stream));
  CK(cudaEventRecord(h->copy_ev[1], h->copy_stream));
  TRY(pisp_factor_perturbed(h, h->in_vals.as<double>(), h->in_D.as<double>(), t, K, precision));
  CK(cudaStreamWaitEvent(h->stream, h->copy_ev[1], 0));
  TRY(pisp_solve(h, h->in_b.as<double>(), R, nullptr, h->out_x.as<double>(), sweeps));
  if (nb) CK(cudaMemcpyAsync(x_host, h->out_x.p, nb, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return PISP_OK;
}

int pisp_profile(pisp_handle* h, int32_t on) {
  if (!h) return fail(h, PISP_ERR_INVALID_ARG, "null handle");
  if (on) {
    DeviceScope dev_scope_;
    TRY(set_device(h, dev_scope_));
    while (h->prof_ev.size() < 2048) {  // events exist before any stream capture
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      h->prof_ev.push_back(e);
    }
    h->prof_on = true;
    h->prof_next = 0;
    h->prof_br.clear();
  } else {
    h->prof_on = false;
  }
  return PISP_OK;
}

int pisp_profile_collect(pisp_handle* h) {
  if (!h) return fail(h, PISP_ERR_INVALID_ARG, "null handle");
  DeviceScope dev_scope_;
  TRY(set_device(h, dev_scope_));
  CK(cudaStreamSynchronize(h->stream));
  bool loop = false;
  for (const auto& b : h->prof_br) loop = loop || b.sweep == -1;
  std::vector<int32_t> nsw;
  std::vector<double> fs, fr;
  if (loop && h->last_adaptive) TRY(sweep_fractions(h, std::max(h->last_sweeps, 1), nsw, fs, fr));
  for (const auto& b : h->prof_br) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->prof_ev[b.e0], h->prof_ev[b.e1]));
    h->prof_ms[b.fam] += ms;
    if (b.sweep == -1) {  // a device-side loop: one iteration per sweep any instance took
      int iters = 0;
      double by = 0.0;
      for (int s = 1; s < (int)fs.size(); ++s)
        if (fr[s] > 0.0) {
          ++iters;
          by += fr[s] * b.bytes_rows + fs[s] * b.bytes_work;
        }
      h->prof_bytes[b.fam] += by;
      h->prof_launches[b.fam] += (int64_t)b.launches * iters;
      continue;
    }
    h->prof_bytes[b.fam] += b.bytes;
    h->prof_launches[b.fam] += b.launches;
  }
  return PISP_OK;
}

int pisp_profile_read(pisp_handle* h, int32_t family, double* ms, double* bytes,
                      int64_t* launches) {
  if (!h || family < 0 || family >= PISP_PROF_FAMILIES)
    return fail(h, PISP_ERR_INVALID_ARG, "bad profiling family");
  if (ms) *ms = h->prof_ms[family];
  if (bytes) *bytes = h->prof_bytes[family];
  if (launches) *launches = h->prof_launches[family];
  return PISP_OK;
}

int pisp_profile_reset(pisp_handle* h) {
  if (!h) return fail(h, PISP_ERR_INVALID_ARG, "null handle");
  for (int f = 0; f < PISP_PROF_FAMILIES; ++f) {
    h->prof_ms[f] = h->prof_bytes[f] = 0.0;
    h->prof_launches[f] = 0;
  }
  return PISP_OK;
}

const char* pisp_profile_name(int32_t family) {
  return (family >= 0 && family < PISP_PROF_FAMILIES) ? kFamilyNames[family] : "";
}

}  // extern "C"
