// Batched triangular solves on the pivot-free factors, the expansion-weighted
// combine (Eq. x_star / Remark 2), FP64 residuals and the adjoint gradient.
//
// Vector layouts (all FP64 unless noted):
//   b, x          [N][R]     original row order (caller-owned)
//   X, Y, Rk, Lam [N][K][R]  permuted row order, one slice per perturbation
//   V             [K][R][F]  per front, factor precision: forward-solve
//                            values of the front's rows (pivot part = y,
//                            update part = contribution to the parent)
// Forward solves run the assembly forest bottom-up, backward solves top-down;
// one CTA handles one (front, perturbation, RHS chunk).
#include <atomic>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "pisp_internal.h"

namespace pisp {
namespace {

constexpr int kSolveThreads = 256;
// The persistent solve is compiled for 2, 3 and 4 resident CTAs per SM
// (register budgets of 128, 80 and 64 per thread); the launch picks one.
// More CTAs hide more of the dependent-load latency of the many small tasks
// of a batch, fewer registers spill more in the blocked path of wide fronts.
// FP32 kernels fit 80 registers with almost no spills, FP64 ones need 128.
constexpr int kSolveSmem = 96 * 1024;

// Forward substitution with L (unit lower, TRANS = false) or with U^T
// (TRANS = true, used by the adjoint), front by front.
template <typename T, bool TRANS>
__global__ void __launch_bounds__(kSolveThreads) k_forward(SymDev sd, const int32_t* __restrict__ list,
                                                          const T* __restrict__ fronts,
                                                          const double* __restrict__ rhs,
                                                          int rhs_mode, T* __restrict__ V, int R,
                                                          int K, int rc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* v = reinterpret_cast<T*>(smraw);
  const int s = list[blockIdx.x];
  const int k = blockIdx.y;
  const int r0 = blockIdx.z * rc;
  if (r0 >= R) return;
  const int nr = min(rc, R - r0);
  const int ns = sd.ns[s], ms = sd.ms[s], F = ns + ms;
  const int c0 = sd.c0[s];
  const int tid = threadIdx.x, nt = blockDim.x;
  const T* f = fronts + (int64_t)K * sd.front_off[s] + (int64_t)k * F * F;
  for (int q = tid; q < nr * ns; q += nt) {
    const int c = q % ns, r = q / ns;
    const double bv = (rhs_mode == RHS_BROADCAST)
                          ? rhs[(int64_t)sd.perm[c0 + c] * R + r0 + r]
                          : rhs[((int64_t)(c0 + c) * K + k) * R + r0 + r];
    v[r * F + c] = (T)bv;
  }
  for (int q = tid; q < nr * ms; q += nt) v[(q / ms) * F + ns + q % ms] = T(0);
  __syncthreads();
  for (int ci = sd.child_off[s]; ci < sd.child_off[s + 1]; ++ci) {
    const int c = sd.child[ci];
    const int cns = sd.ns[c], cms = sd.ms[c], cF = cns + cms;
    const T* cv = V + (int64_t)K * R * sd.vec_off[c] + ((int64_t)k * R + r0) * cF;
    const int32_t* em = sd.emap + sd.row_off[c];
    for (int q = tid; q < nr * cms; q += nt) {
      const int a = q % cms, r = q / cms;
      v[r * F + em[a]] += cv[(int64_t)r * cF + cns + a];
    }
    __syncthreads();
  }
  for (int p = 0; p < ns; ++p) {
    const int m = F - p - 1;
    if (!TRANS) {
      for (int q = tid; q < nr * m; q += nt) {
        const int i = p + 1 + q % m, r = q / m;
        v[r * F + i] -= f[i + (int64_t)p * F] * v[r * F + p];
      }
    } else {
      const T up = f[(int64_t)p * (F + 1)];
      for (int q = tid; q < nr * m; q += nt) {
        const int i = p + 1 + q % m, r = q / m;
        v[r * F + i] -= f[p + (int64_t)i * F] * (v[r * F + p] / up);
      }
    }
    __syncthreads();
  }
  if (TRANS) {
    for (int q = tid; q < nr * ns; q += nt) {
      const int c = q % ns, r = q / ns;
      v[r * F + c] /= f[(int64_t)c * (F + 1)];
    }
    __syncthreads();
  }
  T* out = V + (int64_t)K * R * sd.vec_off[s] + ((int64_t)k * R + r0) * F;
  for (int q = tid; q < nr * F; q += nt) out[q] = v[q];
}

// Backward substitution with U (TRANS = false) or with L^T (TRANS = true),
// top-down.  Reads the already computed solution of the ancestors' rows from
// `out`, writes its own rows to `out` and, if acc != nullptr, adds them to acc.
template <typename T, bool TRANS>
__global__ void __launch_bounds__(kSolveThreads) k_backward(SymDev sd, const int32_t* __restrict__ list,
                                                           const T* __restrict__ fronts,
                                                           const T* __restrict__ V, double* out,
                                                           double* acc, int R, int K, int rc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int s = list[blockIdx.x];
  const int k = blockIdx.y;
  const int r0 = blockIdx.z * rc;
  if (r0 >= R) return;
  const int nr = min(rc, R - r0);
  const int ns = sd.ns[s], ms = sd.ms[s], F = ns + ms;
  const int c0 = sd.c0[s];
  const int tid = threadIdx.x, nt = blockDim.x;
  T* xr = reinterpret_cast<T*>(smraw);
  T* z = xr + nr * ms;
  const T* f = fronts + (int64_t)K * sd.front_off[s] + (int64_t)k * F * F;
  const int32_t* rows = sd.rows + sd.row_off[s];
  for (int q = tid; q < nr * ms; q += nt) {
    const int j = q % ms, r = q / ms;
    xr[q] = (T)out[((int64_t)rows[j] * K + k) * R + r0 + r];
  }
  const T* y = V + (int64_t)K * R * sd.vec_off[s] + ((int64_t)k * R + r0) * F;
  for (int q = tid; q < nr * ns; q += nt) {
    const int p = q % ns, r = q / ns;
    z[q] = y[(int64_t)r * F + p];
  }
  __syncthreads();
  if (ms > 0) {
    for (int q = tid; q < nr * ns; q += nt) {
      const int p = q % ns, r = q / ns;
      T a = z[q];
      const T* xrr = xr + r * ms;
      if (!TRANS) {
        for (int j = 0; j < ms; ++j) a -= f[p + (int64_t)(ns + j) * F] * xrr[j];
      } else {
        const T* lc = f + (int64_t)p * F + ns;
        for (int j = 0; j < ms; ++j) a -= lc[j] * xrr[j];
      }
      z[q] = a;
    }
    __syncthreads();
  }
  for (int p = ns - 1; p >= 1; --p) {
    if (!TRANS) {
      const T up = f[(int64_t)p * (F + 1)];
      for (int q = tid; q < nr * p; q += nt) {
        const int i = q % p, r = q / p;
        z[r * ns + i] -= f[i + (int64_t)p * F] * (z[r * ns + p] / up);
      }
    } else {
      for (int q = tid; q < nr * p; q += nt) {
        const int i = q % p, r = q / p;
        z[r * ns + i] -= f[p + (int64_t)i * F] * z[r * ns + p];
      }
    }
    __syncthreads();
  }
  for (int q = tid; q < nr * ns; q += nt) {
    const int p = q % ns, r = q / ns;
    const T xv = TRANS ? z[q] : z[q] / f[(int64_t)p * (F + 1)];
    const int64_t o = ((int64_t)(c0 + p) * K + k) * R + r0 + r;
    out[o] = (double)xv;
    if (acc) acc[o] += (double)xv;
  }
}

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double load_rhs(const SymDev& sd, const double* rhs, int rhs_mode,
                                           int col, int k, int K, int R, int r) {
  return rhs_mode == RHS_BROADCAST ? rhs[(int64_t)sd.perm[col] * R + r]
                                   : rhs[((int64_t)col * K + k) * R + r];
}

// ---------------------------------------------------------------------------
// Dependency flags of the persistent schedule.  A task (front, k, RHS chunk)
// publishes done[(s*K + k)*nch + ch] = 1 after its results are globally
// visible; consumers spin on it with a bounded number of polls.  A wait that
// gives up sets *err (reported as PISP_ERR_TIMEOUT) and the task proceeds, so
// no wait can hang the GPU.
// ---------------------------------------------------------------------------
constexpr int64_t kWaitPolls = 1 << 22;  // default poll limit of a dependency wait

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// done[s*K + k] counts the finished RHS chunks of (front s, perturbation k).
// Forward solve: a front waits until the counter of each child reaches
// nch[child].  Backward solve: a front waits until its parent's counter
// reaches nch[parent].
struct Sync {
  int* done;          // nullptr: level-synchronous launches, nothing to wait for
  int* err;
  const int* nch;     // [S] RHS chunks per (front, k) in the persistent schedule
  int64_t polls;      // polls before a wait gives up
  __device__ void wait_ge(const int* f, int need) const {
    if (ld_acquire(f) >= need) return;
    for (int64_t i = 0; i < polls; ++i) {
      __nanosleep(64);
      if (ld_acquire(f) >= need) return;
    }
    atomicExch(err, 1);
  }
  __device__ void add(int s, int k, int K) const {
    asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(done + (int64_t)s * K + k) : "memory");
  }
  // backward: front s waits for its parent p (which publishes to itself)
  __device__ void wait_parent(int s, int p, int k, int K) const {
    wait_ge(done + (int64_t)p * K + k, nch[p]);
  }
  __device__ void publish_children(const SymDev& sd, int s, int k, int K) const { add(s, k, K); }
  // forward: the n threads (index 0..n-1) of a CTA or a lane group poll the
  // children's counters in parallel with relaxed loads and then each issues
  // an acquire fence, so a front with many children pays one round trip
  // instead of one per child; the caller's barrier orders the group's later
  // reads after the fences
  __device__ void wait_children(const SymDev& sd, int s, int k, int K, int idx, int n) const {
    const int cb = sd.child_off[s], ce = sd.child_off[s + 1];
    for (int ci = cb + idx; ci < ce; ci += n) {
      const int c = sd.child[ci];
      const int* f = done + (int64_t)c * K + k;
      const int need = nch[c];
      if (ld_relaxed(f) >= need) continue;
      int64_t i = 0;
      for (; i < polls; ++i) {
        __nanosleep(64);
        if (ld_relaxed(f) >= need) break;
      }
      if (i == polls) atomicExch(err, 1);
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
  }
};

// Right-hand side of front s (rows of its pivot part) plus the children's
// contributions to position j, summed in child order: the same order as an
// extend-add that visits children one by one, without a barrier per child.
// NB contributions' loads are in flight at a time; they are added in child
// order whatever NB is.
template <typename T, int NB = 4>
__device__ __forceinline__ T gather_position(const SymDev& sd, int s, int j, int ns, int c0,
                                             const double* rhs, int rhs_mode, const T* V, int k, int K,
                                             int R, int r) {
  T a = (j < ns) ? (T)load_rhs(sd, rhs, rhs_mode, c0 + j, k, K, R, r) : T(0);
  const int64_t e1 = sd.inv_off[sd.vec_off[s] + j + 1];
  const int64_t kr = (int64_t)k * R + r, kR = (int64_t)K * R;
  for (int64_t e = sd.inv_off[sd.vec_off[s] + j]; e < e1; e += NB) {
    const int n = (int)min((int64_t)NB, e1 - e);
    T v[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q)
      v[q] = q < n ? __ldcg(V + kR * sd.inv_vbase[e + q] + kr * sd.inv_cF[e + q] + sd.inv_col[e + q]) : T(0);
#pragma unroll
    for (int q = 0; q < NB; ++q)
      if (q < n) a += v[q];
  }
  return a;
}

// ---------------------------------------------------------------------------
// x[r] = p[r] for r < n (FP64 to T, zero beyond n): the 8 right-hand sides
// of one row are contiguous, so a full aligned chunk is read with 16-byte
// loads (L2 only: the values come from other CTAs of the same launch)
template <typename T>
__device__ __forceinline__ void ld_rhs8(const double* p, int n, T (&x)[kSolveChunk]) {
  if (n == kSolveChunk && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int i = 0; i < kSolveChunk / 2; ++i) {
      const double2 v = __ldcg(q + i);
      x[2 * i] = (T)v.x;
      x[2 * i + 1] = (T)v.y;
    }
  } else {
#pragma unroll
    for (int r = 0; r < kSolveChunk; ++r) x[r] = r < n ? (T)__ldcg(p + r) : T(0);
  }
}

// p[r] = x[r] (and acc[r] += x[r] when acc is given) for r < n, 16-byte
// stores for a full aligned chunk
template <typename T>
__device__ __forceinline__ void st_rhs8(double* p, double* acc, int n, const T (&x)[kSolveChunk]) {
  if (n == kSolveChunk && (reinterpret_cast<uintptr_t>(p) & 15) == 0 &&
      (!acc || (reinterpret_cast<uintptr_t>(acc) & 15) == 0)) {
    double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
    for (int i = 0; i < kSolveChunk / 2; ++i) q[i] = make_double2((double)x[2 * i], (double)x[2 * i + 1]);
    if (acc) {
      double2* qa = reinterpret_cast<double2*>(acc);
#pragma unroll
      for (int i = 0; i < kSolveChunk / 2; ++i) {
        double2 v = qa[i];
        v.x += (double)x[2 * i];
        v.y += (double)x[2 * i + 1];
        qa[i] = v;
      }
    }
  } else {
#pragma unroll
    for (int r = 0; r < kSolveChunk; ++r)
      if (r < n) {
        p[r] = (double)x[r];
        if (acc) acc[r] += (double)x[r];
      }
  }
}

// gather_position for every right-hand side r < nr of one position j at
// once: the index entries of the inverse extend-add map are read once and
// each serves the nr right-hand sides (the same per-RHS order of additions).
// nr = 0 (an inactive lane, or j outside the front) returns zeros.
template <typename T>
__device__ __forceinline__ void gather_position_rhs(const SymDev& sd, int s, int j, int ns, int c0,
                                                    const double* rhs, int rhs_mode, const T* V, int k, int K,
                                                    int R, int r0, int nr, T (&a)[kSolveChunk]) {
  if (j < ns && nr > 0) {
    const double* p = rhs_mode == RHS_BROADCAST ? rhs + (int64_t)sd.perm[c0 + j] * R + r0
                                                : rhs + ((int64_t)(c0 + j) * K + k) * R + r0;
    ld_rhs8<T>(p, nr, a);
  } else {
#pragma unroll
    for (int r = 0; r < kSolveChunk; ++r) a[r] = T(0);
  }
  if (nr <= 0) return;  // no position here (j beyond the front): touch no index array
  const int64_t e1 = sd.inv_off[sd.vec_off[s] + j + 1];
  const int64_t kR = (int64_t)K * R;
  for (int64_t e = sd.inv_off[sd.vec_off[s] + j]; e < e1; ++e) {
    const int cF = sd.inv_cF[e];
    const T* src = V + kR * sd.inv_vbase[e] + ((int64_t)k * R + r0) * cF + sd.inv_col[e];
    T v[kSolveChunk];
#pragma unroll
    for (int r = 0; r < kSolveChunk; ++r) v[r] = r < nr ? __ldcg(src + (int64_t)r * cF) : T(0);
#pragma unroll
    for (int r = 0; r < kSolveChunk; ++r) a[r] += v[r];
  }
}

// Fronts with F <= SEG (SEG = 8, 16 or 32): a warp is split into 32/SEG
// segments and every segment solves one (front, k, chunk of kRW right-hand
// sides).  Lane i of a segment owns row i of its front; the factor entries it
// needs live in registers and the triangular solves are shuffle chains within
// the segment.  Loops run to warp-uniform bounds (entries beyond a front are
// zero), so segments with different fronts never diverge around a shuffle.
// All lanes of a warp call these bodies together.
// ---------------------------------------------------------------------------
constexpr int kRW = 8;

struct SegTask {
  bool active;
  int s, k, r0, nr, ch;
};

__device__ __forceinline__ SegTask seg_task(const SymDev& sd, const int32_t* list, int64_t sg,
                                            int64_t nseg, int R, int K) {
  SegTask t{false, 0, 0, 0, 0, 0};
  const int nch = (R + kRW - 1) / kRW;
  if (sg < nseg) {
    t.active = true;
    t.ch = (int)(sg % nch);
    t.k = (int)((sg / nch) % K);
    t.s = list[sg / ((int64_t)nch * K)];
    t.r0 = t.ch * kRW;
    t.nr = min(kRW, R - t.r0);
  }
  return t;
}

template <typename T, int SEG>
__device__ __forceinline__ void seg_forward(const SymDev& sd, const SegTask& t, int sl,
                                            T (*bw)[SEG + 1], const T* __restrict__ fronts,
                                            const double* __restrict__ rhs, int rhs_mode,
                                            T* __restrict__ V, int R, int K, const Sync& sy) {
  int ns = 0, ms = 0, F = 0, c0 = 0;
  if (t.active) {
    ns = sd.ns[t.s];
    ms = sd.ms[t.s];
    F = ns + ms;
    c0 = sd.c0[t.s];
  }
  const int k = t.k, r0 = t.r0, nr = t.nr;
  const T* f = fronts + (t.active ? (int64_t)K * sd.front_off[t.s] + (int64_t)k * F * F : 0);
  T Lr[SEG];
#pragma unroll
  for (int c = 0; c < SEG; ++c) Lr[c] = (c < ns && sl > c && sl < F) ? f[sl + c * F] : T(0);
  if (sy.done && t.active) sy.wait_children(sd, t.s, k, K, sl, SEG);
  __syncwarp();
  T vv[kRW];
#pragma unroll
  for (int r = 0; r < kRW; ++r)
    vv[r] = (r < nr && sl < F) ? gather_position<T>(sd, t.s, sl, ns, c0, rhs, rhs_mode, V, k, K, R, r0 + r)
                               : T(0);
  // right-hand sides actually present in this warp (uniform): the FP64 pipe
  // is narrow on this GPU, so absent columns must cost nothing
  const int nrw = __reduce_max_sync(kFull, nr);
  const int nsw = __reduce_max_sync(kFull, ns);
#pragma unroll
  for (int c = 0; c < SEG - 1; ++c) {
    if (c >= nsw) break;
#pragma unroll
    for (int r = 0; r < kRW; ++r)
      if (r < nrw) vv[r] -= Lr[c] * __shfl_sync(kFull, vv[r], c, SEG);
  }
  T* Vs = V + (t.active ? (int64_t)K * R * sd.vec_off[t.s] + ((int64_t)k * R + r0) * F : 0);
#pragma unroll
  for (int r = 0; r < kRW; ++r)
    if (r < nr && sl < F) Vs[(int64_t)r * F + sl] = vv[r];
  if (sy.done) {
    __syncwarp();
    if (t.active && sl == 0) {
      __threadfence();
      sy.add(t.s, k, K);
    }
  }
}

template <typename T, int SEG>
__device__ __forceinline__ void seg_backward(const SymDev& sd, const SegTask& t, int sl,
                                             const T* __restrict__ fronts, const T* __restrict__ V,
                                             double* out, double* acc, int R, int K, const Sync& sy) {
  int ns = 0, ms = 0, F = 0, c0 = 0;
  if (t.active) {
    ns = sd.ns[t.s];
    ms = sd.ms[t.s];
    F = ns + ms;
    c0 = sd.c0[t.s];
  }
  const int k = t.k, r0 = t.r0, nr = t.nr;
  const T* f = fronts + (t.active ? (int64_t)K * sd.front_off[t.s] + (int64_t)k * F * F : 0);
  const int myrow = (sl < ms) ? sd.rows[sd.row_off[t.s] + sl] : 0;
  const T* Vs = V + (t.active ? (int64_t)K * R * sd.vec_off[t.s] + ((int64_t)k * R + r0) * F : 0);
  T zt[kRW], xt[kRW];
#pragma unroll
  for (int r = 0; r < kRW; ++r) zt[r] = (r < nr && sl < ns) ? Vs[(int64_t)r * F + sl] : T(0);
  const T rd = (sl < ns) ? T(1) / f[sl * (F + 1)] : T(0);
  if (sy.done && sl == 0 && t.active && ms > 0) sy.wait_parent(t.s, sd.parent[t.s], k, K);
  __syncwarp();
#pragma unroll
  for (int r = 0; r < kRW; ++r)
    xt[r] = (r < nr && sl < ms) ? (T)__ldcg(out + ((int64_t)myrow * K + k) * R + r0 + r) : T(0);
  const int nrw = __reduce_max_sync(kFull, nr);
  const int msw = __reduce_max_sync(kFull, ms);
  const int nsw = __reduce_max_sync(kFull, ns);
  // update part: z -= U12 x_R, one column of U12 at a time
#pragma unroll 4
  for (int j = 0; j < SEG - 1; ++j) {
    if (j >= msw) break;
    const T u = (sl < ns && j < ms) ? f[sl + (ns + j) * F] : T(0);
#pragma unroll
    for (int r = 0; r < kRW; ++r)
      if (r < nrw) zt[r] -= u * __shfl_sync(kFull, xt[r], j, SEG);
  }
  // back substitution with U11, one column at a time
#pragma unroll 4
  for (int c = SEG - 1; c >= 0; --c) {
    if (c >= nsw) continue;
    const T u = (sl < ns && c > sl && c < ns) ? f[sl + c * F] : T(0);
#pragma unroll
    for (int r = 0; r < kRW; ++r) {
      if (r < nrw) {
        if (sl == c) zt[r] *= rd;
        zt[r] -= u * __shfl_sync(kFull, zt[r], c, SEG);
      }
    }
  }
  if (t.active && sl < ns) {
    double* o = out + ((int64_t)(c0 + sl) * K + k) * R + r0;
#pragma unroll
    for (int r = 0; r < kRW; ++r)
      if (r < nr) o[r] = (double)zt[r];
    if (acc) {
      double* a = acc + ((int64_t)(c0 + sl) * K + k) * R + r0;
#pragma unroll
      for (int r = 0; r < kRW; ++r)
        if (r < nr) a[r] += (double)zt[r];
    }
  }
  if (sy.done) {
    __syncwarp();
    if (t.active && sl == 0) {
      __threadfence();
      sy.publish_children(sd, t.s, k, K);
    }
  }
}

// ---------------------------------------------------------------------------
// Fronts with F > 32: a whole CTA per (front, k, RHS chunk), blocked by 32
// pivots.  Warps solve the staged 32x32 diagonal block with shuffles (one
// warp per right-hand side), then every thread updates its rows with the 32
// solved values, reading the factor panel with coalesced column loads.  None
// of the factor entries a step reads depend on the solution, so each step
// issues its first rows' panel loads and the next diagonal block's loads into
// registers before the diagonal solve: the step's memory latency overlaps
// the solve instead of following it.
// ---------------------------------------------------------------------------
constexpr int kBS = 33;  // padded row stride of a staged 32x32 block
// shared memory of the blocked path besides its nr x F vectors (elements):
// two staged diagonal blocks, and the backward solve's partial sums of the
// U12 product for a group of 4 right-hand sides
constexpr int kBlkExtra = 2 * 32 * kBS + 4 * kSolveThreads;

// rows prefetched per thread before the diagonal solve: more would push the
// persistent kernel past its 128-register budget (two CTAs per SM) and spill
template <typename T> struct BlkPF { static constexpr int N = 1; };

// L[c] = f[i + (p0 + c) * F] for c < nb (zero elsewhere or when !ok)
template <typename T>
__device__ __forceinline__ void load_prow(T (&L)[32], const T* f, int F, int i, int p0, int nb, bool ok) {
#pragma unroll
  for (int c = 0; c < 32; ++c) L[c] = (ok && c < nb) ? f[i + (int64_t)(p0 + c) * F] : T(0);
}

// this thread's 4 elements of a 32x32 diagonal block (q = tid + 256 t,
// row q & 31, column q >> 5), kept as stage_block would write them
template <typename T>
__device__ __forceinline__ void load_block_regs(T (&nx)[4], const T* f, int F, int p0, int nb, bool lower,
                                                bool ok, int tid) {
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int q = tid + 256 * t, i = q & 31, c = q >> 5;
    const bool keep = ok && (i < nb && c < nb) && (lower ? (i > c) : (i <= c));
    nx[t] = keep ? f[(p0 + i) + (int64_t)(p0 + c) * F] : T(0);
  }
}

template <typename T>
__device__ __forceinline__ void store_block_regs(T* dst, const T (&nx)[4], int tid) {
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int q = tid + 256 * t;
    dst[(q & 31) * kBS + (q >> 5)] = nx[t];
  }
}

// One warp, one right-hand side: vi (lane = row of the block) becomes
// L11^{-1} v for the unit lower triangle staged in B (strictly lower part,
// zeros elsewhere).  Two pivots per step: every lane forms the second solved
// value itself, as the same operations its owner lane performs, so the
// dependent shuffle chain is half as long and the result is unchanged.
template <typename T>
__device__ __forceinline__ void fwd_block_solve(const T* B, T& vi, int nb, int lane) {
  for (int c = 0; c < nb; c += 2) {
    const T y0 = __shfl_sync(kFull, vi, c);
    const T v1 = __shfl_sync(kFull, vi, (c + 1) & 31);
    vi -= B[lane * kBS + c] * y0;
    if (c + 1 < nb) {
      const T y1 = v1 - B[(c + 1) * kBS + c] * y0;
      vi -= B[lane * kBS + c + 1] * y1;
    }
  }
}

// One warp, one right-hand side: zi becomes U11^{-1} z for the upper triangle
// (with its diagonal) staged in B, one pivot per step from the bottom (unlike
// the forward solve, pairing pivots here costs more shuffles and selects
// than it saves).
template <typename T>
__device__ __forceinline__ void bwd_block_solve(const T* B, T& zi, int nb, int lane) {
  const T rd = (lane < nb) ? T(1) / B[lane * kBS + lane] : T(0);
#pragma unroll
  for (int c = 31; c >= 0; --c) {
    if (c >= nb) continue;
    if (lane == c) zi *= rd;
    const T xc = __shfl_sync(kFull, zi, c);
    if (lane < c) zi -= B[lane * kBS + c] * xc;
  }
}

// vec[r * ld + i] -= sum_{c < nb} L[c] vec[r * ld + p0 + c] for r < nr
template <typename T>
__device__ __forceinline__ void apply_prow(const T (&L)[32], T* vec, int ld, int i, int p0, int nb, int nr) {
  for (int r = 0; r < nr; ++r) {
    const T* yb = vec + r * ld + p0;
    T a = T(0);
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      if (c >= nb) break;
      a += L[c] * yb[c];
    }
    vec[r * ld + i] -= a;
  }
}

template <typename T>
__device__ __forceinline__ void stage_block(T* dst, const T* f, int F, int p0, int nb, bool lower,
                                            int tid, int nt) {
  for (int q = tid; q < 32 * 32; q += nt) {
    const int i = q & 31, c = q >> 5;
    const bool keep = (i < nb && c < nb) && (lower ? (i > c) : (i <= c));
    dst[i * kBS + c] = keep ? f[(p0 + i) + (int64_t)(p0 + c) * F] : T(0);
  }
}

template <typename T>
__device__ __forceinline__ void blk_forward(const SymDev& sd, int s, int k, int r0, int nr, int ch,
                                            unsigned char* smraw, const T* __restrict__ fronts,
                                            const double* __restrict__ rhs, int rhs_mode,
                                            T* __restrict__ V, int R, int K, const Sync& sy) {
  const int ns = sd.ns[s], ms = sd.ms[s], F = ns + ms;
  const int c0 = sd.c0[s];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  T* blk = reinterpret_cast<T*>(smraw);          // 2 x 32 x kBS
  T* v = blk + 2 * 32 * kBS;                      // nr x F
  const T* f = fronts + (int64_t)K * sd.front_off[s] + (int64_t)k * F * F;
  stage_block(blk, f, F, 0, min(32, ns), true, tid, nt);
  if (sy.done) sy.wait_children(sd, s, k, K, tid, nt);
  __syncthreads();
  for (int q = tid; q < nr * F; q += nt) {
    const int j = q % F, r = q / F;
    v[r * F + j] = gather_position<T, 8>(sd, s, j, ns, c0, rhs, rhs_mode, V, k, K, R, r0 + r);
  }
  __syncthreads();
  constexpr int PF = BlkPF<T>::N;
  int cur = 0;
  for (int p0 = 0; p0 < ns; p0 += 32) {
    const int nb = min(32, ns - p0);
    const int ib = p0 + nb;
    const bool more = p0 + 32 < ns;
    T Lp[PF][32], nx[4];
#pragma unroll
    for (int g = 0; g < PF; ++g) load_prow(Lp[g], f, F, ib + g * nt + tid, p0, nb, ib + g * nt + tid < F);
    load_block_regs(nx, f, F, p0 + 32, more ? min(32, ns - p0 - 32) : 0, true, more, tid);
    const T* B = blk + cur * 32 * kBS;
    for (int r = wid; r < nr; r += nw) {
      T vi = (lane < nb) ? v[r * F + p0 + lane] : T(0);
      fwd_block_solve(B, vi, nb, lane);
      if (lane < nb) v[r * F + p0 + lane] = vi;
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < PF; ++g)
      if (ib + g * nt + tid < F) apply_prow(Lp[g], v, F, ib + g * nt + tid, p0, nb, nr);
    // rows beyond the prefetched ones: PF rows per round, loads first
    for (int i0 = ib + PF * nt + tid; i0 < F; i0 += PF * nt) {
#pragma unroll
      for (int g = 0; g < PF; ++g) load_prow(Lp[g], f, F, i0 + g * nt, p0, nb, i0 + g * nt < F);
#pragma unroll
      for (int g = 0; g < PF; ++g)
        if (i0 + g * nt < F) apply_prow(Lp[g], v, F, i0 + g * nt, p0, nb, nr);
    }
    if (more) store_block_regs(blk + (cur ^ 1) * 32 * kBS, nx, tid);
    __syncthreads();
    cur ^= 1;
  }
  T* outv = V + (int64_t)K * R * sd.vec_off[s] + ((int64_t)k * R + r0) * F;
  for (int q = tid; q < nr * F; q += nt) outv[q] = v[q];
  if (sy.done) {
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      sy.add(s, k, K);
    }
  }
}

template <typename T>
__device__ __forceinline__ void blk_backward(const SymDev& sd, int s, int k, int r0, int nr, int ch,
                                             unsigned char* smraw, const T* __restrict__ fronts,
                                             const T* __restrict__ V, double* out, double* acc,
                                             int R, int K, const Sync& sy) {
  const int ns = sd.ns[s], ms = sd.ms[s], F = ns + ms;
  const int c0 = sd.c0[s];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  T* blk = reinterpret_cast<T*>(smraw);
  T* xr = blk + 2 * 32 * kBS;
  T* z = xr + nr * ms;
  const T* f = fronts + (int64_t)K * sd.front_off[s] + (int64_t)k * F * F;
  const int32_t* rows = sd.rows + sd.row_off[s];
  const int last0 = ((ns - 1) / 32) * 32;        // first pivot of the bottom block
  stage_block(blk, f, F, last0, ns - last0, false, tid, nt);
  const T* y = V + (int64_t)K * R * sd.vec_off[s] + ((int64_t)k * R + r0) * F;
  for (int q = tid; q < nr * ns; q += nt) {
    const int p = q % ns, r = q / ns;
    z[q] = y[(int64_t)r * F + p];
  }
  if (sy.done && tid == 0 && ms > 0) sy.wait_parent(s, sd.parent[s], k, K);
  __syncthreads();
  for (int q = tid; q < nr * ms; q += nt) {
    const int j = q % ms, r = q / ms;
    xr[q] = (T)__ldcg(out + ((int64_t)rows[j] * K + k) * R + r0 + r);
  }
  __syncthreads();
  if (ms > 0) {
    // z[r][p] -= sum_j U12[p][j] xr[r][j]; thread (p, jj) takes every JG-th j
    // for a group of 4 right-hand sides.  With JG > 1 the JG partial sums of
    // an (r, p) meet in shared memory and are added in jj order, so that the
    // result does not depend on the order in which threads finish.
    const int JG = max(1, min(32, nt / ns));
    T* part = z + nr * ns;  // [JG][4][ns], JG * ns <= nt
    for (int rr = 0; rr < nr; rr += 4) {
      for (int q = tid; q < ns * JG; q += nt) {
        const int p = q % ns, jj = q / ns;
        T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        for (int j = jj; j < ms; j += JG) {
          const T u = f[p + (int64_t)(ns + j) * F];
          const T* x0 = xr + rr * ms + j;
          a0 += u * x0[0];
          if (rr + 1 < nr) a1 += u * x0[ms];
          if (rr + 2 < nr) a2 += u * x0[2 * ms];
          if (rr + 3 < nr) a3 += u * x0[3 * ms];
        }
        if (JG == 1) {  // one thread per (r, p)
          z[rr * ns + p] -= a0;
          if (rr + 1 < nr) z[(rr + 1) * ns + p] -= a1;
          if (rr + 2 < nr) z[(rr + 2) * ns + p] -= a2;
          if (rr + 3 < nr) z[(rr + 3) * ns + p] -= a3;
        } else {
          T* pq = part + jj * 4 * ns + p;
          pq[0] = a0;
          pq[ns] = a1;
          pq[2 * ns] = a2;
          pq[3 * ns] = a3;
        }
      }
      if (JG > 1) {  // CTA-uniform
        __syncthreads();
        for (int q = tid; q < min(4, nr - rr) * ns; q += nt) {
          const int p = q % ns, r = q / ns;
          T a = 0;
          for (int jj = 0; jj < JG; ++jj) a += part[(jj * 4 + r) * ns + p];
          z[(rr + r) * ns + p] -= a;
        }
        __syncthreads();  // part is reused by the next group
      }
    }
    __syncthreads();
  }
  constexpr int PF = BlkPF<T>::N;
  int cur = 0;
  for (int p0 = last0; p0 >= 0; p0 -= 32) {
    const int nb = min(32, ns - p0);
    T Up[PF][32], nx[4];
#pragma unroll
    for (int g = 0; g < PF; ++g) load_prow(Up[g], f, F, g * nt + tid, p0, nb, g * nt + tid < p0);
    load_block_regs(nx, f, F, p0 - 32, 32, false, p0 > 0, tid);
    const T* B = blk + cur * 32 * kBS;
    for (int r = wid; r < nr; r += nw) {
      T zi = (lane < nb) ? z[r * ns + p0 + lane] : T(0);
      bwd_block_solve(B, zi, nb, lane);
      if (lane < nb) z[r * ns + p0 + lane] = zi;
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < PF; ++g)
      if (g * nt + tid < p0) apply_prow(Up[g], z, ns, g * nt + tid, p0, nb, nr);
    for (int i0 = PF * nt + tid; i0 < p0; i0 += PF * nt) {
#pragma unroll
      for (int g = 0; g < PF; ++g) load_prow(Up[g], f, F, i0 + g * nt, p0, nb, i0 + g * nt < p0);
#pragma unroll
      for (int g = 0; g < PF; ++g)
        if (i0 + g * nt < p0) apply_prow(Up[g], z, ns, i0 + g * nt, p0, nb, nr);
    }
    if (p0 > 0) store_block_regs(blk + (cur ^ 1) * 32 * kBS, nx, tid);
    __syncthreads();
    cur ^= 1;
  }
  for (int q = tid; q < nr * ns; q += nt) {
    const int p = q % ns, r = q / ns;
    const int64_t o = ((int64_t)(c0 + p) * K + k) * R + r0 + r;
    out[o] = (double)z[q];
    if (acc) acc[o] += (double)z[q];
  }
  if (sy.done) {
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      sy.publish_children(sd, s, k, K);
    }
  }
}

// ---- level-synchronous kernels (one launch per level and size class) ----
template <typename T, int SEG>
__global__ void __launch_bounds__(256, 2) k_forward_seg(SymDev sd, const int32_t* __restrict__ list,
                                                        int64_t nseg, const T* __restrict__ fronts,
                                                        const double* __restrict__ rhs, int rhs_mode,
                                                        T* __restrict__ V, int R, int K) {
  __shared__ T buf[256 / SEG][kRW][SEG + 1];
  const int64_t sg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / SEG;
  const SegTask t = seg_task(sd, list, sg, nseg, R, K);
  seg_forward<T, SEG>(sd, t, threadIdx.x % SEG, buf[threadIdx.x / SEG], fronts, rhs, rhs_mode, V, R,
                      K, Sync{nullptr, nullptr, nullptr, 0});
}

template <typename T, int SEG>
__global__ void __launch_bounds__(256, 2) k_backward_seg(SymDev sd, const int32_t* __restrict__ list,
                                                         int64_t nseg, const T* __restrict__ fronts,
                                                         const T* __restrict__ V, double* out,
                                                         double* acc, int R, int K) {
  const int64_t sg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / SEG;
  const SegTask t = seg_task(sd, list, sg, nseg, R, K);
  seg_backward<T, SEG>(sd, t, threadIdx.x % SEG, fronts, V, out, acc, R, K, Sync{nullptr, nullptr, nullptr, 0});
}

template <typename T>
__global__ void __launch_bounds__(kSolveThreads, 2) k_forward_blk(SymDev sd, const int32_t* __restrict__ list,
                                                                  const T* __restrict__ fronts,
                                                                  const double* __restrict__ rhs,
                                                                  int rhs_mode, T* __restrict__ V,
                                                                  int R, int K, int rc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int r0 = blockIdx.z * rc;
  if (r0 >= R) return;
  blk_forward<T>(sd, list[blockIdx.x], blockIdx.y, r0, min(rc, R - r0), 0, smraw, fronts, rhs,
                 rhs_mode, V, R, K, Sync{nullptr, nullptr, nullptr, 0});
}

template <typename T>
__global__ void __launch_bounds__(kSolveThreads, 2) k_backward_blk(SymDev sd, const int32_t* __restrict__ list,
                                                                   const T* __restrict__ fronts,
                                                                   const T* __restrict__ V, double* out,
                                                                   double* acc, int R, int K, int rc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int r0 = blockIdx.z * rc;
  if (r0 >= R) return;
  blk_backward<T>(sd, list[blockIdx.x], blockIdx.y, r0, min(rc, R - r0), 0, smraw, fronts, V, out,
                  acc, R, K, Sync{nullptr, nullptr, nullptr, 0});
}

// ---------------------------------------------------------------------------
// K-fused segment tasks of the persistent schedule.  A segment of SEG lanes
// (SEG = 8, 16 or 32) solves one (front, RHS chunk of up to kRW right-hand
// sides) for ALL K perturbations: the task's ticket, its structure loads and
// its dependency wait are paid once for the K solves, and the index data of
// the gathers is fetched from memory once and re-read from L1 for the other
// shifts.  A front qualifies when its pivots fit the segment (ns <= SEG);
// for SEG < 32 the whole front fits (F <= SEG), for SEG = 32 the update rows
// beyond the first 32 are handled in further blocks of 32 rows: lane i owns
// rows i, i + 32, ...  Loops run to warp-uniform bounds (entries beyond a
// front are zero), so segments with different fronts never diverge around a
// shuffle.  All lanes of a warp call these bodies together.
// ---------------------------------------------------------------------------
struct FTask {
  bool active;
  int s, r0, nr, k0, k1;  // front, RHS chunk [r0, r0 + nr), shifts [k0, k1)
};

// task q of a group: front list[q / (nkg * nch)], shift group (q / nch) % nkg
// of kf shifts, RHS chunk q % nch (nkg = ceil(K / kf) shift groups)
// (act: per-instance flags of the adaptive sweeps; a task of an instance
// that has stopped is inactive, or nullptr: every task is active)
__device__ __forceinline__ FTask ftask(const int32_t* list, int64_t q, int64_t ntasks, int R, int K,
                                       int kf, const int32_t* inst, const uint8_t* act) {
  FTask t{false, 0, 0, 0, 0, 0};
  const int nch = (R + kRW - 1) / kRW;
  const int nkg = (K + kf - 1) / kf;
  if (q < ntasks) {
    t.s = list[q / ((int64_t)nch * nkg)];
    t.active = !act || act[inst[t.s]];
    const int kg = (int)((q / nch) % nkg);
    t.k0 = kg * kf;
    t.k1 = min(K, t.k0 + kf);
    t.r0 = (int)(q % nch) * kRW;
    t.nr = min(kRW, R - t.r0);
  }
  return t;
}

// the n lanes (index idx) of a segment wait for every (child, k) counter,
// k in [k0, k1), of front s, polling in parallel; each polling lane then
// fences (acquire), and the caller's __syncwarp orders the segment's later
// loads after the fences
__device__ __forceinline__ void wait_children_allk(const Sync& sy, const SymDev& sd, int s, int k0, int k1,
                                                   int K, int idx, int n) {
  const int cb = sd.child_off[s], ce = sd.child_off[s + 1];
  const int nk = k1 - k0;
  const int total = (ce - cb) * nk;
  for (int q = idx; q < total; q += n) {
    const int c = sd.child[cb + q / nk], k = k0 + q % nk;
    const int* f = sy.done + (int64_t)c * K + k;
    const int need = sy.nch[c];
    if (ld_relaxed(f) >= need) continue;
    int64_t i = 0;
    for (; i < sy.polls; ++i) {
      __nanosleep(64);
      if (ld_relaxed(f) >= need) break;
    }
    if (i == sy.polls) atomicExch(sy.err, 1);
  }
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

// the parent's counters of every k in [k0, k1) (backward solve)
__device__ __forceinline__ void wait_parent_allk(const Sync& sy, int p, int k0, int k1, int K, int idx, int n) {
  for (int k = k0 + idx; k < k1; k += n) {
    const int* f = sy.done + (int64_t)p * K + k;
    const int need = sy.nch[p];
    if (ld_relaxed(f) >= need) continue;
    int64_t i = 0;
    for (; i < sy.polls; ++i) {
      __nanosleep(64);
      if (ld_relaxed(f) >= need) break;
    }
    if (i == sy.polls) atomicExch(sy.err, 1);
  }
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

// after the segment's stores: one lane per k makes them visible and counts
// the finished chunk of (s, k)
__device__ __forceinline__ void publish_allk(const Sync& sy, bool active, int s, int k0, int k1, int K,
                                             int idx, int n) {
  __syncwarp();
  if (!active) return;
  for (int k = k0 + idx; k < k1; k += n) {
    __threadfence();
    asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(sy.done + (int64_t)s * K + k) : "memory");
  }
}

// Forward solve with L (unit lower) of one front for all K: y = L11^{-1} v on
// the pivot rows (shuffle chain), then v_i -= L21(i, :) y on the update rows;
// V[k][r][0..F) receives the result (pivot part y, update part the
// contribution the parent gathers).  yb: this warp's [32][kRW] staging area
// for y when the front has update rows beyond the first 32.
template <typename T, int SEG>
__device__ __forceinline__ void kseg_forward(const SymDev& sd, const FTask& t, int sl, T* yb,
                                             const T* __restrict__ fronts, const double* __restrict__ rhs,
                                             int rhs_mode, T* __restrict__ V, int R, int K, const Sync& sy) {
  int ns = 0, F = 0, c0 = 0;
  int64_t fo = 0, vo = 0;
  if (t.active) {
    ns = sd.ns[t.s];
    F = ns + sd.ms[t.s];
    c0 = sd.c0[t.s];
    fo = sd.front_off[t.s];
    vo = sd.vec_off[t.s];
  }
  const int r0 = t.r0, nr = t.nr;
  if (sy.done && t.active) wait_children_allk(sy, sd, t.s, t.k0, t.k1, K, sl, SEG);
  __syncwarp();
  const int nrw = __reduce_max_sync(kFull, nr);
  const int nsw = __reduce_max_sync(kFull, ns);
  const int nb = (__reduce_max_sync(kFull, F) + SEG - 1) / SEG;  // > 1 only for SEG = 32
  const int nkw = __reduce_max_sync(kFull, t.k1 - t.k0);          // shifts per task (uniform)
  for (int kk = 0; kk < nkw; ++kk) {
    const int k = t.active ? min(t.k0 + kk, t.k1 - 1) : 0;
    const bool kon = t.active && t.k0 + kk < t.k1;
    const T* f = fronts + (kon ? (int64_t)K * fo + (int64_t)k * F * F : 0);
    T Lr[SEG];
#pragma unroll
    for (int c = 0; c < SEG; ++c) Lr[c] = (kon && c < ns && sl > c && sl < F) ? f[sl + c * F] : T(0);
    T vv[kRW];
    gather_position_rhs<T>(sd, t.s, sl, ns, c0, rhs, rhs_mode, V, k, K, R, r0, (kon && sl < F) ? nr : 0, vv);
#pragma unroll
    for (int c = 0; c < SEG - 1; ++c) {
      if (c >= nsw) break;
#pragma unroll
      for (int r = 0; r < kRW; ++r)
        if (r < nrw) vv[r] -= Lr[c] * __shfl_sync(kFull, vv[r], c, SEG);
    }
    T* Vs = V + (kon ? (int64_t)K * R * vo + ((int64_t)k * R + r0) * F : 0);
#pragma unroll
    for (int r = 0; r < kRW; ++r)
      if (kon && r < nr && sl < F) Vs[(int64_t)r * F + sl] = vv[r];
    if (SEG == 32 && nb > 1) {
#pragma unroll
      for (int r = 0; r < kRW; ++r) yb[sl * kRW + r] = vv[r];
      __syncwarp();
      for (int b = 1; b < nb; ++b) {
        const int i = b * 32 + sl;
        T acc[kRW];
        gather_position_rhs<T>(sd, t.s, i, ns, c0, rhs, rhs_mode, V, k, K, R, r0, (kon && i < F) ? nr : 0, acc);
        for (int c = 0; c < nsw; ++c) {
          const T l = (kon && c < ns && i < F) ? f[i + (int64_t)c * F] : T(0);
#pragma unroll
          for (int r = 0; r < kRW; ++r) acc[r] -= l * yb[c * kRW + r];
        }
#pragma unroll
        for (int r = 0; r < kRW; ++r)
          if (kon && r < nr && i < F) Vs[(int64_t)r * F + i] = acc[r];
      }
      __syncwarp();  // yb is reused by the next k
    }
  }
  if (sy.done) publish_allk(sy, t.active, t.s, t.k0, t.k1, K, sl, SEG);
}

// Backward solve with U of one front for all K: z = y - U12 x_R (update rows
// gathered from the ancestors' solutions SEG at a time and shared by
// shuffles), then x = U11^{-1} z by a shuffle chain; x is written to `out`
// (and added to `acc`).
template <typename T, int SEG>
__device__ __forceinline__ void kseg_backward(const SymDev& sd, const FTask& t, int sl,
                                              const T* __restrict__ fronts, const T* __restrict__ V,
                                              double* out, double* acc, int R, int K, const Sync& sy) {
  int ns = 0, ms = 0, F = 0, c0 = 0;
  int64_t fo = 0, vo = 0, ro = 0;
  if (t.active) {
    ns = sd.ns[t.s];
    ms = sd.ms[t.s];
    F = ns + ms;
    c0 = sd.c0[t.s];
    fo = sd.front_off[t.s];
    vo = sd.vec_off[t.s];
    ro = sd.row_off[t.s];
  }
  const int r0 = t.r0, nr = t.nr;
  if (sy.done && t.active && ms > 0) wait_parent_allk(sy, sd.parent[t.s], t.k0, t.k1, K, sl, SEG);
  __syncwarp();
  const int nrw = __reduce_max_sync(kFull, nr);
  const int msw = __reduce_max_sync(kFull, ms);
  const int nsw = __reduce_max_sync(kFull, ns);
  const int nkw = __reduce_max_sync(kFull, t.k1 - t.k0);          // shifts per task (uniform)
  for (int kk = 0; kk < nkw; ++kk) {
    const int k = t.active ? min(t.k0 + kk, t.k1 - 1) : 0;
    const bool kon = t.active && t.k0 + kk < t.k1;
    const T* f = fronts + (kon ? (int64_t)K * fo + (int64_t)k * F * F : 0);
    const T* Vs = V + (kon ? (int64_t)K * R * vo + ((int64_t)k * R + r0) * F : 0);
    T zt[kRW];
#pragma unroll
    for (int r = 0; r < kRW; ++r) zt[r] = (kon && r < nr && sl < ns) ? Vs[(int64_t)r * F + sl] : T(0);
    const T rd = (kon && sl < ns) ? T(1) / f[sl * (F + 1)] : T(0);
    for (int j0 = 0; j0 < msw; j0 += SEG) {
      const int j = j0 + sl;
      const int64_t row = (j < ms) ? sd.rows[ro + j] : 0;
      T xt[kRW];
      ld_rhs8<T>(out + (row * K + k) * R + r0, (kon && j < ms) ? nr : 0, xt);
#pragma unroll 4
      for (int jj = 0; jj < SEG; ++jj) {
        if (j0 + jj >= msw) break;
        const T u = (kon && sl < ns && j0 + jj < ms) ? f[sl + (int64_t)(ns + j0 + jj) * F] : T(0);
#pragma unroll
        for (int r = 0; r < kRW; ++r)
          if (r < nrw) zt[r] -= u * __shfl_sync(kFull, xt[r], jj, SEG);
      }
    }
#pragma unroll 4
    for (int c = SEG - 1; c >= 0; --c) {
      if (c >= nsw) continue;
      const T u = (kon && sl < ns && c > sl && c < ns) ? f[sl + c * F] : T(0);
#pragma unroll
      for (int r = 0; r < kRW; ++r) {
        if (r < nrw) {
          if (sl == c) zt[r] *= rd;
          zt[r] -= u * __shfl_sync(kFull, zt[r], c, SEG);
        }
      }
    }
    if (kon && sl < ns) {
      const int64_t o = ((int64_t)(c0 + sl) * K + k) * R + r0;
      st_rhs8<T>(out + o, acc ? acc + o : nullptr, nr, zt);
    }
  }
  if (sy.done) publish_allk(sy, t.active, t.s, t.k0, t.k1, K, sl, SEG);
}

// ---- persistent schedule: one launch per direction -------------------------
// CTAs take work units in ticket order (levels bottom-up for the forward
// solve, top-down for the backward solve).  A unit is either one (front, k,
// RHS chunk) of a front with more than 32 pivots, solved by the whole CTA
// (blocked path), or 256/SEG K-fused segment tasks, one per segment of the
// CTA's warps.  A unit only waits for units with smaller tickets, which
// running CTAs already hold, so the schedule cannot deadlock whatever the
// number of resident CTAs.  In the later adaptive sweeps the list is the
// in-order subsequence of the units that hold a front of an instance still
// iterating, which keeps that property.
template <typename T, bool FWD, int MINB>
__global__ void __launch_bounds__(kSolveThreads, MINB)
k_solve_persistent(SymDev sd, const SolveUnit* __restrict__ units, int nunits, const int* __restrict__ ucount,
                   const uint8_t* __restrict__ act, int* ticket, int* done, int* err,
                   const int* __restrict__ nch, const int32_t* __restrict__ all, const T* __restrict__ fronts,
                   const double* __restrict__ rhs, int rhs_mode, T* __restrict__ V, double* out, double* acc,
                   int R, int K, int64_t polls) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_unit;
  const Sync sy{done, err, nch, polls};
  const int tid = threadIdx.x;
  // a compacted unit list (adaptive sweeps) has its length on the device
  if (ucount) nunits = *ucount;
  for (;;) {
    if (tid == 0) s_unit = atomicAdd(ticket, 1);
    __syncthreads();
    const int u = s_unit;
    if (u >= nunits) return;
    const SolveUnit U = units[u];
    if (U.kind == kUnitBlk) {
      // a front of an instance whose sweeps have stopped is skipped: no front
      // of another instance depends on it (CTA-uniform test)
      if (!act || act[sd.inst[U.a]]) {
        const int r0 = U.c * U.d;
        if (FWD)
          blk_forward<T>(sd, U.a, U.b, r0, min(U.d, R - r0), U.c, smraw, fronts, rhs, rhs_mode, V, R, K, sy);
        else
          blk_backward<T>(sd, U.a, U.b, r0, min(U.d, R - r0), U.c, smraw, fronts, V, out, acc, R, K, sy);
      }
    } else {
      const int SEG = U.kind == kUnitSeg8 ? 8 : (U.kind == kUnitSeg16 ? 16 : 32);
      const int64_t q = (int64_t)U.b + tid / SEG;
      const FTask t = ftask(all + U.a, q, (int64_t)U.c, R, K, max(1, U.d), sd.inst, act);
      T* yb = reinterpret_cast<T*>(smraw) + (tid >> 5) * 32 * kRW;
      if (U.kind == kUnitSeg8) {
        if (FWD) kseg_forward<T, 8>(sd, t, tid % 8, yb, fronts, rhs, rhs_mode, V, R, K, sy);
        else kseg_backward<T, 8>(sd, t, tid % 8, fronts, V, out, acc, R, K, sy);
      } else if (U.kind == kUnitSeg16) {
        if (FWD) kseg_forward<T, 16>(sd, t, tid % 16, yb, fronts, rhs, rhs_mode, V, R, K, sy);
        else kseg_backward<T, 16>(sd, t, tid % 16, fronts, V, out, acc, R, K, sy);
      } else {
        if (FWD) kseg_forward<T, 32>(sd, t, tid % 32, yb, fronts, rhs, rhs_mode, V, R, K, sy);
        else kseg_backward<T, 32>(sd, t, tid % 32, fronts, V, out, acc, R, K, sy);
      }
    }
    __syncthreads();
  }
}

// x[perm[i]][r] = sum_k w_k X[i][k][r]   (Eq. x_star; FP64, k ascending)
__global__ void k_combine(SymDev sd, const double* __restrict__ X, Shifts sh, int R,
                          double* __restrict__ x) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= sd.N * R) return;
  const int64_t i = q / R;
  const int r = (int)(q % R);
  const int K = sh.K;
  double a = 0.0;
  for (int k = 0; k < K; ++k) a += sh.w[k] * X[(i * K + k) * R + r];
  x[(int64_t)sd.perm[i] * R + r] = a;
}

// largest q in [0, n] with arow[q] <= a (arow[0] = 0 <= a)
__device__ __forceinline__ int active_slot(const int64_t* arow, int n, int64_t a) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (arow[mid] <= a) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Rk[pi][k][r] = b[i][r] - sum_j A_ij X[pj][k][r] - t_k D_i X[pi][k][r] for one
// row (original index i, permuted pi), FP64, by one warp.
__device__ __forceinline__ void residual_row(const SymDev& sd, const double* __restrict__ vals,
                                             const double* __restrict__ D, const Shifts& sh,
                                             const double* __restrict__ b, const double* __restrict__ X, int R,
                                             double* __restrict__ Rk, int64_t i, int64_t pi, int lane) {
  const int K = sh.K;
  const int KR = K * R;
  const int64_t e0 = sd.row_ptr[i], e1 = sd.row_ptr[i + 1];
  const double di = D[i];
  if (e1 - e0 <= 32) {
    // the row's entries and permuted columns are loaded once, one per lane,
    // and broadcast: the (k, r) columns of the row do not repeat the chain
    // of dependent index loads; the sum keeps the entry order
    const int nz = (int)(e1 - e0);
    double v = 0.0;
    int64_t pc = 0;
    if (lane < nz) {
      v = vals[e0 + lane];
      pc = sd.iperm[sd.col[e0 + lane]];
    }
    for (int q0 = 0; q0 < KR; q0 += 32) {  // warp-uniform: every lane reaches the shuffles
      const int q = q0 + lane;
      const bool act = q < KR;
      const int k = act ? q / R : 0, r = act ? q - k * R : 0;
      double a = act ? b[i * R + r] - sh.t[k] * di * X[(pi * K + k) * R + r] : 0.0;
      for (int e = 0; e < nz; ++e) {
        const double ve = __shfl_sync(kFull, v, e);
        const int64_t pe = __shfl_sync(kFull, pc, e);
        if (act) a -= ve * X[(pe * K + k) * R + r];
      }
      if (act) Rk[(pi * K + k) * R + r] = a;
    }
    return;
  }
  for (int q = lane; q < KR; q += 32) {
    const int k = q / R, r = q % R;
    double a = b[i * R + r] - sh.t[k] * di * X[(pi * K + k) * R + r];
    for (int64_t e = e0; e < e1; ++e)
      a -= vals[e] * X[((int64_t)sd.iperm[sd.col[e]] * K + k) * R + r];
    Rk[(pi * K + k) * R + r] = a;
  }
}

// The FP64 residuals of the perturbed systems, one warp per row, warps
// striding over the rows (rows as ResidualMode selects) in the permuted order,
// where an instance's rows keep its range: the writes of Rk and the reads of
// the row's own X are sequential.

__global__ void k_residual_per_k(SymDev sd, const double* __restrict__ vals,
                                 const double* __restrict__ D, Shifts sh,
                                 const double* __restrict__ b, const double* __restrict__ X, int R,
                                 double* __restrict__ Rk, ActiveSet as, int mode) {
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  int nact = 0;
  int64_t total = sd.N;
  if (mode == kResActive) {
    nact = *as.nact;
    total = as.arow[nact];
  }
  for (int64_t a = w0; a < total; a += nw) {  // warp-uniform
    int64_t pi = a;  // an instance's permuted rows are its original range
    if (mode == kResActive) {
      const int q = active_slot(as.arow, nact, a);
      pi = as.inst_off[as.ai[q]] + (a - as.arow[q]);
    }
    const int64_t i = sd.perm[pi];
    if (mode == kResZeroStopped && !as.act[sd.row_inst[i]]) {
      const int KR = sh.K * R;
      for (int q = lane; q < KR; q += 32) Rk[pi * KR + q] = 0.0;
      continue;
    }
    residual_row(sd, vals, D, sh, b, X, R, Rk, i, pi, lane);
  }
}

// Rk[pj][k][r] = g[j][r] - sum_i A_ij Lam[pi][k][r] - t_k D_j Lam[pj][k][r]  (FP64):
// the residual of the transposed perturbed system (A + t_k D)^T lambda_k = g,
// one warp per original column j (A's columns through the CSC arrays).
__global__ void k_residual_T_per_k(SymDev sd, const double* __restrict__ vals,
                                   const double* __restrict__ D, Shifts sh,
                                   const double* __restrict__ g, const double* __restrict__ Lam, int R,
                                   double* __restrict__ Rk) {
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= sd.N) return;
  const int K = sh.K;
  const int KR = K * R;
  const int64_t pj = sd.iperm[j];
  const int64_t q0 = sd.at_ptr[j], q1 = sd.at_ptr[j + 1];
  const double dj = D[j];
  for (int q = lane; q < KR; q += 32) {
    const int k = q / R, r = q % R;
    double a = g[j * R + r] - sh.t[k] * dj * Lam[(pj * K + k) * R + r];
    for (int64_t e = q0; e < q1; ++e)
      a -= vals[sd.at_src[e]] * Lam[((int64_t)sd.iperm[sd.at_row[e]] * K + k) * R + r];
    Rk[(pj * K + k) * R + r] = a;
  }
}

// r[i][c] = b[i][c] - sum_j A_ij x[j][c]  (FP64, original order), warp per row
__global__ void k_residual(SymDev sd, const double* __restrict__ vals, const double* __restrict__ b,
                           const double* __restrict__ x, int R, double* __restrict__ res) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= sd.N) return;
  const int64_t e0 = sd.row_ptr[i], e1 = sd.row_ptr[i + 1];
  for (int r = lane; r < R; r += 32) {
    double a = b[i * R + r];
    for (int64_t e = e0; e < e1; ++e) a -= vals[e] * x[(int64_t)sd.col[e] * R + r];
    res[i * R + r] = a;
  }
}

// ---- adaptive FP64 residual sweeps -----------------------------------------
// After the correction solves of sweep s, every instance g still iterating
// takes its correction, X += Y (FP64, one addition per entry: the sum the
// backward solve's accumulation would form), and gets the size of the
// correction d_s and of the new solution, per right-hand side r:
//   dmax[g][r] = max over its rows i and over k of |Y[pi][k][r]|,
//   xmax[g][r] = max over its rows i and over k of |X[pi][k][r]|.
// CTAs stride over chunks of kStatRows rows of the active set.  Within an
// instance the rows' (i, k) pairs form a matrix of R columns: thread t keeps
// column c = t % RB of a pass (RB = min(R, 256)) and every (256/RB)-th pair,
// so a warp's loads are contiguous; the per-column maxima meet in shared
// memory and then in one
// 64-bit atomicMax per (g, r) on the bit patterns (non-negative doubles
// order as their bit patterns, and a NaN orders above +inf, so a NaN never
// reads as converged).
constexpr int kStatThreads = 256;
constexpr int kStatRows = 64;

__global__ void __launch_bounds__(kStatThreads)
k_refine_stats(SymDev sd, ActiveSet as, double* __restrict__ X, const double* __restrict__ Y, int K, int R,
               unsigned long long* __restrict__ dmax, unsigned long long* __restrict__ xmax) {
  __shared__ unsigned long long s_d[kStatThreads], s_x[kStatThreads];
  const int nact = *as.nact;
  const int64_t total = as.arow[nact];
  const int tid = threadIdx.x;
  const int RB = min(R, kStatThreads);
  const int nj = kStatThreads / RB;
  const int c = tid % RB, j = tid / RB;
  for (int64_t a0 = (int64_t)blockIdx.x * kStatRows; a0 < total; a0 += (int64_t)gridDim.x * kStatRows) {
    const int64_t a1 = min(total, a0 + kStatRows);
    // the instances overlapping active rows [a0, a1), in order (CTA-uniform)
    int q = active_slot(as.arow, nact, a0);
    for (;; ++q) {
      const int g = as.ai[q];
      const int64_t s0 = as.arow[q], s1 = as.arow[q + 1];
      const int64_t lo = max(a0, s0), hi = min(a1, s1);
      if (lo < hi) {
        // the instance's permuted rows are its original range: its (row, k)
        // pairs from i0 on are contiguous in X and Y
        const int64_t i0 = as.inst_off[g] + (lo - s0);
        const int64_t npair = (hi - lo) * K;
        for (int rb = 0; rb < R; rb += RB) {
          const int r = rb + c;
          unsigned long long md = 0, mx = 0;
          if (j < nj && r < R) {
            for (int64_t m = j; m < npair; m += nj) {
              const int64_t o = (i0 * K + m) * R + r;
              const double y = Y[o];
              const double xn = X[o] + y;
              X[o] = xn;
              md = max(md, (unsigned long long)__double_as_longlong(fabs(y)));
              mx = max(mx, (unsigned long long)__double_as_longlong(fabs(xn)));
            }
          }
          s_d[tid] = md;
          s_x[tid] = mx;
          __syncthreads();
          if (j == 0 && r < R) {
            for (int t = 1; t < nj; ++t) {
              md = max(md, s_d[t * RB + c]);
              mx = max(mx, s_x[t * RB + c]);
            }
            atomicMax(dmax + (int64_t)g * R + r, md);
            atomicMax(xmax + (int64_t)g * R + r, mx);
          }
          __syncthreads();
        }
      }
      if (s1 >= a1) break;
    }
  }
}

// Exclusive prefix sum over the 1024 threads of a CTA (every thread calls);
// total = the sum of all v.
constexpr int kDecideThreads = 1024;

template <typename V>
__device__ V block_excl_scan(V v, V* sh, V& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  V x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const V y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    V y = sh[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const V z = __shfl_up_sync(kFull, y, o);
      if (lane >= o) y += z;
    }
    sh[lane] = y;
  }
  __syncthreads();
  total = sh[31];
  const V r = x - v + (w > 0 ? sh[w - 1] : V(0));
  __syncthreads();  // sh is reused by the next scan
  return r;
}

// One CTA, after sweep s = *sweep + 1 (the count of sweeps done is kept on
// the device, so that the same launch serves every sweep of a device-side
// loop).  For each instance g still iterating: the stopping test of
// extra-precise iterative refinement (Demmel, Hida, Kahan, Li, Mukherjee,
// Riedy, ACM TOMS 2006), with the contraction per sweep estimated from two
// successive corrections, so from the second sweep on.  Per right-hand side,
// rho = |d_s| / |d_{s-1}|: converged when |d_s| = 0, or (s >= 2) when rho <
// 1/2 and rho / (1 - rho) |d_s| <= tol |x| (the error that a contraction by
// rho per sweep leaves); stagnating when rho >= 1/2 (s >= 2: further sweeps
// no longer reduce the error).  After the first sweep only |d_1| = 0 stops:
// |d_1| / |x| is the first solve's error, which can understate the
// contraction by orders of magnitude.  The instance stops when every
// right-hand side has converged or stagnated, or after sweep S; nsw[g] = the
// sweeps it took.  dmax / xmax are zeroed for the next sweep.  Then the
// active set: pre[g] = the active instances before g (pre[G] = their number =
// *nact), ai and arow as in ActiveSet.  With a conditional handle (the sweeps
// as a device-side loop) the loop goes on while an instance is active and s <
// S: at most S sweeps whatever the data.
__global__ void __launch_bounds__(kDecideThreads)
k_refine_decide(int G, int R, double tol, int S, int* __restrict__ sweep, cudaGraphConditionalHandle cond,
                int has_cond, uint8_t* __restrict__ act, unsigned long long* __restrict__ dmax,
                unsigned long long* __restrict__ xmax, double* __restrict__ prevd, int* __restrict__ nsw,
                int* __restrict__ pre, int* __restrict__ nact, int* __restrict__ ai, int64_t* __restrict__ arow,
                const int64_t* __restrict__ inst_off) {
  __shared__ int sh[32];
  __shared__ long long sh64[32];
  const int s = *sweep + 1;
  const bool last = s >= S;
  for (int g = threadIdx.x; g < G; g += kDecideThreads) {
    if (!act[g]) continue;
    bool all = true;
    for (int r = 0; r < R; ++r) {
      const int64_t q = (int64_t)g * R + r;
      const double d = __longlong_as_double((long long)dmax[q]);
      const double x = __longlong_as_double((long long)xmax[q]);
      dmax[q] = 0;
      xmax[q] = 0;
      const double p = prevd[q];
      prevd[q] = d;
      bool done_r = d == 0.0;
      if (!done_r && s >= 2) {
        const double rho = d / p;  // NaN: neither test holds
        done_r = rho < 0.5 ? rho / (1.0 - rho) * d <= tol * x : rho >= 0.5;
      }
      all = all && done_r;
    }
    if (all || last) {
      act[g] = 0;
      nsw[g] = s;
    }
  }
  __syncthreads();
  const int64_t per = ((int64_t)G + kDecideThreads - 1) / kDecideThreads;
  const int64_t b = min((int64_t)G, (int64_t)threadIdx.x * per), e = min((int64_t)G, b + per);
  int c = 0;
  long long rows = 0;
  for (int64_t g = b; g < e; ++g)
    if (act[g]) {
      ++c;
      rows += inst_off[g + 1] - inst_off[g];
    }
  int total;
  long long total_rows;
  int o = block_excl_scan<int>(c, sh, total);
  long long ro = block_excl_scan<long long>(rows, sh64, total_rows);
  for (int64_t g = b; g < e; ++g) {
    pre[g] = o;
    if (act[g]) {
      ai[o] = (int)g;
      arow[o] = ro;
      ++o;
      ro += inst_off[g + 1] - inst_off[g];
    }
  }
  if (threadIdx.x == 0) {
    pre[G] = total;
    *nact = total;
    arow[total] = total_rows;
    *sweep = s;
    if (has_cond) cudaGraphSetConditional(cond, (!last && total > 0) ? 1u : 0u);
  }
}

// Every instance active before the first sweep: act = 1, pre[g] = g,
// *nact = G, ai[g] = g, arow = inst_off, no sweep done yet.
__global__ void k_refine_init(int G, uint8_t* __restrict__ act, int* __restrict__ pre, int* __restrict__ nact,
                              int* __restrict__ ai, int64_t* __restrict__ arow, const int64_t* __restrict__ inst_off,
                              int* __restrict__ sweep) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < G) {
    act[g] = 1;
    ai[g] = g;
  }
  if (g <= G) {
    pre[g] = g;
    arow[g] = inst_off[g];
  }
  if (g == 0) {
    *nact = G;
    *sweep = 0;
  }
}

// In-order compaction of the persistent solves' unit lists (blockIdx.y = 0:
// forward, 1: backward) to the units whose instance range [rng.x, rng.y]
// holds an active instance (pre = running count of active instances), in two
// launches: CTA c counts its kCompactThreads units, then writes them at the
// sum of the counts of CTAs 0..c-1; the last CTA stores the length.
constexpr int kCompactThreads = 256;

__device__ __forceinline__ bool unit_active(const int2* rng, int n, int u, const int* pre) {
  return u < n && pre[rng[u].y + 1] > pre[rng[u].x];
}

__global__ void __launch_bounds__(kCompactThreads)
k_compact_count(const int2* __restrict__ rf, int nf, const int2* __restrict__ rb, int nb, const int* __restrict__ pre,
                int* __restrict__ cnt) {
  const int y = blockIdx.y;
  const int u = blockIdx.x * kCompactThreads + threadIdx.x;
  const int c = __syncthreads_count(unit_active(y ? rb : rf, y ? nb : nf, u, pre));
  if (threadIdx.x == 0) cnt[y * gridDim.x + blockIdx.x] = c;
}

__global__ void __launch_bounds__(kCompactThreads)
k_compact_write(const SolveUnit* __restrict__ uf, const int2* __restrict__ rf, int nf, SolveUnit* __restrict__ cf,
                const SolveUnit* __restrict__ ub, const int2* __restrict__ rb, int nb, SolveUnit* __restrict__ cb,
                const int* __restrict__ pre, const int* __restrict__ cnt, int* __restrict__ ucount) {
  __shared__ int s_part[kCompactThreads / 32], s_keep[kCompactThreads / 32];
  const int y = blockIdx.y;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // offset of this CTA: the kept units of the CTAs before it
  int part = 0;
  for (int c = threadIdx.x; c < (int)blockIdx.x; c += kCompactThreads) part += cnt[y * gridDim.x + c];
  part = __reduce_add_sync(kFull, part);
  const int u = blockIdx.x * kCompactThreads + threadIdx.x;
  const bool keep = unit_active(y ? rb : rf, y ? nb : nf, u, pre);
  const unsigned bal = __ballot_sync(kFull, keep);
  if (lane == 0) {
    s_part[w] = part;
    s_keep[w] = __popc(bal);
  }
  __syncthreads();
  int off = 0, before = 0, kept = 0;
  for (int q = 0; q < kCompactThreads / 32; ++q) {
    off += s_part[q];
    if (q < w) before += s_keep[q];
    kept += s_keep[q];
  }
  if (keep) {
    const int o = off + before + __popc(bal & ((1u << lane) - 1u));
    (y ? cb : cf)[o] = (y ? ub : uf)[u];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) ucount[y] = off + kept;
}

__global__ void k_axpy(int64_t n, const double* __restrict__ y, double* __restrict__ x) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) x[q] += y[q];
}

// grad[e] = - sum_k w_k sum_r Lam[pi][k][r] X[pj][k][r] for entry e = (i, j)
__global__ void k_grad_values(SymDev sd, const double* __restrict__ Lam,
                              const double* __restrict__ X, Shifts sh, int R,
                              double* __restrict__ grad) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= sd.N) return;
  const int K = sh.K;
  const int KR = K * R;
  const int64_t pi = sd.iperm[i];
  const int64_t e0 = sd.row_ptr[i], e1 = sd.row_ptr[i + 1];
  for (int64_t eb = e0; eb < e1; eb += 32) {
    // permuted columns of up to 32 entries loaded at once, one per lane
    const int ne = (int)min((int64_t)32, e1 - eb);
    const int64_t pjl = lane < ne ? (int64_t)sd.iperm[sd.col[eb + lane]] : 0;
    for (int e = 0; e < ne; ++e) {
      const int64_t pj = __shfl_sync(0xffffffffu, pjl, e);
      double a = 0.0;
      for (int q = lane; q < KR; q += 32) {
        const int k = q / R;
        a += sh.w[k] * Lam[pi * KR + q] * X[pj * KR + q];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) grad[eb + e] = -a;
    }
  }
}

__global__ void k_fill_nan_failed(SymDev sd, const int32_t* __restrict__ status, int K, int R,
                                  double* __restrict__ x) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= sd.N * R) return;
  const int g = sd.row_inst[q / R];
  int bad = 0;
  for (int k = 0; k < K; ++k) bad |= status[g * K + k];
  if (bad) x[q] = __longlong_as_double(0x7ff8000000000000LL);
}

template <typename T>
void set_solve_attrs() {
  static std::atomic<bool> done_dev[kMaxDevices];
  const int dev = current_device();
  if (done_dev[dev].load(std::memory_order_acquire)) return;
  cudaFuncSetAttribute(k_forward<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSolveSmem);
  cudaFuncSetAttribute(k_forward<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSolveSmem);
  cudaFuncSetAttribute(k_backward<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSolveSmem);
  cudaFuncSetAttribute(k_backward<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSolveSmem);
  cudaFuncSetAttribute(k_forward_blk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kSolveSmem + kBlkExtra * (int)sizeof(T));
  cudaFuncSetAttribute(k_backward_blk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kSolveSmem + kBlkExtra * (int)sizeof(T));
  done_dev[dev].store(true, std::memory_order_release);
}

// RHS chunk: enough CTAs to fill the GPU, within the shared-memory budget.
int pick_rc(int count, int K, int R, int maxF, int esize) {
  const int target = 2 * 152;
  int chunks = (target + count * K - 1) / (count * K);
  chunks = std::max(1, std::min(chunks, R));
  int rc = (R + chunks - 1) / chunks;
  const int cap = std::max(1, kSolveSmem / std::max(1, maxF * esize));
  return std::max(1, std::min(rc, cap));
}

template <typename T>
int forward_impl(bool trans, const SymDev& sd, const LevelPlan& lp, const int32_t* d_all,
                 const void* fronts, const double* rhs, int rhs_mode, void* V, int R, int K,
                 cudaStream_t st) {
  set_solve_attrs<T>();
  int launches = 0;
  for (int g = 0; g < lp.n_sgroups; ++g) {
    const auto& G = lp.sgroups[g];
    if (!G.count) continue;
    if (!trans && G.maxF <= 32) {
      const int64_t segs = (int64_t)G.count * K * ((R + kRW - 1) / kRW);
      const int SEG = G.maxF <= 8 ? 8 : (G.maxF <= 16 ? 16 : 32);
      const unsigned blocks = (unsigned)((segs * SEG + 255) / 256);
      if (SEG == 8)
        k_forward_seg<T, 8><<<blocks, 256, 0, st>>>(sd, d_all + G.off, segs, (const T*)fronts, rhs, rhs_mode, (T*)V, R, K);
      else if (SEG == 16)
        k_forward_seg<T, 16><<<blocks, 256, 0, st>>>(sd, d_all + G.off, segs, (const T*)fronts, rhs, rhs_mode, (T*)V, R, K);
      else
        k_forward_seg<T, 32><<<blocks, 256, 0, st>>>(sd, d_all + G.off, segs, (const T*)fronts, rhs, rhs_mode, (T*)V, R, K);
      ++launches;
      continue;
    }
    const int rc = pick_rc(G.count, K, R, G.maxF, sizeof(T));
    const dim3 grid(G.count, K, (R + rc - 1) / rc);
    const size_t smem = (size_t)rc * G.maxF * sizeof(T) + (trans ? 0 : kBlkExtra * sizeof(T));
    if (trans)
      k_forward<T, true><<<grid, kSolveThreads, smem, st>>>(sd, d_all + G.off, (const T*)fronts, rhs,
                                                            rhs_mode, (T*)V, R, K, rc);
    else
      k_forward_blk<T><<<grid, kSolveThreads, smem, st>>>(sd, d_all + G.off, (const T*)fronts, rhs,
                                                          rhs_mode, (T*)V, R, K, rc);
    ++launches;
  }
  if (cudaGetLastError() != cudaSuccess) return -1;
  return launches;
}

template <typename T>
int backward_impl(bool trans, const SymDev& sd, const LevelPlan& lp, const int32_t* d_all,
                  const void* fronts, const void* V, double* out, double* acc, int R, int K,
                  cudaStream_t st) {
  set_solve_attrs<T>();
  int launches = 0;
  for (int g = 0; g < lp.n_sgroups; ++g) {
    const auto& G = lp.sgroups[g];
    if (!G.count) continue;
    if (!trans && G.maxF <= 32) {
      const int64_t segs = (int64_t)G.count * K * ((R + kRW - 1) / kRW);
      const int SEG = G.maxF <= 8 ? 8 : (G.maxF <= 16 ? 16 : 32);
      const unsigned blocks = (unsigned)((segs * SEG + 255) / 256);
      if (SEG == 8)
        k_backward_seg<T, 8><<<blocks, 256, 0, st>>>(sd, d_all + G.off, segs, (const T*)fronts, (const T*)V, out, acc, R, K);
      else if (SEG == 16)
        k_backward_seg<T, 16><<<blocks, 256, 0, st>>>(sd, d_all + G.off, segs, (const T*)fronts, (const T*)V, out, acc, R, K);
      else
        k_backward_seg<T, 32><<<blocks, 256, 0, st>>>(sd, d_all + G.off, segs, (const T*)fronts, (const T*)V, out, acc, R, K);
      ++launches;
      continue;
    }
    const int rc = pick_rc(G.count, K, R, G.maxF, sizeof(T));
    const dim3 grid(G.count, K, (R + rc - 1) / rc);
    const size_t smem = (size_t)rc * G.maxF * sizeof(T) + (trans ? 0 : kBlkExtra * sizeof(T));
    if (trans)
      k_backward<T, true><<<grid, kSolveThreads, smem, st>>>(sd, d_all + G.off, (const T*)fronts,
                                                             (const T*)V, out, acc, R, K, rc);
    else
      k_backward_blk<T><<<grid, kSolveThreads, smem, st>>>(sd, d_all + G.off, (const T*)fronts,
                                                           (const T*)V, out, acc, R, K, rc);
    ++launches;
  }
  if (cudaGetLastError() != cudaSuccess) return -1;
  return launches;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// SMs of the current device (read once per device)
unsigned sm_count() {
  static std::atomic<int> nsm_dev[kMaxDevices];
  const int dev = current_device();
  int nsm = nsm_dev[dev].load(std::memory_order_acquire);
  if (!nsm) {
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    nsm = std::max(nsm, 1);
    nsm_dev[dev].store(nsm, std::memory_order_release);
  }
  return (unsigned)nsm;
}

}  // namespace

int max_solve_front(int precision) { return kSolveSmem / (precision == PISP_FP32 ? 4 : 8); }

int pick_chunk(int fronts_in_level, int K, int R) {
  const int target = 2 * 152;
  int chunks = (target + fronts_in_level * K - 1) / std::max(1, fronts_in_level * K);
  chunks = std::max(1, std::min(chunks, R));
  return std::max(1, std::min((R + chunks - 1) / chunks, kSolveChunk));
}

int launch_forward_level(int precision, bool trans, const SymDev& sd, const LevelPlan& lp,
                         const int32_t* d_all, const void* fronts, const double* rhs,
                         int rhs_mode, void* V, int32_t R, int32_t K, cudaStream_t st) {
  if (precision == PISP_FP32)
    return forward_impl<float>(trans, sd, lp, d_all, fronts, rhs, rhs_mode, V, R, K, st);
  return forward_impl<double>(trans, sd, lp, d_all, fronts, rhs, rhs_mode, V, R, K, st);
}

int launch_backward_level(int precision, bool trans, const SymDev& sd, const LevelPlan& lp,
                          const int32_t* d_all, const void* fronts, const void* V, double* out,
                          double* acc, int32_t R, int32_t K, cudaStream_t st) {
  if (precision == PISP_FP32)
    return backward_impl<float>(trans, sd, lp, d_all, fronts, V, out, acc, R, K, st);
  return backward_impl<double>(trans, sd, lp, d_all, fronts, V, out, acc, R, K, st);
}

namespace {
template <typename T, int M>
int persistent_launch(bool forward, const SymDev& sd, const SolveUnit* units, int nunits, const int* ucount,
                      const uint8_t* act, int* ticket, int* done, int* err, const int* nch,
                      const int32_t* d_all, const void* fronts, const double* rhs, int rhs_mode, void* V,
                      double* out, double* acc, int R, int K, size_t smem, int64_t polls, cudaStream_t st) {
  static std::atomic<int> nsm_dev[kMaxDevices];
  const int dev = current_device();
  int nsm = nsm_dev[dev].load(std::memory_order_acquire);
  if (!nsm) {
    cudaFuncSetAttribute(k_solve_persistent<T, true, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_solve_persistent<T, false, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    nsm_dev[dev].store(nsm, std::memory_order_release);
  }
  int occ = 0;
  if (forward)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_solve_persistent<T, true, M>, kSolveThreads, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_solve_persistent<T, false, M>, kSolveThreads, smem);
  const int grid = std::max(1, std::min(nunits, std::max(1, occ) * std::max(nsm, 1)));
  if (forward)
    k_solve_persistent<T, true, M><<<grid, kSolveThreads, smem, st>>>(
        sd, units, nunits, ucount, act, ticket, done, err, nch, d_all, (const T*)fronts, rhs, rhs_mode, (T*)V,
        out, acc, R, K, polls);
  else
    k_solve_persistent<T, false, M><<<grid, kSolveThreads, smem, st>>>(
        sd, units, nunits, ucount, act, ticket, done, err, nch, d_all, (const T*)fronts, rhs, rhs_mode, (T*)V,
        out, acc, R, K, polls);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

template <typename T>
int persistent_impl(bool forward, const SymDev& sd, const SolveUnit* units, int nunits, const int* ucount,
                    const uint8_t* act, int* ticket, int* done, int* err, const int* nch, const int32_t* d_all,
                    const void* fronts, const double* rhs, int rhs_mode, void* V, double* out, double* acc, int R,
                    int K, int max_blk_F, int ctas, int64_t polls, cudaStream_t st) {
  if (polls <= 0) polls = kWaitPolls;
  if (nunits == 0) return 0;
  const size_t seg_smem = (size_t)(kSolveThreads / 32) * 32 * kRW * sizeof(T);  // y staging per warp
  const size_t mF = (size_t)std::max(max_blk_F, 1);
  const size_t blk_smem = (size_t)(kBlkExtra + kSolveChunk * mF) * sizeof(T);
  const size_t smem = std::max(seg_smem, blk_smem);
  if (smem > 200 * 1024) return -1;
  if (ctas <= 0) ctas = sizeof(T) == 4 ? 3 : 2;
  if (ctas >= 4)
    return persistent_launch<T, 4>(forward, sd, units, nunits, ucount, act, ticket, done, err, nch, d_all,
                                   fronts, rhs, rhs_mode, V, out, acc, R, K, smem, polls, st);
  if (ctas == 3)
    return persistent_launch<T, 3>(forward, sd, units, nunits, ucount, act, ticket, done, err, nch, d_all,
                                   fronts, rhs, rhs_mode, V, out, acc, R, K, smem, polls, st);
  return persistent_launch<T, 2>(forward, sd, units, nunits, ucount, act, ticket, done, err, nch, d_all,
                                 fronts, rhs, rhs_mode, V, out, acc, R, K, smem, polls, st);
}

}  // namespace

int launch_solve_persistent(int precision, bool forward, const SymDev& sd, const SolveUnit* units,
                            int nunits, const int* ucount, const uint8_t* act, int* ticket, int* done,
                            int* err, const int* nch, const int32_t* d_all, const void* fronts,
                            const double* rhs, int rhs_mode, void* V, double* out, double* acc, int32_t R,
                            int32_t K, int32_t max_blk_F, int32_t ctas, int64_t polls, cudaStream_t st) {
  if (precision == PISP_FP32)
    return persistent_impl<float>(forward, sd, units, nunits, ucount, act, ticket, done, err, nch, d_all,
                                  fronts, rhs, rhs_mode, V, out, acc, R, K, max_blk_F, ctas, polls, st);
  return persistent_impl<double>(forward, sd, units, nunits, ucount, act, ticket, done, err, nch, d_all,
                                 fronts, rhs, rhs_mode, V, out, acc, R, K, max_blk_F, ctas, polls, st);
}

int launch_combine(const SymDev& sd, const double* X, const Shifts& sh, int32_t R, double* x,
                   cudaStream_t st) {
  const int64_t n = sd.N * R;
  if (n == 0) return 0;
  k_combine<<<blocks_for(n, 256), 256, 0, st>>>(sd, X, sh, R, x);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_residual_per_k(const SymDev& sd, const double* vals, const double* D,
                          const Shifts& sh, const double* b, const double* X, int32_t R,
                          double* Rk, const ActiveSet& as, int mode, cudaStream_t st) {
  if (sd.N == 0) return 0;
  unsigned grid = blocks_for(sd.N * 32, 256);
  if (mode == kResActive) grid = std::min<unsigned>(grid, 16u * sm_count());  // rows known on the device only
  k_residual_per_k<<<grid, 256, 0, st>>>(sd, vals, D, sh, b, X, R, Rk, as, mode);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_refine_stats(const SymDev& sd, const ActiveSet& as, double* X, const double* Y, int32_t K, int32_t R,
                        unsigned long long* dmax, unsigned long long* xmax, cudaStream_t st) {
  if (sd.N == 0 || R < 1) return 0;
  const unsigned grid = std::min<unsigned>((unsigned)((sd.N + kStatRows - 1) / kStatRows), 32u * sm_count());
  k_refine_stats<<<grid, kStatThreads, 0, st>>>(sd, as, X, Y, K, R, dmax, xmax);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_refine_decide(int32_t G, int32_t R, double tol, int32_t S, int32_t* sweep,
                         cudaGraphConditionalHandle cond, int has_cond, uint8_t* act, unsigned long long* dmax,
                         unsigned long long* xmax, double* prevd, int32_t* nsw, int32_t* pre, int32_t* nact,
                         int32_t* ai, int64_t* arow, const int64_t* inst_off, cudaStream_t st) {
  if (G < 1) return 0;
  k_refine_decide<<<1, kDecideThreads, 0, st>>>(G, R, tol, S, sweep, cond, has_cond, act, dmax, xmax, prevd, nsw,
                                                pre, nact, ai, arow, inst_off);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_refine_init(int32_t G, uint8_t* act, int32_t* pre, int32_t* nact, int32_t* ai, int64_t* arow,
                       const int64_t* inst_off, int32_t* sweep, cudaStream_t st) {
  if (G < 1) return 0;
  k_refine_init<<<blocks_for((int64_t)G + 1, 256), 256, 0, st>>>(G, act, pre, nact, ai, arow, inst_off, sweep);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int compact_scratch(int32_t nf, int32_t nb) {
  return 2 * (int)((std::max(nf, nb) + kCompactThreads - 1) / kCompactThreads);
}

int launch_compact_units(const SolveUnit* uf, const int32_t* rf, int32_t nf, SolveUnit* cf, const SolveUnit* ub,
                         const int32_t* rb, int32_t nb, SolveUnit* cb, const int32_t* pre, int32_t* cnt,
                         int32_t* ucount, cudaStream_t st) {
  const int gx = compact_scratch(nf, nb) / 2;
  if (gx == 0) return 0;
  const dim3 grid(gx, 2);
  const int2* f2 = reinterpret_cast<const int2*>(rf);
  const int2* b2 = reinterpret_cast<const int2*>(rb);
  k_compact_count<<<grid, kCompactThreads, 0, st>>>(f2, nf, b2, nb, pre, cnt);
  if (cudaGetLastError() != cudaSuccess) return -1;
  k_compact_write<<<grid, kCompactThreads, 0, st>>>(uf, f2, nf, cf, ub, b2, nb, cb, pre, cnt, ucount);
  return cudaGetLastError() == cudaSuccess ? 2 : -1;
}

int launch_residual_T_per_k(const SymDev& sd, const double* vals, const double* D,
                            const Shifts& sh, const double* g, const double* Lam, int32_t R,
                            double* Rk, cudaStream_t st) {
  if (sd.N == 0) return 0;
  k_residual_T_per_k<<<blocks_for(sd.N * 32, 256), 256, 0, st>>>(sd, vals, D, sh, g, Lam, R, Rk);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_residual(const SymDev& sd, const double* vals, const double* b, const double* x,
                    int32_t R, double* r, cudaStream_t st) {
  if (sd.N == 0) return 0;
  k_residual<<<blocks_for(sd.N * 32, 256), 256, 0, st>>>(sd, vals, b, x, R, r);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_axpy(int64_t n, const double* y, double* x, cudaStream_t st) {
  if (n == 0) return 0;
  k_axpy<<<blocks_for(n, 256), 256, 0, st>>>(n, y, x);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_grad_values(const SymDev& sd, const double* Lam, const double* X, const Shifts& sh,
                       int32_t R, double* grad, cudaStream_t st) {
  if (sd.N == 0) return 0;
  k_grad_values<<<blocks_for(sd.N * 32, 256), 256, 0, st>>>(sd, Lam, X, sh, R, grad);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_fill_nan_failed(const SymDev& sd, const int32_t* status, int32_t K, int32_t R,
                           double* x, cudaStream_t st) {
  const int64_t n = sd.N * R;
  if (n == 0) return 0;
  k_fill_nan_failed<<<blocks_for(n, 256), 256, 0, st>>>(sd, status, K, R, x);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace pisp
