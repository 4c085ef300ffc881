// Pivot-free multifrontal LU of all K perturbed matrices (Alg. 1, Eq. xap / xam).
//
// Each supernode s owns a dense front of size F = ns + ms per perturbation k:
//   1. assembly: P (A + t_k D) P^T entries that belong to s, plus the
//      Schur complements (update blocks) of its children (extend-add);
//   2. ns steps of right-looking elimination WITHOUT pivoting: the pivot
//      order is the static one fixed by the symbolic phase (Sec. II-C).
// Fronts at the same level of the assembly forest are independent; one
// launch covers all of them, all K perturbations (grid.y / grid.z) and all
// instances of a batch.  Small fronts are factored in shared memory, one CTA
// per (front, k); large fronts use a blocked right-looking scheme in global
// memory (panel factorisation, row-block triangular solve, tiled update).
//
// Storage: front s of perturbation k occupies F*F contiguous elements
// (column-major) at K*front_off[s] + k*F*F.  After factorisation it holds
// L11\U11, L21, U12 and the Schur complement F22 that the parent reads.
#include <atomic>
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <type_traits>
#include <vector>

#include "pisp_internal.h"

namespace pisp {
namespace {

constexpr int kSmemCap = 225 * 1024;  // dynamic shared memory budget per CTA
constexpr int kStatusZero = 1;        // status bits: exact zero pivot
constexpr int kStatusNonfinite = 2;   //              Inf / NaN pivot

template <typename T>
__device__ __forceinline__ void check_pivot(T piv, const SymDev& sd, int s, int k, int K,
                                            int col, int32_t* status, int32_t* badcol) {
  const double p = (double)piv;
  int code = 0;
  if (!isfinite(p)) code = kStatusNonfinite;
  else if (p == 0.0) code = kStatusZero;
  if (code) {
    const int g = sd.inst[s];
    atomicOr(&status[g * K + k], code);
    atomicMin(&badcol[g * K + k], col);
  }
}

// Pivot-free LU of a panel in shared memory: rows p0..F-1 of nb <= 32
// columns, P[i + c*ld] = front(i, p0 + c).  Warps take rows; lane j of a warp
// updates column j, so a row costs one instruction group.  The warp that
// finishes row p0+c+1 during step c also copies it to the other half of a
// double-buffered pivot row, so each pivot costs one block barrier.  An odd
// ld keeps the lanes' column accesses on distinct banks.
template <typename T>
__device__ __forceinline__ void panel_factor_rows(T* P, int ld, int F, int p0, int nb,
                                                  T (*prow)[32], const SymDev& sd, int s, int k,
                                                  int K, int colbase, int32_t* status,
                                                  int32_t* badcol) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (wid == 0 && lane < nb) prow[0][lane] = P[p0 + lane * ld];
  for (int c = 0; c < nb; ++c) {
    __syncthreads();
    const T* pr = prow[c & 1];
    const int pc = p0 + c;
    const T piv = pr[c];
    if (threadIdx.x == 0) check_pivot(piv, sd, s, k, K, colbase + c, status, badcol);
    const T rp = T(1) / piv;
    const T pj = (lane > c && lane < nb) ? pr[lane] : T(0);
    for (int i = pc + 1 + wid; i < F; i += nw) {
      const T l = P[i + c * ld] * rp;
      __syncwarp();
      if (lane == c) P[i + c * ld] = l;
      else if (lane > c && lane < nb) P[i + lane * ld] -= l * pj;
      if (i == pc + 1 && c + 1 < nb) {
        __syncwarp();
        if (lane < nb) prow[(c + 1) & 1][lane] = P[i + lane * ld];
      }
    }
  }
  __syncthreads();
}

// Pivot-free elimination of a panel in shared memory: rows 0..Mr-1, nb <= 32
// columns, P[i + c*ld] (ld odd).  Per pivot: scale the column by one
// reciprocal, then lane j of each warp updates column j of the warp's rows;
// the loops carry no integer division.
template <typename T>
__device__ __forceinline__ void panel_eliminate(T* P, int ld, int Mr, int nb, const SymDev& sd,
                                                int s, int k, int K, int colbase, int32_t* status,
                                                int32_t* badcol) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int c = 0; c < nb; ++c) {
    const T piv = P[c + c * ld];
    if (tid == 0) check_pivot(piv, sd, s, k, K, colbase + c, status, badcol);
    const T rp = T(1) / piv;
    for (int i = c + 1 + tid; i < Mr; i += nt) P[i + c * ld] *= rp;
    __syncthreads();
    if (lane > c && lane < nb) {
      const T u = P[c + lane * ld];
      T* col = P + lane * ld;
      const T* lc = P + c * ld;
      for (int i = c + 1 + wid; i < Mr; i += nw) col[i] -= lc[i] * u;
    }
    __syncthreads();
  }
}

// Children's update columns added into the destination columns [d0, d0 + w)
// and rows [R0, R1) of front s, stored at dst[(row - R0) + (col - d0) * ld].  Each destination column
// belongs to one warp (col - d0 = warp, warp + warps, ...), which walks the
// column's inverse extend-add list in child order: every element receives its
// contributions in child order, with no barrier between children, and a
// group of 8 x 32 child rows is loaded before any of them is added.
template <typename T>
__device__ __forceinline__ void extend_add_columns(const SymDev& sd, int s, int k, int K,
                                                   const T* __restrict__ fronts, T* dst, int ld,
                                                   int d0, int w, int R0, int R1, int wid, int nw) {
  const int lane = threadIdx.x & 31;
  const int64_t vo = sd.vec_off[s];
  for (int dc = wid; dc < w; dc += nw) {
    const int64_t e0 = sd.inv_off[vo + d0 + dc], e1 = sd.inv_off[vo + d0 + dc + 1];
    T* dcol = dst + (int64_t)dc * ld;
    for (int64_t eb = e0; eb < e1; eb += 32) {
      const int ne = (int)min((int64_t)32, e1 - eb);
      int ca = 0, cF = 1, ccol = 0;
      int64_t cfo = 0, cro = 0;
      if (lane < ne) {
        const int ch = sd.inv_child[eb + lane];
        ca = sd.inv_a[eb + lane];
        cF = sd.inv_cF[eb + lane];
        ccol = sd.inv_col[eb + lane];
        cfo = sd.front_off[ch];
        cro = sd.row_off[ch];
      }
      for (int e = 0; e < ne; ++e) {
        const int eF = __shfl_sync(0xffffffffu, cF, e);
        const int ecol = __shfl_sync(0xffffffffu, ccol, e);
        const int cns = ecol - __shfl_sync(0xffffffffu, ca, e);
        const int cms = eF - cns;
        const int32_t* em = sd.emap + __shfl_sync(0xffffffffu, cro, e);
        const T* scol = fronts + (int64_t)K * __shfl_sync(0xffffffffu, cfo, e) + (int64_t)k * eF * eF +
                        (int64_t)ecol * eF + cns;
        for (int a0 = 0; a0 < cms; a0 += 256) {
          int r[8];
          T v[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int a = a0 + lane + 32 * t;
            r[t] = a < cms ? em[a] : -1;
            v[t] = a < cms ? scol[a] : T(0);
          }
#pragma unroll
          for (int t = 0; t < 8; ++t)
            if (r[t] >= R0 && r[t] < R1) dcol[r[t] - R0] += v[t];
        }
        __syncwarp();
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Small fronts: whole front in shared memory, one CTA per (front, k).
// ---------------------------------------------------------------------------
// One (front s, perturbation k) in the shared-memory buffer f (F*F
// elements): assembly (original entries, t_k D, children's Schur complements
// in child order per element), ns steps of pivot-free elimination, write to
// the front storage.  Any number of threads that is a multiple of 32.
template <typename T>
__device__ __forceinline__ void front_cta(const SymDev& sd, int s, int k, const double* __restrict__ vals,
                                          const double* __restrict__ D, const Shifts& sh,
                                          T* __restrict__ fronts, int32_t* status, int32_t* badcol, T* f) {
  const int K = sh.K;
  const int ns = sd.ns[s], ms = sd.ms[s], F = ns + ms;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int FF = F * F;
  for (int q = tid; q < FF; q += nt) f[q] = T(0);
  __syncthreads();
  // 1a. entries of A owned by this front (duplicates add up)
  const int64_t a0 = sd.amap_off[s], a1 = sd.amap_off[s + 1];
  for (int64_t q = a0 + tid; q < a1; q += nt) atomicAdd(&f[sd.amap_dst[q]], (T)vals[sd.amap_src[q]]);
  // 1b. the perturbation t_k D on the pivot diagonal
  const double tk = sh.t[k];
  const int c0 = sd.c0[s];
  for (int c = tid; c < ns; c += nt) atomicAdd(&f[c * (F + 1)], (T)(tk * D[sd.perm[c0 + c]]));
  __syncthreads();
  // 1c. extend-add of the children's Schur complements, child by child (each
  // element receives its contributions in child order): the threads take the
  // entries of one child's update block, which land on distinct elements
  for (int ci = sd.child_off[s]; ci < sd.child_off[s + 1]; ++ci) {
    const int c = sd.child[ci];
    const int cns = sd.ns[c], cms = sd.ms[c], cF = cns + cms;
    const T* cf = fronts + (int64_t)K * sd.front_off[c] + (int64_t)k * cF * cF;
    const int32_t* em = sd.emap + sd.row_off[c];
    const int n2 = cms * cms;
    for (int q = tid; q < n2; q += nt) {
      const int a = q % cms, b = q / cms;  // child update row a, column b
      f[em[a] + em[b] * F] += cf[(cns + a) + (int64_t)(cns + b) * cF];
    }
    __syncthreads();
  }
  // 2. ns steps of pivot-free elimination
  for (int p = 0; p < ns; ++p) {
    const T piv = f[p * (F + 1)];
    if (tid == 0) check_pivot(piv, sd, s, k, K, c0 + p, status, badcol);
    const int m = F - p - 1;
    const T rp = T(1) / piv;
    for (int i = tid; i < m; i += nt) f[(p + 1 + i) + p * F] *= rp;
    __syncthreads();
    {
      // lanes run down a column (consecutive i), warps take columns
      const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
      const T* lc = f + p * F;
      for (int j = p + 1 + wid; j < F; j += nw) {
        const T u = f[p + j * F];
        T* col = f + j * F;
        for (int i = p + 1 + lane; i < F; i += 32) col[i] -= lc[i] * u;
      }
    }
    __syncthreads();
  }
  T* out = fronts + (int64_t)K * sd.front_off[s] + (int64_t)k * FF;
  for (int q = tid; q < FF; q += nt) out[q] = f[q];
}

template <typename T>
__global__ void k_front_small(SymDev sd, const int32_t* __restrict__ list,
                              const double* __restrict__ vals, const double* __restrict__ D,
                              Shifts sh, T* __restrict__ fronts, int32_t* status,
                              int32_t* badcol) {
  extern __shared__ __align__(16) unsigned char smraw[];
  front_cta<T>(sd, list[blockIdx.x], blockIdx.y, vals, D, sh, fronts, status, badcol,
               reinterpret_cast<T*>(smraw));
}

// One (front s, perturbation k) with F <= 32 by one warp, in its F x F
// shared-memory area f (column-major): the same assembly and the same
// per-element sequence of operations as front_cta, with the warp's lanes as
// rows and no block barrier.
template <typename T>
__device__ __forceinline__ void front_warp(const SymDev& sd, int s, int k, const double* __restrict__ vals,
                                           const double* __restrict__ D, const Shifts& sh,
                                           T* __restrict__ fronts, int32_t* status, int32_t* badcol, T* f) {
  const int K = sh.K;
  const int lane = threadIdx.x & 31;
  const int ns = sd.ns[s], ms = sd.ms[s], F = ns + ms;
  const int FF = F * F;
  for (int q = lane; q < FF; q += 32) f[q] = T(0);
  __syncwarp();
  const int64_t a0 = sd.amap_off[s], a1 = sd.amap_off[s + 1];
  for (int64_t q = a0 + lane; q < a1; q += 32) atomicAdd(&f[sd.amap_dst[q]], (T)vals[sd.amap_src[q]]);
  const double tk = sh.t[k];
  const int c0 = sd.c0[s];
  for (int c = lane; c < ns; c += 32) atomicAdd(&f[c * (F + 1)], (T)(tk * D[sd.perm[c0 + c]]));
  __syncwarp();
  // extend-add, child by child (each element receives its children's
  // contributions in child order, as in the column-owner form): the lanes
  // take the entries of the child's cms x cms update block, which land on
  // distinct elements of this front
  for (int ci = sd.child_off[s]; ci < sd.child_off[s + 1]; ++ci) {
    const int c = sd.child[ci];
    const int cns = sd.ns[c], cms = sd.ms[c], cF = cns + cms;
    const T* cf = fronts + (int64_t)K * sd.front_off[c] + (int64_t)k * cF * cF;
    const int32_t* em = sd.emap + sd.row_off[c];
    const int n2 = cms * cms;
    for (int q = lane; q < n2; q += 32) {
      const int a = q % cms, b = q / cms;  // child update row a, column b
      f[em[a] + em[b] * F] += cf[(cns + a) + (int64_t)(cns + b) * cF];
    }
    __syncwarp();
  }
  for (int p = 0; p < ns; ++p) {
    const T piv = f[p * (F + 1)];
    if (lane == 0) check_pivot(piv, sd, s, k, K, c0 + p, status, badcol);
    const T rp = T(1) / piv;
    const int i = p + 1 + lane;  // this lane's row (F <= 32: one row per lane)
    T l = T(0);
    if (i < F) {
      l = f[i + p * F] * rp;
      f[i + p * F] = l;
    }
    for (int j = p + 1; j < F; ++j) {
      const T u = f[p + j * F];
      if (i < F) f[i + j * F] -= l * u;
    }
    __syncwarp();
  }
  T* out = fronts + (int64_t)K * sd.front_off[s] + (int64_t)k * FF;
  for (int q = lane; q < FF; q += 32) out[q] = f[q];
}

// ---------------------------------------------------------------------------
// Big fronts, step 1: assembly, one CTA per (column tile, front, k).  Each
// CTA owns TW columns, so children are added in a fixed order: the result is
// deterministic.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t lower_bound_col(const int32_t* dst, int64_t lo, int64_t hi,
                                                   int F, int j) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (dst[mid] / F < j) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int lower_bound_i(const int32_t* a, int n, int x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

template <typename T>
__global__ void __launch_bounds__(256) k_assemble_big(SymDev sd, const int32_t* __restrict__ list,
                                                      const double* __restrict__ vals,
                                                      const double* __restrict__ D, Shifts sh,
                                                      T* __restrict__ fronts, int TW) {
  const int s = list[blockIdx.y];
  const int k = blockIdx.z;
  const int K = sh.K;
  const int ns = sd.ns[s], ms = sd.ms[s], F = ns + ms;
  const int j0 = blockIdx.x * TW;
  if (j0 >= F) return;
  const int j1 = min(F, j0 + TW);
  const int tid = threadIdx.x, nt = blockDim.x;
  T* f = fronts + (int64_t)K * sd.front_off[s] + (int64_t)k * F * F;
  const int64_t nz = (int64_t)F * (j1 - j0);
  for (int64_t q = tid; q < nz; q += nt) f[(int64_t)j0 * F + q] = T(0);
  __syncthreads();
  const int64_t a0 = sd.amap_off[s], a1 = sd.amap_off[s + 1];
  const int64_t lo = lower_bound_col(sd.amap_dst, a0, a1, F, j0);
  const int64_t hi = lower_bound_col(sd.amap_dst, lo, a1, F, j1);
  for (int64_t q = lo + tid; q < hi; q += nt) atomicAdd(&f[sd.amap_dst[q]], (T)vals[sd.amap_src[q]]);
  const double tk = sh.t[k];
  const int c0 = sd.c0[s];
  for (int c = j0 + tid; c < min(j1, ns); c += nt)
    atomicAdd(&f[(int64_t)c * (F + 1)], (T)(tk * D[sd.perm[c0 + c]]));
  __syncthreads();
  for (int ci = sd.child_off[s]; ci < sd.child_off[s + 1]; ++ci) {
    const int c = sd.child[ci];
    const int cns = sd.ns[c], cms = sd.ms[c], cF = cns + cms;
    const int32_t* em = sd.emap + sd.row_off[c];
    const int b0 = lower_bound_i(em, cms, j0);
    const int b1 = lower_bound_i(em, cms, j1);
    if (b1 > b0) {
      const T* cf = fronts + (int64_t)K * sd.front_off[c] + (int64_t)k * cF * cF;
      const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
      for (int b = b0 + wid; b < b1; b += nw) {
        T* dcol = f + (int64_t)em[b] * F;
        const T* scol = cf + (int64_t)(cns + b) * cF + cns;
        for (int a = lane; a < cms; a += 32) dcol[em[a]] += scol[a];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Big fronts, step 2: factor the panel of columns [p0, p0+NB) (rows p0..F-1)
// in shared memory, then solve the row block U[p0:p0+NB, p0+NB:F] with the
// panel's unit lower triangle.  One CTA per (front, k).
// ---------------------------------------------------------------------------
template <typename T, int NB>
__global__ void __launch_bounds__(512) k_panel_big(SymDev sd, const int32_t* __restrict__ list,
                                                   int K, T* __restrict__ fronts, int p0,
                                                   int32_t* status, int32_t* badcol) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* P = reinterpret_cast<T*>(smraw);
  const int s = list[blockIdx.x];
  const int k = blockIdx.y;
  const int ns = sd.ns[s], F = ns + sd.ms[s];
  if (p0 >= ns) return;
  const int nbe = min(NB, ns - p0);
  const int Mr = F - p0;
  const int ld = Mr | 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  T* f = fronts + (int64_t)K * sd.front_off[s] + (int64_t)k * F * F;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int c = wid; c < nbe; c += nw)
    for (int i = lane; i < Mr; i += 32) P[i + c * ld] = f[(p0 + i) + (int64_t)(p0 + c) * F];
  __syncthreads();
  panel_eliminate<T>(P, ld, Mr, nbe, sd, s, k, K, sd.c0[s] + p0, status, badcol);
  for (int c = wid; c < nbe; c += nw)
    for (int i = lane; i < Mr; i += 32) f[(p0 + i) + (int64_t)(p0 + c) * F] = P[i + c * ld];
  // row block of U: columns j >= p0 + nbe
  for (int j = p0 + nbe + tid; j < F; j += nt) {
    T* col = f + (int64_t)j * F + p0;
    T u[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) u[q] = (q < nbe) ? col[q] : T(0);
#pragma unroll
    for (int q = 1; q < NB; ++q) {
      T a = u[q];
#pragma unroll
      for (int r = 0; r < NB - 1; ++r)
        if (r < q) a -= P[q + r * ld] * u[r];
      u[q] = a;
    }
#pragma unroll
    for (int q = 0; q < NB; ++q)
      if (q < nbe) col[q] = u[q];
  }
}

// ---------------------------------------------------------------------------
// Big fronts, step 3: trailing update C -= L_panel * U_panel on 64x64 tiles.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_update_big(SymDev sd, const int32_t* __restrict__ list,
                                                    int K, T* __restrict__ fronts, int p0,
                                                    int nb) {
  const int s = list[blockIdx.y];
  const int k = blockIdx.z;
  const int ns = sd.ns[s], F = ns + sd.ms[s];
  if (p0 >= ns) return;
  const int nbe = min(nb, ns - p0);
  const int t0 = p0 + nbe;
  const int m = F - t0;
  if (m <= 0) return;
  const int tpd = (m + 63) / 64;
  if ((int)blockIdx.x >= tpd * tpd) return;
  const int i0 = t0 + (blockIdx.x % tpd) * 64;
  const int j0 = t0 + (blockIdx.x / tpd) * 64;
  T* f = fronts + (int64_t)K * sd.front_off[s] + (int64_t)k * F * F;
  __shared__ T As[32][64];
  __shared__ T Bs[32][65];
  const int tid = threadIdx.x;
  for (int e = tid; e < 64 * 32; e += 256) {
    const int r = e % 64, q = e / 64;
    As[q][r] = (q < nbe && i0 + r < F) ? f[(i0 + r) + (int64_t)(p0 + q) * F] : T(0);
  }
  for (int e = tid; e < 64 * 32; e += 256) {
    const int q = e % 32, c = e / 32;
    Bs[q][c] = (q < nbe && j0 + c < F) ? f[(p0 + q) + (int64_t)(j0 + c) * F] : T(0);
  }
  __syncthreads();
  const int tx = tid % 16, ty = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int q = 0; q < nbe; ++q) {
    T a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = As[q][tx + 16 * i];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = Bs[q][ty + 16 * j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = i0 + tx + 16 * i, c = j0 + ty + 16 * j;
      if (r < F && c < F) f[r + (int64_t)c * F] -= acc[i][j];
    }
}

// ---------------------------------------------------------------------------
// Mid-size fronts: one thread-block cluster of C CTAs per (front, k).  The
// front's columns are dealt out to the CTAs in widths cw (a multiple of 32)
// and live in their shared memory for the whole factorisation.  For each
// panel of 32 pivots the owning CTA factors it locally, one cluster barrier
// publishes it, and every CTA copies the panel over distributed shared
// memory, solves its part of the U row block and applies a register-tiled
// update to its columns.  Only the owner's panel columns are ever read
// remotely and they are not written after being factored, so one barrier per
// panel suffices; a final barrier keeps every CTA resident until the last
// remote read is done.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int cluster_cw(int F, int C) {
  return (((F + C - 1) / C) + 31) / 32 * 32;
}

template <typename T>
__host__ __device__ __forceinline__ size_t cluster_smem(int F, int C) {
  const size_t cw = (size_t)cluster_cw(F, C);
  return ((size_t)F * cw + (C > 1 ? (size_t)F * 32 : 0) + 32 * 33) * sizeof(T);
}

template <typename T>
__global__ void __launch_bounds__(256) k_front_cluster(SymDev sd, const int32_t* __restrict__ list,
                                                       int C, const double* __restrict__ vals,
                                                       const double* __restrict__ D, Shifts sh,
                                                       T* __restrict__ fronts, int32_t* status,
                                                       int32_t* badcol) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smraw[];
  const int rank = (int)cl.block_rank();
  const int s = list[blockIdx.x / C];
  const int k = blockIdx.y;
  const int K = sh.K;
  const int ns = sd.ns[s], ms = sd.ms[s], F = ns + ms;
  const int cw = cluster_cw(F, C);
  const int j0 = min(F, rank * cw), j1 = min(F, j0 + cw);
  const int nc = j1 - j0;
  T* M = reinterpret_cast<T*>(smraw);                  // my columns, F x cw, ld F
  T* Lp = M + (size_t)F * cw;                           // copy of a remote panel
  T* L11 = Lp + (C > 1 ? (size_t)F * 32 : 0);           // 32 x 33 unit-lower block
  __shared__ T prow[2][32];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int c0 = sd.c0[s];
  // 1. assembly of my columns
  for (int q = tid; q < F * nc; q += nt) M[q] = T(0);
  __syncthreads();
  if (nc > 0) {
    const int64_t a0 = sd.amap_off[s], a1 = sd.amap_off[s + 1];
    const int64_t lo = lower_bound_col(sd.amap_dst, a0, a1, F, j0);
    const int64_t hi = lower_bound_col(sd.amap_dst, lo, a1, F, j1);
    for (int64_t q = lo + tid; q < hi; q += nt)
      atomicAdd(&M[sd.amap_dst[q] - j0 * F], (T)vals[sd.amap_src[q]]);
    const double tk = sh.t[k];
    for (int c = j0 + tid; c < min(j1, ns); c += nt)
      atomicAdd(&M[c + (c - j0) * F], (T)(tk * D[sd.perm[c0 + c]]));
  }
  __syncthreads();
  for (int ci = sd.child_off[s]; ci < sd.child_off[s + 1]; ++ci) {
    const int c = sd.child[ci];
    const int cns = sd.ns[c], cms = sd.ms[c], cF = cns + cms;
    const int32_t* em = sd.emap + sd.row_off[c];
    const int b0 = lower_bound_i(em, cms, j0);
    const int b1 = lower_bound_i(em, cms, j1);
    if (b1 > b0) {
      const T* cf = fronts + (int64_t)K * sd.front_off[c] + (int64_t)k * cF * cF;
      const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
      for (int b = b0 + wid; b < b1; b += nw) {
        T* dcol = M + (size_t)(em[b] - j0) * F;
        const T* scol = cf + (int64_t)(cns + b) * cF + cns;
        for (int a = lane; a < cms; a += 32) dcol[em[a]] += scol[a];
      }
    }
    __syncthreads();
  }
  // 2. blocked right-looking elimination, 32 pivots per panel
  const int tx = tid & 15, ty = tid >> 4;
  for (int p0 = 0; p0 < ns; p0 += 32) {
    const int nb = min(32, ns - p0);
    const int owner = p0 / cw;
    if (rank == owner) panel_factor_rows<T>(M + (size_t)(p0 - j0) * F, F, F, p0, nb, prow, sd, s, k,
                                            K, c0 + p0, status, badcol);
    cl.sync();
    const int jlo = max(j0, p0 + nb);
    if (jlo < j1) {
      const T* Ls;                                       // Ls[i + c*F] = front(i, p0 + c)
      if (rank == owner) {
        Ls = M + (size_t)(p0 - j0) * F;
      } else {
        const T* R = cl.map_shared_rank(M, owner) + (size_t)(p0 - owner * cw) * F;
        const int hr = F - p0;
        for (int e = tid; e < hr * nb; e += nt) {
          const int i = p0 + e % hr, c = e / hr;
          Lp[i + c * F] = R[i + c * F];
        }
        Ls = Lp;
      }
      __syncthreads();
      for (int e = tid; e < 32 * 32; e += nt) {
        const int r = e >> 5, c = e & 31;
        L11[r * 33 + c] = (r < nb && c < r) ? Ls[(p0 + r) + c * F] : T(0);
      }
      __syncthreads();
      // (a) U row block of my columns: unit-lower triangular solve, one column per thread
      for (int j = jlo + tid; j < j1; j += nt) {
        T* col = M + (size_t)(j - j0) * F + p0;
        T u[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) u[r] = (r < nb) ? col[r] : T(0);
#pragma unroll
        for (int r = 1; r < 32; ++r) {
          T a = u[r];
#pragma unroll
          for (int c = 0; c < 31; ++c)
            if (c < r) a -= L11[r * 33 + c] * u[c];
          u[r] = a;
        }
#pragma unroll
        for (int r = 0; r < 32; ++r)
          if (r < nb) col[r] = u[r];
      }
      __syncthreads();
      // (b) trailing update of my columns, 64 x 64 tiles, 4 x 4 per thread
      const int r0 = p0 + nb;
      for (int rb = r0; rb < F; rb += 64) {
        for (int cb = jlo; cb < j1; cb += 64) {
          T acc[4][4];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
          for (int c = 0; c < nb; ++c) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
              const int i = rb + tx + 16 * a;
              av[a] = (i < F) ? Ls[i + c * F] : T(0);
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const int j = cb + ty + 16 * b;
              bv[b] = (j < j1) ? M[(p0 + c) + (size_t)(j - j0) * F] : T(0);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
          }
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const int i = rb + tx + 16 * a, j = cb + ty + 16 * b;
              if (i < F && j < j1) M[i + (size_t)(j - j0) * F] -= acc[a][b];
            }
        }
      }
      __syncthreads();
    }
  }
  cl.sync();
  T* out = fronts + (int64_t)K * sd.front_off[s] + (int64_t)k * F * F + (int64_t)j0 * F;
  for (int e = tid; e < F * nc; e += nt) out[e] = M[e];
}

// ---------------------------------------------------------------------------
// Big fronts as a tile DAG, one persistent launch per level.  Column blocks
// are 32 wide.  Tasks: ASM(j) assembles block j; PANEL(p) factors the panel
// of pivots [32p, 32p+32) in shared memory; UPDATE(p, j) applies panel p to
// block j (unit-lower solve of its 32 U rows, then the trailing update of all
// rows below).  PANEL(p+1) waits only for UPDATE(p, p+1), so the next panel
// starts while the rest of step p is still updating (look-ahead).  CTAs take
// tasks in ticket order and wait only for tasks with smaller tickets; every
// wait is bounded and sets *err when it gives up.
// ---------------------------------------------------------------------------
constexpr int64_t kDagWaitPolls = 1 << 22;

__device__ __forceinline__ int dag_ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void dag_st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void dag_wait(const int* f, int need, int* err) {
  if (dag_ld_acquire(f) >= need) return;
  for (int64_t i = 0; i < kDagWaitPolls; ++i) {
    __nanosleep(64);
    if (dag_ld_acquire(f) >= need) return;
  }
  atomicExch(err, 1);
}

template <typename T>
__global__ void __launch_bounds__(256) k_big_dag(SymDev sd, const int32_t* __restrict__ big,
                                                 const DagTask* __restrict__ tasks, int ntasks,
                                                 int* ticket, int* flags, int* err,
                                                 const double* __restrict__ vals,
                                                 const double* __restrict__ D, Shifts sh,
                                                 T* __restrict__ fronts, int32_t* status,
                                                 int32_t* badcol) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_t;
  const int K = sh.K;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5;
  for (;;) {
    if (tid == 0) s_t = atomicAdd(ticket, 1);
    __syncthreads();
    const int u = s_t;
    __syncthreads();
    if (u >= ntasks) return;
    const DagTask t = tasks[u];
    const int s = big[t.b];
    const int k = t.k;
    const int ns = sd.ns[s], F = ns + sd.ms[s];
    const int J = (F + 31) / 32;
    int* stepdone = flags + t.flags;
    int* paneldone = stepdone + J;
    T* f = fronts + (int64_t)K * sd.front_off[s] + (int64_t)k * F * F;
    int publish_at = -1, publish_val = 0;
    if (t.kind == kDagAsm) {
      const int j0 = 32 * t.j, j1 = min(F, j0 + 32);
      const int64_t nz = (int64_t)F * (j1 - j0);
      for (int64_t q = tid; q < nz; q += nt) f[(int64_t)j0 * F + q] = T(0);
      __syncthreads();
      const int64_t a0 = sd.amap_off[s], a1 = sd.amap_off[s + 1];
      const int64_t lo = lower_bound_col(sd.amap_dst, a0, a1, F, j0);
      const int64_t hi = lower_bound_col(sd.amap_dst, lo, a1, F, j1);
      for (int64_t q = lo + tid; q < hi; q += nt) atomicAdd(&f[sd.amap_dst[q]], (T)vals[sd.amap_src[q]]);
      const double tk = sh.t[k];
      const int c0 = sd.c0[s];
      for (int c = j0 + tid; c < min(j1, ns); c += nt)
        atomicAdd(&f[(int64_t)c * (F + 1)], (T)(tk * D[sd.perm[c0 + c]]));
      __syncthreads();
      for (int ci = sd.child_off[s]; ci < sd.child_off[s + 1]; ++ci) {
        const int c = sd.child[ci];
        const int cns = sd.ns[c], cms = sd.ms[c], cF = cns + cms;
        const int32_t* em = sd.emap + sd.row_off[c];
        const int b0 = lower_bound_i(em, cms, j0);
        const int b1 = lower_bound_i(em, cms, j1);
        if (b1 > b0) {
          const T* cf = fronts + (int64_t)K * sd.front_off[c] + (int64_t)k * cF * cF;
          for (int b = b0 + wid; b < b1; b += (nt >> 5)) {
            T* dcol = f + (int64_t)em[b] * F;
            const T* scol = cf + (int64_t)(cns + b) * cF + cns;
            for (int a = lane; a < cms; a += 32) dcol[em[a]] += scol[a];
          }
        }
        __syncthreads();
      }
      publish_at = t.j;
      publish_val = 1;
    } else if (t.kind == kDagPanel) {
      if (tid == 0) dag_wait(&stepdone[t.p], t.p + 1, err);
      __syncthreads();
      T* P = reinterpret_cast<T*>(smraw);
      const int r0 = 32 * t.p;
      const int nb = min(32, ns - r0);
      const int Mr = F - r0;
      const int ld = Mr | 1;
      for (int c = wid; c < nb; c += (nt >> 5))
        for (int i = lane; i < Mr; i += 32) P[i + c * ld] = __ldcg(f + (r0 + i) + (int64_t)(r0 + c) * F);
      __syncthreads();
      panel_eliminate<T>(P, ld, Mr, nb, sd, s, k, K, sd.c0[s] + r0, status, badcol);
      for (int c = wid; c < nb; c += (nt >> 5))
        for (int i = lane; i < Mr; i += 32) f[(r0 + i) + (int64_t)(r0 + c) * F] = P[i + c * ld];
      publish_at = J + t.p;
      publish_val = 1;
    } else {
      const int p = t.p, j = t.j;
      const int r0 = 32 * p;
      const int nb = min(32, ns - r0);
      const int jc0 = max(32 * j, r0 + nb), jc1 = min(32 * j + 32, F);
      const int w = jc1 - jc0;
      if (tid == 0) {
        dag_wait(&paneldone[p], 1, err);
        dag_wait(&stepdone[j], p + 1, err);
      }
      __syncthreads();
      T* Ls = reinterpret_cast<T*>(smraw);       // 32 x 33: unit-lower L11 of panel p
      T* Us = Ls + 32 * 33;                       // 32 x 33: U rows of this block
      for (int e = tid; e < 32 * 32; e += nt) {
        const int r = e & 31, c = e >> 5;
        Ls[r * 33 + c] = (r < nb && c < r) ? __ldcg(f + (r0 + r) + (int64_t)(r0 + c) * F) : T(0);
        Us[r * 33 + c] = (r < nb && c < w) ? __ldcg(f + (r0 + r) + (int64_t)(jc0 + c) * F) : T(0);
      }
      __syncthreads();
      if (wid == 0) {
        T uu[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) uu[r] = Us[r * 33 + lane];
#pragma unroll
        for (int r = 1; r < 32; ++r) {
          T a = uu[r];
#pragma unroll
          for (int c = 0; c < 31; ++c)
            if (c < r) a -= Ls[r * 33 + c] * uu[c];
          uu[r] = a;
        }
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          Us[r * 33 + lane] = uu[r];
          if (r < nb && lane < w) f[(r0 + r) + (int64_t)(jc0 + lane) * F] = uu[r];
        }
      }
      __syncthreads();
      for (int i = r0 + nb + tid; i < F; i += nt) {
        T l[32], cv[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) l[c] = (c < nb) ? __ldcg(f + i + (int64_t)(r0 + c) * F) : T(0);
#pragma unroll
        for (int col = 0; col < 32; ++col) cv[col] = (col < w) ? __ldcg(f + i + (int64_t)(jc0 + col) * F) : T(0);
#pragma unroll
        for (int col = 0; col < 32; ++col) {
          T a = T(0);
#pragma unroll
          for (int c = 0; c < 32; ++c) a += l[c] * Us[c * 33 + col];
          cv[col] -= a;
        }
#pragma unroll
        for (int col = 0; col < 32; ++col)
          if (col < w) f[i + (int64_t)(jc0 + col) * F] = cv[col];
      }
      publish_at = j;
      publish_val = p + 2;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0 && publish_at >= 0) dag_st_release(&stepdone[publish_at], publish_val);
  }
}

template <typename T>
int big_dag_impl(const SymDev& sd, const LevelPlan& lp, const int32_t* d_big, const DagTask* tasks,
                 int* ticket, int* flags, int* err, const double* vals, const double* D,
                 const Shifts& sh, void* fronts, int32_t* status, int32_t* badcol, cudaStream_t st) {
  if (lp.dag_tasks == 0) return 0;
  static std::atomic<int> nsm_dev[kMaxDevices];
  const int dev = current_device();
  int nsm = nsm_dev[dev].load(std::memory_order_acquire);
  if (!nsm) {
    cudaFuncSetAttribute(k_big_dag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    nsm_dev[dev].store(nsm, std::memory_order_release);
  }
  const size_t smem = std::max((size_t)(lp.big_maxF + 1) * 32, (size_t)2 * 32 * 33) * sizeof(T);
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_big_dag<T>, 256, smem);
  const int grid = std::max(1, std::min(lp.dag_tasks, std::max(1, occ) * std::max(nsm, 1)));
  k_big_dag<T><<<grid, 256, smem, st>>>(sd, d_big + lp.big_off, tasks + lp.dag_task_off, lp.dag_tasks,
                                        ticket, flags, err, vals, D, sh, (T*)fronts, status, badcol);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

// ---------------------------------------------------------------------------
// Big fronts, owner tiles: one persistent launch per level.  A task is a
// tile: the 32-column block j of one (front, k) restricted to a chunk of CH
// rows (CH a multiple of 32; a whole column when CH >= F).  The CTA that takes
// it keeps the tile in shared memory from assembly to its final value:
//   1. assembly of the tile: the original entries (per-column ranges of the
//      assembly map), t_k D on the diagonal, and the children's update
//      columns through the inverse extend-add map.  Each destination column
//      belongs to one warp, which adds its contributions in child order, so
//      the sums are deterministic with no barrier between children;
//   2. every earlier panel p, in pivot order (left-looking form of the
//      static-pivot elimination of Sec. II-C): the tile holding panel p's
//      pivot rows waits for L11(p), solves the block's U rows and releases
//      them for the chunks below; every tile below the pivot rows waits for
//      those U rows and for its own chunk's rows of L21(p), then subtracts
//      L21(p) U(p, j) from its rows;
//   3. if the block holds pivots: the tile holding the diagonal block factors
//      it in shared memory (two pivots per barrier), eliminates its rows below
//      it and releases them; the tiles of the chunks below wait for that,
//      then eliminate their rows with the released U rows and reciprocal
//      pivots.  Tiles are written to the front storage before their release
//      flags (st.release.gpu) are set.
// Every phase runs on all 8 warps with short loop bodies: straight-line code
// run by a single warp is fetched cold and stalls on instruction fetch.
// The same per-element sequence of multiply-adds as panel_eliminate is used
// for the panel, so the pivot block and L21 match the per-panel path.
// Tasks are taken in ticket order from a list sorted by (block, chunk):
// every wait is on a tile earlier in that order, already held by a running
// CTA, so the schedule cannot deadlock whatever the residency, and every wait
// is bounded.
// ---------------------------------------------------------------------------
constexpr int kOwnThreads = 256;
constexpr unsigned kOwnFull = 0xffffffffu;

// U rows r0..r0+nb-1 of the block, solved with the unit lower L11 in Ls
// (row-major, ld 33): warp g takes columns [4g, 4g+4), lane r holds row r and
// receives row q's final values by shuffle.  The loop body is small so one
// warp's instruction stream stays cached.  Us gets the U rows row-major (32
// per row, zero beyond w and nb) for the update.  Needs 8 warps.
template <typename T>
__device__ __forceinline__ void own_trsm(T* Bk, int ld, int r0, int nb, int w, const T* Ls, T* Us) {
  const int lane = threadIdx.x & 31, cb = (threadIdx.x >> 5) * 4;
  T x[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) x[i] = (lane < nb && cb + i < w) ? Bk[r0 + lane + (cb + i) * ld] : T(0);
  for (int q = 0; q + 1 < nb; ++q) {
    T u[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) u[i] = __shfl_sync(kOwnFull, x[i], q);
    if (lane > q) {
      const T l = Ls[lane * 33 + q];
#pragma unroll
      for (int i = 0; i < 4; ++i) x[i] -= l * u[i];
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const bool in = lane < nb && cb + i < w;
    if (in) Bk[r0 + lane + (cb + i) * ld] = x[i];
    Us[lane * 32 + cb + i] = in ? x[i] : T(0);
  }
}

// rows [i0, i1) of the tile (stored from row R0): x(i, :) -= L(i, r0..r0+nb-1) U,
// L read from the front storage (written before its release) straight into
// registers, U from Us; a work item is one row and 16 columns.
template <typename T>
__device__ __forceinline__ void own_update_rows(T* Bt, int ld, int R0, const T* f, int F, int r0, int nb,
                                                const T* Us, int i0, int i1, int w) {
  const int m = i1 - i0;
  for (int q = threadIdx.x; q < 2 * m; q += blockDim.x) {
    const int g = q >= m ? 1 : 0;
    const int i = i0 + q - g * m;
    const int cb = 16 * g;
    if (cb >= w) continue;
    T l[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) l[c] = (c < nb) ? __ldcg(f + i + (int64_t)(r0 + c) * F) : T(0);
    T* row = Bt + (i - R0);
    T x[16];
#pragma unroll
    for (int col = 0; col < 16; ++col) x[col] = row[(cb + col) * ld];
#pragma unroll
    for (int cg = 0; cg < 32; cg += 8) {
      if (cg < nb) {
#pragma unroll
        for (int c = cg; c < cg + 8; ++c) {
          const T* ur = Us + c * 32 + cb;
#pragma unroll
          for (int col = 0; col < 16; ++col) x[col] -= l[c] * ur[col];
        }
      }
    }
#pragma unroll
    for (int col = 0; col < 16; ++col)
      if (cb + col < w) row[(cb + col) * ld] = x[col];
  }
}

// pivot-free LU of the np x w diagonal block D (rows = the block's pivots) in
// shared memory: lane = column, warp g = rows g, g + 8, g + 16, g + 24, and
// two pivots per barrier.  Columns keep their unscaled values during the
// elimination and are scaled once at the end; every thread forms the
// multipliers, the second pivot and the second pivot's row and column entries
// after the first elimination itself, as the same expressions in the same
// order as the one-pivot-at-a-time elimination (so every thread holds the
// values the owners of those entries store).  Writes the reciprocal pivots to
// rinv and the U rows, row-major, to Us.
template <typename T>
__device__ __forceinline__ void own_factor_diag(T* D, int ld, int np, int w, T* Us, T* rinv,
                                                const SymDev& sd, int s, int k, int K, int colbase,
                                                int32_t* status, int32_t* badcol) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int c = 0;
  for (; c + 1 < np; c += 2) {
    const T p0 = D[c + c * ld], b = D[(c + 1) + c * ld], e = D[c + (c + 1) * ld];
    const T p1raw = D[(c + 1) + (c + 1) * ld];
    const T rp0 = T(1) / p0;
    const T l1 = b * rp0;
    const T p1 = p1raw - l1 * e;
    const T rp1 = T(1) / p1;
    if (threadIdx.x == 0) {
      check_pivot(p0, sd, s, k, K, colbase + c, status, badcol);
      check_pivot(p1, sd, s, k, K, colbase + c + 1, status, badcol);
      rinv[c] = rp0;
      rinv[c + 1] = rp1;
    }
    // row c + 1 and column c + 1 are read unmodified by every thread in this
    // step, so their new values are stored only after the barrier (nothing
    // reads them again before the step after next)
    T held[4];
    int hmask = 0;
    if (lane > c && lane < w) {
      const T u0 = D[c + lane * ld];
      const T u1 = D[(c + 1) + lane * ld] - l1 * u0;
      T a0[4], a1[4], d[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = wid + 8 * i;
        a0[i] = r < np ? D[r + c * ld] : T(0);
        a1[i] = r < np ? D[r + (c + 1) * ld] : T(0);
        d[i] = r < np ? D[r + lane * ld] : T(0);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = wid + 8 * i;
        held[i] = T(0);
        if (r > c && r < np) {
          const T m0 = a0[i] * rp0;
          T v = d[i] - m0 * u0;
          if (r > c + 1 && lane > c + 1) {
            const T m1 = (a1[i] - m0 * e) * rp1;
            v = v - m1 * u1;
            D[r + lane * ld] = v;
          } else {
            held[i] = v;
            hmask |= 1 << i;
          }
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (hmask & (1 << i)) D[(wid + 8 * i) + lane * ld] = held[i];
  }
  __syncthreads();
  if (c < np) {  // odd count: the last pivot updates nothing below it
    if (threadIdx.x == 0) {
      const T piv = D[c + c * ld];
      check_pivot(piv, sd, s, k, K, colbase + c, status, badcol);
      rinv[c] = T(1) / piv;
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = wid + 8 * i;
    T v = T(0);
    if (r < np && lane < w) {
      v = D[r + lane * ld];
      if (lane < r) D[r + lane * ld] = v * rinv[lane];
    }
    Us[r * 32 + lane] = (r < np && lane < w && lane >= r) ? v : T(0);
  }
}

// rows [i0, i1) of the tile (stored from row R0), all below the factored
// diagonal block: one thread per row scales by the reciprocal pivots and
// eliminates in pivot order (the remaining columns of a block that straddles
// the end of the pivots are updated too).
template <typename T>
__device__ __forceinline__ void own_eliminate_rows(T* Bt, int ld, int R0, int i0, int i1, int np, int w,
                                                   const T* Us, const T* rinv) {
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    T* row = Bt + (i - R0);
    T x[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) x[c] = (c < w) ? row[c * ld] : T(0);
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      if (c < np) {
        const T l = x[c] * rinv[c];
        x[c] = l;
#pragma unroll
        for (int cc = c + 1; cc < 32; ++cc) x[cc] -= l * Us[c * 32 + cc];
      }
    }
#pragma unroll
    for (int c = 0; c < 32; ++c)
      if (c < w) row[c * ld] = x[c];
  }
}

// ---------------------------------------------------------------------------
// Tensor-core form of an owner tile's trailing update (FP32 factors only):
//     x(i, c) -= sum_{cc < nb} L(i, r0 + cc) U(cc, c)
// for the tile's rows, 128 rows at a time, on the 5th-generation tensor cores
// (tcgen05.mma, kind::tf32, M = 128, N = 32, K = 8 per instruction, FP32
// accumulator in tensor memory).  TF32 keeps 10 mantissa bits, so every FP32
// operand is split as hi + lo (hi = TF32 rounding of x, lo = TF32 rounding of
// x - hi) and the product is formed as hi*hi + hi*lo + lo*hi ("3xTF32"): the
// dropped lo*lo term and the rounding of lo are below FP32 rounding of the
// sum, so the update keeps FP32 accuracy.  Operands are staged in shared
// memory in the no-swizzle K-major core-matrix layout: 8 rows x 16 bytes per
// core matrix, K-adjacent core matrices 128 bytes apart, 8-row groups 1024
// bytes apart.
// ---------------------------------------------------------------------------
struct TcCtx {
  int on;          // 1: owner-tile updates on the tensor cores
  float* sA;       // [2][128 * 32] hi / lo of 128 rows of L
  float* sB;       // [2][32 * 32]  hi / lo of the 32 U rows (as N x K)
  uint32_t tmem;   // 32 tensor-memory columns: the 128 x 32 FP32 accumulator
  uint32_t mbar;   // shared-memory address of the MMA-completion barrier
  uint32_t phase;  // parity of the next completion of that barrier
};
constexpr int kTcSmemFloats = 2 * 128 * 32 + 2 * 32 * 32;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// offset of element (row r, k) of a rows x 32 K-major operand
__device__ __forceinline__ int tc_kmaj(int r, int k) {
  return (r >> 3) * 256 + (k >> 2) * 32 + (r & 7) * 4 + (k & 3);
}

// shared-memory matrix descriptor: start address, leading-dimension (K) and
// stride-dimension (8-row group) byte offsets, fixed field 0b001, no swizzle
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Allocates the CTA's 32 tensor-memory columns (warp 0) and initialises the
// completion barrier; every thread of the CTA calls it.
__device__ __forceinline__ void tc_setup(TcCtx& tc, uint32_t* s_taddr, uint64_t* s_mbar) {
  if (!tc.on) return;
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_addr(s_taddr)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(s_mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  tc.tmem = *s_taddr;
  tc.mbar = smem_addr(s_mbar);
  tc.phase = 0;
}

// Frees the tensor memory; every thread of the CTA calls it before exiting.
__device__ __forceinline__ void tc_teardown(const TcCtx& tc) {
  if (!tc.on) return;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tc.tmem));
}

// rows [i0, i1) of the tile (stored from row R0): x(i, c) -= L(i, r0..r0+nb-1) U
// for c < w, L from the front storage, U from Us (32 x 32 row-major, zero
// beyond nb rows and w columns).  Needs kOwnThreads (8 warps) threads.
__device__ __noinline__ void tc_update_rows(float* Bt, int ld, int R0, const float* f, int F, int r0, int nb,
                                               const float* Us, int i0, int i1, int w, TcCtx& tc, int* err) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5;
  float* sAh = tc.sA;
  float* sAl = tc.sA + 128 * 32;
  float* sBh = tc.sB;
  float* sBl = tc.sB + 32 * 32;
  for (int q = tid; q < 32 * 32; q += nt) {  // B(k, n) = U(k, n), staged as N x K
    const int n = q & 31, k = q >> 5;
    const float u = Us[k * 32 + n], hi = tf32_round(u);
    sBh[tc_kmaj(n, k)] = hi;
    sBl[tc_kmaj(n, k)] = tf32_round(u - hi);
  }
  const int ksteps = (nb + 7) >> 3;
  // instruction descriptor: FP32 accumulator, TF32 A and B, both K-major,
  // N = 32, M = 128
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
  for (int m0 = i0; m0 < i1; m0 += 128) {
    for (int q = tid; q < 128 * 32; q += nt) {  // A(r, k) = L(m0 + r, r0 + k), zero outside
      const int r = q & 127, k = q >> 7, i = m0 + r;
      const float a = (i < i1 && k < nb) ? __ldcg(f + i + (int64_t)(r0 + k) * F) : 0.f;
      const float hi = tf32_round(a);
      sAh[tc_kmaj(r, k)] = hi;
      sAl[tc_kmaj(r, k)] = tf32_round(a - hi);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      uint32_t acc = 0;
      for (int ks = 0; ks < ksteps; ++ks) {
        for (int term = 0; term < 3; ++term) {  // hi*hi, hi*lo, lo*hi
          const uint64_t da = tc_sdesc(smem_addr(term == 2 ? sAl : sAh) + ks * 256);
          const uint64_t db = tc_sdesc(smem_addr(term == 1 ? sBl : sBh) + ks * 256);
          asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                       " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tc.tmem),
                       "l"(da), "l"(db), "r"(idesc), "r"(acc));
          acc = 1;
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc.mbar));
    }
    {  // bounded wait for the MMAs of this block
      uint32_t done = 0;
      for (int it = 0; it < (1 << 24) && !done; ++it)
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(tc.mbar), "r"(tc.phase));
      if (!done && tid == 0) atomicExch(err, 1);
      tc.phase ^= 1;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (rows), columns
    // 16 (w / 4) .. + 15
    uint32_t v[16];
    const uint32_t ta = tc.tmem + ((uint32_t)(32 * (wid & 3)) << 16) + 16 * (wid >> 2);
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                   "=r"(v[15])
                 : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int row = m0 + 32 * (wid & 3) + lane;
    if (row < i1) {
      float* x = Bt + (row - R0);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int col = 16 * (wid >> 2) + c;
        if (col < w) x[col * ld] -= __uint_as_float(v[c]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // sA / the accumulator are reused by the next block
  }
}

// One owner tile: the 32-column block j of front s, perturbation k,
// restricted to the row chunk q of CH rows (see above).  `flags` points at
// the (front, k) pair's release flags.  Needs kOwnThreads threads and the
// shared memory layout of the owner kernels (Us, Ls, Bt, rinv).
template <typename T, bool TC>
__device__ __forceinline__ void owner_tile(const SymDev& sd, int s, int k, int j, int q, int* flags, int CH,
                                           int* err, const double* __restrict__ vals,
                                           const double* __restrict__ D, const Shifts& sh,
                                           T* __restrict__ fronts, int32_t* status, int32_t* badcol,
                                           T* Us, T* Ls, T* Bt, T* rinv, TcCtx& tc) {
  const int K = sh.K;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int ld = CH + 1;
  const int ns = sd.ns[s], F = ns + sd.ms[s];
  const int P = (ns + 31) >> 5, J = (F + 31) >> 5, Q = (F + CH - 1) / CH;
  const int j0 = j << 5, w = min(32, F - j0);
  const int R0 = q * CH, R1 = min(F, R0 + CH);
  int* Lf = flags;            // [P][Q]: rows of chunk q of panel block p final
  int* Uf = Lf + P * Q;       // [P][J]: U rows of panel p in block j final
  T* f = fronts + (int64_t)K * sd.front_off[s] + (int64_t)k * F * F;
  const int64_t vo = sd.vec_off[s];

  // 1. assembly of the tile: rows [R0, R1) of columns [j0, j0 + w)
  for (int e = tid; e < ld * w; e += nt) Bt[e] = T(0);
  __syncthreads();
  {
    const int64_t a0 = sd.amap_coff[vo + j0], a1 = sd.amap_coff[vo + j0 + w];
    for (int64_t e = a0 + tid; e < a1; e += nt) {
      const int d = sd.amap_dst[e];
      const int c = d / F, i = d - c * F;
      if (i >= R0 && i < R1) atomicAdd(&Bt[(i - R0) + (c - j0) * ld], (T)vals[sd.amap_src[e]]);
    }
    const double tk = sh.t[k];
    const int c0 = sd.c0[s];
    for (int c = max(j0, R0) + tid; c < min(min(j0 + w, ns), R1); c += nt)
      atomicAdd(&Bt[(c - R0) + (c - j0) * ld], (T)(tk * D[sd.perm[c0 + c]]));
  }
  __syncthreads();
  extend_add_columns<T>(sd, s, k, K, fronts, Bt, ld, j0, w, R0, R1, (int)(threadIdx.x >> 5), (int)(blockDim.x >> 5));
  __syncthreads();

  // 2. the updates of every earlier panel, in pivot order; panels whose
  //    pivot rows lie below the tile do not touch it
  const int pe = min(j, P);
  for (int p = 0; p < pe; ++p) {
    const int r0 = p << 5, nb = min(32, ns - r0), qp = r0 / CH;
    if (q < qp) break;
    if (q == qp) {
      // the tile holds panel p's pivot rows: solve this block's U rows
      if (tid == 0) dag_wait(Lf + p * Q + qp, 1, err);
      __syncthreads();
      for (int e = tid; e < 32 * 32; e += nt) {
        const int r = e & 31, c = e >> 5;
        Ls[r * 33 + c] = (r < nb && c < r) ? __ldcg(f + (r0 + r) + (int64_t)(r0 + c) * F) : T(0);
      }
      __syncthreads();
      own_trsm<T>(Bt + (r0 - R0), ld, 0, nb, w, Ls, Us);
      __syncthreads();
      if (qp + 1 < Q) {  // chunks below read these U rows
        for (int c = wid; c < w; c += nw)
          for (int r = lane; r < nb; r += 32) f[(r0 + r) + (int64_t)(j0 + c) * F] = Bt[(r0 - R0 + r) + c * ld];
        __threadfence();
        __syncthreads();
        if (tid == 0) dag_st_release(Uf + p * J + j, 1);
      }
      if constexpr (TC && std::is_same<T, float>::value)
        tc_update_rows(Bt, ld, R0, f, F, r0, nb, Us, r0 + nb, R1, w, tc, err);
      else
        own_update_rows<T>(Bt, ld, R0, f, F, r0, nb, Us, r0 + nb, R1, w);
      __syncthreads();
    } else {
      // a chunk below panel p: its U rows of this block come from the
      // chunk holding the pivot rows, its L rows from this chunk's tile of
      // panel p
      if (tid == 0) {
        dag_wait(Uf + p * J + j, 1, err);
        dag_wait(Lf + p * Q + q, 1, err);
      }
      __syncthreads();
      for (int e = tid; e < 32 * 32; e += nt) {
        const int r = e >> 5, c = e & 31;
        Us[e] = (r < nb && c < w) ? __ldcg(f + (r0 + r) + (int64_t)(j0 + c) * F) : T(0);
      }
      __syncthreads();
      if constexpr (TC && std::is_same<T, float>::value)
        tc_update_rows(Bt, ld, R0, f, F, r0, nb, Us, R0, R1, w, tc, err);
      else
        own_update_rows<T>(Bt, ld, R0, f, F, r0, nb, Us, R0, R1, w);
      __syncthreads();
    }
  }

  // 3. the block's own pivots
  const int qj = j0 / CH;
  if (j < P) {
    const int np = min(32, ns - j0);
    if (q == qj) {
      own_factor_diag<T>(Bt + (j0 - R0), ld, np, w, Us, rinv, sd, s, k, K, sd.c0[s] + j0, status, badcol);
      __syncthreads();
      own_eliminate_rows<T>(Bt, ld, R0, j0 + np, R1, np, w, Us, rinv);
      __syncthreads();
    } else if (q > qj) {
      // rows below the diagonal block's chunk: its factored rows come from
      // the front storage once that tile has released them
      if (tid == 0) dag_wait(Lf + j * Q + qj, 1, err);
      __syncthreads();
      for (int e = tid; e < 32 * 32; e += nt) {
        const int r = e >> 5, c = e & 31;
        Us[e] = (r < np && c < w && c >= r) ? __ldcg(f + (j0 + r) + (int64_t)(j0 + c) * F) : T(0);
      }
      if (tid < np) rinv[tid] = T(1) / __ldcg(f + (int64_t)(j0 + tid) * (F + 1));
      __syncthreads();
      own_eliminate_rows<T>(Bt, ld, R0, R0, R1, np, w, Us, rinv);
      __syncthreads();
    }
  }

  // 4. write the tile; tiles holding L rows of this block release them
  //    (rows from the first pivot down first, then the U rows above)
  const bool rel = j < P && q >= qj;
  const int rs = (rel && q == qj) ? j0 : R0;
  for (int c = wid; c < w; c += nw) {
    T* dst = f + (int64_t)(j0 + c) * F;
    const T* src = Bt + c * ld;
    for (int i = rs + lane; i < R1; i += 32) dst[i] = src[i - R0];
  }
  if (rel) {
    __threadfence();
    __syncthreads();
    if (tid == 0) dag_st_release(Lf + j * Q + q, 1);
  }
  for (int c = wid; c < w; c += nw) {
    T* dst = f + (int64_t)(j0 + c) * F;
    const T* src = Bt + c * ld;
    for (int i = R0 + lane; i < rs; i += 32) dst[i] = src[i - R0];
  }
}

template <typename T, bool TC>
__global__ void __launch_bounds__(kOwnThreads) k_front_owner(SymDev sd, const int32_t* __restrict__ big,
                                                             const DagTask* __restrict__ tasks, int ntasks,
                                                             int* ticket, int* flags, int* err,
                                                             const double* __restrict__ vals,
                                                             const double* __restrict__ D, Shifts sh,
                                                             T* __restrict__ fronts, int32_t* status,
                                                             int32_t* badcol, int CH) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_t;
  __shared__ T rinv[32];
  __shared__ uint32_t s_taddr;
  __shared__ __align__(8) uint64_t s_mbar;
  T* Us = reinterpret_cast<T*>(smraw);  // 32 x 32 row-major: U rows of the current panel
  T* Ls = Us + 32 * 32;                 // 32 x 33 row-major: unit-lower L11 of the current panel
  T* Bt = Ls + 32 * 33;                 // (CH + 1) x 32 column-major: the owned tile
  float* tcs = reinterpret_cast<float*>(Bt + (size_t)(CH + 1) * 32);  // tensor-core staging (FP32 only)
  TcCtx tc{TC ? 1 : 0, tcs, tcs + 2 * 128 * 32, 0, 0, 0};
  if constexpr (TC) tc_setup(tc, &s_taddr, &s_mbar);
  const int tid = threadIdx.x;
  for (;;) {
    __syncthreads();  // the previous task is done with shared memory and s_t
    if (tid == 0) s_t = atomicAdd(ticket, 1);
    __syncthreads();
    const int u = s_t;
    if (u >= ntasks) break;
    const DagTask t = tasks[u];
    owner_tile<T, TC>(sd, big[t.b], t.k, t.j, t.p, flags + t.flags, CH, err, vals, D, sh, fronts, status, badcol,
                  Us, Ls, Bt, rinv, tc);
  }
  if constexpr (TC) tc_teardown(tc);
}

// ---------------------------------------------------------------------------
// The whole factorisation as ONE persistent launch over every level of the
// assembly forest, all K shifts and all instances of a batch.  Tasks, taken in
// ticket order (levels bottom-up; within a level the owner tiles first, then
// the shared-memory fronts, then the warp fronts):
//   kFacWarp : up to 8 (front, k) pairs with F <= 32, one per warp, each in
//              its warp's shared-memory area (front_warp);
//   kFacCta  : one (front, k) pair of a front that fits in shared memory
//              (front_cta);
//   kFacOwner: one owner tile of a wider front (owner_tile).
// Before its assembly a task waits until every child's completion counter
// for its k, fdone[child * K + k], has reached need[child] (1 for warp and
// shared-memory fronts, the number of tiles for an owner front); a finished
// task adds 1 to its own counter after its writes are visible.  Every wait is
// on a task with a smaller ticket (a child, or an earlier tile of the same
// front), which a running CTA already holds, so the schedule cannot deadlock
// whatever the residency, and every wait is bounded.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fac_wait_children(const SymDev& sd, const int* fdone, const int* need, int s,
                                                  int k, int K, int idx, int n, int* err, int64_t polls) {
  const int cb = sd.child_off[s], ce = sd.child_off[s + 1];
  for (int ci = cb + idx; ci < ce; ci += n) {
    const int c = sd.child[ci];
    const int* f = fdone + (int64_t)c * K + k;
    const int want = need[c];
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
    if (v >= want) continue;
    int64_t i = 0;
    for (; i < polls; ++i) {
      __nanosleep(64);
      asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
      if (v >= want) break;
    }
    if (i == polls) atomicExch(err, 1);
  }
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

__device__ __forceinline__ void fac_publish(int* fdone, int s, int k, int K) {
  __threadfence();
  asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(fdone + (int64_t)s * K + k) : "memory");
}

template <typename T, bool TC, int MINB>
__global__ void __launch_bounds__(kOwnThreads, MINB)
k_factor_persistent(SymDev sd, const FactorTask* __restrict__ tasks, int ntasks, int* ticket, int* fdone,
                    const int* __restrict__ need, int* flags, int* err, const int32_t* __restrict__ wlist,
                    const double* __restrict__ vals, const double* __restrict__ D, Shifts sh,
                    T* __restrict__ fronts, int32_t* status, int32_t* badcol, int CH, int64_t polls,
                    size_t tc_off) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_t;
  __shared__ T rinv[32];
  __shared__ uint32_t s_taddr;
  __shared__ __align__(8) uint64_t s_mbar;
  T* sm = reinterpret_cast<T*>(smraw);
  float* tcs = reinterpret_cast<float*>(smraw + tc_off);  // tensor-core staging (FP32 owner tiles)
  TcCtx tc{TC ? 1 : 0, tcs, tcs + 2 * 128 * 32, 0, 0, 0};
  if constexpr (TC) tc_setup(tc, &s_taddr, &s_mbar);
  const int K = sh.K;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5;
  for (;;) {
    __syncthreads();  // the previous task is done with shared memory and s_t
    if (tid == 0) s_t = atomicAdd(ticket, 1);
    __syncthreads();
    const int u = s_t;
    if (u >= ntasks) break;
    const FactorTask t = tasks[u];
    if (t.kind == kFacWarp) {
      const int q = t.q + wid;
      if (q < t.j) {
        const int s = wlist[t.s + q / K], k = q % K;
        fac_wait_children(sd, fdone, need, s, k, K, lane, 32, err, polls);
        __syncwarp();
        front_warp<T>(sd, s, k, vals, D, sh, fronts, status, badcol, sm + wid * 32 * 32);
        __syncwarp();
        if (lane == 0) fac_publish(fdone, s, k, K);
      }
    } else {
      fac_wait_children(sd, fdone, need, t.s, t.k, K, tid, nt, err, polls);
      __syncthreads();
      if (t.kind == kFacCta)
        front_cta<T>(sd, t.s, t.k, vals, D, sh, fronts, status, badcol, sm);
      else
        owner_tile<T, TC>(sd, t.s, t.k, t.j, t.q, flags + t.flags, CH, err, vals, D, sh, fronts, status,
                          badcol, sm, sm + 32 * 32, sm + 32 * 32 + 32 * 33, rinv, tc);
      __syncthreads();
      if (tid == 0) fac_publish(fdone, t.s, t.k, K);
    }
  }
  if constexpr (TC) tc_teardown(tc);
}

template <typename T, bool TC, int M>
int factor_persistent_launch(const SymDev& sd, const FactorTask* tasks, int ntasks, int* ticket, int* fdone,
                             const int* need, int* flags, int* err, const int32_t* wlist, const double* vals,
                             const double* D, const Shifts& sh, void* fronts, int32_t* status, int32_t* badcol,
                             int CH, size_t smem, size_t tc_off, int64_t polls, cudaStream_t st) {
  static std::atomic<int> nsm_dev[kMaxDevices];
  const int dev = current_device();
  int nsm = nsm_dev[dev].load(std::memory_order_acquire);
  if (!nsm) {
    cudaFuncSetAttribute(k_factor_persistent<T, TC, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    nsm_dev[dev].store(nsm, std::memory_order_release);
  }
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_factor_persistent<T, TC, M>, kOwnThreads, smem);
  const int grid = std::max(1, std::min(ntasks, std::max(1, occ) * std::max(nsm, 1)));
  k_factor_persistent<T, TC, M><<<grid, kOwnThreads, smem, st>>>(sd, tasks, ntasks, ticket, fdone, need, flags,
                                                                 err, wlist, vals, D, sh, (T*)fronts, status,
                                                                 badcol, CH, polls > 0 ? polls : kDagWaitPolls,
                                                                 tc_off);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

// ctas: resident CTAs per SM the kernel is compiled for, 2 (128 registers per
// thread) or 3 (80; the owner tiles' register arrays then spill a little)
template <typename T>
int factor_persistent_impl(const SymDev& sd, const FactorTask* tasks, int ntasks, int* ticket, int* fdone,
                           const int* need, int* flags, int* err, const int32_t* wlist, const double* vals,
                           const double* D, const Shifts& sh, void* fronts, int32_t* status, int32_t* badcol,
                           int CH, size_t smem, int64_t polls, int tc, int ctas, cudaStream_t st) {
  if (ntasks == 0) return 0;
  const int tc_on = tc && sizeof(T) == 4 ? 1 : 0;
  const size_t tc_off = smem;  // the staging follows everything the other task kinds use
  if (tc_on) smem += (size_t)kTcSmemFloats * sizeof(float);
  if (smem > (size_t)kSmemCap) return -1;
  if (tc_on)
    return factor_persistent_launch<T, true, 2>(sd, tasks, ntasks, ticket, fdone, need, flags, err, wlist, vals, D,
                                                sh, fronts, status, badcol, CH, smem, tc_off, polls, st);
  if (ctas >= 3)
    return factor_persistent_launch<T, false, 3>(sd, tasks, ntasks, ticket, fdone, need, flags, err, wlist, vals,
                                                 D, sh, fronts, status, badcol, CH, smem, tc_off, polls, st);
  return factor_persistent_launch<T, false, 2>(sd, tasks, ntasks, ticket, fdone, need, flags, err, wlist, vals, D,
                                               sh, fronts, status, badcol, CH, smem, tc_off, polls, st);
}

template <typename T>
int owner_impl(const SymDev& sd, const LevelPlan& lp, const int32_t* d_big, const DagTask* tasks,
               int* ticket, int* flags, int* err, const double* vals, const double* D,
               const Shifts& sh, void* fronts, int32_t* status, int32_t* badcol, int tc, cudaStream_t st) {
  static std::atomic<int> nsm_dev[kMaxDevices];
  const int dev = current_device();
  int nsm = nsm_dev[dev].load(std::memory_order_acquire);
  if (!nsm) {
    cudaFuncSetAttribute(k_front_owner<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
    cudaFuncSetAttribute(k_front_owner<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    nsm_dev[dev].store(nsm, std::memory_order_release);
  }
  const int tc_on = tc && sizeof(T) == 4 ? 1 : 0;
  const size_t smem = ((size_t)(lp.own_ch + 1) * 32 + 32 * 32 + 32 * 33) * sizeof(T) +
                      (tc_on ? (size_t)kTcSmemFloats * sizeof(float) : 0);
  if (lp.own_ch < 32 || lp.own_ch % 32 || smem > (size_t)kSmemCap) return -1;
  int occ = 1;
  if (tc_on) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_front_owner<T, true>, kOwnThreads, smem);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_front_owner<T, false>, kOwnThreads, smem);
  const int grid = std::max(1, std::min(lp.dag_tasks, std::max(1, occ) * std::max(nsm, 1)));
  if (tc_on)
    k_front_owner<T, true><<<grid, kOwnThreads, smem, st>>>(sd, d_big + lp.big_off, tasks + lp.dag_task_off,
                                                            lp.dag_tasks, ticket, flags, err, vals, D, sh,
                                                            (T*)fronts, status, badcol, lp.own_ch);
  else
    k_front_owner<T, false><<<grid, kOwnThreads, smem, st>>>(sd, d_big + lp.big_off, tasks + lp.dag_task_off,
                                                             lp.dag_tasks, ticket, flags, err, vals, D, sh,
                                                             (T*)fronts, status, badcol, lp.own_ch);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

template <typename T>
int small_threads(int maxF) {
  if (maxF <= 16) return 64;
  if (maxF <= 32) return 128;
  if (maxF <= 96) return 256;
  return 512;
}

template <typename T>
void set_smem_attrs() {
  static std::atomic<bool> done_dev[kMaxDevices];
  const int dev = current_device();
  if (done_dev[dev].load(std::memory_order_acquire)) return;
  cudaFuncSetAttribute(k_front_small<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
  cudaFuncSetAttribute(k_front_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
  cudaFuncSetAttribute(k_panel_big<T, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
  cudaFuncSetAttribute(k_panel_big<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
  cudaFuncSetAttribute(k_panel_big<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
  cudaFuncSetAttribute(k_panel_big<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap);
  done_dev[dev].store(true, std::memory_order_release);
}

template <typename T, int NB>
int run_panels(const SymDev& sd, const LevelPlan& lp, const int32_t* d_big,
               const BigFrontHost* bh, int K, T* fr, int32_t* status, int32_t* badcol,
               cudaStream_t st) {
  int launches = 0;
  for (int p0 = 0; p0 < lp.big_maxns; p0 += NB) {
    int maxMr = 0, mmax = 0;
    for (int b = 0; b < lp.big_count; ++b) {
      if (p0 >= bh[b].ns) continue;
      maxMr = std::max(maxMr, bh[b].F - p0);
      mmax = std::max(mmax, bh[b].F - p0 - std::min(NB, bh[b].ns - p0));
    }
    if (maxMr == 0) continue;
    const size_t smem = (size_t)(maxMr + 1) * NB * sizeof(T);
    k_panel_big<T, NB><<<dim3(lp.big_count, K), 512, smem, st>>>(sd, d_big, K, fr, p0, status, badcol);
    ++launches;
    if (mmax > 0) {
      const int tpd = (mmax + 63) / 64;
      k_update_big<T><<<dim3(tpd * tpd, lp.big_count, K), 256, 0, st>>>(sd, d_big, K, fr, p0, NB);
      ++launches;
    }
  }
  return launches;
}

template <typename T>
int factor_small_group(const SymDev& sd, const LevelPlan& lp, int g, const int32_t* d_small,
                       const double* vals, const double* D, const Shifts& sh, void* fronts,
                       int32_t* status, int32_t* badcol, cudaStream_t st) {
  set_smem_attrs<T>();
  T* fr = reinterpret_cast<T*>(fronts);
  const int K = sh.K;
  int launches = 0;
  {
    const auto& G = lp.groups[g];
    if (G.count == 0) return 0;
    if (G.cluster == 0) {
      const size_t smem = (size_t)G.maxF * G.maxF * sizeof(T);
      k_front_small<T><<<dim3(G.count, K), small_threads<T>(G.maxF), smem, st>>>(
          sd, d_small + G.off, vals, D, sh, fr, status, badcol);
    } else {
      const int C = G.cluster;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(G.count * C, K, 1);
      cfg.blockDim = dim3(256, 1, 1);
      cfg.dynamicSmemBytes = cluster_smem<T>(G.maxF, C);
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = C;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      const int32_t* lst = d_small + G.off;
      if (cudaLaunchKernelEx(&cfg, k_front_cluster<T>, sd, lst, C, vals, D, sh, fr, status, badcol) !=
          cudaSuccess)
        return -1;
    }
    ++launches;
  }
  if (cudaGetLastError() != cudaSuccess) return -1;
  return launches;
}

template <typename T>
int factor_small_impl(const SymDev& sd, const LevelPlan& lp, const int32_t* d_small,
                      const double* vals, const double* D, const Shifts& sh, void* fronts,
                      int32_t* status, int32_t* badcol, cudaStream_t st) {
  int launches = 0;
  for (int g = 0; g < lp.n_groups; ++g) {
    const int n = factor_small_group<T>(sd, lp, g, d_small, vals, D, sh, fronts, status, badcol, st);
    if (n < 0) return -1;
    launches += n;
  }
  return launches;
}

template <typename T>
int factor_big_impl(const SymDev& sd, const LevelPlan& lp, const int32_t* d_big,
                    const BigFrontHost* bh, const double* vals, const double* D, const Shifts& sh,
                    void* fronts, int32_t* status, int32_t* badcol, cudaStream_t st) {
  set_smem_attrs<T>();
  T* fr = reinterpret_cast<T*>(fronts);
  const int K = sh.K;
  int launches = 0;
  if (lp.big_count > 0) {
    const int TW = 32;
    const int big = lp.big_count;
    const int32_t* lst = d_big + lp.big_off;
    k_assemble_big<T><<<dim3((lp.big_maxF + TW - 1) / TW, big, K), 256, 0, st>>>(
        sd, lst, vals, D, sh, fr, TW);
    ++launches;
    const BigFrontHost* b = bh + lp.big_off;
    if ((size_t)(lp.big_maxF + 1) * 32 * sizeof(T) <= (size_t)kSmemCap)
      launches += run_panels<T, 32>(sd, lp, lst, b, K, fr, status, badcol, st);
    else if ((size_t)(lp.big_maxF + 1) * 16 * sizeof(T) <= (size_t)kSmemCap)
      launches += run_panels<T, 16>(sd, lp, lst, b, K, fr, status, badcol, st);
    else if ((size_t)(lp.big_maxF + 1) * 8 * sizeof(T) <= (size_t)kSmemCap)
      launches += run_panels<T, 8>(sd, lp, lst, b, K, fr, status, badcol, st);
    else
      launches += run_panels<T, 4>(sd, lp, lst, b, K, fr, status, badcol, st);
  }
  if (cudaGetLastError() != cudaSuccess) return -1;
  return launches;
}

}  // namespace

int small_front_limit(int precision) { return precision == PISP_FP32 ? 224 : 160; }

int front_cluster_size(int F, int precision) {
  if (F <= 64) return 0;
  for (int C = 1; C <= 8; C *= 2) {
    const size_t need = precision == PISP_FP32 ? cluster_smem<float>(F, C) : cluster_smem<double>(F, C);
    if (need <= (size_t)kSmemCap) return C;
  }
  return -1;
}

int max_big_front(int precision) {
  return kSmemCap / (4 * (precision == PISP_FP32 ? 4 : 8)) - 1;
}

int launch_factor_small(int precision, const SymDev& sd, const LevelPlan& lp,
                        const int32_t* d_small, const double* vals, const double* D,
                        const Shifts& sh, void* fronts, int32_t* status, int32_t* badcol,
                        cudaStream_t st) {
  if (precision == PISP_FP32)
    return factor_small_impl<float>(sd, lp, d_small, vals, D, sh, fronts, status, badcol, st);
  return factor_small_impl<double>(sd, lp, d_small, vals, D, sh, fronts, status, badcol, st);
}

int launch_factor_small_group(int precision, const SymDev& sd, const LevelPlan& lp, int g,
                              const int32_t* d_small, const double* vals, const double* D,
                              const Shifts& sh, void* fronts, int32_t* status, int32_t* badcol,
                              cudaStream_t st) {
  if (precision == PISP_FP32)
    return factor_small_group<float>(sd, lp, g, d_small, vals, D, sh, fronts, status, badcol, st);
  return factor_small_group<double>(sd, lp, g, d_small, vals, D, sh, fronts, status, badcol, st);
}

int max_dag_front(int precision) { return kSmemCap / (32 * (precision == PISP_FP32 ? 4 : 8)) - 1; }

int owner_chunk_rows(int precision, int maxF, int tc) {
  // Rows per tile.  FP64 elimination runs at a small fraction of the FP32
  // rate on this part, so one SM per 32-column block is the bottleneck of a
  // panel step: 32-row tiles spread a block's update and elimination over
  // its chunks (1354-bus root: 0.66 ms against 0.82 with whole columns).  In
  // FP32 the extra hand-offs and reloads of row chunks cost more than they
  // save (10000-bus: 3.2-5.1 ms with 256- to 96-row tiles against 3.0), so a
  // tile is a whole column block while it fits in shared memory.
  const int full = (maxF + 31) / 32 * 32;
  if (precision != PISP_FP32) return std::min(32, full);
  // (CH + 1) * 32 + 2080 floats, plus the tensor-core staging when it is on
  const int fit = ((kSmemCap / 4 - 32 * 32 - 32 * 33 - (tc ? kTcSmemFloats : 0)) / 32 - 1) / 32 * 32;
  return std::min(full, fit);
}

void build_owner_tasks(const BigFrontHost* big, int32_t nbig, int32_t K, int32_t CH,
                       std::vector<DagTask>& out, int32_t& nflags) {
  out.clear();
  std::vector<int32_t> foff((size_t)nbig * K);
  nflags = 0;
  int maxJ = 0, maxQ = 0;
  for (int b = 0; b < nbig; ++b) {
    const int P = (big[b].ns + 31) / 32, J = (big[b].F + 31) / 32, Q = (big[b].F + CH - 1) / CH;
    maxJ = std::max(maxJ, J);
    maxQ = std::max(maxQ, Q);
    for (int k = 0; k < K; ++k) {
      foff[(size_t)b * K + k] = nflags;
      nflags += P * (Q + J);
    }
  }
  // (block, chunk) order: every wait of a tile is on a tile earlier in it
  for (int j = 0; j < maxJ; ++j)
    for (int q = 0; q < maxQ; ++q)
      for (int b = 0; b < nbig; ++b) {
        if (j >= (big[b].F + 31) / 32 || q >= (big[b].F + CH - 1) / CH) continue;
        for (int k = 0; k < K; ++k) out.push_back({kDagOwner, b, k, q, j, foff[(size_t)b * K + k]});
      }
}

void build_dag_tasks(const BigFrontHost* big, int32_t nbig, int32_t K, std::vector<DagTask>& out,
                     int32_t& nflags) {
  out.clear();
  std::vector<int32_t> foff((size_t)nbig * K);
  nflags = 0;
  int maxP = 0;
  for (int b = 0; b < nbig; ++b) {
    const int J = (big[b].F + 31) / 32, P = (big[b].ns + 31) / 32;
    maxP = std::max(maxP, P);
    for (int k = 0; k < K; ++k) {
      foff[(size_t)b * K + k] = nflags;
      nflags += J + P;
    }
  }
  for (int b = 0; b < nbig; ++b)
    for (int k = 0; k < K; ++k)
      for (int j = 0; j < (big[b].F + 31) / 32; ++j)
        out.push_back({kDagAsm, b, k, 0, j, foff[(size_t)b * K + k]});
  for (int p = 0; p < maxP; ++p) {
    for (int b = 0; b < nbig; ++b) {
      const int F = big[b].F, ns = big[b].ns;
      const int J = (F + 31) / 32, P = (ns + 31) / 32;
      if (p >= P) continue;
      const int nb = std::min(32, ns - 32 * p);
      for (int k = 0; k < K; ++k) {
        const int fo = foff[(size_t)b * K + k];
        if (p == 0) out.push_back({kDagPanel, b, k, 0, 0, fo});
        if (p + 1 < J) out.push_back({kDagUpdate, b, k, p, p + 1, fo});
        if (p + 1 < P) out.push_back({kDagPanel, b, k, p + 1, 0, fo});
        if (32 * p + nb < std::min(32 * p + 32, F)) out.push_back({kDagUpdate, b, k, p, p, fo});
        for (int j = p + 2; j < J; ++j) out.push_back({kDagUpdate, b, k, p, j, fo});
      }
    }
  }
}

int launch_factor_big_dag(int precision, const SymDev& sd, const LevelPlan& lp, const int32_t* d_big,
                          const DagTask* tasks, int* ticket, int* flags, int* err,
                          const double* vals, const double* D, const Shifts& sh, void* fronts,
                          int32_t* status, int32_t* badcol, int tc, cudaStream_t st) {
  if (lp.dag_owner) {
    if (precision == PISP_FP32)
      return owner_impl<float>(sd, lp, d_big, tasks, ticket, flags, err, vals, D, sh, fronts, status,
                               badcol, tc, st);
    return owner_impl<double>(sd, lp, d_big, tasks, ticket, flags, err, vals, D, sh, fronts, status,
                              badcol, tc, st);
  }
  if (precision == PISP_FP32)
    return big_dag_impl<float>(sd, lp, d_big, tasks, ticket, flags, err, vals, D, sh, fronts, status,
                               badcol, st);
  return big_dag_impl<double>(sd, lp, d_big, tasks, ticket, flags, err, vals, D, sh, fronts, status,
                              badcol, st);
}

int persistent_cta_front_limit(int precision) { return precision == PISP_FP32 ? 160 : 112; }

size_t factor_persistent_smem(int precision, int CH, bool has_owner, int maxCtaF) {
  const size_t es = precision == PISP_FP32 ? 4 : 8;
  size_t e = (size_t)(kOwnThreads / 32) * 32 * 32;                          // warp fronts
  e = std::max(e, (size_t)maxCtaF * maxCtaF);                                // shared-memory fronts
  if (has_owner) e = std::max(e, (size_t)(CH + 1) * 32 + 32 * 32 + 32 * 33);  // owner tiles
  return e * es;
}

int launch_factor_persistent(int precision, const SymDev& sd, const FactorTask* tasks, int ntasks, int* ticket,
                             int* fdone, const int* need, int* flags, int* err, const int32_t* wlist,
                             const double* vals, const double* D, const Shifts& sh, void* fronts,
                             int32_t* status, int32_t* badcol, int CH, size_t smem, int64_t polls, int tc,
                             int ctas, cudaStream_t st) {
  if (precision == PISP_FP32)
    return factor_persistent_impl<float>(sd, tasks, ntasks, ticket, fdone, need, flags, err, wlist, vals, D, sh,
                                         fronts, status, badcol, CH, smem, polls, tc, ctas, st);
  return factor_persistent_impl<double>(sd, tasks, ntasks, ticket, fdone, need, flags, err, wlist, vals, D, sh,
                                        fronts, status, badcol, CH, smem, polls, tc, ctas, st);
}

int launch_factor_big(int precision, const SymDev& sd, const LevelPlan& lp, const int32_t* d_big,
                      const BigFrontHost* big_host, const double* vals, const double* D,
                      const Shifts& sh, void* fronts, int32_t* status, int32_t* badcol,
                      cudaStream_t st) {
  if (precision == PISP_FP32)
    return factor_big_impl<float>(sd, lp, d_big, big_host, vals, D, sh, fronts, status, badcol, st);
  return factor_big_impl<double>(sd, lp, d_big, big_host, vals, D, sh, fronts, status, badcol, st);
}

}  // namespace pisp
