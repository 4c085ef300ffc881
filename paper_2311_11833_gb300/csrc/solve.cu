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
#include <cuda_runtime.h>

#include <algorithm>

#include "pisp_internal.h"

namespace pisp {
namespace {

constexpr int kSolveThreads = 256;
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

// Rk[pi][k][r] = b[i][r] - sum_j A_ij X[pj][k][r] - t_k D_i X[pi][k][r]  (FP64),
// one warp per original row i.
__global__ void k_residual_per_k(SymDev sd, const double* __restrict__ vals,
                                 const double* __restrict__ D, Shifts sh,
                                 const double* __restrict__ b, const double* __restrict__ X, int R,
                                 double* __restrict__ Rk) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= sd.N) return;
  const int K = sh.K;
  const int KR = K * R;
  const int64_t pi = sd.iperm[i];
  const int64_t e0 = sd.row_ptr[i], e1 = sd.row_ptr[i + 1];
  const double di = D[i];
  for (int q = lane; q < KR; q += 32) {
    const int k = q / R, r = q % R;
    double a = b[i * R + r] - sh.t[k] * di * X[(pi * K + k) * R + r];
    for (int64_t e = e0; e < e1; ++e)
      a -= vals[e] * X[((int64_t)sd.iperm[sd.col[e]] * K + k) * R + r];
    Rk[(pi * K + k) * R + r] = a;
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
  for (int64_t e = sd.row_ptr[i]; e < sd.row_ptr[i + 1]; ++e) {
    const int64_t pj = sd.iperm[sd.col[e]];
    double a = 0.0;
    for (int q = lane; q < KR; q += 32) {
      const int k = q / R;
      a += sh.w[k] * Lam[pi * KR + q] * X[pj * KR + q];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) grad[e] = -a;
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
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(k_forward<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSolveSmem);
  cudaFuncSetAttribute(k_forward<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSolveSmem);
  cudaFuncSetAttribute(k_backward<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSolveSmem);
  cudaFuncSetAttribute(k_backward<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSolveSmem);
  done = true;
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
    const int rc = pick_rc(G.count, K, R, G.maxF, sizeof(T));
    const dim3 grid(G.count, K, (R + rc - 1) / rc);
    const size_t smem = (size_t)rc * G.maxF * sizeof(T);
    if (trans)
      k_forward<T, true><<<grid, kSolveThreads, smem, st>>>(sd, d_all + G.off, (const T*)fronts, rhs,
                                                            rhs_mode, (T*)V, R, K, rc);
    else
      k_forward<T, false><<<grid, kSolveThreads, smem, st>>>(sd, d_all + G.off, (const T*)fronts, rhs,
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
    const int rc = pick_rc(G.count, K, R, G.maxF, sizeof(T));
    const dim3 grid(G.count, K, (R + rc - 1) / rc);
    const size_t smem = (size_t)rc * G.maxF * sizeof(T);
    if (trans)
      k_backward<T, true><<<grid, kSolveThreads, smem, st>>>(sd, d_all + G.off, (const T*)fronts,
                                                             (const T*)V, out, acc, R, K, rc);
    else
      k_backward<T, false><<<grid, kSolveThreads, smem, st>>>(sd, d_all + G.off, (const T*)fronts,
                                                              (const T*)V, out, acc, R, K, rc);
    ++launches;
  }
  if (cudaGetLastError() != cudaSuccess) return -1;
  return launches;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int max_solve_front(int precision) { return kSolveSmem / (precision == PISP_FP32 ? 4 : 8); }

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

int launch_combine(const SymDev& sd, const double* X, const Shifts& sh, int32_t R, double* x,
                   cudaStream_t st) {
  const int64_t n = sd.N * R;
  if (n == 0) return 0;
  k_combine<<<blocks_for(n, 256), 256, 0, st>>>(sd, X, sh, R, x);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_residual_per_k(const SymDev& sd, const double* vals, const double* D,
                          const Shifts& sh, const double* b, const double* X, int32_t R,
                          double* Rk, cudaStream_t st) {
  if (sd.N == 0) return 0;
  k_residual_per_k<<<blocks_for(sd.N * 32, 256), 256, 0, st>>>(sd, vals, D, sh, b, X, R, Rk);
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
