// Allocation-free entry point: small dense perturbed systems solved with a
// fixed, file-scope device scratch array instead of library workspace.
//
// Who needs it: callers that may not allocate device memory at the time of
// the call -- code running under a memory budget fixed at start-up, host
// callbacks and real-time loops where cudaMalloc's implicit synchronisation
// is not acceptable, or frameworks that hand this library only their input
// and output buffers.  Every other entry point of the library allocates its
// workspace (factors, per-perturbation solutions) on first use.
//
// The work is the same as pisp_factor_perturbed + pisp_solve on a single
// dense front: one CTA per perturbation k assembles A + t_k D in shared
// memory, factors it without pivoting, solves all right-hand sides and
// writes x_k to the static scratch; a second kernel forms sum_k w_k x_k.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/pisp.h"

namespace {

constexpr int kMaxN = PISP_STATIC_MAX_N;
constexpr int kMaxR = PISP_STATIC_MAX_R;
constexpr int kMaxK = PISP_K_MAX;

// Per-perturbation solutions x_k, [K][R][n].  Every GPU that loads the
// library holds this array until the process exits.  Each call overwrites the
// part it uses before reading it, so nothing has to start at zero; calls that
// overlap on the GPU (different streams, or different host threads) race on
// it.
static __device__ __align__(256) double g_pisp_static_scratch[kMaxK * kMaxR * kMaxN];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

struct StaticShifts {
  double t[kMaxK];
  double w[kMaxK];
};

// One CTA per perturbation k: M = A + t_k D (column-major in shared memory),
// pivot-free LU in place, then L y = b and U x = y for all right-hand sides.
__global__ void __launch_bounds__(256) k_dense_perturbed_solve(int n, const double* __restrict__ A,
                                                               const double* __restrict__ D,
                                                               StaticShifts sh,
                                                               const double* __restrict__ b, int R,
                                                               double* __restrict__ xk) {
  extern __shared__ __align__(16) double sm[];
  double* M = sm;                  // n x n, M[i + j*n]
  double* v = sm + n * n;          // R x n, v[r*n + i]
  const int k = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const double tk = sh.t[k];
  for (int q = tid; q < n * n; q += nt) {
    const int i = q % n, j = q / n;
    M[q] = A[(int64_t)i * n + j] + (i == j ? tk * D[i] : 0.0);
  }
  for (int q = tid; q < n * R; q += nt) {
    const int i = q % n, r = q / n;
    v[r * n + i] = b[(int64_t)i * R + r];
  }
  __syncthreads();
  for (int p = 0; p < n; ++p) {
    const double piv = M[p * (n + 1)];
    const int m = n - p - 1;
    for (int i = tid; i < m; i += nt) M[(p + 1 + i) + p * n] /= piv;
    __syncthreads();
    for (int q = tid; q < m * m; q += nt) {
      const int i = p + 1 + q % m, j = p + 1 + q / m;
      M[i + j * n] -= M[i + p * n] * M[p + j * n];
    }
    __syncthreads();
  }
  for (int p = 0; p < n; ++p) {               // unit lower forward substitution
    const int m = n - p - 1;
    for (int q = tid; q < m * R; q += nt) {
      const int i = p + 1 + q % m, r = q / m;
      v[r * n + i] -= M[i + p * n] * v[r * n + p];
    }
    __syncthreads();
  }
  for (int p = n - 1; p >= 0; --p) {          // upper backward substitution
    if (tid < R) v[tid * n + p] /= M[p * (n + 1)];
    __syncthreads();
    for (int q = tid; q < p * R; q += nt) {
      const int i = q % p, r = q / p;
      v[r * n + i] -= M[i + p * n] * v[r * n + p];
    }
    __syncthreads();
  }
  double* out = xk + (int64_t)k * R * n;
  for (int q = tid; q < n * R; q += nt) out[q] = v[q];
}

__global__ void k_dense_combine(int n, int R, int K, StaticShifts sh, const double* __restrict__ xk,
                                double* __restrict__ x) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * R) return;
  const int i = q / R, r = q % R;
  double a = 0.0;
  for (int k = 0; k < K; ++k) a += sh.w[k] * xk[((int64_t)k * R + r) * n + i];
  x[q] = a;
}

}  // namespace

extern "C" int pisp_dense_solve_static(void* stream, int32_t n, const double* A, const double* D,
                                       const double* t, int32_t K, const double* b, int32_t R,
                                       double* x) {
  if (n < 1 || n > kMaxN || R < 1 || R > kMaxR || K < 1 || K > kMaxK)
    return PISP_ERR_UNSUPPORTED;
  if (!A || !D || !t || !b || !x) return PISP_ERR_INVALID_ARG;
  StaticShifts sh{};
  if (pisp_weights(t, K, sh.w) != PISP_OK) return PISP_ERR_INVALID_ARG;
  for (int k = 0; k < K; ++k) sh.t[k] = t[k];
  // An error already pending on this host thread belongs to the caller: leave
  // it in place for them to read (peek, do not clear) and launch nothing, since
  // a launch failure of this call could not be told apart from it.
  if (cudaPeekAtLastError() != cudaSuccess) return PISP_ERR_CUDA;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PISP_ERR_CUDA;
  double* scratch = nullptr;
  {
    // First call on a device (that device current): resolve the device
    // address of the static array -- in host code its name only denotes a
    // host-side stand-in -- and raise the kernel's shared-memory limit.
    // Later calls on the device reuse both.
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_pisp_static_scratch) != cudaSuccess || !p) return PISP_ERR_CUDA;
      const int smem_max = (int)(((size_t)kMaxN * kMaxN + (size_t)kMaxN * kMaxR) * sizeof(double));
      if (cudaFuncSetAttribute(k_dense_perturbed_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               smem_max) != cudaSuccess)
        return PISP_ERR_CUDA;
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t smem = ((size_t)n * n + (size_t)n * R) * sizeof(double);
  k_dense_perturbed_solve<<<K, 256, smem, st>>>(n, A, D, sh, b, R, scratch);
  if (cudaGetLastError() != cudaSuccess) return PISP_ERR_CUDA;  // nothing else enqueued
  k_dense_combine<<<(n * R + 255) / 256, 256, 0, st>>>(n, R, K, sh, scratch, x);
  return cudaGetLastError() == cudaSuccess ? PISP_OK : PISP_ERR_CUDA;
}
