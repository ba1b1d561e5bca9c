// Fermi level from a caller-owned moment table without any device allocation.
//
// Some callers cannot call cudaMalloc: code running while an allocator is locked or inside
// a memory-pool budget that forbids growth, plug-ins that must not touch the process's device
// heap, or host threads that already hold every byte of HBM they were given. For them this
// entry point keeps its scratch (the node sums R^j, the cosine sums F_k and a status word) in
// one file-scope __device__ array of fixed size, which every GPU that loads the library holds
// until the process exits. The scratch is fully rewritten by each call, so nothing in it has
// to start at zero; calls that overlap on the GPU (different streams, or several host threads)
// share the array and race.
#include <cmath>
#include <mutex>

#include "sq_internal.h"

namespace sq {

// defined in sq_reduce.cu
__global__ void k_rsum(const double* __restrict__ mom, int Nd, int n_pl, double* __restrict__ R);
__global__ void k_cosF(const double* __restrict__ R, int n_pl, int M, double* __restrict__ F);

constexpr int kNoAllocScratch = SQ_NOALLOC_MAX_NPL + 1 + SQ_NOALLOC_MAX_M + 32;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratch];

namespace {

std::mutex g_mu;
double* g_scratch_ptr[256] = {nullptr};   // device address of the scratch, per device ordinal

__device__ __forceinline__ double fermi_na(double x) {
  const double ex = exp(-fabs(x));
  return (x > 0.0) ? ex / (1.0 + ex) : 1.0 / (1.0 + ex);
}

__device__ double sum_block(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__device__ double count_na(const double* F, int M, double chi_q, double zeta_q, double kT, double mu, double* sh) {
  double s = 0.0;
  for (int k = threadIdx.x; k < M; k += blockDim.x)
    s += fermi_na((chi_q + zeta_q * cos(M_PI * (k + 0.5) / M) - mu) / kT) * F[k];
  return 4.0 / M * sum_block(s, sh);
}

// Same bisection rule as sq_fermi_level, with the bounds passed by value and mu written to
// the caller's device pointer (NaN when N(mu) - N_e has no sign change on the bracket).
__global__ void k_bisect_noalloc(const double* __restrict__ F, int M, double lam_lo, double lam_hi, double kT,
                                 double n_e, double* __restrict__ mu_out) {
  __shared__ double sh[1024];
  const double chi_q = 0.5 * (lam_hi + lam_lo), zeta_q = 0.5 * (lam_hi - lam_lo);
  double lo = lam_lo - 40.0 * kT, hi = lam_hi + 40.0 * kT;
  const double nlo = count_na(F, M, chi_q, zeta_q, kT, lo, sh);
  const double nhi = count_na(F, M, chi_q, zeta_q, kT, hi, sh);
  if (!(nlo < n_e && n_e < nhi)) {
    if (threadIdx.x == 0) *mu_out = NAN;
    return;
  }
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count_na(F, M, chi_q, zeta_q, kT, mid, sh) < n_e) lo = mid;
    else hi = mid;
    if (hi - lo < 1e-13 * fmax(1.0, fabs(mid))) break;
  }
  if (threadIdx.x == 0) *mu_out = 0.5 * (lo + hi);
}

}  // namespace
}  // namespace sq

extern "C" int sq_fermi_level_noalloc(const double* mom_dev, int n_nodes, int n_pl, double lambda_lo,
                                      double lambda_hi, double kT, double n_e, int cheb_quad_M, void* stream,
                                      double* mu_dev) {
  const int M = cheb_quad_M > 0 ? cheb_quad_M : 2048;
  if (!mom_dev || !mu_dev || n_nodes < 1 || n_pl < 1 || n_pl > SQ_NOALLOC_MAX_NPL || M > SQ_NOALLOC_MAX_M ||
      !(lambda_lo < lambda_hi) || !std::isfinite(lambda_lo) || !std::isfinite(lambda_hi) || !(kT > 0.0) ||
      !std::isfinite(kT) || !(n_e > 0.0) || !(n_e < 2.0 * double(n_nodes)))
    return SQ_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return SQ_ERR_CUDA;
  double* scratch = nullptr;
  {
    // once per device, with that device current: the device address of the scratch array
    std::lock_guard<std::mutex> lock(sq::g_mu);
    if (!sq::g_scratch_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, sq::g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return SQ_ERR_CUDA;
      }
      sq::g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scratch = sq::g_scratch_ptr[dev];
  }
  double* R = scratch;                            // [n_pl + 1]
  double* F = scratch + SQ_NOALLOC_MAX_NPL + 1;   // [M]
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  sq::k_rsum<<<n_pl + 1, 256, 0, s>>>(mom_dev, n_nodes, n_pl, R);
  sq::k_cosF<<<(M + 255) / 256, 256, 0, s>>>(R, n_pl, M, F);
  sq::k_bisect_noalloc<<<1, 1024, 0, s>>>(F, M, lambda_lo, lambda_hi, kT, n_e, mu_dev);
  return cudaGetLastError() == cudaSuccess ? SQ_OK : SQ_ERR_CUDA;
}
