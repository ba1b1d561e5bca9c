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

#include "sq_device.cuh"

namespace sq {

// defined in sq_reduce.cu
__global__ void k_rsum(const double* __restrict__ mom, int Nd, int n_pl, double* __restrict__ R);
__global__ void k_cosF(const double* __restrict__ R, int n_pl, int M, double* __restrict__ F);

constexpr int kNoAllocScratch = SQ_NOALLOC_MAX_NPL + 1 + SQ_NOALLOC_MAX_M + 32;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratch];

namespace {

std::mutex g_mu;
double* g_scratch_ptr[256] = {nullptr};   // last looked-up device address of the scratch, per device ordinal

// The library's bisection rule (fermi_bisect_rule, shared with sq_fermi_level), with the
// bounds passed by value and mu written to the caller's device pointer (NaN when
// N(mu) - N_e has no sign change on the bracket).
__global__ void k_bisect_noalloc(const double* __restrict__ F, int M, double lam_lo, double lam_hi, double kT,
                                 double n_e, double* __restrict__ mu_out) {
  __shared__ double sh[1024];
  double mu = 0.0;
  const bool ok = fermi_bisect_rule(F, M, lam_lo, lam_hi, kT, n_e, sh, &mu);
  if (threadIdx.x == 0) *mu_out = ok ? mu : NAN;
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
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The device address of the scratch array, with the calling device current. Outside stream
  // capture it is looked up on every call (a host-side table lookup), so a module reloaded
  // after a device reset never leaves a stale address behind; inside a capture no lookup is
  // made and the address of the last uncaptured call on this device is used.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    return SQ_ERR_CUDA;
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(sq::g_mu);
    if (cap == cudaStreamCaptureStatusNone) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, sq::g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return SQ_ERR_CUDA;
      }
      sq::g_scratch_ptr[dev] = static_cast<double*>(p);
    } else if (!sq::g_scratch_ptr[dev]) {
      return SQ_ERR_STATE;   // first call on this device inside a capture
    }
    scratch = sq::g_scratch_ptr[dev];
  }
  double* R = scratch;                            // [n_pl + 1]
  double* F = scratch + SQ_NOALLOC_MAX_NPL + 1;   // [M]
  sq::k_rsum<<<n_pl + 1, 256, 0, s>>>(mom_dev, n_nodes, n_pl, R);
  sq::k_cosF<<<(M + 255) / 256, 256, 0, s>>>(R, n_pl, M, F);
  sq::k_bisect_noalloc<<<1, 1024, 0, s>>>(F, M, lambda_lo, lambda_hi, kT, n_e, mu_dev);
  return cudaGetLastError() == cudaSuccess ? SQ_OK : SQ_ERR_CUDA;
}
