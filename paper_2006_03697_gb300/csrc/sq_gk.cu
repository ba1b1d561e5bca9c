// Green-Kubo shear viscosity from a stress time series (Sec. 5.2, Eq. viscosity):
//   eta(t) = |Omega| / (k_B T) int_0^t (1/5) sum_i <s_i(t') s_i(0)> dt'
// with s_i the independent deviatoric components sigma_12, sigma_23, sigma_31,
// (sigma_11 - sigma_22)/2, (sigma_22 - sigma_33)/2. The average <.> is taken over every time
// origin of every trajectory; the time integral is the trapezoid rule on the sampled lags.
#include "sq_device.cuh"

namespace sq {

// s[traj][step][5] from sigma[traj][step][9] (row-major 3 x 3)
__global__ void k_gk_deviatoric(const double* __restrict__ sigma, long long n, double* __restrict__ s) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double* a = sigma + 9 * i;
    double* o = s + 5 * i;
    o[0] = a[1];
    o[1] = a[5];
    o[2] = a[6];
    o[3] = 0.5 * (a[0] - a[4]);
    o[4] = 0.5 * (a[4] - a[8]);
  }
}

// acf[k] = (1/5) mean over (traj, origin t < n_steps - k) of sum_i s_i(t + k) s_i(t); one block
// per lag, fixed-order block reduction (deterministic)
__global__ void __launch_bounds__(256) k_gk_acf(const double* __restrict__ s, int n_traj, int n_steps,
                                                double* __restrict__ acf) {
  __shared__ double sh[256];
  const int k = blockIdx.x;
  const int no = n_steps - k;
  double acc = 0.0;
  for (long long idx = threadIdx.x; idx < (long long)n_traj * no; idx += blockDim.x) {
    const int tr = int(idx / no), t = int(idx % no);
    const double* a = s + 5 * ((long long)tr * n_steps + t);
    const double* b = a + 5 * (long long)k;
#pragma unroll
    for (int i = 0; i < 5; ++i) acc += a[i] * b[i];
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) acf[k] = sh[0] / (5.0 * double(n_traj) * double(no));
}

// eta[k] = (|Omega| / kT) * trapezoid integral of acf over [0, k dt] (serial, fixed order)
__global__ void k_gk_integrate(const double* __restrict__ acf, int max_lag, double dt, double scale,
                               double* __restrict__ eta) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double run = 0.0;
  eta[0] = 0.0;
  for (int k = 1; k <= max_lag; ++k) {
    run += 0.5 * dt * (acf[k - 1] + acf[k]);
    eta[k] = scale * run;
  }
}

}  // namespace sq

extern "C" int sq_green_kubo(const double* sigma_host, int n_traj, int n_steps, double dt, double volume, double kT,
                  int max_lag, void* stream, double* eta_out, double* acf_out) {
  using sq::fail;
  if (!sigma_host || !eta_out) return fail(nullptr, SQ_ERR_INVALID_ARG, "sigma or eta_out is NULL");
  if (n_traj < 1 || n_steps < 2 || max_lag < 0 || max_lag >= n_steps)
    return fail(nullptr, SQ_ERR_INVALID_ARG, "need n_traj >= 1, n_steps >= 2, 0 <= max_lag < n_steps");
  if (!(dt > 0.0) || !(volume > 0.0) || !(kT > 0.0))
    return fail(nullptr, SQ_ERR_INVALID_ARG, "dt, volume and kT must be positive");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long n = (long long)n_traj * n_steps;
  double *d_sig = nullptr, *d_s = nullptr, *d_acf = nullptr, *d_eta = nullptr;
  int rc = SQ_OK;
  auto cleanup = [&]() {
    cudaFree(d_sig);
    cudaFree(d_s);
    cudaFree(d_acf);
    cudaFree(d_eta);
  };
  if (cudaMalloc(&d_sig, sizeof(double) * 9 * n) != cudaSuccess || cudaMalloc(&d_s, sizeof(double) * 5 * n) != cudaSuccess ||
      cudaMalloc(&d_acf, sizeof(double) * (max_lag + 1)) != cudaSuccess ||
      cudaMalloc(&d_eta, sizeof(double) * (max_lag + 1)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(nullptr, SQ_ERR_OOM, "device allocation for the stress series failed");
  }
  if (cudaMemcpyAsync(d_sig, sigma_host, sizeof(double) * 9 * n, cudaMemcpyHostToDevice, s) != cudaSuccess) rc = SQ_ERR_CUDA;
  if (rc == SQ_OK) {
    sq::k_gk_deviatoric<<<1024, 256, 0, s>>>(d_sig, n, d_s);
    sq::k_gk_acf<<<max_lag + 1, 256, 0, s>>>(d_s, n_traj, n_steps, d_acf);
    sq::k_gk_integrate<<<1, 32, 0, s>>>(d_acf, max_lag, dt, volume / kT, d_eta);
    if (cudaGetLastError() != cudaSuccess) rc = SQ_ERR_CUDA;
  }
  if (rc == SQ_OK && cudaMemcpyAsync(eta_out, d_eta, sizeof(double) * (max_lag + 1), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    rc = SQ_ERR_CUDA;
  if (rc == SQ_OK && acf_out &&
      cudaMemcpyAsync(acf_out, d_acf, sizeof(double) * (max_lag + 1), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    rc = SQ_ERR_CUDA;
  if (rc == SQ_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = SQ_ERR_CUDA;
  cleanup();
  if (rc != SQ_OK) return fail(nullptr, rc, "CUDA error in sq_green_kubo");
  return SQ_OK;
}
