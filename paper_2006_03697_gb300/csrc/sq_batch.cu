// Concurrent evaluation of many SQ instances (uneven quantum-MD snapshots) on one GPU.
//
// Each instance runs its whole pipeline - Lanczos bounds, Chebyshev sweep with moments,
// Fermi level, contraction - on its own host thread and its own CUDA stream, so the tile
// kernels of different instances overlap on the device while each instance's arithmetic
// (and hence its result) is exactly what it would be alone.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <thread>
#include <vector>

#include "sq_internal.h"

extern "C" int sq_batch_evaluate(sq_handle* const* hs, int n, int max_concurrent, double* mu_out,
                                 sq_energies* e_out, double* sigma_out) {
  if (n < 0 || (n > 0 && !hs)) return SQ_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    if (!hs[i]) return SQ_ERR_INVALID_ARG;
  if (n == 0) return SQ_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SQ_ERR_CUDA;
  const int nthr = std::max(1, std::min(n, max_concurrent > 0 ? max_concurrent : n));
  std::vector<int> rc(n, SQ_OK);
  std::atomic<int> next(0);
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (int i = next.fetch_add(1); i < n; i = next.fetch_add(1)) {
      sq_handle* h = hs[i];
      int r = sq_moments(h);
      double mu = 0.0;
      if (r == SQ_OK) r = sq_fermi_level(h, &mu);
      sq_energies e;
      std::memset(&e, 0, sizeof(e));
      double sig[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      if (r == SQ_OK) r = sq_density_energy_stress(h, mu, nullptr, &e, sig);
      rc[i] = r;
      if (mu_out) mu_out[i] = mu;
      if (e_out) e_out[i] = e;
      if (sigma_out) std::memcpy(sigma_out + 9 * (size_t)i, sig, sizeof(sig));
    }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < nthr; ++t) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  for (int i = 0; i < n; ++i)
    if (rc[i] != SQ_OK) return rc[i];
  return SQ_OK;
}
