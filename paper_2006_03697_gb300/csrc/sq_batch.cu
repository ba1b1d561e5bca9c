// Evaluation of many SQ instances (uneven quantum-MD snapshots) on one GPU.
//
// sq_batch_evaluate: each instance runs its whole pipeline - Lanczos bounds, Chebyshev sweep
// with moments, Fermi level, contraction - on its own host thread and CUDA stream, so the tile
// kernels of different instances overlap on the device while each instance's arithmetic (and
// hence its result) is exactly what it would be alone.
//
// sq_batch_create / sq_batch_run: the same pipelines captured once into one CUDA graph, one
// branch per instance (forked from and joined into one stream), and launched as a single graph:
// no host round trip anywhere between the first Lanczos kernel and the last contraction kernel
// of any instance (the spectral scaling, the wave layout and the Fermi level stay on the
// device). After sq_update_atoms on member handles the graph is launched again as is, or
// captured anew when a wave layout needs more shared memory than the captured one.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <string>
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

struct sq_batch {
  std::vector<sq_handle*> hs;
  int chains = 0;                       // parallel branches of the graph (members round-robin)
  std::vector<std::vector<int>> rows;   // wave layouts the graph was captured with
  std::vector<std::vector<int>> recs;   // and the brick image counts (staged step)
  cudaStream_t s0 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> evs;
  std::string err;
};

namespace {

void drop_graph(sq_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// one handle's evaluation with nothing crossing to the host
int pipeline_device(sq_handle* h) {
  if (cudaMemsetAsync(h->d.status, 0, sizeof(int) * sq::kStCount, h->stream) != cudaSuccess)
    return sq::fail(h, SQ_ERR_CUDA, "status reset failed");
  int rc = SQ_OK;
  if (h->bounds_mode == SQ_BOUNDS_LANCZOS) {
    rc = sq::run_lanczos(h);
    if (rc != SQ_OK) return rc;
  } else {
    // given bounds: re-scale from scal[8], scal[9] (kept by set_bounds) after the status reset
    rc = sq::set_bounds_device(h);
    if (rc != SQ_OK) return rc;
  }
  rc = sq::run_sweep(h);
  if (rc != SQ_OK) return rc;
  return sq::run_fermi_contraction_device(h);
}

int capture(sq_batch* b) {
  drop_graph(b);
  const int n = int(b->hs.size());
  if (cudaStreamBeginCapture(b->s0, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    b->err = "cudaStreamBeginCapture failed";
    return SQ_ERR_CUDA;
  }
  int rc = SQ_OK;
  if (cudaEventRecord(b->evs[0], b->s0) != cudaSuccess) rc = SQ_ERR_CUDA;
  // members i, i + C, i + 2C, ... form chain i (each waits for the previous one of its chain);
  // the chains run side by side and all join the origin stream at the end
  const int C = std::max(1, std::min(n, b->chains > 0 ? b->chains : n));
  std::vector<cudaEvent_t> last(C, b->evs[0]);
  for (int i = 0; i < n && rc == SQ_OK; ++i) {
    sq_handle* h = b->hs[i];
    if (cudaStreamWaitEvent(h->stream, last[i % C], 0) != cudaSuccess) { rc = SQ_ERR_CUDA; break; }
    rc = pipeline_device(h);
    if (rc != SQ_OK) {
      b->err = std::string("instance ") + std::to_string(i) + ": " + sq_last_error(h);
      break;
    }
    if (cudaEventRecord(b->evs[i + 1], h->stream) != cudaSuccess) rc = SQ_ERR_CUDA;
    last[i % C] = b->evs[i + 1];
  }
  for (int c = 0; c < C && rc == SQ_OK; ++c)
    if (cudaStreamWaitEvent(b->s0, last[c], 0) != cudaSuccess) rc = SQ_ERR_CUDA;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->s0, &g);   // always leave capture mode
  if (rc == SQ_OK && e != cudaSuccess) rc = SQ_ERR_CUDA;
  if (rc != SQ_OK) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (b->err.empty()) b->err = "graph capture failed";
    return rc;
  }
  b->graph = g;
  if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) {
    cudaGetLastError();
    drop_graph(b);
    b->err = "cudaGraphInstantiate failed";
    return SQ_ERR_CUDA;
  }
  b->rows.clear();
  b->recs.clear();
  for (sq_handle* h : b->hs) {
    b->rows.push_back(h->wave_rows);
    b->recs.push_back(h->wave_recs);
  }
  return SQ_OK;
}

}  // namespace

extern "C" {

int sq_batch_create(sq_handle* const* hs, int n, sq_batch** out) {
  if (!out || n < 1 || !hs) return SQ_ERR_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!hs[i] || !hs[i]->stream) return SQ_ERR_INVALID_ARG;   // every member on its own stream
    if (hs[i]->bounds_mode == SQ_BOUNDS_PER_NODE) return SQ_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i] || hs[j]->stream == hs[i]->stream) return SQ_ERR_INVALID_ARG;
  }
  sq_batch* b = new sq_batch();
  b->hs.assign(hs, hs + n);
  int rc = SQ_OK;
  if (cudaStreamCreateWithFlags(&b->s0, cudaStreamNonBlocking) != cudaSuccess) rc = SQ_ERR_CUDA;
  b->evs.assign(n + 1, nullptr);
  for (int i = 0; i <= n && rc == SQ_OK; ++i)
    if (cudaEventCreateWithFlags(&b->evs[i], cudaEventDisableTiming) != cudaSuccess) rc = SQ_ERR_CUDA;
  // nothing of the members may still be running when the capture starts
  for (int i = 0; i < n && rc == SQ_OK; ++i)
    if (cudaStreamSynchronize(hs[i]->stream) != cudaSuccess) rc = SQ_ERR_CUDA;
  if (rc == SQ_OK) rc = capture(b);
  if (rc != SQ_OK) {
    cudaGetLastError();
    sq_batch_destroy(b);
    return rc;
  }
  *out = b;
  return SQ_OK;
}

int sq_batch_run(sq_batch* b, double* mu_out, sq_energies* e_out, double* sigma_out) {
  if (!b) return SQ_ERR_INVALID_ARG;
  sq::NvtxRange nvtx("sq_batch_run");
  const int n = int(b->hs.size());
  bool stale = !b->exec;
  for (int i = 0; i < n; ++i)
    for (size_t w = 0; w < b->hs[i]->wave_rows.size(); ++w)
      if (b->rows[i].size() != b->hs[i]->wave_rows.size() || b->hs[i]->wave_rows[w] > b->rows[i][w] ||
          b->recs[i].size() != b->hs[i]->wave_recs.size() || b->hs[i]->wave_recs[w] > b->recs[i][w])
        stale = true;
  if (stale) {
    const int rc = capture(b);
    if (rc != SQ_OK) return rc;
  }
  if (cudaGraphLaunch(b->exec, b->s0) != cudaSuccess || cudaStreamSynchronize(b->s0) != cudaSuccess) {
    cudaGetLastError();
    b->err = "graph launch failed";
    return SQ_ERR_CUDA;
  }
  int first = SQ_OK;
  for (int i = 0; i < n; ++i) {
    sq_handle* h = b->hs[i];
    double sc[31];
    int st[sq::kStCount];
    if (cudaMemcpy(sc, h->d.scal, sizeof(sc), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(st, h->d.status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return SQ_ERR_CUDA;
    }
    int rc = SQ_OK;
    if (st[sq::kStBadBounds]) rc = sq::fail(h, SQ_ERR_CUDA, "spectral bounds are not finite or empty");
    else if (st[sq::kStOverflow]) rc = sq::fail(h, SQ_ERR_CUDA, "internal list capacity exceeded");
    else if (st[sq::kStTimeout]) rc = sq::fail(h, SQ_ERR_TIMEOUT, "a staged step block's copy wait ran out");
    else if (st[sq::kStNoBracket]) rc = sq::fail(h, SQ_ERR_NO_BRACKET, "N(mu) - N_e has no sign change on the bisection bracket");
    h->bounds_ready = true;
    h->moments_ready = (rc == SQ_OK);
    if (rc != SQ_OK && first == SQ_OK) {
      first = rc;
      b->err = std::string("instance ") + std::to_string(i) + ": " + sq_last_error(h);
    }
    const double* o = sc + 16;
    if (mu_out) mu_out[i] = sc[2];
    if (e_out) {
      e_out[i].E_band = o[0];
      e_out[i].E_s = o[1];
      e_out[i].E_nl = o[2];
      e_out[i].F = o[0] + o[1];
      e_out[i].N_check = o[3];
      e_out[i].mu = sc[2];
    }
    if (sigma_out) std::memcpy(sigma_out + 9 * (size_t)i, o + 4, 9 * sizeof(double));
  }
  return first;
}

int sq_batch_set_chains(sq_batch* b, int chains) {
  if (!b || chains < 0) return SQ_ERR_INVALID_ARG;
  b->chains = chains;
  for (sq_handle* h : b->hs)
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
      cudaGetLastError();
      return SQ_ERR_CUDA;
    }
  return capture(b);
}

const char* sq_batch_last_error(const sq_batch* b) {
  if (!b) return "batch is NULL";
  return b->err.empty() ? "no error" : b->err.c_str();
}

void sq_batch_destroy(sq_batch* b) {
  if (!b) return;
  if (b->s0) cudaStreamSynchronize(b->s0);
  drop_graph(b);
  for (cudaEvent_t e : b->evs)
    if (e) cudaEventDestroy(e);
  if (b->s0) cudaStreamDestroy(b->s0);
  delete b;
}

}  // extern "C"
