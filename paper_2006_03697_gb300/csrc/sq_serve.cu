// Request loop for energy / stress evaluations with continuous batching on one GPU.
//
// Requests (instance descriptors, inputs copied at submit) wait in a FIFO. A dispatcher admits
// the oldest request as soon as the device bytes it needs (sq_footprint_bytes) fit under the
// budget next to the requests in flight and a worker slot is free; admitted requests run
// their whole pipeline on their own worker thread and CUDA stream, so requests that arrive
// while others are on the GPU overlap with them. A request larger than the whole budget is
// answered with SQ_ERR_OOM without touching the device. Results are collected with
// sq_server_poll; each carries its latency from submit to completion.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "sq_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  long long tag = 0;
  sq_instance_desc desc;
  std::vector<double> v, pos;
  std::vector<int> species, proj_offset;
  std::vector<sq_proj> proj;
  size_t bytes = 0;
  Clock::time_point t_submit;
};

}  // namespace

struct sq_server {
  size_t budget = 0;
  int max_inflight = 1;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;          // dispatcher wake-ups
  std::condition_variable cv_done;     // result arrivals
  std::deque<Request*> queue;
  std::deque<sq_result> results;
  size_t in_use = 0;
  int inflight = 0;
  bool stop = false;
  std::thread dispatcher;
};

namespace {

void run_request(sq_server* s, Request* rq) {
  cudaSetDevice(s->device);
  sq_result res;
  std::memset(&res, 0, sizeof(res));
  res.tag = rq->tag;
  cudaStream_t st = nullptr;
  int rc = (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess) ? SQ_OK : SQ_ERR_CUDA;
  sq_handle* h = nullptr;
  if (rc == SQ_OK) {
    rq->desc.stream = st;
    rc = sq_setup(&rq->desc, &h);
  }
  if (rc == SQ_OK) rc = sq_moments(h);
  if (rc == SQ_OK) rc = sq_fermi_level(h, &res.mu);
  if (rc == SQ_OK) rc = sq_density_energy_stress(h, res.mu, nullptr, &res.energies, res.sigma);
  if (rc != SQ_OK) std::strncpy(res.error, sq_last_error(h), sizeof(res.error) - 1);
  if (h) sq_destroy(h);
  if (st) cudaStreamDestroy(st);
  res.status = rc;
  res.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - rq->t_submit).count();
  const size_t bytes = rq->bytes;
  delete rq;
  // everything that touches the server happens under its lock, so sq_server_destroy (which
  // waits for inflight == 0 under the same lock) never frees it while this thread uses it
  std::lock_guard<std::mutex> lk(s->mu);
  s->in_use -= bytes;
  s->inflight -= 1;
  s->results.push_back(res);
  s->cv.notify_all();
  s->cv_done.notify_all();
}

void dispatch_loop(sq_server* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv.wait(lk, [&] {
      if (s->stop && s->queue.empty()) return true;
      if (s->queue.empty()) return false;
      const Request* rq = s->queue.front();
      return rq->bytes > s->budget ||
             (s->inflight < s->max_inflight && s->in_use + rq->bytes <= s->budget);
    });
    if (s->queue.empty()) break;   // stop requested and nothing left
    Request* rq = s->queue.front();
    s->queue.pop_front();
    if (rq->bytes > s->budget) {   // can never fit: refuse
      sq_result res;
      std::memset(&res, 0, sizeof(res));
      res.tag = rq->tag;
      res.status = SQ_ERR_OOM;
      std::strncpy(res.error, "device footprint exceeds the server's budget", sizeof(res.error) - 1);
      res.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - rq->t_submit).count();
      s->results.push_back(res);
      delete rq;
      s->cv_done.notify_all();
      continue;
    }
    s->in_use += rq->bytes;
    s->inflight += 1;
    std::thread(run_request, s, rq).detach();   // sq_server_destroy waits for inflight == 0
  }
}

}  // namespace

extern "C" {

int sq_server_create(size_t hbm_budget_bytes, int max_inflight, sq_server** out) {
  if (!out || hbm_budget_bytes == 0 || max_inflight < 1) return SQ_ERR_INVALID_ARG;
  sq_server* s = new sq_server();
  s->budget = hbm_budget_bytes;
  s->max_inflight = max_inflight;
  if (cudaGetDevice(&s->device) != cudaSuccess) {   // no device yet: refusals still work
    cudaGetLastError();
    s->device = 0;
  }
  s->dispatcher = std::thread(dispatch_loop, s);
  *out = s;
  return SQ_OK;
}

int sq_server_submit(sq_server* s, const sq_instance_desc* d, long long tag) {
  if (!s || !d) return SQ_ERR_INVALID_ARG;
  const size_t bytes = sq_footprint_bytes(d);
  if (bytes == 0) return SQ_ERR_INVALID_ARG;   // the descriptor does not validate
  Request* rq = new Request();
  rq->tag = tag;
  rq->desc = *d;
  const size_t nd = size_t(d->n[0]) * d->n[1] * d->n[2];
  rq->v.assign(d->v_eff, d->v_eff + nd);
  rq->desc.v_eff = rq->v.data();
  if (d->n_atoms > 0) {
    rq->pos.assign(d->pos, d->pos + 3 * size_t(d->n_atoms));
    rq->species.assign(d->species, d->species + d->n_atoms);
    rq->proj_offset.assign(d->proj_offset, d->proj_offset + d->n_species + 1);
    rq->proj.assign(d->proj, d->proj + d->proj_offset[d->n_species]);
    rq->desc.pos = rq->pos.data();
    rq->desc.species = rq->species.data();
    rq->desc.proj_offset = rq->proj_offset.data();
    rq->desc.proj = rq->proj.empty() ? nullptr : rq->proj.data();
  }
  rq->desc.stream = nullptr;
  rq->bytes = bytes;
  rq->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete rq;
      return SQ_ERR_STATE;
    }
    s->queue.push_back(rq);
  }
  s->cv.notify_all();
  return SQ_OK;
}

int sq_server_poll(sq_server* s, sq_result* out, int max_results, int timeout_ms, int* n_out) {
  if (!s || !n_out || (max_results > 0 && !out)) return SQ_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->results.empty() && timeout_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return !s->results.empty(); });
  int k = 0;
  while (k < max_results && !s->results.empty()) {
    out[k++] = s->results.front();
    s->results.pop_front();
  }
  *n_out = k;
  return SQ_OK;
}

int sq_server_pending(sq_server* s) {
  if (!s) return -1;
  std::lock_guard<std::mutex> lk(s->mu);
  return int(s->queue.size()) + s->inflight;
}

void sq_server_destroy(sq_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  s->dispatcher.join();
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv.wait(lk, [&] { return s->inflight == 0; });
  lk.unlock();
  delete s;
}

}  // extern "C"
