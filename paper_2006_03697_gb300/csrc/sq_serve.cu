// Request loop for energy / stress evaluations with continuous batching on one GPU.
//
// Requests (instance descriptors, inputs copied at submit) wait in a queue. A dispatcher
// admits requests in submission order as soon as the device bytes they need
// (sq_footprint_bytes) fit under the budget next to the requests in flight and a worker slot
// is free; admitted requests run their pipeline on their own worker thread and CUDA stream, so
// requests that arrive while others are on the GPU overlap with them. A request larger than
// the whole budget is answered with SQ_ERR_OOM without touching the device. Results are
// collected with sq_server_poll; each carries its latency from submit to completion.
//
// Trajectories (sq_server_submit_traj): the requests of one trajectory are successive
// snapshots of one cell. Its first request sets up a handle that stays resident on the device
// (buffers, stream, projector-table slots); later requests move the atoms and V_eff of that
// handle in place (sq_update_atoms) instead of a setup and a teardown. A trajectory runs one
// request at a time, in submission order; requests of other trajectories may overtake a
// request whose trajectory is busy. Idle resident handles count against the budget and are
// released, least recently used first, when a request needs their memory.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "sq_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  long long tag = 0;
  long long traj = -1;
  sq_instance_desc desc;
  std::vector<double> v, pos;
  std::vector<int> species, proj_offset;
  std::vector<sq_proj> proj;
  size_t bytes = 0;
  Clock::time_point t_submit;
};

// A trajectory's handle kept on the device between its requests.
struct Resident {
  sq_handle* h = nullptr;
  cudaStream_t st = nullptr;
  size_t bytes = 0;
  bool busy = false;
  long long last_use = 0;
  Request* shape = nullptr;   // the request that created it (descriptor fields reuse must match)
};

// Everything but the atom positions and V_eff must match for a request to reuse a handle.
bool same_shape(const Request& a, const Request& b) {
  const sq_instance_desc &x = a.desc, &y = b.desc;
  for (int i = 0; i < 3; ++i)
    if (x.L[i] != y.L[i] || x.n[i] != y.n[i]) return false;
  if (x.n_o != y.n_o || x.n_atoms != y.n_atoms || x.n_species != y.n_species || x.kT != y.kT || x.n_e != y.n_e ||
      x.r_cut != y.r_cut || x.n_pl != y.n_pl || x.precision != y.precision || x.bounds_mode != y.bounds_mode ||
      x.cheb_quad_M != y.cheb_quad_M || x.lanczos_k != y.lanczos_k || x.part_rank != y.part_rank ||
      x.part_count != y.part_count)
    return false;
  if (x.bounds_mode == SQ_BOUNDS_GIVEN && (x.lambda_lo != y.lambda_lo || x.lambda_hi != y.lambda_hi)) return false;
  if (a.species != b.species || a.proj_offset != b.proj_offset || a.proj.size() != b.proj.size()) return false;
  for (size_t i = 0; i < a.proj.size(); ++i)
    if (a.proj[i].l != b.proj[i].l || a.proj[i].width != b.proj[i].width || a.proj[i].gamma != b.proj[i].gamma ||
        a.proj[i].rcut != b.proj[i].rcut)
      return false;
  return true;
}

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
  std::map<long long, Resident> resident;
  long long clock = 0;
  size_t in_use = 0;                   // bytes of running requests and resident handles
  int inflight = 0;
  bool stop = false;
  std::thread dispatcher;
};

namespace {

void finish(sq_server* s, sq_result& res, Request* rq) {
  res.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - rq->t_submit).count();
  s->results.push_back(res);
  s->cv.notify_all();
  s->cv_done.notify_all();
}

void evaluate(sq_handle* h, sq_result& res, int rc) {
  sq::NvtxRange nvtx("served request");
  if (rc == SQ_OK) rc = sq_moments(h);
  if (rc == SQ_OK) rc = sq_fermi_level(h, &res.mu);
  if (rc == SQ_OK) rc = sq_density_energy_stress(h, res.mu, nullptr, &res.energies, res.sigma);
  if (rc != SQ_OK) std::strncpy(res.error, sq_last_error(h), sizeof(res.error) - 1);
  res.status = rc;
}

// A request without a trajectory: setup, evaluation, teardown.
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
  if (h) evaluate(h, res, rc);
  else {
    res.status = rc;
    std::strncpy(res.error, sq_last_error(nullptr), sizeof(res.error) - 1);
  }
  if (h) sq_destroy(h);
  if (st) cudaStreamDestroy(st);
  // everything that touches the server happens under its lock, so sq_server_destroy (which
  // waits for inflight == 0 under the same lock) never frees it while this thread uses it
  std::lock_guard<std::mutex> lk(s->mu);
  s->in_use -= rq->bytes;
  s->inflight -= 1;
  finish(s, res, rq);
  delete rq;
}

// A request of a trajectory on its resident handle (fresh: set it up first).
void run_traj(sq_server* s, Request* rq, Resident* r, bool fresh) {
  cudaSetDevice(s->device);
  sq_result res;
  std::memset(&res, 0, sizeof(res));
  res.tag = rq->tag;
  int rc = SQ_OK;
  if (fresh) {
    if (cudaStreamCreateWithFlags(&r->st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      r->st = nullptr;
      rc = SQ_ERR_CUDA;
    }
    if (rc == SQ_OK) {
      rq->desc.stream = r->st;
      rc = sq_setup(&rq->desc, &r->h);
    }
  } else {
    rc = sq_update_atoms(r->h, rq->pos.empty() ? nullptr : rq->pos.data(), rq->v.data());
  }
  if (r->h) evaluate(r->h, res, rc);
  else {
    res.status = rc;
    std::strncpy(res.error, sq_last_error(nullptr), sizeof(res.error) - 1);
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->inflight -= 1;
  r->busy = false;
  r->last_use = ++s->clock;
  finish(s, res, rq);
  if (fresh) r->shape = rq;     // kept: later requests are compared with it
  else delete rq;
  if (!r->h) {                  // setup failed: nothing stays resident
    if (r->st) cudaStreamDestroy(r->st);
    s->in_use -= r->bytes;
    delete r->shape;
    for (auto it = s->resident.begin(); it != s->resident.end(); ++it)
      if (&it->second == r) {
        s->resident.erase(it);
        break;
      }
  }
}

// Frees idle resident handles (least recently used first, never `keep`) until `need` more
// bytes fit under the budget; the handles to destroy are returned (destroyed off the lock).
bool make_room(sq_server* s, size_t need, long long keep, std::vector<Resident>& drop) {
  while (s->in_use + need > s->budget) {
    auto victim = s->resident.end();
    for (auto it = s->resident.begin(); it != s->resident.end(); ++it)
      if (!it->second.busy && it->first != keep && it->second.h &&
          (victim == s->resident.end() || it->second.last_use < victim->second.last_use))
        victim = it;
    if (victim == s->resident.end()) return false;
    s->in_use -= victim->second.bytes;
    drop.push_back(victim->second);
    s->resident.erase(victim);
  }
  return true;
}

void release(std::vector<Resident>& drop) {
  for (Resident& r : drop) {
    if (r.h) sq_destroy(r.h);
    if (r.st) cudaStreamDestroy(r.st);
    delete r.shape;
  }
  drop.clear();
}

void dispatch_loop(sq_server* s) {
  cudaSetDevice(s->device);   // released resident handles are destroyed on this thread
  std::unique_lock<std::mutex> lk(s->mu);
  std::vector<Resident> drop;
  for (;;) {
    bool progress = false;
    for (auto qi = s->queue.begin(); qi != s->queue.end();) {
      Request* rq = *qi;
      if (rq->bytes > s->budget) {   // can never fit: refuse
        sq_result res;
        std::memset(&res, 0, sizeof(res));
        res.tag = rq->tag;
        res.status = SQ_ERR_OOM;
        std::strncpy(res.error, "device footprint exceeds the server's budget", sizeof(res.error) - 1);
        finish(s, res, rq);
        delete rq;
        qi = s->queue.erase(qi);
        progress = true;
        continue;
      }
      if (s->inflight >= s->max_inflight) break;
      if (rq->traj >= 0) {
        auto it = s->resident.find(rq->traj);
        if (it != s->resident.end() && it->second.busy) {   // its trajectory is running: later
          ++qi;
          continue;
        }
        if (it != s->resident.end() && it->second.h && same_shape(*it->second.shape, *rq)) {
          Resident* r = &it->second;
          r->busy = true;
          s->inflight += 1;
          qi = s->queue.erase(qi);
          std::thread(run_traj, s, rq, r, false).detach();
          progress = true;
          continue;
        }
        if (it != s->resident.end()) {                      // another cell under the same id
          s->in_use -= it->second.bytes;
          drop.push_back(it->second);
          s->resident.erase(it);
        }
        if (!make_room(s, rq->bytes, rq->traj, drop)) break;   // waits for memory, in order
        Resident& r = s->resident[rq->traj];
        r.bytes = rq->bytes;
        r.busy = true;
        s->in_use += rq->bytes;
        s->inflight += 1;
        qi = s->queue.erase(qi);
        std::thread(run_traj, s, rq, &r, true).detach();
        progress = true;
        continue;
      }
      if (!make_room(s, rq->bytes, -1, drop)) break;
      s->in_use += rq->bytes;
      s->inflight += 1;
      qi = s->queue.erase(qi);
      std::thread(run_request, s, rq).detach();   // sq_server_destroy waits for inflight == 0
      progress = true;
    }
    if (!drop.empty()) {   // destroy released handles without holding the lock
      lk.unlock();
      release(drop);
      lk.lock();
      continue;
    }
    if (s->stop && s->queue.empty()) break;
    if (!progress) s->cv.wait(lk);
  }
}

int submit(sq_server* s, const sq_instance_desc* d, long long tag, long long traj) {
  if (!s || !d) return SQ_ERR_INVALID_ARG;
  const size_t bytes = sq_footprint_bytes(d);
  if (bytes == 0) return SQ_ERR_INVALID_ARG;   // the descriptor does not validate
  Request* rq = new Request();
  rq->tag = tag;
  rq->traj = traj;
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

int sq_server_submit(sq_server* s, const sq_instance_desc* d, long long tag) { return submit(s, d, tag, -1); }

int sq_server_submit_traj(sq_server* s, const sq_instance_desc* d, long long tag, long long traj) {
  if (traj < 0) return SQ_ERR_INVALID_ARG;
  return submit(s, d, tag, traj);
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

int sq_server_resident(sq_server* s) {
  if (!s) return -1;
  std::lock_guard<std::mutex> lk(s->mu);
  return int(s->resident.size());
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
  std::vector<Resident> drop;
  for (auto& kv : s->resident) drop.push_back(kv.second);
  s->resident.clear();
  lk.unlock();
  release(drop);
  delete s;
}

}  // extern "C"
