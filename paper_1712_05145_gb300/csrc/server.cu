// Continuous-batching request server for RVE solves (hom_server_*, see include/hom.h).
//
// Requests (a voxel RVE, an order, a tolerance) are queued on submission.  Worker threads admit
// queued requests as soon as a worker is free and the device-memory budget allows, so a request
// that arrives while others run starts without waiting for them:
//
//  * Batching.  An admitted order-0 request takes with it up to max_batch - 1 further queued
//    order-0 requests of the same grid, precision, scheme and tolerance.  They are solved in one
//    handle with one RVE slot each (hom_options.n_rve), so every Lippmann-Schwinger launch carries
//    the loads of all of them.  Each load's arithmetic is that of its RVE alone (per-load solver
//    state, per-slot material tables and reference media, per-load refinement decisions), so a
//    request gets the same result alone and in a batch.
//  * Resident handles.  Handles are kept per (grid, precision, scheme, slots) after use and
//    refilled with the next requests' microstructures by hom_set_rve, so steady-state admission
//    allocates no device memory.  Idle handles of other kinds are destroyed, least recently used
//    first, when a new kind does not fit the budget.
//  * Overlap.  Every handle runs on its own CUDA stream, so the launches of different grids and
//    of requests admitted by different workers overlap on the device.
//
// Order-1 requests run in one-slot handles (order 0, then order 1 from its correctors).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "hom.h"

namespace {

constexpr int kMaxBatch = 10;   // RVE slots of a handle (hom_options.n_rve)

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct ServerRequest {
  int64_t id = 0;
  int32_t grid[3] = {0, 0, 0};
  std::vector<uint8_t> phase;
  std::vector<double> lame;
  double lam0 = 0, mu0 = 0, tol = 1e-6;
  int32_t order = 0, precision = HOM_FP32_REFINE, scheme = HOM_CG;
  hom_result res{};
  double t_submit = 0, t_start = 0, t_end = 0;
};

// what a resident handle can serve: grid, precision, scheme, order (0, or 1 with its order 0) and
// RVE slots
struct Kind {
  int32_t grid[3];
  int32_t precision, scheme, order, slots;
  bool operator==(const Kind& o) const {
    return std::memcmp(grid, o.grid, sizeof(grid)) == 0 && precision == o.precision && scheme == o.scheme &&
           order == o.order && slots == o.slots;
  }
};

struct Resident {
  hom_t h = nullptr;
  Kind kind{};
  size_t bytes = 0;
  double last_use = 0;
};

}  // namespace

struct hom_server_ctx {
  int device = 0;
  size_t budget = 0, in_use = 0;
  int max_active = 1, active = 0, max_batch = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<ServerRequest*> queue;
  std::map<int64_t, std::unique_ptr<ServerRequest>> reqs;
  std::vector<Resident> idle;          // resident handles not in use
  int64_t next_id = 1;
  int64_t n_batches = 0, n_batched = 0, n_created = 0;
  bool stop = false;
  std::vector<std::thread> workers;
};

namespace {

// device bytes a new handle of kind k is expected to hold (its first solve included)
size_t kind_bytes(const Kind& k) {
  const int64_t one = hom_estimate_bytes(k.grid, k.order, k.precision);
  return one <= 0 ? 0 : (size_t)one * (size_t)k.slots;
}

// order-0 requests get handles of max_batch slots, fewer where the budget cannot hold that many
Kind kind_of(const hom_server_ctx* s, const ServerRequest* r) {
  Kind k{};
  std::memcpy(k.grid, r->grid, sizeof(k.grid));
  k.precision = r->precision;
  k.scheme = r->scheme;
  k.order = r->order;
  k.slots = 1;
  if (r->order == 0) {
    const size_t one = kind_bytes(k);
    const size_t fit = one > 0 ? s->budget / one : 1;
    k.slots = (int32_t)std::max<size_t>(1, std::min<size_t>((size_t)s->max_batch, fit));
  }
  return k;
}

bool same_batch(const ServerRequest* a, const ServerRequest* b) {
  return a->order == 0 && b->order == 0 && std::memcmp(a->grid, b->grid, sizeof(a->grid)) == 0 &&
         a->precision == b->precision && a->scheme == b->scheme && a->tol == b->tol;
}

// A unit of work taken from the queue under the lock: the requests, and either an idle resident
// handle or the bytes reserved for a new one.
struct Work {
  std::vector<ServerRequest*> reqs;
  Resident res;
  bool fresh = false;
  size_t reserved = 0;
};

// First queued request that can start (first-fit), with its batch.  Evicts least recently used idle
// handles of other kinds into `evicted` when a new handle would not fit otherwise.
bool take_work(hom_server_ctx* s, Work& w, std::vector<Resident>& evicted) {
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
    ServerRequest* r = *it;
    const Kind k = kind_of(s, r);
    int found = -1;
    for (size_t i = 0; i < s->idle.size(); ++i)
      if (s->idle[i].kind == k && (found < 0 || s->idle[i].last_use > s->idle[(size_t)found].last_use)) found = (int)i;
    if (found < 0) {
      const size_t need = kind_bytes(k);
      size_t freeable = 0;
      for (const Resident& x : s->idle) freeable += x.bytes;
      if (need == 0 || s->in_use + need > s->budget + freeable) continue;
      while (s->in_use + need > s->budget) {   // evict idle handles, least recently used first
        auto lru = std::min_element(s->idle.begin(), s->idle.end(),
                                    [](const Resident& a, const Resident& b) { return a.last_use < b.last_use; });
        s->in_use -= lru->bytes;
        evicted.push_back(*lru);
        s->idle.erase(lru);
      }
      s->in_use += need;
      w.fresh = true;
      w.reserved = need;
      w.res.kind = k;
    } else {
      w.res = s->idle[(size_t)found];
      s->idle.erase(s->idle.begin() + found);
    }
    w.reqs.push_back(r);
    s->queue.erase(it);
    // the rest of the batch: queued order-0 requests of the same grid, precision, scheme and tol
    if (r->order == 0) {
      for (auto jt = s->queue.begin(); jt != s->queue.end() && (int)w.reqs.size() < k.slots;) {
        if (same_batch(r, *jt)) {
          w.reqs.push_back(*jt);
          jt = s->queue.erase(jt);
        } else {
          ++jt;
        }
      }
    }
    return true;
  }
  return false;
}

void fail_all(Work& w, hom_status st, const char* msg) {
  for (ServerRequest* r : w.reqs) {
    r->res.status = st;
    std::snprintf(r->res.message, sizeof(r->res.message), "%s", msg ? msg : "");
  }
}

// Runs the requests of `w` on its handle (created here if fresh).  Returns false if the handle is
// unusable afterwards (it is then destroyed rather than kept resident).
bool run_work(Work& w) {
  ServerRequest* r0 = w.reqs.front();
  const int n = (int)w.reqs.size();
  hom_status st = HOM_OK;
  if (w.fresh) {
    hom_options o;
    hom_default_options(&o);
    o.precision = r0->precision;
    o.scheme = r0->scheme;
    o.n_rve = w.res.kind.slots;
    st = hom_create(r0->grid, r0->phase.data(), (int32_t)(r0->lame.size() / 2), r0->lame.data(), r0->lam0, r0->mu0,
                    &o, &w.res.h);
    if (st != HOM_OK) {
      w.res.h = nullptr;
      fail_all(w, st, hom_status_string(st));
      return false;
    }
  }
  hom_t h = w.res.h;
  for (int i = 0; i < n && st == HOM_OK; ++i) {
    ServerRequest* r = w.reqs[(size_t)i];
    st = hom_set_rve(h, i, r->phase.data(), (int32_t)(r->lame.size() / 2), r->lame.data(), r->lam0, r->mu0);
  }
  std::vector<hom_solve_info> info(6 * (size_t)n + 18);
  if (st == HOM_OK) st = hom_solve(h, 0, 6 * n, nullptr, r0->tol, info.data());
  std::vector<double> eff(36 * (size_t)n, 0.0);
  if (st == HOM_OK) st = hom_effective(h, 0, eff.data());
  if (st == HOM_OK) {
    for (int i = 0; i < n; ++i) {
      hom_result& res = w.reqs[(size_t)i]->res;
      int iters = 0;
      for (int j = 0; j < 6; ++j) iters += info[(size_t)(6 * i + j)].iterations;
      res.iterations = iters;
      for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) res.c_eff[a * 6 + b] = eff[(size_t)a * 6 * n + 6 * i + b];
    }
  }
  if (st == HOM_OK && r0->order >= 1) {   // one request per one-slot handle
    st = hom_solve(h, 1, 18, nullptr, r0->tol, info.data());
    for (int i = 0; i < 18; ++i) r0->res.iterations += info[(size_t)i].iterations;
    if (st == HOM_OK) st = hom_effective(h, 1, r0->res.d1);
  }
  for (ServerRequest* r : w.reqs) {
    r->res.status = st;
    r->res.order = r->order;
    if (st != HOM_OK) std::snprintf(r->res.message, sizeof(r->res.message), "%s", hom_last_error(h));
    r->phase.clear();
    r->phase.shrink_to_fit();
  }
  // a solve that stops at its iteration cap or on a NaN leaves the handle sound; a CUDA error may not
  return st == HOM_OK || st == HOM_ERR_NOT_CONVERGED || st == HOM_ERR_NUMERIC || st == HOM_ERR_ARG;
}

void worker_main(hom_server_ctx* s) {
  cudaSetDevice(s->device);
  for (;;) {
    Work w;
    std::vector<Resident> evicted;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || (!s->queue.empty() && take_work(s, w, evicted)); });
      if (s->stop && w.reqs.empty()) {
        for (const Resident& x : evicted) hom_destroy(x.h);
        return;
      }
      s->active += (int)w.reqs.size();
      s->n_batches += 1;
      s->n_batched += (int64_t)w.reqs.size();
      if (w.fresh) s->n_created += 1;
      const double t = now_ms();
      for (ServerRequest* r : w.reqs) r->t_start = t;
    }
    for (const Resident& x : evicted) hom_destroy(x.h);
    const bool keep = run_work(w);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      const double t = now_ms();
      for (ServerRequest* r : w.reqs) {
        r->t_end = t;
        r->res.queue_ms = r->t_start - r->t_submit;
        r->res.run_ms = r->t_end - r->t_start;
        r->res.latency_ms = r->t_end - r->t_submit;
        r->res.done = 1;
      }
      s->active -= (int)w.reqs.size();
      if (w.fresh) s->in_use -= w.reserved;
      else s->in_use -= w.res.bytes;
      if (keep && w.res.h) {
        w.res.bytes = (size_t)hom_device_bytes(w.res.h);
        w.res.last_use = t;
        s->in_use += w.res.bytes;
        s->idle.push_back(w.res);
        w.res.h = nullptr;
      }
    }
    if (w.res.h) hom_destroy(w.res.h);
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

HOM_API hom_status hom_server_create_batched(int64_t budget_bytes, int32_t max_active, int32_t max_batch,
                                             hom_server_t* out) {
  if (!out || max_active < 1 || max_active > 64 || max_batch < 1 || max_batch > kMaxBatch) return HOM_ERR_ARG;
  auto* s = new hom_server_ctx();
  cudaGetDevice(&s->device);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return HOM_ERR_CUDA;
  }
  const size_t cap = (size_t)(0.85 * (double)free_b);
  s->budget = (budget_bytes > 0 && (size_t)budget_bytes < cap) ? (size_t)budget_bytes : cap;
  s->max_active = max_active;
  s->max_batch = max_batch;
  for (int i = 0; i < max_active; ++i) s->workers.emplace_back(worker_main, s);
  *out = s;
  return HOM_OK;
}

HOM_API hom_status hom_server_create(int64_t budget_bytes, int32_t max_active, hom_server_t* out) {
  return hom_server_create_batched(budget_bytes, max_active, 8, out);
}

HOM_API hom_status hom_server_submit(hom_server_t s, const hom_request* q, int64_t* id) {
  if (!s || !q || !id || !q->phase || !q->lame || q->n_phase < 1 || q->n_phase > 256) return HOM_ERR_ARG;
  if (q->order < 0 || q->order > 1 || !(q->tol > 0)) return HOM_ERR_ARG;
  if (q->scheme != HOM_CG && q->scheme != HOM_BASIC && q->scheme != HOM_BICGSTAB) return HOM_ERR_ARG;
  const long long M = (long long)q->grid[0] * q->grid[1] * q->grid[2];
  if (q->grid[0] < 1 || q->grid[1] < 1 || q->grid[2] < 1) return HOM_ERR_SIZE;
  if (hom_estimate_bytes(q->grid, q->order, q->precision) <= 0) return HOM_ERR_SIZE;
  auto r = std::make_unique<ServerRequest>();
  std::memcpy(r->grid, q->grid, sizeof(r->grid));
  r->phase.assign(q->phase, q->phase + M);
  r->lame.assign(q->lame, q->lame + 2 * q->n_phase);
  r->lam0 = q->lambda0;
  r->mu0 = q->mu0;
  r->tol = q->tol;
  r->order = q->order;
  r->precision = q->precision;
  r->scheme = q->scheme;
  r->t_submit = now_ms();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (kind_bytes(kind_of(s, r.get())) > s->budget) return HOM_ERR_NOMEM;
    r->id = s->next_id++;
    *id = r->id;
    s->queue.push_back(r.get());
    s->reqs[r->id] = std::move(r);
  }
  s->cv_work.notify_one();
  return HOM_OK;
}

HOM_API hom_status hom_server_poll(hom_server_t s, int64_t id, hom_result* out) {
  if (!s || !out) return HOM_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return HOM_ERR_ARG;
  if (it->second->res.done) *out = it->second->res;
  else {
    std::memset(out, 0, sizeof(*out));
    out->done = 0;
  }
  return HOM_OK;
}

HOM_API hom_status hom_server_wait(hom_server_t s, int64_t id, hom_result* out) {
  if (!s || !out) return HOM_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return HOM_ERR_ARG;
  ServerRequest* r = it->second.get();
  s->cv_done.wait(lk, [&] { return r->res.done != 0; });
  *out = r->res;
  return HOM_OK;
}

HOM_API hom_status hom_server_stats(hom_server_t s, int64_t* queued, int64_t* running, int64_t* bytes_in_use) {
  if (!s) return HOM_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (queued) *queued = (int64_t)s->queue.size();
  if (running) *running = s->active;
  if (bytes_in_use) *bytes_in_use = (int64_t)s->in_use;
  return HOM_OK;
}

HOM_API hom_status hom_server_counters(hom_server_t s, int64_t* batches, int64_t* requests_run,
                                       int64_t* handles_created) {
  if (!s) return HOM_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (batches) *batches = s->n_batches;
  if (requests_run) *requests_run = s->n_batched;
  if (handles_created) *handles_created = s->n_created;
  return HOM_OK;
}

HOM_API void hom_server_destroy(hom_server_t s) {
  if (!s) return;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    // let queued and running requests finish
    s->cv_done.wait(lk, [&] { return s->queue.empty() && s->active == 0; });
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (const Resident& x : s->idle) hom_destroy(x.h);
  delete s;
}

}  // extern "C"
