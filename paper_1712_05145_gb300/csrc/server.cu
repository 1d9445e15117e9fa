// Continuous-batching request server for RVE solves (hom_server_*, see include/hom.h).
//
// Requests (a voxel RVE, an order, a tolerance) are queued on submission.  Worker threads,
// each owning one CUDA stream, admit queued requests first-fit against a device-memory budget
// (the estimate of hom_estimate_bytes), so a request that arrives while others run starts as
// soon as a worker and enough memory are free, and the kernels of all admitted requests overlap
// on the device through their streams.  A finished request releases its memory at once, which
// admits the next.  Every request runs the same handle-based solve as hom_create / hom_solve /
// hom_effective, so its result does not depend on what else was running.
#include <cuda_runtime.h>

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
  size_t est = 0;
  hom_result res{};
  double t_submit = 0, t_start = 0, t_end = 0;
};

}  // namespace

struct hom_server_ctx {
  int device = 0;
  size_t budget = 0, in_use = 0;
  int max_active = 1, active = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<ServerRequest*> queue;
  std::map<int64_t, std::unique_ptr<ServerRequest>> reqs;
  int64_t next_id = 1;
  bool stop = false;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
};

namespace {

// first queued request that fits the free budget (first-fit admission), removed from the queue
ServerRequest* take_fitting(hom_server_ctx* s) {
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
    if ((*it)->est + s->in_use <= s->budget) {
      ServerRequest* r = *it;
      s->queue.erase(it);
      return r;
    }
  }
  return nullptr;
}

bool any_fitting(const hom_server_ctx* s) {
  for (const ServerRequest* r : s->queue)
    if (r->est + s->in_use <= s->budget) return true;
  return false;
}

void run_request(ServerRequest* r, cudaStream_t stream) {
  hom_options o;
  hom_default_options(&o);
  o.precision = r->precision;
  o.scheme = r->scheme;
  o.cuda_stream = stream;
  hom_t h = nullptr;
  hom_result& res = r->res;
  hom_status st = hom_create(r->grid, r->phase.data(), (int32_t)(r->lame.size() / 2), r->lame.data(), r->lam0,
                             r->mu0, &o, &h);
  r->phase.clear();
  r->phase.shrink_to_fit();
  int iters = 0;
  if (st == HOM_OK) {
    hom_solve_info info[18] = {};
    st = hom_solve(h, 0, 6, nullptr, r->tol, info);
    for (int i = 0; i < 6; ++i) iters += info[i].iterations;
    if (st == HOM_OK) st = hom_effective(h, 0, res.c_eff);
    if (st == HOM_OK && r->order >= 1) {
      st = hom_solve(h, 1, 18, nullptr, r->tol, info);
      for (int i = 0; i < 18; ++i) iters += info[i].iterations;
      if (st == HOM_OK) st = hom_effective(h, 1, res.d1);
    }
  }
  if (st != HOM_OK) {
    const char* m = h ? hom_last_error(h) : hom_status_string(st);
    std::snprintf(res.message, sizeof(res.message), "%s", m ? m : "");
  }
  if (h) hom_destroy(h);
  res.status = st;
  res.iterations = iters;
  res.order = r->order;
}

void worker_main(hom_server_ctx* s, int wi) {
  cudaSetDevice(s->device);
  for (;;) {
    ServerRequest* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || any_fitting(s); });
      if (s->stop) return;
      r = take_fitting(s);
      if (!r) continue;
      s->in_use += r->est;
      s->active += 1;
      r->t_start = now_ms();
    }
    run_request(r, s->streams[wi]);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      r->t_end = now_ms();
      r->res.queue_ms = r->t_start - r->t_submit;
      r->res.run_ms = r->t_end - r->t_start;
      r->res.latency_ms = r->t_end - r->t_submit;
      r->res.done = 1;
      s->in_use -= r->est;
      s->active -= 1;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

HOM_API hom_status hom_server_create(int64_t budget_bytes, int32_t max_active, hom_server_t* out) {
  if (!out || max_active < 1 || max_active > 64) return HOM_ERR_ARG;
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
  s->streams.resize(max_active);
  for (int i = 0; i < max_active; ++i) {
    if (cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      for (int j = 0; j < i; ++j) cudaStreamDestroy(s->streams[j]);
      delete s;
      return HOM_ERR_CUDA;
    }
  }
  for (int i = 0; i < max_active; ++i) s->workers.emplace_back(worker_main, s, i);
  *out = s;
  return HOM_OK;
}

HOM_API hom_status hom_server_submit(hom_server_t s, const hom_request* q, int64_t* id) {
  if (!s || !q || !id || !q->phase || !q->lame || q->n_phase < 1 || q->n_phase > 256) return HOM_ERR_ARG;
  if (q->order < 0 || q->order > 1 || !(q->tol > 0)) return HOM_ERR_ARG;
  const long long M = (long long)q->grid[0] * q->grid[1] * q->grid[2];
  if (q->grid[0] < 1 || q->grid[1] < 1 || q->grid[2] < 1) return HOM_ERR_SIZE;
  const int64_t est = hom_estimate_bytes(q->grid, q->order, q->precision);
  if (est <= 0) return HOM_ERR_SIZE;
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
  r->est = (size_t)est;
  r->t_submit = now_ms();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if ((size_t)est > s->budget) return HOM_ERR_NOMEM;
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
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  delete s;
}

}  // extern "C"
