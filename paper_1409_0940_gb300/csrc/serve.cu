// Serving loop: solve and scoring requests of different sizes admitted by device-
// memory budget, run side by side, models kept resident for scoring.
//
// A pool of worker threads (one per concurrently active request) takes requests
// from one queue.  A request is admitted as soon as a worker is free and its
// device memory fits the budget: a solve reserves its peak bytes (data, state,
// cached factors and set-up scratch, from rff_admm_estimate_bytes) and gives back
// the set-up part when its factors are ready; a scoring request needs its model
// to be solved.  Each admitted request runs on its own CUDA stream, so work of
// requests that arrived at different times overlaps on the device (continuous
// batching); results do not depend on what else runs, because every request owns
// its handle and the kernels are deterministic.  Completions carry queueing,
// running and total latency.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/rff_admm.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Model {
  rff_admm_t h = nullptr;
  size_t resident = 0;
  bool ready = false;
  bool failed = false;
  int64_t d = 0;
  int32_t m = 0;
  std::mutex use;   // one request at a time on a handle
  cudaStream_t score_stream = nullptr;   // highest priority: scoring is not queued behind solves
  ~Model() {
    if (h) rff_admm_destroy(h);
    if (score_stream) cudaStreamDestroy(score_stream);
  }
};

struct Request {
  int64_t id = 0;
  int32_t kind = 0;   // RFF_REQ_SOLVE or RFF_REQ_SCORE
  rff_admm_params params{};
  std::vector<float> X, Y;
  int64_t n = 0, d = 0;
  int32_t iters = 0;
  size_t peak = 0, resident = 0;
  int64_t model = 0;
  int64_t q = 0;
  float* out = nullptr;
  Clock::time_point t_submit;
};

}  // namespace

struct rff_server_s {
  int device = 0;
  size_t budget = 0, used = 0;
  int max_active = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::unique_ptr<Request>> queue;
  std::deque<rff_completion> done;
  std::map<int64_t, std::shared_ptr<Model>> models;
  std::vector<std::thread> workers;
  bool stop = false;
  int64_t next_id = 1;

  // first queued request that can start now (caller holds mu); null if none
  std::unique_ptr<Request> take_admissible() {
    for (auto it = queue.begin(); it != queue.end(); ++it) {
      Request& r = **it;
      bool ok = false;
      if (r.kind == RFF_REQ_SOLVE) {
        ok = used + r.peak <= budget;
      } else {
        auto m = models.find(r.model);
        if (m != models.end()) {
          ok = m->second->ready || m->second->failed;
        } else {
          // a model whose solve is still queued is waited for; an unknown one fails at once
          ok = true;
          for (auto& other : queue)
            if (other->kind == RFF_REQ_SOLVE && other->id == r.model) ok = false;
        }
      }
      if (ok) {
        std::unique_ptr<Request> out = std::move(*it);
        queue.erase(it);
        if (out->kind == RFF_REQ_SOLVE) used += out->peak;
        return out;
      }
    }
    return nullptr;
  }

  void complete(const Request& r, rff_status st, Clock::time_point t_start) {
    const auto t_end = Clock::now();
    rff_completion c{};
    c.id = r.id;
    c.kind = r.kind;
    c.status = st;
    c.queue_ms = ms_between(r.t_submit, t_start);
    c.run_ms = ms_between(t_start, t_end);
    c.latency_ms = ms_between(r.t_submit, t_end);
    std::lock_guard<std::mutex> lock(mu);
    done.push_back(c);
    cv_done.notify_all();
  }

  void run_solve(Request& r) {
    auto model = std::make_shared<Model>();
    model->d = r.d;
    model->m = r.params.m;
    model->resident = r.resident;
    {
      std::lock_guard<std::mutex> lock(mu);
      models[r.id] = model;
    }
    const auto t0 = Clock::now();
    rff_status st = rff_admm_create(&r.params, nullptr, &model->h);
    if (st == RFF_OK) st = rff_admm_set_memory_limit(model->h, r.peak);
    if (st == RFF_OK) st = rff_admm_set_data(model->h, r.X.data(), r.Y.data(), r.n, r.d, 0);
    if (st == RFF_OK) st = rff_admm_solve(model->h, r.iters, nullptr);
    if (st == RFF_OK) {
      // a solved model scores on a stream of the highest priority, so the blocks of its
      // scoring kernels are scheduled ahead of those of solves still running
      int lo = 0, hi = 0;
      if (cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess &&
          cudaStreamCreateWithPriority(&model->score_stream, cudaStreamNonBlocking, hi) == cudaSuccess)
        st = rff_admm_set_stream(model->h, model->score_stream);
      else
        cudaGetLastError();
    }
    std::vector<float>().swap(r.X);
    std::vector<float>().swap(r.Y);
    {
      std::lock_guard<std::mutex> lock(mu);
      // the set-up scratch is gone; a failed solve gives back everything
      used -= (st == RFF_OK) ? (r.peak - r.resident) : r.peak;
      if (st == RFF_OK) {
        model->ready = true;
      } else {
        model->failed = true;
        model->resident = 0;
      }
      cv_work.notify_all();
    }
    complete(r, st, t0);
  }

  void run_score(Request& r) {
    const auto t0 = Clock::now();
    std::shared_ptr<Model> model;
    {
      std::lock_guard<std::mutex> lock(mu);
      auto it = models.find(r.model);
      if (it != models.end()) model = it->second;
    }
    rff_status st = RFF_EINVAL;
    if (model && model->ready) {
      std::lock_guard<std::mutex> use(model->use);
      st = rff_admm_predict(model->h, r.X.data(), r.q, r.out, 0);
    } else if (model) {
      st = RFF_ENOTREADY;
    }
    complete(r, st, t0);
  }

  void worker() {
    cudaSetDevice(device);
    while (true) {
      std::unique_ptr<Request> r;
      {
        std::unique_lock<std::mutex> lock(mu);
        cv_work.wait(lock, [&] {
          if (stop) return true;
          r = take_admissible();
          return r != nullptr;
        });
        if (!r) return;   // stopping
      }
      if (r->kind == RFF_REQ_SOLVE) run_solve(*r);
      else run_score(*r);
      std::lock_guard<std::mutex> lock(mu);
      cv_work.notify_all();
    }
  }
};

extern "C" {

rff_status rff_server_create(size_t budget_bytes, int32_t max_active, rff_server_t* out) {
  if (!out || max_active < 1 || max_active > 256) return RFF_EINVAL;
  *out = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return RFF_ECUDA;
  }
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return RFF_ECUDA;
  }
  auto* s = new rff_server_s();
  s->device = dev;
  s->budget = budget_bytes ? std::min(budget_bytes, fr) : (size_t)(fr * 0.9);
  s->max_active = max_active;
  for (int i = 0; i < max_active; ++i) s->workers.emplace_back([s] { s->worker(); });
  *out = s;
  return RFF_OK;
}

rff_status rff_server_cancel(rff_server_t srv, int64_t request_id) {
  if (!srv) return RFF_EINVAL;
  std::unique_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    for (auto it = srv->queue.begin(); it != srv->queue.end(); ++it)
      if ((*it)->id == request_id) {
        r = std::move(*it);
        srv->queue.erase(it);
        break;
      }
    if (!r) return (request_id >= 1 && request_id < srv->next_id) ? RFF_ENOTREADY : RFF_EINVAL;
    srv->cv_work.notify_all();   // a score that waited on this solve can now be taken (and fail)
  }
  srv->complete(*r, RFF_ECANCELLED, Clock::now());
  return RFF_OK;
}

rff_status rff_server_submit_solve(rff_server_t srv, const rff_admm_params* params, const float* X, const float* Y,
                                   int64_t n, int64_t d, int32_t iters, int64_t* request_id) {
  if (!srv || !params || !X || !Y || iters < 0) return RFF_EINVAL;
  auto r = std::make_unique<Request>();
  const rff_status st = rff_admm_estimate_bytes(params, n, d, &r->resident, &r->peak);
  if (st != RFF_OK) return st;
  if (r->peak > srv->budget) return RFF_ENOMEM;   // could never be admitted
  r->kind = RFF_REQ_SOLVE;
  r->params = *params;
  r->X.assign(X, X + n * d);
  r->Y.assign(Y, Y + n * params->m);
  r->n = n;
  r->d = d;
  r->iters = iters;
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lock(srv->mu);
  r->id = srv->next_id++;
  if (request_id) *request_id = r->id;
  srv->queue.push_back(std::move(r));
  srv->cv_work.notify_all();
  return RFF_OK;
}

rff_status rff_server_submit_score(rff_server_t srv, int64_t model, const float* Xq, int64_t q, float* scores,
                                   int64_t* request_id) {
  if (!srv || q < 0 || (q > 0 && (!Xq || !scores))) return RFF_EINVAL;
  std::lock_guard<std::mutex> lock(srv->mu);
  auto it = srv->models.find(model);
  int64_t d = 0;
  if (it != srv->models.end()) {
    d = it->second->d;
  } else {
    // the solve may still be queued: take d from the queued request
    for (auto& r : srv->queue)
      if (r->kind == RFF_REQ_SOLVE && r->id == model) d = r->d;
  }
  if (d == 0) return RFF_EINVAL;
  auto r = std::make_unique<Request>();
  r->kind = RFF_REQ_SCORE;
  r->model = model;
  r->X.assign(Xq, Xq + q * d);
  r->q = q;
  r->out = scores;
  r->t_submit = Clock::now();
  r->id = srv->next_id++;
  if (request_id) *request_id = r->id;
  srv->queue.push_back(std::move(r));
  srv->cv_work.notify_all();
  return RFF_OK;
}

rff_status rff_server_poll(rff_server_t srv, rff_completion* out, int32_t max, int32_t* count, int32_t wait_ms) {
  if (!srv || !count || max < 0 || (max > 0 && !out)) return RFF_EINVAL;
  std::unique_lock<std::mutex> lock(srv->mu);
  if (srv->done.empty() && wait_ms > 0)
    srv->cv_done.wait_for(lock, std::chrono::milliseconds(wait_ms), [&] { return !srv->done.empty(); });
  int32_t k = 0;
  while (k < max && !srv->done.empty()) {
    out[k++] = srv->done.front();
    srv->done.pop_front();
  }
  *count = k;
  return RFF_OK;
}

rff_status rff_server_get_weights(rff_server_t srv, int64_t model, float* W) {
  if (!srv || !W) return RFF_EINVAL;
  std::shared_ptr<Model> m;
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    auto it = srv->models.find(model);
    if (it == srv->models.end()) return RFF_EINVAL;
    m = it->second;
  }
  if (!m->ready) return RFF_ENOTREADY;
  std::lock_guard<std::mutex> use(m->use);
  return rff_admm_get_weights(m->h, W, 0);
}

rff_status rff_server_release(rff_server_t srv, int64_t model) {
  if (!srv) return RFF_EINVAL;
  std::shared_ptr<Model> m;
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    auto it = srv->models.find(model);
    if (it == srv->models.end() || !(it->second->ready || it->second->failed)) return RFF_EINVAL;
    m = it->second;
    srv->models.erase(it);
    srv->used -= m->resident;
    srv->cv_work.notify_all();
  }
  std::lock_guard<std::mutex> use(m->use);   // a running scoring request finishes first
  return RFF_OK;
}

rff_status rff_server_memory(rff_server_t srv, size_t* used, size_t* budget) {
  if (!srv) return RFF_EINVAL;
  std::lock_guard<std::mutex> lock(srv->mu);
  if (used) *used = srv->used;
  if (budget) *budget = srv->budget;
  return RFF_OK;
}

void rff_server_destroy(rff_server_t srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->stop = true;
    srv->cv_work.notify_all();
  }
  for (auto& t : srv->workers) t.join();
  delete srv;
}

}  // extern "C"
