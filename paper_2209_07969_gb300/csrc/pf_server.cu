// Continuous-batching request server of libpf (host code; C ABI in include/pf.h).
//
// `slots` worker threads share one FIFO queue.  A worker takes the queue head when the
// head's device footprint fits in the budget left by the running simulations, runs its
// whole load path on its own pf_ctx (own CUDA stream), and returns the reserved bytes.
// The head blocks the queue (first come, first served).  Per-request results (reaction and
// staggered passes per step, device time per step) are kept until the request is released
// or the server destroyed.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pf.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
  int64_t id = 0;
  pf_mesh mesh{};
  std::vector<uint8_t> flags, active;
  double E = 0, nu = 0, Gc = 0, l = 0, k_res = 0;
  std::vector<double> increments;
  int scheme = PF_ST;
  double tol = 0;
  pf_options opt{};
  size_t footprint = 0;
  // progress, guarded by the server mutex
  int state = PF_REQ_QUEUED;
  int status = PF_OK;
  bool cancel = false;
  int64_t admit_seq = -1;
  std::vector<double> reactions, step_ms;
  std::vector<int> stag_iters;
  int converged = 0;
  Clock::time_point t_submit, t_start, t_end;
};

}  // namespace

struct pf_server {
  int device = 0;
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request *> queue;
  std::map<int64_t, std::unique_ptr<Request>> reqs;
  size_t in_use = 0, peak_in_use = 0;
  int running = 0, peak_running = 0;
  int64_t next_id = 1, next_admit = 0;
  bool closing = false, paused = false;
  std::vector<std::thread> workers;
};

namespace {

// Run one request's load path on the worker's thread (no lock held).  The final state is
// returned, not published: the worker publishes it in the same critical section that
// returns the request's footprint, because a client may release a finished request (and
// free its record) as soon as it sees the final state.
struct Outcome {
  int state, status;
};

Outcome run_request(pf_server *s, Request *r) {
  cudaSetDevice(s->device);
  pf_ctx *ctx = nullptr;
  pf_status st = pf_create(&r->mesh, r->E, r->nu, r->Gc, r->l, r->k_res, &ctx);
  if (st == PF_OK) st = pf_set_options(ctx, &r->opt);
  bool stopped = false;
  if (st == PF_OK) {
    for (size_t k = 0; k < r->increments.size(); ++k) {
      {
        std::lock_guard<std::mutex> lk(s->mu);
        if (r->cancel) {
          stopped = true;
          break;
        }
      }
      pf_step_result res{};
      const pf_status ss = pf_load_step(ctx, r->increments[k], r->scheme, r->tol, &res);
      if (ss != PF_OK && ss != PF_ENOTCONV) {
        st = ss;
        break;
      }
      std::lock_guard<std::mutex> lk(s->mu);
      r->reactions.push_back(res.reaction);
      r->stag_iters.push_back(res.stag_iters);
      r->step_ms.push_back(res.ms);
      r->converged += res.converged ? 1 : 0;
    }
  }
  if (ctx) pf_destroy(ctx);
  return {st != PF_OK ? PF_REQ_FAILED : stopped ? PF_REQ_CANCELLED : PF_REQ_DONE, (int)st};
}

void worker(pf_server *s) {
  for (;;) {
    Request *r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->closing) return;
        if (!s->paused && !s->queue.empty() &&
            s->in_use + s->queue.front()->footprint <= s->budget) {
          r = s->queue.front();
          s->queue.pop_front();
          s->in_use += r->footprint;
          s->running += 1;
          s->peak_in_use = std::max(s->peak_in_use, s->in_use);
          s->peak_running = std::max(s->peak_running, s->running);
          r->state = PF_REQ_RUNNING;
          r->admit_seq = s->next_admit++;
          r->t_start = Clock::now();
          break;
        }
        s->cv.wait(lk);
      }
    }
    const Outcome o = run_request(s, r);
    {
      // r may be released by a client right after this block: nothing touches it later
      std::lock_guard<std::mutex> lk(s->mu);
      s->in_use -= r->footprint;
      s->running -= 1;
      r->status = o.status;
      r->state = o.state;
      r->t_end = Clock::now();
    }
    s->cv.notify_all();
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  size_t i = (size_t)(q * (double)v.size());
  if (i >= v.size()) i = v.size() - 1;
  return v[i];
}

}  // namespace

extern "C" {

pf_status pf_server_create(size_t hbm_budget, int slots, pf_server **out) {
  if (!out) return PF_EINVAL;
  *out = nullptr;
  if (hbm_budget == 0 || slots < 1 || slots > 4096) return PF_EINVAL;
  pf_server *s = new (std::nothrow) pf_server();
  if (!s) return PF_ENOMEM;
  if (cudaGetDevice(&s->device) != cudaSuccess) s->device = 0;
  s->budget = hbm_budget;
  try {
    for (int i = 0; i < slots; ++i) s->workers.emplace_back(worker, s);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->closing = true;
    }
    s->cv.notify_all();
    for (std::thread &t : s->workers) t.join();
    delete s;
    return PF_ENOMEM;
  }
  *out = s;
  return PF_OK;
}

pf_status pf_server_submit(pf_server *s, const pf_request *req, int64_t *id) {
  if (!s || !req || !id) return PF_EINVAL;
  const pf_mesh &m = req->mesh;
  if (!m.node_flags || m.nx < 1 || m.ny < 1 || !req->increments || req->n_steps < 1 ||
      req->scheme < PF_ST || req->scheme > PF_S3 || !(req->tol > 0.0))
    return PF_EINVAL;
  const size_t fp = pf_footprint_bytes(&m);
  if (fp == 0 || fp > s->budget) return PF_EINVAL;
  std::unique_ptr<Request> r(new (std::nothrow) Request());
  if (!r) return PF_ENOMEM;
  try {
    const size_t nn = (size_t)(m.nx + 1) * (m.ny + 1), ne = (size_t)m.nx * m.ny;
    r->flags.assign(m.node_flags, m.node_flags + nn);
    if (m.elem_active) r->active.assign(m.elem_active, m.elem_active + ne);
    r->increments.assign(req->increments, req->increments + req->n_steps);
    r->reactions.reserve(req->n_steps);
    r->stag_iters.reserve(req->n_steps);
    r->step_ms.reserve(req->n_steps);
  } catch (...) {
    return PF_ENOMEM;
  }
  r->mesh = m;
  r->mesh.node_flags = r->flags.data();
  r->mesh.elem_active = m.elem_active ? r->active.data() : nullptr;
  r->E = req->E;
  r->nu = req->nu;
  r->Gc = req->Gc;
  r->l = req->l;
  r->k_res = req->k_res;
  r->scheme = req->scheme;
  r->tol = req->tol;
  if (req->options)
    r->opt = *req->options;
  else
    pf_default_options(&r->opt);
  r->footprint = fp;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->closing) return PF_EBUSY;
    const int64_t rid = s->next_id++;
    r->id = rid;
    r->t_submit = Clock::now();
    *id = rid;
    s->queue.push_back(r.get());
    s->reqs[rid] = std::move(r);
  }
  s->cv.notify_all();
  return PF_OK;
}

pf_status pf_server_poll(pf_server *s, int64_t id, pf_request_info *info, double *reactions,
                         int *stag_iters) {
  if (!s) return PF_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return PF_EINVAL;
  const Request &r = *it->second;
  if (info) {
    const Clock::time_point now = Clock::now();
    info->state = r.state;
    info->status = r.status;
    info->steps_done = (int)r.reactions.size();
    info->steps_converged = r.converged;
    info->admit_seq = r.admit_seq;
    info->footprint = r.footprint;
    info->queue_ms = r.state == PF_REQ_QUEUED ? ms_between(r.t_submit, now)
                                              : ms_between(r.t_submit, r.t_start);
    const bool done = r.state >= PF_REQ_DONE;   // done, failed or cancelled
    info->path_ms = done ? ms_between(r.t_submit, r.t_end) : 0.0;
    info->step_ms_p50 = percentile(r.step_ms, 0.5);
    info->step_ms_p99 = percentile(r.step_ms, 0.99);
  }
  for (size_t k = 0; k < r.reactions.size(); ++k) {
    if (reactions) reactions[k] = r.reactions[k];
    if (stag_iters) stag_iters[k] = r.stag_iters[k];
  }
  return PF_OK;
}

pf_status pf_server_drain(pf_server *s, double timeout_s) {
  if (!s) return PF_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto idle = [s]() { return s->queue.empty() && s->running == 0; };
  if (timeout_s < 0.0) {
    s->cv.wait(lk, idle);
    return PF_OK;
  }
  const auto limit = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                        std::chrono::duration<double>(timeout_s));
  return s->cv.wait_until(lk, limit, idle) ? PF_OK : PF_ETIMEOUT;
}

pf_status pf_server_stats(pf_server *s, size_t *peak_bytes, int *peak_running) {
  if (!s) return PF_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (peak_bytes) *peak_bytes = s->peak_in_use;
  if (peak_running) *peak_running = s->peak_running;
  return PF_OK;
}

pf_status pf_server_cancel(pf_server *s, int64_t id) {
  if (!s) return PF_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return PF_EINVAL;
    Request *r = it->second.get();
    if (r->state == PF_REQ_QUEUED) {
      s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
      r->state = PF_REQ_CANCELLED;
      r->t_start = r->t_end = Clock::now();
    } else if (r->state == PF_REQ_RUNNING) {
      r->cancel = true;
    }
  }
  s->cv.notify_all();
  return PF_OK;
}

pf_status pf_server_release(pf_server *s, int64_t id) {
  if (!s) return PF_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return PF_EINVAL;
  if (it->second->state < PF_REQ_DONE) return PF_EBUSY;
  s->reqs.erase(it);
  return PF_OK;
}

pf_status pf_server_pause(pf_server *s, int paused) {
  if (!s) return PF_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->paused = paused != 0;
  }
  s->cv.notify_all();
  return PF_OK;
}

void pf_server_destroy(pf_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->closing = true;
  }
  s->cv.notify_all();
  for (std::thread &t : s->workers) t.join();
  delete s;
}

}  // extern "C"
