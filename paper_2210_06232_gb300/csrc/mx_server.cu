// Serving form (C ABI): a request loop that solves problems of different
// grids, eps/mu, precisions and end times as they arrive.
//
// A worker thread admits queued requests while the HBM budget and the slot
// limit allow, each into a resident spectral-form context taken from a pool
// of contexts of its shape (or created; idle contexts are destroyed, least
// recently used first, when a new shape needs the memory).  Every context
// owns a CUDA stream, so the load (host->device copy + 3D forward transform),
// the steps and the read-out (inverse transform + device->host copy) of
// different requests overlap on the device, and a request admitted while
// others run starts at once.  Completion is detected with an event per
// request; latency is completion minus submission, on the host clock.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "mx_ctx.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  long long id;
  mx_request r;
  Clock::time_point t_submit, t_admit, t_done;
  int state = 0;  // 0 queued, 1 running, 2 done, < 0 failed (-status)
  mx_ctx* ctx = nullptr;
  cudaEvent_t done_ev = nullptr;
  size_t bytes = 0;
  std::vector<mx_invariants> inv;
};

struct PoolEntry {
  mx_ctx* ctx;
  size_t bytes;
  std::string key;
  Clock::time_point last_used;
};

// Contexts are pooled by everything their buffers and tables depend on:
// precision, grid and domain (eps and mu are set per request).
std::string shape_key(const mx_request& r) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%d:%d:%d:%d:%.17g:%.17g:%.17g:%.17g:%.17g:%.17g", r.precision, r.nx, r.ny, r.nz, r.lo[0],
           r.lo[1], r.lo[2], r.hi[0], r.hi[1], r.hi[2]);
  return std::string(buf);
}

void destroy_ctx(mx_ctx* c) {
  cudaStream_t st = c->stream;
  mx_destroy(c);
  if (st) cudaStreamDestroy(st);
}

}  // namespace

struct mx_server {
  size_t budget = 0;
  int max_active = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<long long> queue;
  std::map<long long, Req*> reqs;
  std::vector<Req*> active;
  std::list<PoolEntry> idle;  // front = least recently used
  size_t in_use = 0, high_water = 0;
  long long next_id = 1;
  long long admitted = 0, completed = 0, rejected = 0;
  // device concurrency: time-weighted count of admitted, unfinished requests
  Clock::time_point last_change = Clock::now();
  double busy_s = 0.0, conc_area = 0.0, request_s_sum = 0.0;
  long long max_conc = 0;
  bool stop = false;
  int device = 0;
  std::thread worker;
};

namespace {

size_t req_bytes(const mx_request& r) {
  size_t b = 0;
  if (mx_footprint_bytes(r.nx, r.ny, r.nz, r.precision, MX_FORM_SPECTRAL, &b) != MX_OK) return 0;
  return b;
}

// Take or make a context for r; caller holds the lock.  Returns nullptr when the
// budget does not allow it now.
mx_ctx* acquire_ctx(mx_server* s, Req* q, mx_status* err) {
  const std::string key = shape_key(q->r);
  for (auto it = s->idle.begin(); it != s->idle.end(); ++it) {
    if (it->key == key) {
      mx_ctx* c = it->ctx;
      // the pooled context keeps its grid; eps, mu and domain are per request
      q->bytes = it->bytes;
      s->idle.erase(it);
      *err = MX_OK;
      return c;
    }
  }
  const size_t need = req_bytes(q->r);
  if (need == 0) {
    *err = MX_E_INVAL;
    return nullptr;
  }
  if (need > s->budget) {
    *err = MX_E_NOMEM;
    return nullptr;
  }
  while (s->in_use + need > s->budget && !s->idle.empty()) {  // evict least recently used idle contexts
    PoolEntry e = s->idle.front();
    s->idle.pop_front();
    destroy_ctx(e.ctx);
    s->in_use -= e.bytes;
  }
  if (s->in_use + need > s->budget) {
    *err = MX_OK;
    return nullptr;  // wait for memory
  }
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    *err = MX_E_CUDA;
    return nullptr;
  }
  mx_ctx* c = nullptr;
  mx_status cs = mx_create(&c, q->r.nx, q->r.ny, q->r.nz, q->r.lo, q->r.hi, q->r.eps, q->r.mu, q->r.precision,
                           MX_FORM_SPECTRAL, st);
  if (cs != MX_OK) {
    cudaStreamDestroy(st);
    *err = cs;
    return nullptr;
  }
  mx_autotune(c);  // first context of a shape picks its FFT schedules (cached per process)
  s->in_use += need;
  s->high_water = std::max(s->high_water, s->in_use);
  q->bytes = need;
  *err = MX_OK;
  return c;
}

void release_ctx(mx_server* s, Req* q) {
  PoolEntry e{q->ctx, q->bytes, shape_key(q->r), Clock::now()};
  s->idle.push_back(e);
  q->ctx = nullptr;
}

// Enqueue load, steps and read of request q on its context's stream.
mx_status launch_request(Req* q) {
  mx_ctx* c = q->ctx;
  // per-request eps and mu on a pooled context of the right grid and domain
  c->eps = q->r.eps;
  c->mu = q->r.mu;
  mx::set_material(c->g, q->r.eps, q->r.mu);
  c->tab_t = NAN;  // coefficients depend on eps, mu and the domain
  mx_status st = mx_load_fields_async(c, q->r.E0, q->r.H0);
  if (st != MX_OK) return st;
  const long long n = q->r.nsteps;
  st = mx_step(c, q->r.t_end / (double)n, n, q->r.invariants_every > 0 ? q->r.invariants_every : (int)std::min<long long>(n, 1 << 30));
  if (st != MX_OK) return st;
  st = mx_read_fields_async(c, q->r.E_out, q->r.H_out);
  if (st != MX_OK) return st;
  if (cudaEventCreateWithFlags(&q->done_ev, cudaEventDisableTiming) != cudaSuccess) return MX_E_CUDA;
  if (cudaEventRecord(q->done_ev, c->stream) != cudaSuccess) return MX_E_CUDA;
  return MX_OK;
}

// Before the active set changes: add the time since the last change, weighted by its size.
void account(mx_server* s) {
  const Clock::time_point now = Clock::now();
  const double dt = std::chrono::duration<double>(now - s->last_change).count();
  if (!s->active.empty()) {
    s->busy_s += dt;
    s->conc_area += dt * (double)s->active.size();
  }
  s->last_change = now;
}

void finish_request(mx_server* s, Req* q, mx_status st) {
  q->t_done = Clock::now();
  if (q->state == 1) s->request_s_sum += std::chrono::duration<double>(q->t_done - q->t_admit).count();
  if (st == MX_OK && q->ctx) {
    long long nrec = 0;
    st = mx_read_invariants(q->ctx, nullptr, 0, &nrec);
    if (st == MX_OK && nrec > 0) {
      q->inv.resize((size_t)nrec);
      st = mx_read_invariants(q->ctx, q->inv.data(), nrec, &nrec);
    }
  }
  if (q->done_ev) {
    cudaEventDestroy(q->done_ev);
    q->done_ev = nullptr;
  }
  if (q->ctx) {
    if (st == MX_OK) {
      release_ctx(s, q);
    } else {  // a context that failed is not reused
      s->in_use -= q->bytes;
      destroy_ctx(q->ctx);
      q->ctx = nullptr;
    }
  }
  q->state = st == MX_OK ? 2 : -(int)st;
  if (st == MX_OK) ++s->completed;
  else ++s->rejected;
}

void worker_loop(mx_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  while (!s->stop) {
    // admit
    while (!s->queue.empty() && (int)s->active.size() < s->max_active) {
      Req* q = s->reqs[s->queue.front()];
      mx_status err = MX_OK;
      mx_ctx* c = acquire_ctx(s, q, &err);
      if (!c) {
        if (err != MX_OK) {  // cannot ever run (or creation failed)
          s->queue.pop_front();
          finish_request(s, q, err);
          s->cv_done.notify_all();
          continue;
        }
        break;  // wait for memory
      }
      s->queue.pop_front();
      q->ctx = c;
      q->state = 1;
      q->t_admit = Clock::now();
      ++s->admitted;
      const mx_status st = launch_request(q);
      if (st != MX_OK) {
        finish_request(s, q, st);
        s->cv_done.notify_all();
        continue;
      }
      account(s);
      s->active.push_back(q);
      s->max_conc = std::max(s->max_conc, (long long)s->active.size());
    }
    // complete
    bool any = false;
    for (size_t i = 0; i < s->active.size();) {
      Req* q = s->active[i];
      const cudaError_t e = cudaEventQuery(q->done_ev);
      if (e == cudaErrorNotReady) {
        ++i;
        continue;
      }
      finish_request(s, q, e == cudaSuccess ? mx_sync(q->ctx) : MX_E_CUDA);
      account(s);
      s->active.erase(s->active.begin() + (long)i);
      any = true;
    }
    if (any) s->cv_done.notify_all();
    if (s->active.empty() && s->queue.empty()) {
      s->cv_work.wait(lock);
    } else if (!any) {
      lock.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(50));
      lock.lock();
    }
  }
}

}  // namespace

extern "C" {

mx_status mx_server_create(mx_server** out, size_t hbm_budget_bytes, int max_active) {
  if (!out || hbm_budget_bytes == 0 || max_active < 1) return MX_E_INVAL;
  mx_server* s = new mx_server();
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return MX_E_CUDA;
  }
  s->budget = hbm_budget_bytes;
  s->max_active = max_active;
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return MX_OK;
}

mx_status mx_server_submit(mx_server* s, const mx_request* r, long long* id) {
  if (!s || !r || !id) return MX_E_INVAL;
  if (!r->E0 || !r->H0 || !r->E_out || !r->H_out || r->nsteps < 1 || !isfinite(r->t_end)) return MX_E_INVAL;
  if (r->precision != MX_FP32 && r->precision != MX_FP64) return MX_E_INVAL;
  size_t b = 0;
  const mx_status fs = mx_footprint_bytes(r->nx, r->ny, r->nz, r->precision, MX_FORM_SPECTRAL, &b);
  if (fs != MX_OK) return fs;
  Req* q = new Req();
  q->r = *r;
  q->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    q->id = s->next_id++;
    s->reqs[q->id] = q;
    s->queue.push_back(q->id);
    *id = q->id;
  }
  s->cv_work.notify_one();
  return MX_OK;
}

mx_status mx_server_poll(mx_server* s, long long id, int* state) {
  if (!s || !state) return MX_E_INVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return MX_E_INVAL;
  *state = it->second->state;
  return MX_OK;
}

mx_status mx_server_wait(mx_server* s, long long id, double timeout_s, int* state) {
  if (!s || !state) return MX_E_INVAL;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return MX_E_INVAL;
  Req* q = it->second;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
  while (q->state == 0 || q->state == 1) {
    if (s->cv_done.wait_until(lock, deadline) == std::cv_status::timeout) break;
  }
  *state = q->state;
  return (q->state == 0 || q->state == 1) ? MX_E_TIMEOUT : MX_OK;
}

mx_status mx_server_result(mx_server* s, long long id, mx_invariants* inv, long long max, long long* n, double* latency_s,
                           int release) {
  if (!s || !n) return MX_E_INVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return MX_E_INVAL;
  Req* q = it->second;
  if (q->state < 0) return (mx_status)(-q->state);
  if (q->state != 2) return MX_E_STATE;
  const long long cnt = std::min<long long>(max, (long long)q->inv.size());
  for (long long i = 0; i < cnt; ++i) inv[i] = q->inv[(size_t)i];
  *n = max == 0 ? (long long)q->inv.size() : cnt;
  if (latency_s) *latency_s = std::chrono::duration<double>(q->t_done - q->t_submit).count();
  if (release) {
    delete q;
    s->reqs.erase(it);
  }
  return MX_OK;
}

mx_status mx_server_stats(mx_server* s, mx_server_info* out) {
  if (!s || !out) return MX_E_INVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  out->submitted = s->next_id - 1;
  out->admitted = s->admitted;
  out->completed = s->completed;
  out->rejected = s->rejected;
  out->queued = (long long)s->queue.size();
  out->active = (long long)s->active.size();
  out->hbm_in_use = s->in_use;
  out->hbm_high_water = s->high_water;
  out->hbm_budget = s->budget;
  out->pooled_contexts = (long long)s->idle.size();
  out->max_concurrent = s->max_conc;
  out->busy_s = s->busy_s;
  out->mean_concurrent = s->busy_s > 0.0 ? s->conc_area / s->busy_s : 0.0;
  out->request_s_sum = s->request_s_sum;
  return MX_OK;
}

void mx_server_destroy(mx_server* s) {
  if (!s) return;
  {
    std::unique_lock<std::mutex> lock(s->mu);
    // let running requests finish
    while (!s->active.empty()) {
      lock.unlock();
      std::this_thread::sleep_for(std::chrono::milliseconds(1));
      lock.lock();
    }
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& e : s->idle) destroy_ctx(e.ctx);
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
}

}  // extern "C"
