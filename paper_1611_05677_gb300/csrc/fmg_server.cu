// Request server: continuous batching of independent solves on one GPU.
//
// A worker thread owns all device work.  Requests wait in a FIFO queue; the worker admits the
// head request as soon as an in-flight slot is free and the device memory budget allows its
// level hierarchy, launches it on the stream of a context of its shape (a cached one when an
// idle context of the same shape exists, so hierarchies and captured graphs stay on the
// device), and retires requests whose completion event has fired.  Requests in flight run
// concurrently on the device: every context uses the cluster-variant Newton kernel, which any
// number of solves may run side by side.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "fmg_internal.cuh"

using namespace fmg;

namespace {

long long now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// Contexts are interchangeable when every parameter that shapes the hierarchy or the captured
// graph agrees (g is data: it is loaded per request).
bool same_shape(const fmg_params& a, const fmg_params& b) {
  return a.dim == b.dim && a.coarse_cells == b.coarse_cells && a.refinements == b.refinements && a.f == b.f &&
         a.f_scale == b.f_scale && a.m_vcycles == b.m_vcycles && a.nu_pre == b.nu_pre && a.nu_post == b.nu_post &&
         a.p_corrections == b.p_corrections && a.precision == b.precision && a.newton_tol == b.newton_tol &&
         a.newton_maxit == b.newton_maxit && a.level1_tol == b.level1_tol && a.level1_maxit == b.level1_maxit &&
         a.smoother == b.smoother && a.nonlinear == b.nonlinear;
}

struct Cached {
  fmg_ctx* ctx = nullptr;
  fmg_params p{};
  size_t bytes = 0;
  long long last_used = 0;
  bool busy = false;
};

struct Request {
  unsigned long long ticket = 0;
  fmg_params p{};
  const double* g = nullptr;
  double* u = nullptr;
  long long t_submit = 0, t_start = 0, t_done = 0;
  fmg_status status = FMG_OK;
  std::string err;  // what went wrong, for a failed request (handed to the polling thread)
  fmg_stats stats{};
};

struct Slot {
  cudaEvent_t done = nullptr;
  DevState* state = nullptr;  // pinned host copy of the solve's DevState
  Request* req = nullptr;
  Cached* cc = nullptr;
};

}  // namespace

struct fmg_server {
  fmg_server_config cfg{};
  int device = 0;
  // shared between the worker and callers: under mu
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::deque<Request*> finished;
  unsigned long long next_ticket = 1;
  size_t submitted = 0, completed = 0;
  fmg_server_info pub{};  // the worker's counters as last published
  // the worker's own state: read and written by the worker thread only
  std::vector<Cached*> cache;
  std::vector<Slot> slots;
  size_t bytes_held = 0;
  int in_flight = 0;
  fmg_server_info info{};
  std::atomic<bool> stop{false};
  std::thread worker;
};

namespace {

thread_local std::string t_srv_err;

fmg_status srv_fail(fmg_status s, const std::string& m) {
  t_srv_err = m;
  set_thread_error(m);
  return s;
}

// Copies the worker's counters where callers read them (fmg_server_get_info).  Worker thread,
// with mu held.
void publish_locked(fmg_server* sv) {
  sv->pub.contexts_created = sv->info.contexts_created;
  sv->pub.contexts_evicted = sv->info.contexts_evicted;
  sv->pub.bytes_held = sv->bytes_held;
  sv->pub.contexts_cached = (int)sv->cache.size();
  sv->pub.in_flight = sv->in_flight;
}

void publish(fmg_server* sv) {
  std::lock_guard<std::mutex> lk(sv->mu);
  publish_locked(sv);
}

// Hands a finished request (its slot already released) to the callers.  Worker thread.  The
// counters are published with it, so a caller that sees the request completed (a drain) also
// sees the state it left.
void finish(fmg_server* sv, Request* r) {
  r->t_done = now_ns();
  std::lock_guard<std::mutex> lk(sv->mu);
  try {
    sv->finished.push_back(r);
  } catch (...) {
    delete r;  // out of host memory: the result is lost, but the request counts as finished
  }
  publish_locked(sv);
  ++sv->completed;
  sv->cv_done.notify_all();
}

// Destroys least recently used idle contexts until `need` more bytes fit the budget.
// Called by the worker only.
void evict_for(fmg_server* sv, size_t need) {
  while (sv->bytes_held + need > sv->cfg.hbm_budget) {
    Cached* victim = nullptr;
    for (Cached* c : sv->cache)
      if (!c->busy && (!victim || c->last_used < victim->last_used)) victim = c;
    if (!victim) return;
    fmg_destroy(victim->ctx);
    sv->bytes_held -= victim->bytes;
    sv->cache.erase(std::find(sv->cache.begin(), sv->cache.end(), victim));
    delete victim;
    ++sv->info.contexts_evicted;
  }
}

// An idle context for r (cached or new), or nullptr when the budget does not allow one now.
// Sets r->status when the request cannot be served at all.
Cached* context_for(fmg_server* sv, Request* r, const double* g) {
  for (Cached* c : sv->cache)
    if (!c->busy && same_shape(c->p, r->p)) return c;
  size_t need = 0;
  if (fmg_workspace_bytes(&r->p, &need) != FMG_OK) {
    r->status = FMG_ERR_INVALID;
    r->err = std::string("invalid parameters: ") + fmg_last_error(nullptr);
    return nullptr;
  }
  if (need > sv->cfg.hbm_budget) {
    r->status = FMG_ERR_OOM;
    r->err = "the hierarchy needs " + std::to_string(need) + " bytes, more than the server's HBM budget of " +
             std::to_string(sv->cfg.hbm_budget);
    return nullptr;
  }
  evict_for(sv, need);
  if (sv->bytes_held + need > sv->cfg.hbm_budget) return nullptr;  // wait for a busy one to finish
  fmg_ctx* ctx = nullptr;
  fmg_status s = fmg_create(&r->p, g, 0, nullptr, nullptr, 0, &ctx);
  if (s == FMG_OK) s = ctx_make_concurrent(ctx);
  if (s != FMG_OK) {
    r->err = ctx ? ctx_error(ctx) : fmg_last_error(nullptr);
    if (ctx) fmg_destroy(ctx);
    r->status = s;
    return nullptr;
  }
  Cached* c = new (std::nothrow) Cached();
  bool stored = false;
  if (c) {
    try {
      sv->cache.push_back(c);
      stored = true;
    } catch (...) {
    }
  }
  if (!stored) {
    delete c;
    fmg_destroy(ctx);
    r->status = FMG_ERR_OOM;
    r->err = "host allocation failed";
    return nullptr;
  }
  c->ctx = ctx;
  c->p = r->p;
  c->bytes = ctx_bytes(ctx);
  sv->bytes_held += c->bytes;
  ++sv->info.contexts_created;
  return c;
}

void retire(fmg_server* sv) {
  for (Slot& sl : sv->slots) {
    if (!sl.req) continue;
    const cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    Request* r = sl.req;
    if (q != cudaSuccess) {
      r->status = FMG_ERR_CUDA;
      r->err = cudaGetErrorString(q);
    } else {
      r->status = ctx_decode(sl.cc->ctx, *sl.state, &r->stats);
      if (r->status != FMG_OK) r->err = ctx_error(sl.cc->ctx);
    }
    sl.cc->busy = false;
    sl.cc->last_used = now_ns();
    sl.req = nullptr;
    sl.cc = nullptr;
    --sv->in_flight;
    finish(sv, r);
  }
}

// Admits queued requests in arrival order while slots and memory allow.
bool admit(fmg_server* sv) {
  bool any = false;
  for (;;) {
    Slot* free_slot = nullptr;
    for (Slot& sl : sv->slots)
      if (!sl.req) {
        free_slot = &sl;
        break;
      }
    if (!free_slot) return any;
    Request* r = nullptr;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      if (sv->queue.empty()) return any;
      r = sv->queue.front();
    }
    Cached* cc = context_for(sv, r, r->g);
    if (!cc && r->status == FMG_OK) return any;  // head waits for memory (FIFO)
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->queue.pop_front();
    }
    any = true;
    if (!cc) {
      finish(sv, r);
      continue;
    }
    cc->busy = true;
    r->t_start = now_ns();
    fmg_status s = ctx_enqueue(cc->ctx, r->g, r->u, free_slot->state);
    cudaError_t e = cudaSuccess;
    if (s == FMG_OK) e = cudaEventRecord(free_slot->done, ctx_stream(cc->ctx));
    if (s != FMG_OK || e != cudaSuccess) {
      r->status = s != FMG_OK ? s : FMG_ERR_CUDA;
      r->err = s != FMG_OK ? std::string(ctx_error(cc->ctx)) : std::string(cudaGetErrorString(e));
      cc->busy = false;
      finish(sv, r);
      continue;
    }
    free_slot->req = r;
    free_slot->cc = cc;
    ++sv->in_flight;
  }
}

void worker_main(fmg_server* sv) {
  cudaSetDevice(sv->device);
  for (;;) {
    retire(sv);
    const bool admitted = admit(sv);
    publish(sv);
    bool idle;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      idle = sv->in_flight == 0 && sv->queue.empty();
      if (idle) {
        if (sv->stop.load()) break;
        sv->cv_work.wait_for(lk, std::chrono::milliseconds(50));
        continue;
      }
    }
    if (!admitted) std::this_thread::sleep_for(std::chrono::microseconds(sv->cfg.poll_us));
  }
}

}  // namespace

extern "C" {

fmg_status fmg_server_create(const fmg_server_config* cfg, fmg_server** out) {
  if (!out) return srv_fail(FMG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  fmg_server* sv = new (std::nothrow) fmg_server();
  if (!sv) return srv_fail(FMG_ERR_OOM, "host allocation failed");
  if (cfg) sv->cfg = *cfg;
  if (sv->cfg.max_inflight <= 0) sv->cfg.max_inflight = 8;
  if (sv->cfg.max_inflight > 64) sv->cfg.max_inflight = 64;
  if (sv->cfg.poll_us <= 0) sv->cfg.poll_us = 20;
  cudaError_t e = cudaGetDevice(&sv->device);
  size_t free_b = 0, total_b = 0;
  if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) {
    delete sv;
    return srv_fail(FMG_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  }
  if (sv->cfg.hbm_budget == 0) sv->cfg.hbm_budget = free_b / 10 * 8;
  sv->slots.resize(sv->cfg.max_inflight);
  for (Slot& sl : sv->slots) {
    e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.state, sizeof(DevState));
    if (e != cudaSuccess) break;
  }
  if (e != cudaSuccess) {
    for (Slot& sl : sv->slots) {
      if (sl.done) cudaEventDestroy(sl.done);
      if (sl.state) cudaFreeHost(sl.state);
    }
    delete sv;
    return srv_fail(FMG_ERR_CUDA, std::string("server setup: ") + cudaGetErrorString(e));
  }
  sv->worker = std::thread(worker_main, sv);
  *out = sv;
  return FMG_OK;
}

fmg_status fmg_server_submit(fmg_server* sv, const fmg_params* p, const double* g_host, double* u_host,
                             unsigned long long* ticket) {
  if (!sv || !p || !g_host || !u_host) return srv_fail(FMG_ERR_INVALID, "NULL argument");
  if (p->coefficient) return srv_fail(FMG_ERR_INVALID, "the server takes A = I only (no coefficient)");
  size_t need = 0;
  if (fmg_status s = fmg_workspace_bytes(p, &need)) return s;
  Request* r = new (std::nothrow) Request();
  if (!r) return srv_fail(FMG_ERR_OOM, "host allocation failed");
  r->p = *p;
  r->g = g_host;
  r->u = u_host;
  r->t_submit = now_ns();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    r->ticket = sv->next_ticket++;
    sv->queue.push_back(r);
    ++sv->submitted;
  }
  sv->cv_work.notify_one();
  if (ticket) *ticket = r->ticket;
  return FMG_OK;
}

int fmg_server_poll(fmg_server* sv, fmg_server_result* out, int max) {
  if (!sv || !out || max <= 0) return 0;
  int n = 0;
  std::lock_guard<std::mutex> lk(sv->mu);
  while (n < max && !sv->finished.empty()) {
    Request* r = sv->finished.front();
    sv->finished.pop_front();
    fmg_server_result& o = out[n++];
    std::memset(&o, 0, sizeof(o));
    o.ticket = r->ticket;
    o.status = r->status;
    if (r->status != FMG_OK)
      t_srv_err = "request " + std::to_string(r->ticket) + ": " +
                  (r->err.empty() ? "status " + std::to_string((int)r->status) : r->err);
    o.stats = r->stats;
    o.queue_ms = (r->t_start > 0 ? r->t_start - r->t_submit : r->t_done - r->t_submit) * 1e-6;
    o.latency_ms = (r->t_done - r->t_submit) * 1e-6;
    delete r;
  }
  return n;
}

fmg_status fmg_server_drain(fmg_server* sv, double timeout_s) {
  if (!sv) return srv_fail(FMG_ERR_INVALID, "server is NULL");
  std::unique_lock<std::mutex> lk(sv->mu);
  const bool ok = sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                       [&] { return sv->completed == sv->submitted; });
  if (!ok) return srv_fail(FMG_ERR_TIMEOUT, "requests still pending when the drain timed out");
  return FMG_OK;
}

fmg_status fmg_server_get_info(fmg_server* sv, fmg_server_info* info) {
  if (!sv || !info) return srv_fail(FMG_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  *info = sv->pub;
  info->hbm_budget = sv->cfg.hbm_budget;
  info->queued = (int)sv->queue.size();
  info->submitted = sv->submitted;
  info->completed = sv->completed;
  return FMG_OK;
}

const char* fmg_server_last_error(void) { return t_srv_err.c_str(); }

fmg_status fmg_server_destroy(fmg_server* sv) {
  if (!sv) return FMG_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop.store(true);
  }
  sv->cv_work.notify_all();
  // the worker finishes what was submitted, then exits
  if (sv->worker.joinable()) sv->worker.join();
  cudaSetDevice(sv->device);
  for (Request* r : sv->finished) delete r;
  for (Cached* c : sv->cache) {
    fmg_destroy(c->ctx);
    delete c;
  }
  for (Slot& sl : sv->slots) {
    cudaEventDestroy(sl.done);
    cudaFreeHost(sl.state);
  }
  delete sv;
  return FMG_OK;
}

}  // extern "C"
