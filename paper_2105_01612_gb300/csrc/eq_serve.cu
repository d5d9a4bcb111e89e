// eq_serve.cu - request loop with continuous admission (eq_server_* / eq_serve_* of eq.h).
//
// A scheduler thread owns the device work.  Submitted requests wait in a FIFO queue; the head is
// admitted as soon as a slot (a CUDA stream) is free, its plan is ready and its device footprint
// (input + output field) fits under the HBM budget next to the requests in flight and the plans
// alive.  An admitted request gets device buffers from the stream-ordered allocator and runs
// H2D copy -> projection -> D2H copy -> norms on its slot's stream, so requests that arrive while
// others run overlap with them on the device.  Completion is seen by polling each slot's event;
// results are handed to eq_serve_poll.  Every wait is bounded.
//
// Plans come from a second thread, so that no plan is built while the scheduler holds the lock:
// it walks the first queued requests in order and gives each one a plan, an idle one of the same
// grid and options from the cache if there is one, else a new one built outside the lock.  A
// finished request's plan goes back to the cache, which keeps at most `max_idle_plans` idle plans
// in least-recently-used order.  The budget covers the request buffers in flight and the device
// bytes of the plans in flight and in the cache; the scheduler asks for idle plans to be
// released when the head request (buffers and plan) would not fit otherwise, and admits a head
// whose buffers fit an empty server once nothing else is alive, whatever its plan's size (plans
// prepared for queued requests are few, `lookahead` at most, and counted apart).  Releasing a
// plan frees device memory, which waits for the device, so that too happens on the plan thread.
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/eq.h"

#include <nvtx3/nvToolsExt.h>

namespace eqk {
void set_last_error(const std::string& msg);   // eq_api.cu
void log(int level, const char* fmt, ...);     // eq_api.cu
}

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { QUEUED, RUNNING, DONE, FAILED };

struct Request {
  unsigned long long id = 0;
  eq_plan* plan = nullptr;        // set by the plan thread before admission
  size_t plan_bytes = 0;
  bool plan_pending = false;      // being built outside the lock
  int nx = 0, ny = 0, nz = 0;
  eq_dtype dtype = EQ_F32;
  eq_plan_opts opts{};
  const void* host_in = nullptr;
  void* host_out = nullptr;
  size_t bytes = 0;
  Clock::time_point t_submit;
  double latency = 0.0;
  nvtxRangeId_t trace = 0;        // trace range from admission to completion
  ReqState state = QUEUED;
  eq_status status = EQ_OK;
  std::string error;
  eq_norms_t norms{};
};

using PlanKey = std::tuple<int, int, int, int, int, double, double, double, int, int, int>;

PlanKey key_of(const Request& r) {
  return PlanKey(r.nx, r.ny, r.nz, (int)r.dtype, (int)r.opts.op, r.opts.hx, r.opts.hy, r.opts.hz,
                 (int)r.opts.nyq, r.opts.want_linf, (int)r.opts.target);
}

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  Request* req = nullptr;
  eq_plan* plan = nullptr;
  void* d_in = nullptr;
  void* d_out = nullptr;
  eq_norms_t* h_norms = nullptr;   // pinned
};

}  // namespace

struct IdlePlan {
  PlanKey key;
  eq_plan* plan;
  size_t bytes;
};

struct eq_server {
  int device = 0;
  size_t budget = 0;
  size_t in_use = 0;              // request buffers in flight + device bytes of the plans in
                                  // flight, cached or waiting to be released
  size_t queued_plan_bytes = 0;   // plans prepared for queued requests
  int max_queue = 65536;
  size_t max_idle_plans = 64;
  int lookahead = 8;              // queued requests the plan thread prepares ahead of admission
  std::vector<Slot> slots;
  std::deque<Request*> queue;
  std::unordered_map<unsigned long long, Request*> reqs;
  std::list<IdlePlan> lru;        // idle plans, most recently used first
  std::multimap<PlanKey, std::list<IdlePlan>::iterator> idle;
  std::vector<eq_plan*> to_release;   // evicted plans, destroyed by the plan thread
  size_t release_bytes = 0;           // their bytes (still counted in in_use until destroyed)
  bool want_release = false;          // the scheduler needs room: evict idle plans
  unsigned long long next_id = 1;
  std::mutex mu;
  std::condition_variable cv_done;
  std::condition_variable cv_work;
  std::condition_variable cv_plans;
  bool stop = false;
  std::thread worker;
  std::thread planner;
  eq_server_stats_t st{};
};

namespace {

eq_status sfail(eq_status st, const std::string& m) {
  eqk::set_last_error(m);
  return st;
}

// An idle plan for key k from the cache (with the lock held), or nullptr.
bool take_idle(eq_server* s, const PlanKey& k, eq_plan** p, size_t* bytes) {
  auto it = s->idle.find(k);
  if (it == s->idle.end()) return false;
  *p = it->second->plan;
  *bytes = it->second->bytes;
  s->lru.erase(it->second);
  s->idle.erase(it);
  return true;
}

// Move the least recently used idle plan to the release list (with the lock held).
bool evict_one(eq_server* s) {
  if (s->lru.empty()) return false;
  IdlePlan& ip = s->lru.back();
  for (auto it = s->idle.lower_bound(ip.key); it != s->idle.end() && it->first == ip.key; ++it)
    if (it->second == std::prev(s->lru.end())) { s->idle.erase(it); break; }
  s->to_release.push_back(ip.plan);
  s->release_bytes += ip.bytes;
  s->st.plans_evicted++;
  s->lru.pop_back();
  return true;
}

void put_idle(eq_server* s, const PlanKey& k, eq_plan* p, size_t bytes) {
  s->lru.push_front(IdlePlan{k, p, bytes});
  s->idle.emplace(k, s->lru.begin());
  while (s->lru.size() > s->max_idle_plans) evict_one(s);
  if (!s->to_release.empty()) s->cv_plans.notify_one();
}

void update_peaks(eq_server* s) {
  if ((unsigned long long)s->in_use > s->st.hbm_in_use_peak) s->st.hbm_in_use_peak = s->in_use;
}

// The plan thread: prepares plans for the first queued requests (cache or a new plan built
// outside the lock) and destroys evicted plans, also outside the lock.
void planner_loop(eq_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    if (!s->to_release.empty()) {
      std::vector<eq_plan*> rel;
      rel.swap(s->to_release);
      const size_t rb = s->release_bytes;
      s->release_bytes = 0;
      lk.unlock();
      for (eq_plan* p : rel) eq_plan_destroy(p);
      eqk::log(2, "serve: released %zu idle plans (%zu bytes)", rel.size(), rb);
      lk.lock();
      s->in_use -= rb;
      s->cv_work.notify_one();
      continue;
    }
    if (s->want_release) {
      s->want_release = false;
      if (evict_one(s)) continue;
    }
    Request* r = nullptr;
    int seen = 0;
    for (Request* q : s->queue) {
      if (++seen > s->lookahead) break;
      if (!q->plan && !q->plan_pending) { r = q; break; }
    }
    if (!r) {
      if (s->stop) break;
      s->cv_plans.wait_for(lk, std::chrono::milliseconds(5));
      continue;
    }
    const PlanKey k = key_of(*r);
    eq_plan* p = nullptr;
    size_t bytes = 0;
    if (take_idle(s, k, &p, &bytes)) {
      r->plan = p;
      r->plan_bytes = bytes;
      s->in_use -= bytes;
      s->queued_plan_bytes += bytes;
      s->st.plans_reused++;
      s->cv_work.notify_one();
      continue;
    }
    r->plan_pending = true;
    eq_plan_opts o = r->opts;
    o.graph = 0;   // buffers change with every request
    const int nx = r->nx, ny = r->ny, nz = r->nz;
    const eq_dtype dt = r->dtype;
    lk.unlock();
    const Clock::time_point t0 = Clock::now();
    const eq_status cst = eq_plan_create(nx, ny, nz, dt, 1, &o, &p);
    const double dt_s = std::chrono::duration<double>(Clock::now() - t0).count();
    const std::string err = cst == EQ_OK ? std::string() : std::string(eq_last_error());
    bytes = cst == EQ_OK ? eq_plan_workspace_bytes(p) : 0;
    lk.lock();
    s->st.plans_created++;
    s->st.plan_create_seconds += dt_s;
    bool queued = false;                       // still queued (destroy clears the queue)
    for (Request* q : s->queue) queued = queued || q == r;
    if (!queued) {
      if (cst == EQ_OK) {
        s->to_release.push_back(p);
        s->release_bytes += bytes;
        s->in_use += bytes;
      }
      continue;
    }
    r->plan_pending = false;
    if (cst != EQ_OK) {
      // the request fails where it stands in the queue
      for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
        if (*it == r) { s->queue.erase(it); break; }
      r->state = FAILED;
      r->status = cst;
      r->error = err;
      r->latency = std::chrono::duration<double>(Clock::now() - r->t_submit).count();
      s->st.failed++;
      s->cv_done.notify_all();
      continue;
    }
    r->plan = p;
    r->plan_bytes = bytes;
    s->queued_plan_bytes += bytes;
    s->cv_work.notify_one();
  }
  // shutting down: the scheduler has finished every request on the device
  lk.unlock();
}

void finish(eq_server* s, Slot& sl, bool ok, const std::string& err) {
  Request* r = sl.req;
  r->latency = std::chrono::duration<double>(Clock::now() - r->t_submit).count();
  if (ok) {
    r->norms = *sl.h_norms;
    r->state = DONE;
    r->status = EQ_OK;
  } else {
    r->state = FAILED;
    r->status = EQ_ERR_CUDA;
    r->error = err;
  }
  if (ok) s->st.completed++;
  else s->st.failed++;
  if (r->trace) nvtxRangeEnd(r->trace);
  eqk::log(2, "serve: request %llu %dx%dx%d %s after %.3f ms", r->id, r->nx, r->ny, r->nz,
           ok ? "done" : "failed", 1e3 * r->latency);
  if (sl.d_in) cudaFreeAsync(sl.d_in, sl.stream);
  if (sl.d_out) cudaFreeAsync(sl.d_out, sl.stream);
  sl.d_in = sl.d_out = nullptr;
  if (sl.plan) put_idle(s, key_of(*r), sl.plan, r->plan_bytes);
  sl.plan = nullptr;
  r->plan = nullptr;
  s->in_use -= 2 * r->bytes;
  s->st.inflight--;
  sl.req = nullptr;
}

// Start request r on slot sl (called with the lock held).
bool start(eq_server* s, Slot& sl, Request* r) {
  std::string err;
  sl.req = r;
  r->state = RUNNING;
  s->in_use += 2 * r->bytes + r->plan_bytes;
  s->queued_plan_bytes -= r->plan_bytes;
  s->st.admitted++;
  s->st.inflight++;
  if (s->st.inflight > s->st.inflight_peak) s->st.inflight_peak = s->st.inflight;
  update_peaks(s);
  sl.plan = r->plan;
  if (!sl.plan) err = "serve: no plan";
  {
    char name[64];
    snprintf(name, sizeof(name), "eq request %llu", r->id);
    r->trace = nvtxRangeStartA(name);
  }
  eqk::log(2, "serve: admit request %llu %dx%dx%d (%zu bytes in use)", r->id, r->nx, r->ny, r->nz,
           s->in_use);
  cudaError_t e = cudaSuccess;
  if (sl.plan) {
    e = cudaMallocAsync(&sl.d_in, r->bytes, sl.stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&sl.d_out, r->bytes, sl.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.d_in, r->host_in, r->bytes, cudaMemcpyHostToDevice, sl.stream);
    if (e != cudaSuccess) err = std::string("serve: ") + cudaGetErrorString(e);
  }
  bool ok = sl.plan && e == cudaSuccess;
  if (ok && eq_project(sl.plan, sl.d_in, sl.d_out, sl.stream) != EQ_OK) {
    ok = false;
    err = eq_last_error();
  }
  if (ok) {
    e = cudaMemcpyAsync(r->host_out, sl.d_out, r->bytes, cudaMemcpyDeviceToHost, sl.stream);
    if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
    if (e != cudaSuccess) { ok = false; err = std::string("serve: ") + cudaGetErrorString(e); }
  }
  if (!ok) {
    cudaGetLastError();
    finish(s, sl, false, err);
    return false;
  }
  return true;
}

void worker_loop(eq_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    bool progressed = false;
    // completions
    for (Slot& sl : s->slots) {
      if (!sl.req) continue;
      cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      bool ok = q == cudaSuccess;
      std::string err;
      if (ok) {
        // the plan's norms are ready once its work is done (same stream)
        if (eq_norms(sl.plan, sl.h_norms) != EQ_OK) { ok = false; err = eq_last_error(); }
      } else {
        err = std::string("serve: ") + cudaGetErrorString(q);
        cudaGetLastError();
      }
      finish(s, sl, ok, err);
      progressed = true;
    }
    if (progressed) s->cv_done.notify_all();
    // admission: FIFO head while a slot is free, its plan is ready and the footprint fits
    while (!s->queue.empty() && !s->stop) {
      Request* r = s->queue.front();
      Slot* free_slot = nullptr;
      for (Slot& sl : s->slots)
        if (!sl.req) { free_slot = &sl; break; }
      if (!free_slot || !r->plan) break;
      if (s->in_use + 2 * r->bytes + r->plan_bytes > s->budget) {
        // room held by idle plans: ask the plan thread to release the least recently used
        if (!s->lru.empty() || !s->to_release.empty()) {
          s->want_release = !s->lru.empty();
          s->cv_plans.notify_one();
          break;
        }
        bool others = false;                   // anything else in flight?
        for (Slot& sl : s->slots) others = others || sl.req;
        if (others) break;
        // nothing else alive: the buffers fit the budget (checked at submit), admit
      }
      s->queue.pop_front();
      if (!start(s, *free_slot, r)) s->cv_done.notify_all();
      progressed = true;
    }
    if (!s->queue.empty()) s->cv_plans.notify_one();
    bool busy = false;
    for (Slot& sl : s->slots) busy = busy || sl.req;
    if (s->stop && !busy) {
      s->cv_plans.notify_all();
      break;
    }
    if (!progressed) {
      if (busy) {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
      } else {
        s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
      }
    }
  }
}

}  // namespace

extern "C" {

eq_status eq_server_create(size_t hbm_budget_bytes, int max_inflight, eq_server** out) {
  if (!out) return sfail(EQ_ERR_INVALID, "eq_server_create: out is NULL");
  *out = nullptr;
  if (max_inflight < 1 || max_inflight > 256 || hbm_budget_bytes == 0)
    return sfail(EQ_ERR_INVALID, "eq_server_create: max_inflight must be 1..256 and the budget > 0");
  eq_server* s = new (std::nothrow) eq_server();
  if (!s) return sfail(EQ_ERR_OOM, "eq_server_create: host allocation failed");
  s->budget = hbm_budget_bytes;
  cudaError_t e = cudaGetDevice(&s->device);
  // keep freed request buffers cached in the device's stream-ordered pool (up to the budget)
  cudaMemPool_t pool;
  if (e == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
    unsigned long long thr = hbm_budget_bytes;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  s->slots.resize(max_inflight);
  for (Slot& sl : s->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.h_norms, sizeof(eq_norms_t));
  }
  if (e != cudaSuccess) {
    for (Slot& sl : s->slots) {
      if (sl.stream) cudaStreamDestroy(sl.stream);
      if (sl.done) cudaEventDestroy(sl.done);
      if (sl.h_norms) cudaFreeHost(sl.h_norms);
    }
    delete s;
    return sfail(EQ_ERR_CUDA, std::string("eq_server_create: ") + cudaGetErrorString(e));
  }
  s->worker = std::thread(worker_loop, s);
  s->planner = std::thread(planner_loop, s);
  *out = s;
  return EQ_OK;
}

eq_status eq_serve_submit(eq_server* s, int nx, int ny, int nz, eq_dtype dtype,
                          const eq_plan_opts* opts, const void* host_in, void* host_out,
                          unsigned long long* ticket) {
  if (!s || !host_in || !host_out || !ticket) return sfail(EQ_ERR_INVALID, "eq_serve_submit: NULL argument");
  if (nx < 1 || ny < 1 || nz < 1 || nx > 1024 || ny > 1024 || nz > 1024 ||
      (dtype != EQ_F32 && dtype != EQ_F64))
    return sfail(EQ_ERR_INVALID, "eq_serve_submit: bad size or dtype");
  Request* r = new (std::nothrow) Request();
  if (!r) return sfail(EQ_ERR_OOM, "eq_serve_submit: host allocation failed");
  r->nx = nx; r->ny = ny; r->nz = nz; r->dtype = dtype;
  eq_plan_opts_default(&r->opts);
  if (opts) r->opts = *opts;
  r->host_in = host_in;
  r->host_out = host_out;
  r->bytes = (size_t)6 * nx * ny * nz * (dtype == EQ_F32 ? 4 : 8);
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) { delete r; return sfail(EQ_ERR_INVALID, "eq_serve_submit: server is shutting down"); }
  if (2 * r->bytes > s->budget) {
    delete r;
    s->st.rejected++;
    return sfail(EQ_ERR_OOM, "eq_serve_submit: request footprint exceeds the server's HBM budget");
  }
  if ((int)s->queue.size() >= s->max_queue) {
    delete r;
    s->st.rejected++;
    return sfail(EQ_ERR_BUSY, "eq_serve_submit: queue full");
  }
  r->id = s->next_id++;
  s->reqs[r->id] = r;
  s->queue.push_back(r);
  s->st.submitted++;
  *ticket = r->id;
  s->cv_work.notify_one();
  s->cv_plans.notify_one();
  return EQ_OK;
}

eq_status eq_serve_cancel(eq_server* s, unsigned long long ticket) {
  if (!s) return sfail(EQ_ERR_INVALID, "eq_serve_cancel: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return sfail(EQ_ERR_NOT_FOUND, "eq_serve_cancel: unknown ticket");
  Request* r = it->second;
  if (r->state != QUEUED || r->plan_pending)
    return sfail(EQ_ERR_BUSY, "eq_serve_cancel: the request has started (or its plan is being built)");
  for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
    if (*q == r) { s->queue.erase(q); break; }
  if (r->plan) {                              // a prepared plan goes back to the cache
    s->queued_plan_bytes -= r->plan_bytes;
    s->in_use += r->plan_bytes;
    put_idle(s, key_of(*r), r->plan, r->plan_bytes);
    r->plan = nullptr;
  }
  s->reqs.erase(it);
  delete r;
  s->st.cancelled++;
  return EQ_OK;
}

eq_status eq_server_stats(eq_server* s, eq_server_stats_t* out) {
  if (!s || !out) return sfail(EQ_ERR_INVALID, "eq_server_stats: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->queued = (long long)s->queue.size();
  out->hbm_in_use = s->in_use + s->queued_plan_bytes;
  out->hbm_budget = s->budget;
  out->plans_cached = (long long)s->lru.size();
  return EQ_OK;
}

eq_status eq_serve_poll(eq_server* s, unsigned long long ticket, int timeout_us,
                        eq_norms_t* out, double* latency_s) {
  if (!s) return sfail(EQ_ERR_INVALID, "eq_serve_poll: NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return sfail(EQ_ERR_NOT_FOUND, "eq_serve_poll: unknown ticket");
  Request* r = it->second;
  if (timeout_us > 0)
    s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us),
                        [&] { return r->state == DONE || r->state == FAILED; });
  if (r->state != DONE && r->state != FAILED) return EQ_PENDING;
  const eq_status st = r->status;
  if (st == EQ_OK) {
    if (out) *out = r->norms;
    if (latency_s) *latency_s = r->latency;
  } else {
    eqk::set_last_error(r->error);
  }
  s->reqs.erase(it);
  delete r;
  return st;
}

void eq_server_destroy(eq_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (Request* r : s->queue) {           // cancel what has not started
      r->state = FAILED;
      r->status = EQ_ERR_INVALID;
      r->error = "cancelled: server destroyed";
    }
    s->queue.clear();
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();   // running requests finish (bounded GPU work)
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->cv_plans.notify_all();
  }
  if (s->planner.joinable()) s->planner.join();  // a plan being built completes first
  cudaSetDevice(s->device);
  for (Slot& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.h_norms) cudaFreeHost(sl.h_norms);
  }
  for (IdlePlan& ip : s->lru) eq_plan_destroy(ip.plan);
  for (eq_plan* p : s->to_release) eq_plan_destroy(p);
  for (auto& kv : s->reqs) {
    if (kv.second->plan) eq_plan_destroy(kv.second->plan);
    delete kv.second;
  }
  delete s;
}

}  // extern "C"
