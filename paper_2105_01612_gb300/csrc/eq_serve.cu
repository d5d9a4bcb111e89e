// eq_serve.cu - request loop with continuous admission (eq_server_* / eq_serve_* of eq.h).
//
// A scheduler thread owns the device work.  Submitted requests wait in a FIFO queue; the head is
// admitted as soon as a slot (a CUDA stream) is free and its device footprint (input + output
// field) fits under the HBM budget next to the requests already in flight.  An admitted request
// gets device buffers from the stream-ordered allocator, a plan for its grid size from a cache
// of idle plans, and runs H2D copy -> projection -> D2H copy -> norms on its slot's stream, so
// requests that arrive while others run overlap with them on the device.  Completion is seen by
// polling each slot's event; results are handed to eq_serve_poll.  Every wait is bounded.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/eq.h"

namespace eqk {
void set_last_error(const std::string& msg);   // eq_api.cu
}

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { QUEUED, RUNNING, DONE, FAILED };

struct Request {
  unsigned long long id = 0;
  int nx = 0, ny = 0, nz = 0;
  eq_dtype dtype = EQ_F32;
  eq_plan_opts opts{};
  const void* host_in = nullptr;
  void* host_out = nullptr;
  size_t bytes = 0;
  Clock::time_point t_submit;
  double latency = 0.0;
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

struct eq_server {
  int device = 0;
  size_t budget = 0;
  size_t in_use = 0;
  int max_queue = 65536;
  std::vector<Slot> slots;
  std::deque<Request*> queue;
  std::unordered_map<unsigned long long, Request*> reqs;
  std::multimap<PlanKey, eq_plan*> idle_plans;
  unsigned long long next_id = 1;
  std::mutex mu;
  std::condition_variable cv_done;
  std::condition_variable cv_work;
  bool stop = false;
  std::thread worker;
};

namespace {

eq_status sfail(eq_status st, const std::string& m) {
  eqk::set_last_error(m);
  return st;
}

eq_plan* take_plan(eq_server* s, const Request& r, std::string* err) {
  const PlanKey k = key_of(r);
  auto it = s->idle_plans.find(k);
  if (it != s->idle_plans.end()) {
    eq_plan* p = it->second;
    s->idle_plans.erase(it);
    return p;
  }
  eq_plan* p = nullptr;
  eq_plan_opts o = r.opts;
  o.graph = 0;   // buffers change with every request
  if (eq_plan_create(r.nx, r.ny, r.nz, r.dtype, 1, &o, &p) != EQ_OK) {
    *err = eq_last_error();
    return nullptr;
  }
  return p;
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
  if (sl.d_in) cudaFreeAsync(sl.d_in, sl.stream);
  if (sl.d_out) cudaFreeAsync(sl.d_out, sl.stream);
  sl.d_in = sl.d_out = nullptr;
  if (sl.plan) s->idle_plans.emplace(key_of(*r), sl.plan);
  sl.plan = nullptr;
  s->in_use -= 2 * r->bytes;
  sl.req = nullptr;
}

// Start request r on slot sl (called with the lock held).
bool start(eq_server* s, Slot& sl, Request* r) {
  std::string err;
  sl.req = r;
  r->state = RUNNING;
  s->in_use += 2 * r->bytes;
  sl.plan = take_plan(s, *r, &err);
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
    // admission: FIFO head while a slot is free and the footprint fits
    while (!s->queue.empty() && !s->stop) {
      Request* r = s->queue.front();
      Slot* free_slot = nullptr;
      for (Slot& sl : s->slots)
        if (!sl.req) { free_slot = &sl; break; }
      if (!free_slot || s->in_use + 2 * r->bytes > s->budget) break;
      s->queue.pop_front();
      if (!start(s, *free_slot, r)) s->cv_done.notify_all();
      progressed = true;
    }
    bool busy = false;
    for (Slot& sl : s->slots) busy = busy || sl.req;
    if (s->stop && !busy) break;
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
    return sfail(EQ_ERR_OOM, "eq_serve_submit: request footprint exceeds the server's HBM budget");
  }
  if ((int)s->queue.size() >= s->max_queue) { delete r; return sfail(EQ_ERR_BUSY, "eq_serve_submit: queue full"); }
  r->id = s->next_id++;
  s->reqs[r->id] = r;
  s->queue.push_back(r);
  *ticket = r->id;
  s->cv_work.notify_one();
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
  cudaSetDevice(s->device);
  for (Slot& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.h_norms) cudaFreeHost(sl.h_norms);
  }
  for (auto& kv : s->idle_plans) eq_plan_destroy(kv.second);
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
}

}  // extern "C"
