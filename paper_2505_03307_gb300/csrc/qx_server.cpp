// Request loop with continuous batching for many circuits (qx_server_*).
//
// Requests (circuits) are queued as they arrive.  `slots` host workers, each
// with its own non-blocking CUDA stream, take requests in arrival order as
// soon as a slot and memory are free, so the device work of several circuits
// overlaps.  Admission follows the memory side of the feasibility region of
// Sec. IV (n1* <= M_max / (c n)): every slot may hold hbm_budget / slots bytes of
// term storage; a request that needs more stops with QX_EBUDGET inside its
// share, goes back to the head of the queue marked exclusive, and runs alone
// with the whole budget once the other slots have drained.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "qx_common.h"

using namespace qx;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  int n = 0;
  std::vector<qx_instr> ins;
  Clock::time_point submitted;
  bool exclusive = false;
  bool done = false;
  qx_status status = QX_OK;
  std::string error;
  qx_result* result = nullptr;
  double latency_ms = 0.0;
};

}  // namespace

struct qx_server {
  qx_server_opts opts{};
  std::mutex mu;
  std::condition_variable cv_work;  // workers: a request or a slot became available
  std::condition_variable cv_done;  // waiters: a request finished
  std::deque<std::shared_ptr<Request>> queue;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  std::vector<std::thread> workers;
  uint64_t next_ticket = 1;
  int running = 0;
  bool exclusive_running = false;
  bool stopping = false;
  uint64_t completed = 0, failed = 0, retried = 0;
  std::vector<double> latencies;
  int device = 0;
};

namespace {

void run_one(qx_server* s, const std::shared_ptr<Request>& r, cudaStream_t stream, size_t budget) {
  qx_circuit* c = nullptr;
  qx_plan* p = nullptr;
  qx_status st = qx_load_circuit(r->n, r->ins.data(), r->ins.size(), &c);
  if (st == QX_OK) st = qx_group_ops(c, &p);
  qx_result* res = nullptr;
  if (st == QX_OK) {
    qx_prop_opts o;
    qx_default_opts(&o);
    o.precision = s->opts.precision;
    o.eps = s->opts.eps;
    o.hbm_budget = budget;
    o.stream = stream;
    st = qx_propagate(p, &o, &res);
  }
  const std::string msg = st == QX_OK ? std::string() : std::string(qx_last_error());
  qx_free_plan(p);
  qx_free_circuit(c);
  std::lock_guard<std::mutex> lock(s->mu);
  s->running--;
  if (r->exclusive) s->exclusive_running = false;
  if (st == QX_EBUDGET && !r->exclusive && s->opts.slots > 1) {
    // over its share: run again alone with the whole budget
    r->exclusive = true;
    s->queue.push_front(r);
    s->retried++;
    s->cv_work.notify_all();
    return;
  }
  r->status = st;
  r->error = msg;
  r->result = res;
  r->latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - r->submitted).count();
  r->done = true;
  if (st == QX_OK) {
    s->completed++;
    s->latencies.push_back(r->latency_ms);
  } else {
    s->failed++;
  }
  s->cv_done.notify_all();
  s->cv_work.notify_all();
}

void worker_main(qx_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t stream = nullptr;
  const bool have_stream = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess;
  if (!have_stream) {
    cudaGetLastError();
    stream = nullptr;  // requests then fail with the library's own error (no device)
  }
  const size_t share = s->opts.hbm_budget ? s->opts.hbm_budget / size_t(s->opts.slots) : 0;
  while (true) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv_work.wait(lock, [&] {
        if (s->stopping) return true;
        if (s->queue.empty() || s->exclusive_running) return false;
        // an exclusive request waits until it is alone
        return !s->queue.front()->exclusive || s->running == 0;
      });
      if (s->stopping && s->queue.empty()) break;
      if (s->stopping) {  // drain: fail what is still queued
        r = s->queue.front();
        s->queue.pop_front();
        r->status = QX_EINVAL;
        r->error = "server stopped";
        r->done = true;
        s->failed++;
        s->cv_done.notify_all();
        continue;
      }
      r = s->queue.front();
      s->queue.pop_front();
      s->running++;
      if (r->exclusive) s->exclusive_running = true;
    }
    run_one(s, r, stream, r->exclusive ? s->opts.hbm_budget : share);
  }
  if (stream) cudaStreamDestroy(stream);
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * double(v.size() - 1);
  const size_t lo = size_t(pos);
  const size_t hi = std::min(lo + 1, v.size() - 1);
  return v[lo] + (v[hi] - v[lo]) * (pos - double(lo));
}

}  // namespace

extern "C" {

void qx_server_default_opts(qx_server_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->slots = 4;
  o->precision = 64;
}

qx_status qx_server_create(const qx_server_opts* o, qx_server** out) {
  clear_error();
  if (!out) return fail(QX_EINVAL, "out is NULL");
  qx_server_opts opts;
  qx_server_default_opts(&opts);
  if (o) opts = *o;
  if (opts.slots < 1 || opts.slots > 256) return fail(QX_EINVAL, "slots must be in 1..256");
  if (opts.precision != 64 && opts.precision != 32)
    return fail(QX_EINVAL, "precision must be 64 or 32");
  if (!(opts.eps >= 0.0)) return fail(QX_EINVAL, "eps must be >= 0");
  auto* s = new (std::nothrow) qx_server;
  if (!s) return fail(QX_ENOMEM, "host allocation failed");
  s->opts = opts;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    cudaGetLastError();
    s->device = 0;
  }
  for (int k = 0; k < opts.slots; ++k) s->workers.emplace_back(worker_main, s);
  *out = s;
  return QX_OK;
}

qx_status qx_server_submit(qx_server* s, int n, const qx_instr* ins, size_t m, uint64_t* ticket) {
  clear_error();
  if (!s || !ticket) return fail(QX_EINVAL, "NULL argument");
  if (m && !ins) return fail(QX_EINVAL, "ins is NULL");
  auto r = std::make_shared<Request>();
  r->n = n;
  r->ins.assign(ins, ins + m);
  r->submitted = Clock::now();
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->stopping) return fail(QX_EINVAL, "server is stopping");
  if (s->opts.max_queue && s->queue.size() >= s->opts.max_queue)
    return fail(QX_ECAP, "request queue is full");
  r->ticket = s->next_ticket++;
  s->all[r->ticket] = r;
  s->queue.push_back(r);
  *ticket = r->ticket;
  s->cv_work.notify_one();
  return QX_OK;
}

qx_status qx_server_poll(qx_server* s, uint64_t ticket, int* done) {
  clear_error();
  if (!s || !done) return fail(QX_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(QX_EINVAL, "unknown ticket");
  *done = it->second->done ? 1 : 0;
  return QX_OK;
}

qx_status qx_server_wait(qx_server* s, uint64_t ticket, qx_result** out, double* latency_ms) {
  clear_error();
  if (!s || !out) return fail(QX_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(QX_EINVAL, "unknown ticket");
  std::shared_ptr<Request> r = it->second;
  s->cv_done.wait(lock, [&] { return r->done; });
  s->all.erase(ticket);
  if (latency_ms) *latency_ms = r->latency_ms;
  if (r->status != QX_OK) return fail(r->status, "request " + std::to_string(ticket) + ": " + r->error);
  // the worker's stream dies with the server: later work on the result goes
  // to the default stream (the worker synchronised its stream already)
  result_set_stream(r->result, nullptr);
  *out = r->result;
  return QX_OK;
}

qx_status qx_server_stats(qx_server* s, qx_serve_stats* st) {
  clear_error();
  if (!s || !st) return fail(QX_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  st->completed = s->completed;
  st->failed = s->failed;
  st->retried_exclusive = s->retried;
  st->queued = s->queue.size();
  st->running = uint64_t(s->running);
  st->p50_ms = percentile(s->latencies, 0.50);
  st->p99_ms = percentile(s->latencies, 0.99);
  st->max_ms = s->latencies.empty() ? 0.0 : *std::max_element(s->latencies.begin(), s->latencies.end());
  return QX_OK;
}

void qx_server_destroy(qx_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& kv : s->all)
    if (kv.second->result) qx_free_result(kv.second->result);
  delete s;
}

}  // extern "C"
