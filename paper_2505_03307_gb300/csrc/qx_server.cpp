// Request loop with continuous batching for many circuits (qx_server_*).
//
// Requests (circuits) are queued as they arrive.  Planner threads turn each
// into a push-through plan (its non-Clifford gates as Pauli rotations, then
// one Clifford pass) and a reservation: an upper bound on the bytes of term
// storage it can need, from its generator count and rotation count (each
// rotation at most doubles a generator's terms).  Engine threads, each with
// its own CUDA stream, admit planned requests in arrival order into a batch
// while the live ledger of reserved bytes stays within hbm_budget (the memory
// side of the feasibility region of Sec. IV, n1* <= M_max / (c n)), and
// propagate the whole batch in one term store (qx::batch_propagate: the
// generator id becomes (request, generator), every rotation step is one
// launch sequence for all requests).  Requests that arrive while batches run
// join the next batch as soon as an engine and memory are free; several
// batches run on the device at once.  A request whose bound alone exceeds the
// budget runs by itself once nothing else runs, with the budget enforced on
// its exact counted sizes (QX_EBUDGET if it really needs more).
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
  qx_plan* plan = nullptr;
  size_t reserve = 0;  // bytes the ledger holds for it while it runs
  int W = 1;
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
  std::condition_variable cv_plan;   // planners: a request arrived
  std::condition_variable cv_ready;  // engines: a request was planned or memory came free
  std::condition_variable cv_done;   // waiters: a request finished
  std::deque<std::shared_ptr<Request>> to_plan;
  std::map<uint64_t, std::shared_ptr<Request>> ready;  // planned, by arrival
  std::map<uint64_t, std::shared_ptr<Request>> all;
  std::vector<std::thread> planners, engines;
  uint64_t next_ticket = 1;
  size_t in_use = 0, peak_in_use = 0;  // the ledger: bytes reserved by running batches
  int running = 0;                     // batches on the device
  bool alone_running = false;          // a request over the budget runs by itself
  bool stopping = false;
  uint64_t completed = 0, failed = 0, alone = 0, batches = 0, batched = 0;
  std::vector<double> latencies;
  int device = 0;
};

namespace {

// Upper bound on the bytes of term storage of a push-through plan: each of
// its R rotations at most doubles each of its n generators (and no generator
// holds more than 4^n - 1 strings); a rotation step holds its input, its
// output of at most twice as many terms, the index (two 16-byte slots per
// input term) and two 8-byte words per input term, and the results are
// written beside the last step's output.
size_t reservation(const qx_plan* p, int precision) {
  size_t rot = 0;
  for (const Step& s : p->program) rot += s.kind == kStepRot ? 1 : 0;
  const int lg = int(std::min<size_t>(rot, 40));
  unsigned long long per = 1ull << lg;
  if (p->n < 20) per = std::min<unsigned long long>(per, (1ull << (2 * p->n)) - 1);
  const size_t tb = size_t(16 * p->W + (precision == 32 ? 4 : 8) + 4);
  return size_t(per) * size_t(p->n) * (2 * tb + 40) + size_t(p->n) * 64 + 4096;
}

void finish(qx_server* s, const std::shared_ptr<Request>& r, qx_status st, const std::string& msg,
            qx_result* res) {
  r->status = st;
  r->error = msg;
  r->result = res;
  r->latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - r->submitted).count();
  r->done = true;
  qx_free_plan(r->plan);
  r->plan = nullptr;
  if (st == QX_OK) {
    s->completed++;
    s->latencies.push_back(r->latency_ms);
  } else {
    s->failed++;
  }
}

void planner_main(qx_server* s) {
  while (true) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv_plan.wait(lock, [&] { return s->stopping || !s->to_plan.empty(); });
      if (s->to_plan.empty()) break;  // stopping
      r = s->to_plan.front();
      s->to_plan.pop_front();
      if (s->stopping) {
        finish(s, r, QX_EINVAL, "server stopped", nullptr);
        s->cv_done.notify_all();
        continue;
      }
    }
    // the checks of qx_load_circuit, then the plan takes the request's
    // instructions over (nothing else reads them)
    qx_plan* p = nullptr;
    qx::clear_error();
    qx_status st = qx::validate_instrs(r->n, r->ins.data(), r->ins.size());
    if (st == QX_OK) st = qx::build_plan_pushthrough(r->n, std::move(r->ins), &p);
    const std::string msg = st == QX_OK ? std::string() : std::string(qx_last_error());
    std::lock_guard<std::mutex> lock(s->mu);
    if (st != QX_OK) {
      finish(s, r, st, msg, nullptr);
      s->cv_done.notify_all();
      continue;
    }
    r->plan = p;
    r->W = p->W;
    r->reserve = reservation(p, s->opts.precision);
    s->ready[r->ticket] = r;
    s->cv_ready.notify_one();
  }
}

// Whether an engine can start a batch now (the lock is held).
bool admissible(const qx_server* s) {
  if (s->ready.empty() || s->alone_running) return false;
  const size_t budget = s->opts.hbm_budget;
  const size_t first = s->ready.begin()->second->reserve;
  if (budget && first > budget) return s->running == 0;  // runs alone
  return !budget || s->in_use + first <= budget;
}

void engine_main(qx_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t stream = nullptr;
  if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    stream = nullptr;  // requests then fail with the library's own error (no device)
  }
  const size_t budget = s->opts.hbm_budget;
  const size_t max_batch = size_t(s->opts.max_batch > 0 ? s->opts.max_batch : 256);
  while (true) {
    std::vector<std::shared_ptr<Request>> batch;
    size_t reserved = 0;
    bool alone = false;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv_ready.wait(lock, [&] { return s->stopping || admissible(s); });
      if (s->stopping) {  // fail what waits for admission; running batches finish
        for (auto& kv : s->ready) finish(s, kv.second, QX_EINVAL, "server stopped", nullptr);
        s->ready.clear();
        s->cv_done.notify_all();
        break;
      }
      const auto& first = s->ready.begin()->second;
      if (budget && first->reserve > budget) {
        alone = true;
        batch.push_back(first);
        s->alone_running = true;
        s->alone++;
      } else {
        const int W = first->W;
        for (const auto& kv : s->ready) {  // in arrival order, stop at the first that waits
          const auto& r = kv.second;
          if (r->W != W || batch.size() >= max_batch) break;
          if (budget && (r->reserve > budget || s->in_use + reserved + r->reserve > budget)) break;
          batch.push_back(r);
          reserved += r->reserve;
        }
      }
      for (const auto& r : batch) s->ready.erase(r->ticket);
      s->in_use += reserved;
      s->peak_in_use = std::max(s->peak_in_use, s->in_use);
      s->running++;
      s->batches++;
      s->batched += batch.size();
    }
    std::vector<BatchRequest> br(batch.size());
    for (size_t k = 0; k < batch.size(); ++k) br[k].plan = batch[k]->plan;
    const qx_status st =
        batch_propagate(br, s->opts.precision, s->opts.eps, alone ? budget : 0, stream);
    const std::string msg = st == QX_OK ? std::string() : std::string(qx_last_error());
    std::lock_guard<std::mutex> lock(s->mu);
    s->in_use -= reserved;
    s->running--;
    if (alone) s->alone_running = false;
    for (size_t k = 0; k < batch.size(); ++k)
      finish(s, batch[k], st, msg, st == QX_OK ? br[k].result : nullptr);
    s->cv_done.notify_all();
    s->cv_ready.notify_all();
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
  o->slots = 2;
  o->precision = 64;
  o->max_batch = 256;
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
  if (opts.max_batch < 0) return fail(QX_EINVAL, "max_batch must be >= 0");
  auto* s = new (std::nothrow) qx_server;
  if (!s) return fail(QX_ENOMEM, "host allocation failed");
  s->opts = opts;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    cudaGetLastError();
    s->device = 0;
  }
  // Planning is host work that bounds the loop's throughput once requests
  // queue up; idle planners sleep on a condition variable.  They get the
  // cores left after the engines and two more (the caller and the rest of
  // the process), at least one and at most 16.
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const unsigned spare = unsigned(opts.slots) + 2u;
  const int planners = int(std::min(16u, hw > spare ? hw - spare : 1u));
  for (int k = 0; k < planners; ++k) s->planners.emplace_back(planner_main, s);
  for (int k = 0; k < opts.slots; ++k) s->engines.emplace_back(engine_main, s);
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
  if (s->opts.max_queue && s->to_plan.size() + s->ready.size() >= s->opts.max_queue)
    return fail(QX_ECAP, "request queue is full");
  r->ticket = s->next_ticket++;
  s->all[r->ticket] = r;
  s->to_plan.push_back(r);
  *ticket = r->ticket;
  s->cv_plan.notify_one();
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
  // the engine's stream dies with the server: later work on the result goes
  // to the default stream (the engine synchronised its stream already)
  result_set_stream(r->result, nullptr);
  *out = r->result;
  r->result = nullptr;
  return QX_OK;
}

qx_status qx_server_stats(qx_server* s, qx_serve_stats* st) {
  clear_error();
  if (!s || !st) return fail(QX_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  st->completed = s->completed;
  st->failed = s->failed;
  st->alone = s->alone;
  st->queued = s->to_plan.size() + s->ready.size();
  st->running = uint64_t(s->running);
  st->p50_ms = percentile(s->latencies, 0.50);
  st->p99_ms = percentile(s->latencies, 0.99);
  st->max_ms = s->latencies.empty() ? 0.0 : *std::max_element(s->latencies.begin(), s->latencies.end());
  st->batches = s->batches;
  st->mean_batch = s->batches ? double(s->batched) / double(s->batches) : 0.0;
  st->peak_reserved = s->peak_in_use;
  return QX_OK;
}

void qx_server_destroy(qx_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stopping = true;
  }
  s->cv_plan.notify_all();
  s->cv_ready.notify_all();
  for (auto& t : s->planners) t.join();
  for (auto& t : s->engines) t.join();
  for (auto& kv : s->all) {
    qx_free_result(kv.second->result);
    qx_free_plan(kv.second->plan);
  }
  delete s;
}

}  // extern "C"
