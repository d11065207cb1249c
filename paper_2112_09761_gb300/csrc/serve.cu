// serve.cu — a query server over resident graphs with continuous batching.
//
// Queries (graph, pattern, induced) are submitted from any host thread and get
// a ticket.  A scheduler thread admits pending queries in arrival order
// whenever a stream slot is free and the query's execution memory (its plan's
// DFS buffers, counters and root lists; Section 7.2 (3) adaptive buffering)
// fits in the remaining budget; a query that does not fit yet is passed over
// so that smaller ones behind it can start (they overlap on the device).
// Plans are built on first use and kept per (graph, pattern, induced) key;
// several in-flight queries of one key use separate plan instances.  Every
// wait on the device is an event query polled by the host, so nothing spins on
// the GPU.  Latency = completion - submission, host steady clock.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "gpm_internal.cuh"

namespace gpm {
cudaError_t plan_launch_async(gpm_plan_t* p, uint64_t lo, uint64_t hi, uint32_t* list_out,
                              uint64_t cap, cudaStream_t s);
gpm_status plan_finish(gpm_plan_t* p, Control* res);
size_t plan_exec_bytes(const gpm_plan_t* p);
gpm_status api_fail(gpm_status st, const std::string& msg);
}  // namespace gpm

using namespace gpm;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum QState { kPending = 0, kRunning = 1, kDone = 2 };

struct Query {
  gpm_graph* g = nullptr;
  gpm_pattern pat{};
  int induced = 0;
  double t_submit = 0, t_start = 0, t_done = 0;
  QState state = kPending;
  gpm_status status = GPM_OK;
  uint64_t result = 0;
  size_t bytes = 0;
  int slot = -1;
  gpm_plan_t* plan = nullptr;
  std::string key;
};

std::string key_of(const gpm_graph* g, const gpm_pattern& p, int induced) {
  std::string k((const char*)&g, sizeof(g));
  k.append((const char*)&p, sizeof(p));
  k.push_back((char)induced);
  return k;
}

}  // namespace

struct gpm_server_s {
  size_t budget = 0, used = 0;
  int device = 0;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<uint64_t> slot_ticket;  // 0 = free
  std::deque<uint64_t> pending;
  std::unordered_map<uint64_t, Query> queries;
  std::map<std::string, std::vector<gpm_plan_t*>> free_plans;
  std::vector<gpm_plan_t*> all_plans;
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false;
  uint64_t next_ticket = 1;
  uint64_t completed = 0, admitted = 0, peak_inflight = 0;
};

namespace {

// One scheduler pass under the lock: retire finished slots, admit pending
// queries.  Returns true if anything changed.
bool step(gpm_server_s* S) {
  bool changed = false;
  const int nslots = (int)S->streams.size();
  for (int i = 0; i < nslots; i++) {
    const uint64_t t = S->slot_ticket[i];
    if (!t) continue;
    const cudaError_t q = cudaEventQuery(S->events[i]);
    if (q == cudaErrorNotReady) continue;
    Query& Q = S->queries[t];
    Q.t_done = now_s();
    if (q != cudaSuccess) {
      Q.status = GPM_E_CUDA;
    } else {
      Control r;
      Q.status = plan_finish(Q.plan, &r);
      Q.result = r.result;
    }
    Q.state = kDone;
    S->used -= Q.bytes;
    S->free_plans[Q.key].push_back(Q.plan);
    Q.plan = nullptr;
    S->slot_ticket[i] = 0;
    S->completed++;
    changed = true;
  }
  for (auto it = S->pending.begin(); it != S->pending.end();) {
    int slot = -1;
    for (int i = 0; i < nslots; i++)
      if (!S->slot_ticket[i]) { slot = i; break; }
    if (slot < 0) break;
    const uint64_t t = *it;
    Query& Q = S->queries[t];
    gpm_plan_t* p = nullptr;
    auto& fl = S->free_plans[Q.key];
    if (!fl.empty()) {
      p = fl.back();
      fl.pop_back();
    } else {
      gpm_plan_t* np = nullptr;
      const gpm_status st =
          gpm_plan(Q.g, &Q.pat, Q.induced, GPM_COUNT, nullptr, S->streams[slot], &np);
      if (st != GPM_OK) {
        Q.status = st;
        Q.state = kDone;
        Q.t_done = now_s();
        it = S->pending.erase(it);
        changed = true;
        continue;
      }
      S->all_plans.push_back(np);
      p = np;
    }
    const size_t bytes = plan_exec_bytes(p);
    const bool idle = (S->used == 0);
    if (S->used + bytes > S->budget && !idle) {
      fl.push_back(p);  // does not fit yet: let smaller queries behind it go
      ++it;
      continue;
    }
    Q.plan = p;
    Q.bytes = bytes;
    Q.slot = slot;
    Q.t_start = now_s();
    cudaError_t e = plan_launch_async(p, 0, ~0ull, nullptr, 0, S->streams[slot]);
    if (e == cudaSuccess) e = cudaEventRecord(S->events[slot], S->streams[slot]);
    if (e != cudaSuccess) {
      Q.status = GPM_E_CUDA;
      Q.state = kDone;
      Q.t_done = now_s();
      fl.push_back(p);
      Q.plan = nullptr;
      it = S->pending.erase(it);
      changed = true;
      continue;
    }
    Q.state = kRunning;
    S->used += bytes;
    S->slot_ticket[slot] = t;
    S->admitted++;
    uint64_t inflight = 0;
    for (int i = 0; i < nslots; i++) inflight += S->slot_ticket[i] != 0;
    if (inflight > S->peak_inflight) S->peak_inflight = inflight;
    it = S->pending.erase(it);
    changed = true;
  }
  return changed;
}

void worker_main(gpm_server_s* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop) {
    const bool changed = step(S);
    if (changed) S->cv.notify_all();
    bool busy = !S->pending.empty();
    for (uint64_t t : S->slot_ticket) busy |= t != 0;
    if (busy) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(changed ? 0 : 20));
      lk.lock();
    } else {
      S->cv.wait_for(lk, std::chrono::milliseconds(50));
    }
  }
}

}  // namespace

extern "C" {

gpm_status gpm_server_create(size_t mem_budget, uint32_t max_inflight, gpm_server_t** out) {
  if (!out || max_inflight == 0 || max_inflight > 256)
    return api_fail(GPM_E_INVALID_ARG, "gpm_server_create: bad arguments");
  gpm_server_s* S = new gpm_server_s();
  S->budget = mem_budget;
  cudaError_t e = cudaGetDevice(&S->device);
  for (uint32_t i = 0; i < max_inflight && e == cudaSuccess; i++) {
    cudaStream_t st;
    cudaEvent_t ev;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) break;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) { cudaStreamDestroy(st); break; }
    S->streams.push_back(st);
    S->events.push_back(ev);
    S->slot_ticket.push_back(0);
  }
  if (e != cudaSuccess) {
    gpm_server_free(S);
    return api_fail(GPM_E_CUDA, std::string("gpm_server_create: ") + cudaGetErrorString(e));
  }
  S->worker = std::thread(worker_main, S);
  *out = S;
  return GPM_OK;
}

gpm_status gpm_server_submit(gpm_server_t* S, gpm_graph* g, const gpm_pattern* p, int induced,
                             uint64_t* ticket) {
  if (!S || !g || !p || !ticket) return api_fail(GPM_E_INVALID_ARG, "gpm_server_submit: NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  const uint64_t t = S->next_ticket++;
  Query& Q = S->queries[t];
  Q.g = g;
  Q.pat = *p;
  Q.induced = induced ? 1 : 0;
  Q.t_submit = now_s();
  Q.key = key_of(g, *p, Q.induced);
  S->pending.push_back(t);
  *ticket = t;
  S->cv.notify_all();
  return GPM_OK;
}

gpm_status gpm_server_poll(gpm_server_t* S, uint64_t ticket, int* done, uint64_t* count,
                           double* latency_s) {
  if (!S || !done) return api_fail(GPM_E_INVALID_ARG, "gpm_server_poll: NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->queries.find(ticket);
  if (it == S->queries.end()) return api_fail(GPM_E_INVALID_ARG, "gpm_server_poll: unknown ticket");
  const Query& Q = it->second;
  *done = Q.state == kDone;
  if (!*done) return GPM_OK;
  if (Q.status != GPM_OK) return Q.status;
  if (count) *count = Q.result;
  if (latency_s) *latency_s = Q.t_done - Q.t_submit;
  return GPM_OK;
}

gpm_status gpm_server_wait(gpm_server_t* S, uint64_t ticket, double timeout_s, uint64_t* count,
                           double* latency_s) {
  if (!S) return api_fail(GPM_E_INVALID_ARG, "gpm_server_wait: NULL server");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->queries.find(ticket);
  if (it == S->queries.end()) return api_fail(GPM_E_INVALID_ARG, "gpm_server_wait: unknown ticket");
  const double deadline = now_s() + timeout_s;
  while (it->second.state != kDone) {
    if (now_s() >= deadline) return api_fail(GPM_E_TIMEOUT, "gpm_server_wait: timed out");
    S->cv.wait_for(lk, std::chrono::milliseconds(5));
  }
  const Query& Q = it->second;
  if (Q.status != GPM_OK) return Q.status;
  if (count) *count = Q.result;
  if (latency_s) *latency_s = Q.t_done - Q.t_submit;
  return GPM_OK;
}

gpm_status gpm_server_stats(gpm_server_t* S, uint64_t* completed, uint64_t* pending,
                            uint64_t* peak_inflight, size_t* bytes_in_use) {
  if (!S) return api_fail(GPM_E_INVALID_ARG, "gpm_server_stats: NULL server");
  std::lock_guard<std::mutex> lk(S->mu);
  if (completed) *completed = S->completed;
  if (pending) *pending = S->pending.size();
  if (peak_inflight) *peak_inflight = S->peak_inflight;
  if (bytes_in_use) *bytes_in_use = S->used;
  return GPM_OK;
}

void gpm_server_free(gpm_server_t* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto st : S->streams) cudaStreamSynchronize(st);
  for (auto p : S->all_plans) gpm_plan_free(p);
  for (auto ev : S->events) cudaEventDestroy(ev);
  for (auto st : S->streams) cudaStreamDestroy(st);
  delete S;
}

}  // extern "C"
