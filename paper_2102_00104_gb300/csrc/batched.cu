// batched.cu -- batched and serve forms: many independent TT-SVDs (Alg. 2 each).
//
// Batched: every job runs the single-tensor driver (tt_svd_ex) on one of a pool
// of library-owned streams, forked from the caller's stream and joined back
// into it with events; the call stays asynchronous and graph-capturable.
//
// Serve: a host scheduler thread implements continuous batching over slots
// (one stream each) and an HBM budget; workspaces are carved first-fit out of
// one arena allocated at creation.  Completion is observed with
// cudaEventQuery, never by a device-side wait.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "engine.h"
#include "tt_svd.h"

namespace tt {
namespace {

size_t align256b(size_t x) { return (x + 255) & ~(size_t)255; }

__global__ void k_copy_status(const int* status_word, int* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = *status_word;
}

tt_status job_work_bytes(const tt_job& j, size_t* wb) {
  size_t cb = 0;
  return tt_query(j.d, j.n, j.r_max, j.tol, j.dtype, &cb, wb);
}

tt_status run_job(const tt_job& j, void* work, size_t wbytes, cudaStream_t s) {
  tt_status st = tt_svd(j.X, j.dtype, j.d, j.n, j.r_max, j.tol, j.cores_out, j.ranks_out,
                        j.sigma_out, j.err2_out, work, wbytes, s);
  if (st != TT_OK) return st;
  if (j.status_out) {
    // the device status word sits at the start of the job's workspace
    k_copy_status<<<1, 32, 0, s>>>(static_cast<const int*>(work), j.status_out);
    if (cudaGetLastError() != cudaSuccess) return TT_ECUDA;
  }
  return TT_OK;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ---- the pool of streams used by tt_svd_batched -----------------------------------
// (tt_svd_batched uses the first "batched.streams" of them, 64 by default: measured on
// GB300 for the 256-job batch, 183 / 141 / 131 / 132 ms with 16 / 32 / 64 / 128 streams)
constexpr int kPoolStreams = 128;
struct StreamPool {
  int dev = -1;
  cudaStream_t s[kPoolStreams];
  cudaEvent_t fork, join[kPoolStreams];
};
std::mutex g_pool_mu;
std::map<int, StreamPool*> g_pools;

cudaError_t get_pool(StreamPool** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  auto it = g_pools.find(dev);
  if (it != g_pools.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  StreamPool* p = new StreamPool;
  p->dev = dev;
  for (int i = 0; i < kPoolStreams; ++i) {
    if ((e = cudaStreamCreateWithFlags(&p->s[i], cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&p->join[i], cudaEventDisableTiming)) != cudaSuccess) return e;
  }
  if ((e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming)) != cudaSuccess) return e;
  g_pools[dev] = p;
  *out = p;
  return cudaSuccess;
}

}  // namespace
}  // namespace tt

using namespace tt;

extern "C" {

tt_status tt_batched_query(int batch, const tt_job* jobs, size_t* work_bytes) {
  if (batch < 0 || (batch > 0 && !jobs) || !work_bytes) return TT_EINVAL;
  size_t total = 0;
  for (int i = 0; i < batch; ++i) {
    size_t wb = 0;
    tt_status st = job_work_bytes(jobs[i], &wb);
    if (st != TT_OK) return st;
    total += align256b(wb);
  }
  *work_bytes = total;
  return TT_OK;
}

tt_status tt_svd_batched(int batch, const tt_job* jobs, void* work, size_t work_bytes,
                         void* stream) {
  if (batch < 0 || (batch > 0 && (!jobs || !work)) || ((uintptr_t)work & 255)) return TT_EINVAL;
  if (batch == 0) return TT_OK;
  std::vector<size_t> wb(batch), off(batch);
  size_t total = 0;
  for (int i = 0; i < batch; ++i) {
    tt_status st = job_work_bytes(jobs[i], &wb[i]);
    if (st != TT_OK) return st;
    off[i] = total;
    total += align256b(wb[i]);
  }
  if (work_bytes < total) return TT_ENOMEM;
  StreamPool* P = nullptr;
  if (get_pool(&P) != cudaSuccess) return TT_ECUDA;
  cudaStream_t cs = (cudaStream_t)stream;
  // longest jobs first, each onto the stream with the least estimated work so far
  // (greedy LPT on a rough per-job time from the plan)
  std::vector<double> cost(batch);
  for (int i = 0; i < batch; ++i)
    cost[i] = job_cost_estimate(jobs[i].d, jobs[i].n, jobs[i].r_max, jobs[i].tol, (int)jobs[i].dtype);
  std::vector<int> order(batch);
  for (int i = 0; i < batch; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  const int ns = std::min(batch, std::max(1, std::min(kPoolStreams, tune_get("batched.streams", 64))));
  std::vector<double> load(ns, 0.0);
  if (cudaEventRecord(P->fork, cs) != cudaSuccess) return TT_ECUDA;
  for (int k = 0; k < ns; ++k)
    if (cudaStreamWaitEvent(P->s[k], P->fork, 0) != cudaSuccess) return TT_ECUDA;
  tt_status result = TT_OK;
  for (int t = 0; t < batch; ++t) {
    const int i = order[t];
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[k] += cost[i];
    tt_status st = run_job(jobs[i], static_cast<char*>(work) + off[i], wb[i], P->s[k]);
    if (st != TT_OK && result == TT_OK) result = st;
  }
  for (int k = 0; k < ns; ++k) {
    if (cudaEventRecord(P->join[k], P->s[k]) != cudaSuccess) return TT_ECUDA;
    if (cudaStreamWaitEvent(cs, P->join[k], 0) != cudaSuccess) return TT_ECUDA;
  }
  return result;
}

}  // extern "C"

// ---- serve ------------------------------------------------------------------------------
struct tt_server {
  struct Req {
    uint64_t ticket;
    tt_job job;
    size_t ws;          // workspace bytes
    size_t acct;        // accounted bytes: input + cores + workspace
    size_t arena_off = 0;
    int slot = -1;
    tt_job_result res{};
    bool done = false;
    cudaEvent_t ready = nullptr;  // recorded on the submitter's stream: inputs and outputs ready
    double cost = 0.0;            // estimated device seconds (job_cost_estimate)
  };
  size_t budget = 0, arena_bytes = 0, accounted = 0;
  double timeout_s = 60.0;
  int policy = TT_SERVE_FIFO;
  double max_wait_s = 1.0;
  char* arena = nullptr;
  std::vector<std::pair<size_t, size_t>> free_list;  // (offset, size), sorted by offset
  std::vector<cudaStream_t> slot_stream;
  std::vector<cudaEvent_t> slot_event;
  std::vector<uint64_t> slot_ticket;                 // 0 = free
  std::vector<cudaEvent_t> spare_events;             // recycled ready events
  std::map<uint64_t, Req> reqs;
  std::deque<uint64_t> queue;
  uint64_t next_ticket = 1;
  std::mutex mu;
  std::condition_variable cv;                        // wakes the scheduler and pollers
  bool stop = false;
  int device = 0;
  std::thread worker;

  bool arena_alloc(size_t n, size_t* off) {
    n = (n + 255) & ~(size_t)255;
    for (size_t i = 0; i < free_list.size(); ++i) {
      if (free_list[i].second >= n) {
        *off = free_list[i].first;
        free_list[i].first += n;
        free_list[i].second -= n;
        if (free_list[i].second == 0) free_list.erase(free_list.begin() + i);
        return true;
      }
    }
    return false;
  }
  void arena_free(size_t off, size_t n) {
    n = (n + 255) & ~(size_t)255;
    auto it = std::lower_bound(free_list.begin(), free_list.end(), std::make_pair(off, (size_t)0));
    it = free_list.insert(it, {off, n});
    // merge with neighbours
    size_t i = it - free_list.begin();
    if (i + 1 < free_list.size() && free_list[i].first + free_list[i].second == free_list[i + 1].first) {
      free_list[i].second += free_list[i + 1].second;
      free_list.erase(free_list.begin() + i + 1);
    }
    if (i > 0 && free_list[i - 1].first + free_list[i - 1].second == free_list[i].first) {
      free_list[i - 1].second += free_list[i].second;
      free_list.erase(free_list.begin() + i);
    }
  }

  // one scheduler pass under the lock: retire finished slots, admit queued requests
  void pass() {
    for (size_t k = 0; k < slot_stream.size(); ++k) {
      const uint64_t t = slot_ticket[k];
      if (!t) continue;
      const cudaError_t q = cudaEventQuery(slot_event[k]);
      if (q == cudaErrorNotReady) continue;
      Req& r = reqs[t];
      r.res.t_done = now_s();
      if (q != cudaSuccess && r.res.status == TT_OK) r.res.status = TT_ECUDA;
      if (r.res.status == TT_OK && r.job.status_out == nullptr) {
        int v = 0;  // the job's device status word (start of its workspace), on its own stream
        if (cudaMemcpyAsync(&v, arena + r.arena_off, sizeof(int), cudaMemcpyDeviceToHost,
                            slot_stream[k]) == cudaSuccess &&
            cudaStreamSynchronize(slot_stream[k]) == cudaSuccess && v)
          r.res.status = (v & DEV_ERR_SHAPE)     ? TT_EINVAL
                         : (v & DEV_ERR_TIMEOUT) ? TT_ETIMEOUT
                                                 : TT_ENUMERIC;
      }
      r.done = true;
      if (r.ready) { spare_events.push_back(r.ready); r.ready = nullptr; }
      arena_free(r.arena_off, r.ws);
      accounted -= r.acct;
      slot_ticket[k] = 0;
      cv.notify_all();
    }
    while (!queue.empty()) {
      int slot = -1;
      for (size_t k = 0; k < slot_ticket.size(); ++k)
        if (!slot_ticket[k]) { slot = (int)k; break; }
      if (slot < 0) break;
      // the next request: the head of the queue, or (SHORTEST) the least estimated work
      // unless the head has waited max_wait_s
      size_t pick = 0;
      if (policy == TT_SERVE_SHORTEST && now_s() - reqs[queue.front()].res.t_submit < max_wait_s) {
        for (size_t q = 1; q < queue.size(); ++q)
          if (reqs[queue[q]].cost < reqs[queue[pick]].cost) pick = q;
      }
      Req& r = reqs[queue[pick]];
      if (accounted + r.acct > budget) break;   // wait for memory to free up
      size_t off = 0;
      if (!arena_alloc(r.ws, &off)) break;
      queue.erase(queue.begin() + (std::ptrdiff_t)pick);
      r.arena_off = off;
      r.slot = slot;
      r.res.t_start = now_s();
      accounted += r.acct;
      slot_ticket[slot] = r.ticket;
      // the job's kernels start only after the submitter's stream has reached the submit
      tt_status st = TT_OK;
      if (r.ready && cudaStreamWaitEvent(slot_stream[slot], r.ready, 0) != cudaSuccess) st = TT_ECUDA;
      if (st == TT_OK) st = run_job(r.job, arena + off, r.ws, slot_stream[slot]);
      if (st != TT_OK) r.res.status = st;
      cudaEventRecord(slot_event[slot], slot_stream[slot]);
    }
  }

  void loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
      pass();
      bool busy = false;
      for (uint64_t t : slot_ticket) busy |= (t != 0);
      // short sleeps while work is in flight, longer ones when idle (both bounded)
      cv.wait_for(lk, busy ? std::chrono::microseconds(20) : std::chrono::milliseconds(2));
    }
  }
};

namespace {
size_t job_bytes_accounted(const tt_job& j, size_t ws) {
  int64_t caps[TT_MAX_D], ss = 0, sc = 0;
  size_t b = ws;
  if (tt_core_caps(j.d, j.n, j.r_max, caps, &ss, &sc) == TT_OK)
    for (int i = 0; i < j.d; ++i) b += (size_t)caps[i] * 8;
  double entries = 1;
  for (int i = 0; i < j.d; ++i) entries *= (double)j.n[i];
  b += (size_t)(entries * (j.dtype == TT_F32 ? 4 : 8));
  return b;
}
}  // namespace

extern "C" {

tt_status tt_serve_create(size_t hbm_budget_bytes, const tt_serve_opts* opts, tt_server** out) {
  if (!out || hbm_budget_bytes == 0) return TT_EINVAL;
  *out = nullptr;
  const int slots = opts && opts->max_inflight > 0 ? opts->max_inflight : 8;
  if (slots > 256) return TT_EINVAL;
  tt_server* s = new tt_server;
  s->budget = hbm_budget_bytes;
  s->arena_bytes = opts && opts->arena_bytes ? opts->arena_bytes : hbm_budget_bytes / 4;
  s->arena_bytes = (s->arena_bytes + 255) & ~(size_t)255;
  s->timeout_s = opts && opts->timeout_s > 0 ? opts->timeout_s : 60.0;
  if (opts && opts->policy != TT_SERVE_FIFO && opts->policy != TT_SERVE_SHORTEST) {
    delete s;
    return TT_EINVAL;
  }
  s->policy = opts ? opts->policy : TT_SERVE_FIFO;
  s->max_wait_s = opts && opts->max_wait_s > 0 ? opts->max_wait_s : 1.0;
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaMalloc(&s->arena, s->arena_bytes) != cudaSuccess) {
    delete s;
    return TT_ENOMEM;
  }
  s->free_list.push_back({0, s->arena_bytes});
  s->slot_stream.resize(slots);
  s->slot_event.resize(slots);
  s->slot_ticket.assign(slots, 0);
  for (int k = 0; k < slots; ++k) {
    if (cudaStreamCreateWithFlags(&s->slot_stream[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->slot_event[k], cudaEventDisableTiming) != cudaSuccess) {
      cudaFree(s->arena);
      delete s;
      return TT_ECUDA;
    }
  }
  s->worker = std::thread([s] { s->loop(); });
  *out = s;
  return TT_OK;
}

tt_status tt_serve_submit(tt_server* s, const tt_job* job, void* ready_stream, uint64_t* ticket) {
  if (!s || !job || !ticket) return TT_EINVAL;
  size_t ws = 0;
  tt_status st = job_work_bytes(*job, &ws);
  if (st != TT_OK) return st;
  const size_t acct = job_bytes_accounted(*job, ws);
  if (acct > s->budget || ((ws + 255) & ~(size_t)255) > s->arena_bytes) return TT_ENOMEM;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return TT_ECANCELLED;
  // mark the point of the submitter's stream after which the inputs and outputs are ready
  cudaEvent_t ready = nullptr;
  if (!s->spare_events.empty()) {
    ready = s->spare_events.back();
    s->spare_events.pop_back();
  } else if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess) {
    set_last_error_text("tt_serve_submit: cudaEventCreateWithFlags failed");
    return TT_ECUDA;
  }
  if (cudaEventRecord(ready, (cudaStream_t)ready_stream) != cudaSuccess) {
    s->spare_events.push_back(ready);
    set_last_error_text("tt_serve_submit: cudaEventRecord on the ready stream failed");
    return TT_ECUDA;
  }
  tt_server::Req r;
  r.ready = ready;
  r.ticket = s->next_ticket++;
  r.job = *job;
  r.ws = ws;
  r.acct = acct;
  r.res.status = TT_OK;
  r.res.t_submit = now_s();
  r.cost = job_cost_estimate(job->d, job->n, job->r_max, job->tol, (int)job->dtype);
  s->reqs[r.ticket] = r;
  s->queue.push_back(r.ticket);
  *ticket = r.ticket;
  s->cv.notify_all();
  return TT_OK;
}

tt_status tt_serve_poll(tt_server* s, uint64_t ticket, int wait, tt_job_result* out) {
  if (!s || !out) return TT_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return TT_EINVAL;
  if (!it->second.done) {
    if (!wait) return TT_EAGAIN;
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::duration<double>(s->timeout_s);
    while (!it->second.done) {
      if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout && !it->second.done)
        return TT_ETIMEOUT;
      it = s->reqs.find(ticket);
      if (it == s->reqs.end()) return TT_EINVAL;
    }
  }
  *out = it->second.res;
  return TT_OK;
}

tt_status tt_serve_release(tt_server* s, uint64_t ticket) {
  if (!s) return TT_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return TT_EINVAL;
  if (!it->second.done) return TT_EAGAIN;
  s->reqs.erase(it);
  return TT_OK;
}

tt_status tt_serve_destroy(tt_server* s) {
  if (!s) return TT_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (uint64_t t : s->queue) {
      tt_server::Req& r = s->reqs[t];
      r.res.status = TT_ECANCELLED;
      r.res.t_done = now_s();
      r.done = true;
      if (r.ready) { s->spare_events.push_back(r.ready); r.ready = nullptr; }
    }
    s->queue.clear();
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  tt_status result = TT_OK;
  // running requests: bounded wait for their streams, then release everything
  for (size_t k = 0; k < s->slot_stream.size(); ++k) {
    if (s->slot_ticket[k]) {
      const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(s->timeout_s);
      while (cudaEventQuery(s->slot_event[k]) == cudaErrorNotReady) {
        if (std::chrono::steady_clock::now() > deadline) { result = TT_ETIMEOUT; break; }
        std::this_thread::sleep_for(std::chrono::microseconds(100));
      }
    }
  }
  if (result == TT_OK) {
    for (size_t k = 0; k < s->slot_stream.size(); ++k) {
      cudaStreamDestroy(s->slot_stream[k]);
      cudaEventDestroy(s->slot_event[k]);
    }
    for (cudaEvent_t e : s->spare_events) cudaEventDestroy(e);
    for (auto& kv : s->reqs)
      if (kv.second.ready) cudaEventDestroy(kv.second.ready);
    cudaFree(s->arena);
    delete s;
  }
  return result;
}

}  // extern "C"
