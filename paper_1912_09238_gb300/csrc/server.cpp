// server.cpp -- continuous-batching request server (ipm_server_*, declared in include/ipm.h).
//
// Two host threads per server drive the device:
//   admission thread: waiting requests, in arrival order, are taken while a slot is free and the sum
//      of the admitted requests' ipm_footprint stays within the memory cap (the oldest request is never
//      passed over, so admission is FIFO); each gets its context (ipm_init: stream-ordered allocations
//      from the library's memory pool, initial data, dual solve, graph capture) and its own stream, and
//      is handed to the worker. Set-up thus runs beside the worker's launches instead of between them.
//   worker thread, each loop iteration:
//   1. it takes the contexts the admission thread has readied;
//   2. launch: every active request without work in flight gets its next batch of time steps
//      (ipm_step graph launches on the request's own stream) and an event after the batch;
//   3. completion: requests whose event has fired are checked (t >= t_end, max_steps, or a per-cell
//      failure); finished requests copy their moments to the host, free their context (stream-ordered
//      frees, no device-wide synchronisation) and slot, and wake the admission thread and ipm_poll /
//      ipm_server_drain callers.
// Batches are sized from the last time step so that a request stops within a few steps of t_end.
// The kernels of all active requests overlap on the GPU through their separate streams; no request
// reads another's memory, and every kernel's result is independent of the order in which CTAs run,
// so a request's moments are the same alone and in any mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ipm.h"

namespace {

constexpr int64_t kFirstBatch = 4;     // steps launched before the first dt is known
constexpr int64_t kMaxBatch = 64;      // steps per batch at most (bounds the overshoot past t_end)

struct Job {
  uint64_t ticket = 0;
  ipm_request req{};
  size_t footprint = 0;
  double t_submit = 0, t_start = 0, t_finish = 0;
  ipm_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  int64_t launched = 0;
  bool in_flight = false;
  bool done = false;
  int32_t status = IPM_OK;
  ipm_stats stats{};
  ipm_dims dims{};
  std::vector<double> moments;
  std::string error;
};

}  // namespace

struct ipm_server {
  size_t mem_cap = 0;
  int max_active = 1;
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work;   // worker waits for submissions
  std::condition_variable cv_done;   // drain waits for completions
  std::condition_variable cv_admit; // admission thread waits for submissions and freed capacity
  std::deque<std::shared_ptr<Job>> waiting;
  std::deque<std::shared_ptr<Job>> ready;   // contexts set up by the admission thread, not yet active
  std::map<uint64_t, std::shared_ptr<Job>> jobs;
  uint64_t next_ticket = 1;
  size_t outstanding = 0;            // submitted and not yet done
  int admitted = 0;                  // requests holding a slot (being set up, ready or active)
  size_t in_use = 0;                 // their footprints
  bool admitting = false;            // the admission thread is setting up a request
  bool stop = false;
  std::thread worker, admitter;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  void run();
  void admit();
};

static void finish(ipm_server* s, const std::shared_ptr<Job>& j, int32_t status, const std::string& why = "") {
  j->status = status;
  if (status != IPM_OK && j->error.empty()) j->error = why;
  if (j->ctx) {
    ipm_get_dims(j->ctx, &j->dims);
    ipm_sync_stats(j->ctx, &j->stats);
    if (status == IPM_OK) {
      j->moments.resize((size_t)j->dims.n_cells * j->dims.N * j->dims.m);
      const ipm_status st = ipm_get_moments(j->ctx, j->moments.data(), j->moments.size());
      if (st != IPM_OK) {
        j->status = st;
        j->error = std::string("ipm_get_moments: ") + ipm_last_error(j->ctx);
      }
    }
    ipm_destroy(j->ctx);
    j->ctx = nullptr;
  }
  if (j->ev) cudaEventDestroy(j->ev);
  if (j->stream) cudaStreamDestroy(j->stream);
  j->ev = nullptr;
  j->stream = nullptr;
  j->t_finish = s->now();
  std::lock_guard<std::mutex> lk(s->mu);
  j->done = true;
  --s->outstanding;
  --s->admitted;
  s->in_use -= j->footprint;
  s->cv_done.notify_all();
  s->cv_admit.notify_all();
}

// Admission thread: FIFO by slots and memory; sets up each admitted request's context.
void ipm_server::admit() {
  cudaSetDevice(device);
  for (;;) {
    std::shared_ptr<Job> j;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_admit.wait(lk, [&] {
        return stop || (!waiting.empty() && admitted < max_active && in_use + waiting.front()->footprint <= mem_cap);
      });
      if (stop) {
        // drop the waiting requests; the running ones finish
        for (auto& w : waiting) {
          w->status = IPM_EAGAIN;
          w->done = true;
          --outstanding;
        }
        waiting.clear();
        cv_done.notify_all();
        return;
      }
      j = waiting.front();
      waiting.pop_front();
      ++admitted;
      in_use += j->footprint;
      admitting = true;
    }
    j->t_start = now();
    std::string why;
    ipm_status st = ipm_init(&j->req.problem, &j->req.basis, &j->req.quad, &j->req.entropy, &j->req.options, &j->ctx);
    if (st != IPM_OK) why = std::string("ipm_init: ") + ipm_last_error(nullptr);
    cudaError_t ce = cudaSuccess;
    if (st == IPM_OK && (ce = cudaStreamCreateWithFlags(&j->stream, cudaStreamNonBlocking)) != cudaSuccess) {
      st = IPM_ECUDA;
      why = std::string("cudaStreamCreate: ") + cudaGetErrorString(ce);
    }
    if (st == IPM_OK && (ce = cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming)) != cudaSuccess) {
      st = IPM_ECUDA;
      why = std::string("cudaEventCreate: ") + cudaGetErrorString(ce);
    }
    if (st == IPM_OK && (st = ipm_set_stream(j->ctx, j->stream)) != IPM_OK)
      why = std::string("ipm_set_stream: ") + ipm_last_error(j->ctx);
    if (st != IPM_OK) {
      finish(this, j, st, why);
      std::lock_guard<std::mutex> lk(mu);
      admitting = false;
      continue;
    }
    std::lock_guard<std::mutex> lk(mu);
    ready.push_back(j);
    admitting = false;
    cv_work.notify_one();
  }
}

void ipm_server::run() {
  cudaSetDevice(device);
  std::vector<std::shared_ptr<Job>> active;
  for (;;) {
    // 1. contexts the admission thread has set up
    {
      std::unique_lock<std::mutex> lk(mu);
      if (active.empty() && ready.empty()) {
        // idle: wait for a readied request, or for the end (nothing waiting, admitted or being set up)
        cv_work.wait(lk, [&] { return !ready.empty() || (stop && admitted == 0 && !admitting); });
        if (ready.empty()) break;
      }
      while (!ready.empty()) {
        active.push_back(ready.front());
        ready.pop_front();
      }
    }
    // 2. launch the next batch of every idle active request
    for (auto& j : active) {
      if (j->in_flight) continue;
      int64_t batch = kFirstBatch;
      const double t_end = j->req.problem.t_end;
      if (j->launched > 0 && t_end > 0.0 && j->stats.dt > 0.0)
        batch = (int64_t)std::ceil((t_end - j->stats.t) / j->stats.dt);
      batch = std::max<int64_t>(1, std::min<int64_t>({batch, kMaxBatch, j->req.max_steps - j->launched}));
      ipm_status st = IPM_OK;
      for (int64_t k = 0; k < batch && st == IPM_OK; ++k) st = ipm_step(j->ctx, nullptr);
      if (st != IPM_OK) j->error = std::string("ipm_step: ") + ipm_last_error(j->ctx);
      cudaError_t ce = cudaSuccess;
      if (st == IPM_OK && (ce = cudaEventRecord(j->ev, j->stream)) != cudaSuccess) {
        st = IPM_ECUDA;
        j->error = std::string("cudaEventRecord: ") + cudaGetErrorString(ce);
      }
      if (st != IPM_OK) {
        j->status = st;
        continue;
      }
      j->launched += batch;
      j->in_flight = true;
    }
    // 3. completions
    bool progressed = false;
    for (size_t k = 0; k < active.size();) {
      auto j = active[k];
      bool done = false;
      int32_t status = j->status;
      if (status != IPM_OK) {
        done = true;
      } else if (j->in_flight) {
        const cudaError_t q = cudaEventQuery(j->ev);
        if (q == cudaErrorNotReady) {
          ++k;
          continue;
        }
        j->in_flight = false;
        progressed = true;
        if (q != cudaSuccess) {
          status = IPM_ECUDA;
          j->error = std::string("cudaEventQuery: ") + cudaGetErrorString(q);
          done = true;
        } else if (ipm_sync_stats(j->ctx, &j->stats) != IPM_OK) {
          status = IPM_ECUDA;
          j->error = std::string("ipm_sync_stats: ") + ipm_last_error(j->ctx);
          done = true;
        } else if (j->stats.failed_cells > 0) {
          status = j->stats.first_status;
          done = true;
        } else {
          const double t_end = j->req.problem.t_end;
          const bool at_end = t_end > 0.0 && (j->stats.t >= t_end || j->stats.dt <= 0.0);
          done = at_end || j->launched >= j->req.max_steps;
        }
      }
      if (done) {
        finish(this, j, status);
        active.erase(active.begin() + k);
        progressed = true;
      } else {
        ++k;
      }
    }
    if (!progressed && !active.empty()) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

extern "C" {

ipm_status ipm_server_create(size_t mem_cap_bytes, int max_active, ipm_server** out) {
  if (!out || max_active < 1) return IPM_EINVAL;
  *out = nullptr;
  ipm_server* s = new ipm_server();
  s->t0 = std::chrono::steady_clock::now();
  s->max_active = max_active;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return IPM_ECUDA;
  }
  if (mem_cap_bytes == 0) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      delete s;
      return IPM_ECUDA;
    }
    mem_cap_bytes = free_b / 10 * 9;
  }
  s->mem_cap = mem_cap_bytes;
  s->worker = std::thread([s] { s->run(); });
  s->admitter = std::thread([s] { s->admit(); });
  *out = s;
  return IPM_OK;
}

ipm_status ipm_submit(ipm_server* s, const ipm_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return IPM_EINVAL;
  if (req->max_steps < 1) return IPM_EINVAL;
  auto j = std::make_shared<Job>();
  j->req = *req;
  const ipm_status st = ipm_footprint(&req->problem, &req->basis, &req->quad, &req->entropy, &req->options, &j->footprint);
  if (st != IPM_OK) return st;
  if (j->footprint > s->mem_cap) return IPM_ENOMEM;
  j->t_submit = s->now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return IPM_EINVAL;
  j->ticket = s->next_ticket++;
  s->jobs[j->ticket] = j;
  s->waiting.push_back(j);
  ++s->outstanding;
  *ticket = j->ticket;
  s->cv_admit.notify_one();
  return IPM_OK;
}

ipm_status ipm_poll(ipm_server* s, uint64_t ticket, ipm_result* out, double* moments, size_t count) {
  if (!s) return IPM_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return IPM_EINVAL;
  const auto& j = it->second;
  if (!j->done) return IPM_EAGAIN;
  if (out) {
    std::memset(out, 0, sizeof(*out));
    out->status = j->status;
    out->dims = j->dims;
    out->stats = j->stats;
    out->submit_s = j->t_submit;
    out->start_s = j->t_start;
    out->finish_s = j->t_finish;
    out->footprint_bytes = j->footprint;
    std::strncpy(out->error, j->error.c_str(), sizeof(out->error) - 1);
  }
  if (moments) {
    if (count != j->moments.size()) return IPM_EINVAL;
    std::memcpy(moments, j->moments.data(), count * sizeof(double));
    s->jobs.erase(it);
  }
  return IPM_OK;
}

ipm_status ipm_server_drain(ipm_server* s, double timeout_s) {
  if (!s) return IPM_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return s->outstanding == 0; });
  return ok ? IPM_OK : IPM_ETIMEOUT;
}

void ipm_server_destroy(ipm_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
    s->cv_admit.notify_all();
  }
  if (s->admitter.joinable()) s->admitter.join();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  delete s;
}

}  // extern "C"
