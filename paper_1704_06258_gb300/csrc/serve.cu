// Continuous-batching serving loop for GA solve requests of differing n and p.
//
// Requests wait in a FIFO until they fit: at most `max_active` are admitted
// or running at once and the device bytes of those stay within the HBM
// budget.  An admitted request gets its own instance handle (W, C and the GA
// state stay on the device until it finishes).  Every tick runs up to 8
// generations of every running request with one launch per kernel and
// generation over all of them (offspring, allocation + access terms,
// transfer term, reduction + selection), so the work of requests that
// arrived at different times overlaps on the device.  Each request's
// arithmetic depends only on its own data, so its result is the same alone
// and in any mix.
//
// The tick itself does no device-memory management and waits for no request:
// a worker thread makes each admitted request's handle (stream-ordered
// allocations from the server's memory pool, set-up kernels and the initial
// solution on the handle's own stream; the tick's stream waits on an event
// before the request's first generation) and finishes each request whose
// last generation has been enqueued (its stream waits on an event of the
// tick's stream, then the fp64 rescoring, the copy-out and the stream-ordered
// frees of the handle).  The host runs at most two ticks ahead of the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "usaphmp.h"
#include "common.cuh"
#include "kernels.cuh"

using namespace usaphmp;

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
  int64_t ticket = 0;
  int n = 0, p = 0, R = 0, P = 0, G = 0;
  double chi = 0, alpha = 0, delta = 0;
  uint64_t seed = 0;
  std::vector<float> W, C;
  Clock::time_point t_submit;
  usaphmp_t h = nullptr;
  int gens = 0;
  size_t bytes = 0;
  cudaEvent_t ready = nullptr;   // the handle's stream, after the initial solution
  cudaEvent_t last = nullptr;    // the server's stream, after the request's last generation
  int status = USAPHMP_OK;       // of the admission (worker)
  std::string error;
  bool cancelled = false;
};

struct Finished {
  int status = USAPHMP_OK;
  std::string error;
  std::vector<int32_t> hubs, S;
  double cost_fp64 = 0;
  float cost_fp32 = 0;
  int64_t evals = 0;
  double ms = 0;
};

enum JobKind { kAdmit, kFinish };
struct Job {
  JobKind kind;
  Request* r;
  int status;  // kFinish: USAPHMP_OK (result wanted) or the status to report
  std::string error;
};

}  // namespace

// Generations a step runs for the running requests at most: fewer host round
// trips per generation at the cost of admitting new requests only between
// steps.  A step's generations are replayed from a CUDA graph of the running
// set (captured again only when the set changes).
constexpr int kGensPerTick = 8;

struct usaphmp_server_s {
  size_t budget = 0;
  int max_active = 0, path = 0, num_sms = 0, device = 0;
  cudaStream_t stream = nullptr;
  cudaMemPool_t pool = nullptr;
  uint32_t* d_status = nullptr;
  Task* d_tasks = nullptr;
  std::vector<Task> h_tasks;
  bool tasks_dirty = true;                 // the device task table no longer matches `active`
  cudaGraphExec_t gexec = nullptr;         // the tick's generations for the current running set
  bool graph_valid = false;
  int graph_k = 0;
  cudaEvent_t tick_ev[2] = {nullptr, nullptr};
  int64_t ticks = 0;
  std::deque<Request*> pending;            // tick thread only
  std::vector<Request*> active;            // tick thread only
  int64_t next_ticket = 1;
  // shared with the worker thread (under mu)
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Job> jobs;
  bool stop = false;
  std::vector<Request*> admitting;         // handed to the worker, not yet picked up
  std::vector<Request*> admitted;          // made by the worker, waiting for the tick
  std::map<int64_t, Finished> done;
  size_t used = 0;                         // device bytes of admitted and running requests
  int finishing = 0;                       // requests handed to the worker to finish
  int64_t jobs_done = 0;                   // jobs the worker has completed
  usaphmp_server_counters stats{};
  std::thread worker;
};

namespace {

void release_request(usaphmp_server_s* s, Request* r) {
  if (r->ready) cudaEventDestroy(r->ready);
  if (r->last) cudaEventDestroy(r->last);
  delete r;
  (void)s;
}

// Worker: make the handle of an admitted request (its stream only).
void do_admit(usaphmp_server_s* s, Request* r) {
  int rc = create_pooled(r->n, r->p, r->W.data(), r->C.data(), r->chi, r->alpha, r->delta, s->pool, &r->h);
  cudaStream_t hs = r->h ? handle_stream(r->h) : nullptr;
  if (rc == USAPHMP_OK) {
    usaphmp_params prm;
    usaphmp_get_params(r->h, &prm);
    prm.islands = r->R;
    prm.island_size = r->P;
    prm.path = s->path;
    prm.use_graph = 0;
    rc = usaphmp_set_params(r->h, &prm);
  }
  if (rc == USAPHMP_OK) rc = usaphmp_ga_begin(r->h, r->seed, hs);
  cudaError_t e = cudaSuccess;
  if (rc == USAPHMP_OK) e = cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming);
  if (rc == USAPHMP_OK && e == cudaSuccess) e = cudaEventCreateWithFlags(&r->last, cudaEventDisableTiming);
  if (rc == USAPHMP_OK && e == cudaSuccess) e = cudaEventRecord(r->ready, hs);
  if (rc == USAPHMP_OK && e != cudaSuccess) {
    rc = e == cudaErrorMemoryAllocation ? USAPHMP_ENOMEM : USAPHMP_ECUDA;
    report_error(rc, std::string("admission: ") + cudaGetErrorString(e));
  }
  std::vector<float>().swap(r->W);
  std::vector<float>().swap(r->C);
  if (rc != USAPHMP_OK) {
    r->status = rc;
    r->error = usaphmp_last_error();
    if (r->h) {
      usaphmp_destroy(r->h);
      r->h = nullptr;
    }
  }
}

// Worker: result and release of a request whose last generation (or
// cancellation point) is r->last on the server's stream.
void do_finish(usaphmp_server_s* s, Request* r, int status, const std::string& err) {
  Finished f;
  f.status = status;
  f.error = err;
  if (r->h) {
    cudaStream_t hs = handle_stream(r->h);
    if (r->last) cudaStreamWaitEvent(hs, r->last, 0);
    if (status == USAPHMP_OK) {
      f.hubs.resize(r->p);
      f.S.resize(r->n);
      usaphmp_result res{};
      res.hubs = f.hubs.data();
      res.S = f.S.data();
      const int rc = usaphmp_ga_result(r->h, &res, hs);
      if (rc != USAPHMP_OK) {
        f.status = rc;
        f.error = usaphmp_last_error();
      } else {
        f.cost_fp64 = res.cost_fp64;
        f.cost_fp32 = res.cost_fp32;
        f.evals = res.evals;
      }
    }
    usaphmp_destroy(r->h);   // synchronises the handle's stream; frees are stream-ordered
    r->h = nullptr;
  }
  f.ms = ms_between(r->t_submit, Clock::now());
  std::lock_guard<std::mutex> lock(s->mu);
  s->used -= r->bytes;
  s->finishing -= 1;
  s->done[r->ticket] = std::move(f);
  release_request(s, r);
}

void worker_loop(usaphmp_server_s* s) {
  cudaSetDevice(s->device);   // the server's device, current for this thread too
  for (;;) {
    Job job;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv.wait(lock, [&] { return s->stop || !s->jobs.empty(); });
      if (s->jobs.empty()) return;   // stop requested and nothing left
      job = std::move(s->jobs.front());
      s->jobs.pop_front();
    }
    if (job.kind == kAdmit) {
      const auto t0 = Clock::now();
      do_admit(s, job.r);
      std::lock_guard<std::mutex> lock(s->mu);
      s->stats.admit_ms_total += ms_between(t0, Clock::now());
      s->admitting.erase(std::find(s->admitting.begin(), s->admitting.end(), job.r));
      s->admitted.push_back(job.r);
    } else {
      do_finish(s, job.r, job.status, job.error);
    }
    {
      std::lock_guard<std::mutex> lock(s->mu);
      s->jobs_done += 1;
    }
    s->cv.notify_all();
  }
}

// Tick thread: hand a request that leaves the running set to the worker.
int enqueue_finish(usaphmp_server_s* s, Request* r, int status, const std::string& err) {
  if (r->last) {
    const cudaError_t e = cudaEventRecord(r->last, s->stream);
    if (e != cudaSuccess) return report_error(USAPHMP_ECUDA, std::string("finish event: ") + cudaGetErrorString(e));
  }
  std::lock_guard<std::mutex> lock(s->mu);
  s->finishing += 1;
  s->jobs.push_back(Job{kFinish, r, status, err});
  s->cv.notify_all();
  return USAPHMP_OK;
}

}  // namespace

extern "C" {

int usaphmp_server_footprint(int32_t n, int32_t p, int32_t islands, int32_t island_size, int64_t* bytes) {
  if (!bytes || n < 2 || p < 1 || islands < 1 || island_size < 2) return report_error(USAPHMP_EINVAL, "bad argument");
  *bytes = (int64_t)handle_device_bytes(n, p, islands, island_size);
  return USAPHMP_OK;
}

int usaphmp_server_create(int64_t hbm_budget_bytes, int32_t max_active, int32_t path, usaphmp_server_t* out) {
  if (!out) return report_error(USAPHMP_EINVAL, "out is NULL");
  *out = nullptr;
  if (hbm_budget_bytes <= 0 || max_active < 1 || max_active > kMaxTasks)
    return report_error(USAPHMP_EINVAL, "budget must be > 0 and max_active in [1, 64]");
  if (path != USAPHMP_PATH_PLAIN_FP32 && path != USAPHMP_PATH_SPLIT_BF16)
    return report_error(USAPHMP_EINVAL, "unknown path");
  usaphmp_server_s* s = new usaphmp_server_s();
  s->budget = (size_t)hbm_budget_bytes;
  s->max_active = max_active;
  s->path = path;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  s->device = dev;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_status, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(s->d_status, 0, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_tasks, sizeof(Task) * kMaxTasks);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&s->tick_ev[k], cudaEventDisableTiming);
  if (e == cudaSuccess) {
    // the requests' device memory: a pool of this device that keeps up to the
    // budget once allocated, so requests coming and going reuse it
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    e = cudaMemPoolCreate(&s->pool, &props);
    if (e == cudaSuccess) {
      uint64_t keep = (uint64_t)hbm_budget_bytes;
      e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
  }
  if (e != cudaSuccess) {
    usaphmp_server_destroy(s);
    return report_error(e == cudaErrorMemoryAllocation ? USAPHMP_ENOMEM : USAPHMP_ECUDA,
                        std::string("server set-up: ") + cudaGetErrorString(e));
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return USAPHMP_OK;
}

int usaphmp_server_submit(usaphmp_server_t s, int32_t n, int32_t p, const float* W, const float* C, double chi,
                          double alpha, double delta, int32_t islands, int32_t island_size, int32_t generations,
                          uint64_t seed, int64_t* ticket) {
  if (!s || !W || !C || !ticket) return report_error(USAPHMP_EINVAL, "NULL argument");
  if (n < 2 || n > kMaxN || p < 1 || p > n || p > kMaxP) return report_error(USAPHMP_EINVAL, "bad n or p");
  if (islands < 1 || island_size < 2 || (island_size & 1) || generations < 0)
    return report_error(USAPHMP_EINVAL, "bad islands, island_size or generations");
  Request* r = new Request();
  r->ticket = s->next_ticket++;
  r->n = n; r->p = p; r->R = islands; r->P = island_size; r->G = generations;
  r->chi = chi; r->alpha = alpha; r->delta = delta; r->seed = seed;
  r->W.assign(W, W + (size_t)n * n);
  r->C.assign(C, C + (size_t)n * n);
  r->bytes = handle_device_bytes(n, p, islands, island_size);
  r->t_submit = Clock::now();
  *ticket = r->ticket;
  if (r->bytes > s->budget) {
    Finished f;
    f.status = USAPHMP_EBUSY;
    f.error = "request needs more device memory than the server budget";
    std::lock_guard<std::mutex> lock(s->mu);
    s->done[r->ticket] = std::move(f);
    delete r;
    return USAPHMP_OK;
  }
  s->pending.push_back(r);
  return USAPHMP_OK;
}

int usaphmp_server_step(usaphmp_server_t s, int32_t* n_active, int32_t* n_pending) {
  const NvtxRange nvtx_range("usaphmp_server_step");
  if (!s) return report_error(USAPHMP_EINVAL, "NULL server");
  const auto t_tick = Clock::now();
  std::vector<Request*> fresh;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    // admission, FIFO, by slots (admitting and running) and by device bytes
    while (!s->pending.empty() && (int)(s->active.size() + s->admitting.size() + s->admitted.size()) < s->max_active &&
           s->used + s->pending.front()->bytes <= s->budget) {
      Request* r = s->pending.front();
      s->pending.pop_front();
      s->used += r->bytes;
      s->admitting.push_back(r);
      s->jobs.push_back(Job{kAdmit, r, USAPHMP_OK, ""});
      s->cv.notify_all();
    }
    fresh.swap(s->admitted);
  }
  // requests the worker has made join the running set
  for (Request* r : fresh) {
    const auto now = Clock::now();
    if (r->status != USAPHMP_OK || r->cancelled) {
      const int st = r->status != USAPHMP_OK ? r->status : USAPHMP_ECANCELED;
      const int rc = enqueue_finish(s, r, st, r->status != USAPHMP_OK ? r->error : "cancelled");
      if (rc != USAPHMP_OK) return rc;
      continue;
    }
    const cudaError_t e = cudaStreamWaitEvent(s->stream, r->ready, 0);
    if (e != cudaSuccess) return report_error(USAPHMP_ECUDA, std::string("admission event: ") + cudaGetErrorString(e));
    const double wait = ms_between(r->t_submit, now);
    s->stats.admitted += 1;
    s->stats.admit_wait_ms_total += wait;
    s->stats.admit_wait_ms_max = std::max(s->stats.admit_wait_ms_max, wait);
    s->active.push_back(r);
    s->tasks_dirty = true;
  }
  // requests asking for no generation finish at once
  for (size_t i = 0; i < s->active.size();) {
    if (s->active[i]->gens >= s->active[i]->G) {
      const int rc = enqueue_finish(s, s->active[i], USAPHMP_OK, "");
      if (rc != USAPHMP_OK) return rc;
      s->active.erase(s->active.begin() + i);
      s->tasks_dirty = true;
    } else {
      ++i;
    }
  }
  if (!s->active.empty()) {
    // at most two ticks in flight: wait for the one two ticks back
    cudaEvent_t slot_ev = s->tick_ev[s->ticks & 1];
    if (s->ticks >= 2) {
      const cudaError_t e = cudaEventSynchronize(slot_ev);
      if (e != cudaSuccess) return report_error(USAPHMP_ECUDA, std::string("tick wait: ") + cudaGetErrorString(e));
    }
    // up to kGensPerTick generations of every running request (no more than
    // any of them still needs), one launch per kernel over all of them; the
    // task table goes to the device only when the running set has changed
    // (from pageable memory: staged before the call returns, and ordered on
    // the stream after the previous tick's kernels)
    bool tc = false;
    if (s->tasks_dirty) {
      s->h_tasks.clear();
      for (Request* r : s->active) s->h_tasks.push_back(handle_ga_task(r->h));
      const cudaError_t e = cudaMemcpyAsync(s->d_tasks, s->h_tasks.data(), sizeof(Task) * s->h_tasks.size(),
                                            cudaMemcpyHostToDevice, s->stream);
      if (e != cudaSuccess) return report_error(USAPHMP_ECUDA, std::string("task upload: ") + cudaGetErrorString(e));
      s->tasks_dirty = false;
      s->graph_valid = false;
    }
    int k = kGensPerTick;
    for (Request* r : s->active) {
      tc = handle_uses_tc(r->h);
      k = std::min(k, r->G - r->gens);
    }
    // The tick's generations (k x 4 launches over the running set, with
    // programmatic edges) are captured into a CUDA graph when the running
    // set or k changes -- the executable graph is updated in place when only
    // its launch parameters differ -- and replayed otherwise.
    cudaError_t e = cudaSuccess;
    if (!s->graph_valid || s->graph_k != k) {
      const TaskSet ts{s->d_tasks, s->h_tasks.data(), (int)s->h_tasks.size()};
      e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        for (int g = 0; g < k; ++g) {
          launch_children(ts, s->stream);
          launch_alloc(ts, true, tc, s->stream);
          if (tc)
            launch_eval_tc(ts, s->num_sms, s->d_status, s->stream);
          else
            launch_eval_plain(ts, s->stream);
          launch_reduce_select(ts, s->stream);
        }
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(s->stream, &g);
        if (e == cudaSuccess) {
          cudaGraphExecUpdateResultInfo info;
          if (!s->gexec || cudaGraphExecUpdate(s->gexec, g, &info) != cudaSuccess) {
            cudaGetLastError();   // an update that does not apply is not an error
            if (s->gexec) cudaGraphExecDestroy(s->gexec);
            s->gexec = nullptr;
            e = cudaGraphInstantiate(&s->gexec, g, 0);
          }
          cudaGraphDestroy(g);
        }
      }
      if (e != cudaSuccess)
        return report_error(USAPHMP_ECUDA, std::string("tick graph: ") + cudaGetErrorString(e));
      s->graph_valid = true;
      s->graph_k = k;
      s->stats.graph_builds += 1;
    }
    e = cudaGraphLaunch(s->gexec, s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(slot_ev, s->stream);
    if (e != cudaSuccess) return report_error(USAPHMP_ECUDA, std::string("generation launch: ") + cudaGetErrorString(e));
    ++s->ticks;
    for (Request* r : s->active) {
      r->gens += k;
      handle_note_generations(r->h, k);
    }
    for (size_t i = 0; i < s->active.size();) {
      if (s->active[i]->gens >= s->active[i]->G) {
        const int rc = enqueue_finish(s, s->active[i], USAPHMP_OK, "");
        if (rc != USAPHMP_OK) return rc;
        s->active.erase(s->active.begin() + i);
        s->tasks_dirty = true;
      } else {
        ++i;
      }
    }
  }
  const double tick_ms = ms_between(t_tick, Clock::now());
  std::unique_lock<std::mutex> lock(s->mu);
  if (s->active.empty() && s->admitted.empty() && (!s->admitting.empty() || s->finishing > 0)) {
    // nothing to run until the worker has made or finished a request: wait
    // for its next completed job (at most 10 ms) instead of returning at once
    const int64_t seen = s->jobs_done;
    s->cv.wait_for(lock, std::chrono::milliseconds(10), [&] { return s->jobs_done != seen; });
  }
  s->stats.ticks += 1;
  s->stats.tick_ms_total += tick_ms;
  s->stats.tick_ms_max = std::max(s->stats.tick_ms_max, tick_ms);
  if (n_active) *n_active = (int32_t)(s->active.size() + s->admitting.size() + s->admitted.size());
  if (n_pending) *n_pending = (int32_t)s->pending.size() + s->finishing;
  return USAPHMP_OK;
}

int usaphmp_server_cancel(usaphmp_server_t s, int64_t ticket) {
  if (!s) return report_error(USAPHMP_EINVAL, "NULL server");
  for (auto it = s->pending.begin(); it != s->pending.end(); ++it)
    if ((*it)->ticket == ticket) {
      Request* r = *it;
      s->pending.erase(it);
      Finished f;
      f.status = USAPHMP_ECANCELED;
      f.error = "cancelled";
      f.ms = ms_between(r->t_submit, Clock::now());
      std::lock_guard<std::mutex> lock(s->mu);
      s->done[ticket] = std::move(f);
      delete r;
      return USAPHMP_OK;
    }
  for (size_t i = 0; i < s->active.size(); ++i)
    if (s->active[i]->ticket == ticket) {
      // its generations already enqueued finish first (the worker waits for
      // the event recorded here before it frees the request's memory)
      Request* r = s->active[i];
      s->active.erase(s->active.begin() + i);
      s->tasks_dirty = true;
      return enqueue_finish(s, r, USAPHMP_ECANCELED, "cancelled");
    }
  {
    std::lock_guard<std::mutex> lock(s->mu);
    for (Request* r : s->admitting)
      if (r->ticket == ticket && !r->cancelled) {
        r->cancelled = true;   // released when the worker has made it
        return USAPHMP_OK;
      }
    for (Request* r : s->admitted)
      if (r->ticket == ticket && !r->cancelled) {
        r->cancelled = true;
        return USAPHMP_OK;
      }
  }
  return report_error(USAPHMP_EINVAL, "cancel: ticket " + std::to_string(ticket) + " is not queued or running");
}

int usaphmp_server_poll(usaphmp_server_t s, int64_t ticket, usaphmp_result* out) {
  if (!s || !out) return report_error(USAPHMP_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->done.find(ticket);
  if (it == s->done.end()) return 0;
  Finished& f = it->second;
  const int status = f.status;
  if (status != USAPHMP_OK) {
    report_error(status, "request " + std::to_string(ticket) + ": " + f.error);
    s->done.erase(it);
    return status;
  }
  if (out->hubs) std::copy(f.hubs.begin(), f.hubs.end(), out->hubs);
  if (out->S) std::copy(f.S.begin(), f.S.end(), out->S);
  out->cost_fp64 = f.cost_fp64;
  out->cost_fp32 = f.cost_fp32;
  out->evals = f.evals;
  out->ms = f.ms;
  s->done.erase(it);
  return 1;
}

int usaphmp_server_stats(usaphmp_server_t s, usaphmp_server_counters* out) {
  if (!s || !out) return report_error(USAPHMP_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  *out = s->stats;
  return USAPHMP_OK;
}

void usaphmp_server_destroy(usaphmp_server_t s) {
  if (!s) return;
  if (s->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lock(s->mu);
      s->stop = true;
      s->cv.notify_all();
    }
    s->worker.join();   // finishes the jobs already handed over
  }
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (Request* r : s->active) {
    if (r->h) usaphmp_destroy(r->h);
    release_request(s, r);
  }
  for (Request* r : s->admitted) {
    if (r->h) usaphmp_destroy(r->h);
    release_request(s, r);
  }
  for (Request* r : s->pending) delete r;
  for (cudaEvent_t& ev : s->tick_ev)
    if (ev) cudaEventDestroy(ev);
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  if (s->d_tasks) cudaFree(s->d_tasks);
  if (s->d_status) cudaFree(s->d_status);
  if (s->pool) {
    cudaDeviceSynchronize();   // every stream-ordered free of the requests has run
    cudaMemPoolDestroy(s->pool);
  }
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

}  // extern "C"
