// Continuous-batching serving loop for GA solve requests of differing n and p.
//
// Requests wait in a FIFO until they fit: at most `max_active` run at once
// and the device bytes of the running ones stay within the HBM budget.  An
// admitted request gets its own instance handle (W, C and the GA state stay
// on the device until it finishes).  Every tick runs one generation of every
// running request with one launch per kernel over all of them (offspring,
// allocation + access terms, transfer term, reduction, selection), so the
// work of requests that arrived at different times overlaps on the device;
// a request whose last generation has run is rescored in fp64, its result
// kept for polling and its device memory released.  Each request's
// arithmetic depends only on its own data, so its result is the same alone
// and in any mix.
#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include "usaphmp.h"
#include "common.cuh"
#include "kernels.cuh"

using namespace usaphmp;

namespace {

using Clock = std::chrono::steady_clock;

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

}  // namespace

// Generations a step runs for the running requests at most: fewer host round
// trips per generation at the cost of admitting new requests only between
// steps.
constexpr int kGensPerTick = 8;

struct usaphmp_server_s {
  size_t budget = 0, used = 0;
  int max_active = 0, path = 0, num_sms = 0;
  cudaStream_t stream = nullptr;
  uint32_t* d_status = nullptr;
  Task* d_tasks = nullptr;
  std::vector<Task> h_tasks;
  bool tasks_dirty = true;  // the device task table no longer matches `active`
  std::deque<Request> pending;
  std::vector<Request> active;
  std::map<int64_t, Finished> done;
  int64_t next_ticket = 1;
};

namespace {

int finish(usaphmp_server_s* s, Request& r, int status, const std::string& err) {
  Finished f;
  f.status = status;
  f.error = err;
  if (status == USAPHMP_OK && r.h) {
    f.hubs.resize(r.p);
    f.S.resize(r.n);
    usaphmp_result res{};
    res.hubs = f.hubs.data();
    res.S = f.S.data();
    const int rc = usaphmp_ga_result(r.h, &res, s->stream);
    if (rc != USAPHMP_OK) {
      f.status = rc;
      f.error = usaphmp_last_error();
    } else {
      f.cost_fp64 = res.cost_fp64;
      f.cost_fp32 = res.cost_fp32;
      f.evals = res.evals;
    }
  }
  f.ms = std::chrono::duration<double, std::milli>(Clock::now() - r.t_submit).count();
  if (r.h) {
    usaphmp_destroy(r.h);
    r.h = nullptr;
    s->used -= r.bytes;
  }
  s->done[r.ticket] = std::move(f);
  return USAPHMP_OK;
}

// Admission: instance set-up and GA start state of one request.
int admit(usaphmp_server_s* s, Request& r) {
  int rc = usaphmp_create(r.n, r.p, r.W.data(), r.C.data(), r.chi, r.alpha, r.delta, &r.h);
  if (rc == USAPHMP_OK) {
    usaphmp_params prm;
    usaphmp_get_params(r.h, &prm);
    prm.islands = r.R;
    prm.island_size = r.P;
    prm.path = s->path;
    prm.use_graph = 0;
    rc = usaphmp_set_params(r.h, &prm);
  }
  if (rc == USAPHMP_OK) rc = usaphmp_ga_begin(r.h, r.seed, s->stream);
  std::vector<float>().swap(r.W);
  std::vector<float>().swap(r.C);
  if (rc != USAPHMP_OK) {
    const std::string err = usaphmp_last_error();
    if (r.h) { usaphmp_destroy(r.h); r.h = nullptr; }
    return finish(s, r, rc, err);
  }
  s->used += r.bytes;
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
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_status, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(s->d_status, 0, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_tasks, sizeof(Task) * kMaxTasks);
  if (e != cudaSuccess) {
    usaphmp_server_destroy(s);
    return report_error(e == cudaErrorMemoryAllocation ? USAPHMP_ENOMEM : USAPHMP_ECUDA,
                        std::string("server set-up: ") + cudaGetErrorString(e));
  }
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
  Request r;
  r.ticket = s->next_ticket++;
  r.n = n; r.p = p; r.R = islands; r.P = island_size; r.G = generations;
  r.chi = chi; r.alpha = alpha; r.delta = delta; r.seed = seed;
  r.W.assign(W, W + (size_t)n * n);
  r.C.assign(C, C + (size_t)n * n);
  r.bytes = handle_device_bytes(n, p, islands, island_size);
  r.t_submit = Clock::now();
  *ticket = r.ticket;
  if (r.bytes > s->budget) {
    finish(s, r, USAPHMP_EBUSY, "request needs more device memory than the server budget");
    return USAPHMP_OK;
  }
  s->pending.push_back(std::move(r));
  return USAPHMP_OK;
}

int usaphmp_server_step(usaphmp_server_t s, int32_t* n_active, int32_t* n_pending) {
  const NvtxRange nvtx_range("usaphmp_server_step");
  if (!s) return report_error(USAPHMP_EINVAL, "NULL server");
  // admission, FIFO, by slots and by device bytes
  while (!s->pending.empty() && (int)s->active.size() < s->max_active &&
         s->used + s->pending.front().bytes <= s->budget) {
    Request r = std::move(s->pending.front());
    s->pending.pop_front();
    const int rc = admit(s, r);
    if (rc != USAPHMP_OK) return rc;
    if (r.h) {
      s->active.push_back(std::move(r));
      s->tasks_dirty = true;
    }
  }
  // requests asking for no generation finish at once
  for (size_t i = 0; i < s->active.size();) {
    if (s->active[i].gens >= s->active[i].G) {
      finish(s, s->active[i], USAPHMP_OK, "");
      s->active.erase(s->active.begin() + i);
      s->tasks_dirty = true;
    } else {
      ++i;
    }
  }
  if (!s->active.empty()) {
    // up to kGensPerTick generations of every running request (no more than
    // any of them still needs), one launch per kernel over all of them; the
    // task table goes to the device only when the running set has changed
    bool tc = false;
    if (s->tasks_dirty) {
      s->h_tasks.clear();
      for (auto& r : s->active) s->h_tasks.push_back(handle_ga_task(r.h));
      cudaError_t e = cudaMemcpyAsync(s->d_tasks, s->h_tasks.data(), sizeof(Task) * s->h_tasks.size(),
                                      cudaMemcpyHostToDevice, s->stream);
      if (e != cudaSuccess) return report_error(USAPHMP_ECUDA, std::string("task upload: ") + cudaGetErrorString(e));
      s->tasks_dirty = false;
    }
    int k = kGensPerTick;
    for (auto& r : s->active) {
      tc = handle_uses_tc(r.h);
      k = std::min(k, r.G - r.gens);
    }
    const TaskSet ts{s->d_tasks, s->h_tasks.data(), (int)s->h_tasks.size()};
    for (int g = 0; g < k; ++g) {
      launch_children(ts, s->stream);
      launch_alloc(ts, true, tc, s->stream);
      if (tc)
        launch_eval_tc(ts, s->num_sms, s->d_status, s->stream);
      else
        launch_eval_plain(ts, s->stream);
      launch_reduce_select(ts, s->stream);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return report_error(USAPHMP_ECUDA, std::string("generation launch: ") + cudaGetErrorString(e));
    for (auto& r : s->active) {
      r.gens += k;
      handle_note_generations(r.h, k);
    }
    for (size_t i = 0; i < s->active.size();) {
      if (s->active[i].gens >= s->active[i].G) {
        finish(s, s->active[i], USAPHMP_OK, "");
        s->active.erase(s->active.begin() + i);
        s->tasks_dirty = true;
      } else {
        ++i;
      }
    }
  }
  if (n_active) *n_active = (int32_t)s->active.size();
  if (n_pending) *n_pending = (int32_t)s->pending.size();
  return USAPHMP_OK;
}

int usaphmp_server_cancel(usaphmp_server_t s, int64_t ticket) {
  if (!s) return report_error(USAPHMP_EINVAL, "NULL server");
  for (auto it = s->pending.begin(); it != s->pending.end(); ++it)
    if (it->ticket == ticket) {
      finish(s, *it, USAPHMP_ECANCELED, "cancelled");
      s->pending.erase(it);
      return USAPHMP_OK;
    }
  for (size_t i = 0; i < s->active.size(); ++i)
    if (s->active[i].ticket == ticket) {
      // its last generations may still run on the server's stream
      const cudaError_t e = cudaStreamSynchronize(s->stream);
      if (e != cudaSuccess) return report_error(USAPHMP_ECUDA, std::string("cancel: ") + cudaGetErrorString(e));
      finish(s, s->active[i], USAPHMP_ECANCELED, "cancelled");
      s->active.erase(s->active.begin() + i);
      s->tasks_dirty = true;
      return USAPHMP_OK;
    }
  return report_error(USAPHMP_EINVAL, "cancel: ticket " + std::to_string(ticket) + " is not queued or running");
}

int usaphmp_server_poll(usaphmp_server_t s, int64_t ticket, usaphmp_result* out) {
  if (!s || !out) return report_error(USAPHMP_EINVAL, "NULL argument");
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

void usaphmp_server_destroy(usaphmp_server_t s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (auto& r : s->active)
    if (r.h) usaphmp_destroy(r.h);
  if (s->d_tasks) cudaFree(s->d_tasks);
  if (s->d_status) cudaFree(s->d_status);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

}  // extern "C"
