// C ABI and host engine: instance set-up, workspaces, the evaluation
// pipeline (canonical form -> allocation / access terms -> transfer term ->
// fixed-order reduction) and the GA driver (§5) with CUDA-graph replay of
// generations.  Every arithmetic step runs in the library's kernels.
#include "usaphmp.h"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

using namespace usaphmp;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();
  return fail(e == cudaErrorMemoryAllocation ? USAPHMP_ENOMEM : USAPHMP_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(x)                                                   \
  do {                                                          \
    cudaError_t e_ = (x);                                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x);            \
  } while (0)

#define RET(x)                  \
  do {                          \
    int r_ = (x);               \
    if (r_ != USAPHMP_OK) return r_; \
  } while (0)

// Testing hook (usaphmp_debug_fail_allocations): device allocations left
// before one fails; negative = never.
std::atomic<int> g_fail_after{-1};

// Device allocations of a handle: cudaMalloc / cudaFree, or, for a handle
// created with a memory pool (the serving loop's), stream-ordered
// allocations from that pool on the handle's stream, which neither
// allocate from nor return memory to the device nor synchronise it.
struct AllocCtx {
  cudaMemPool_t pool = nullptr;
  cudaStream_t stream = nullptr;
};

template <class T>
cudaError_t dalloc(const AllocCtx& a, T** p, size_t count) {
  int left = g_fail_after.load();
  while (left >= 0) {
    if (left == 0) return cudaErrorMemoryAllocation;
    if (g_fail_after.compare_exchange_weak(left, left - 1)) break;
  }
  const size_t bytes = sizeof(T) * std::max<size_t>(count, 1);
  if (a.pool) return cudaMallocFromPoolAsync(reinterpret_cast<void**>(p), bytes, a.pool, a.stream);
  return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

template <class T>
void dfree(const AllocCtx& a, T*& p) {
  if (p) {
    if (a.pool)
      cudaFreeAsync(p, a.stream);
    else
      cudaFree(p);
  }
  p = nullptr;
}

// Device buffers of a population of up to `cap` chromosomes.
struct Pop {
  int cap = 0;
  size_t part_cap = 0;
  uint32_t* mask = nullptr;
  int32_t* hubs = nullptr;
  uint8_t* slot = nullptr;
  float* t12 = nullptr;
  float* chub = nullptr;
  float* part = nullptr;
  float* fit = nullptr;
  void release(const AllocCtx& a) {
    dfree(a, mask); dfree(a, hubs); dfree(a, slot); dfree(a, t12); dfree(a, chub); dfree(a, part); dfree(a, fit);
    cap = 0;
    part_cap = 0;
  }
};

}  // namespace

struct usaphmp_s {
  AllocCtx ac;  // how this handle allocates device memory (pool and stream, or cudaMalloc)
  int n = 0, p = 0, ldw = 0, ns = 0, nw = 0;
  double chi = 0, alpha = 0, delta = 0;
  int symmetric = 0;
  float* W = nullptr;
  float* C = nullptr;
  float* CTbuf = nullptr;
  float* Ufold = nullptr;   // fp32 folded W (symmetric C): the plain evaluator's operand
  float* O = nullptr;
  float* D = nullptr;
  __nv_bfloat16* Whi = nullptr;
  __nv_bfloat16* Wlo = nullptr;
  char* tmaps = nullptr;  // two CUtensorMap in device memory
  usaphmp_params prm{};
  TcTile tile{};  // tile shape of the tensor-core evaluator (usaphmp_set_tile / usaphmp_autotune)
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  uint32_t* d_status = nullptr;
  int* d_bad = nullptr;
  uint32_t* h_status = nullptr;  // pinned (pageable for a pool handle: no host-allocation synchronisation)
  int* h_bad = nullptr;
  double* d_dscratch = nullptr;
  double* d_cost = nullptr;
  double* d_rpart = nullptr;
  int rpart_cap = 0;
  double* d_dist64 = nullptr;  // p*p fp64 hub-path table of the returned solution (hub-path routing)
  double* d_total = nullptr;   // sum of W, fp64 (device)
  double* d_ls = nullptr;      // local-search scratch of the returned solution
  double* d_ls_batch = nullptr;  // usaphmp_local_search_dev scratch (grows, kept)
  size_t ls_batch_cap = 0;
  float* d_WT = nullptr;       // local search: W transposed and fp64 flow sums [O; D]
  double* d_OD64 = nullptr;    //   (made on first use)
  double* d_part64 = nullptr;  // fp64 reference path: per-chromosome partial sums,
  double* d_cost64 = nullptr;  //   costs and hub-path tables, for up to cap64 chromosomes
  double* d_paths64 = nullptr;
  int cap64 = 0;
  int32_t* d_ls_count = nullptr;  // its moves and sweeps
  double total_flow = 0.0;     // the same on the host
  // evaluation workspace and host-call staging
  Pop ev;
  int32_t* d_hubs_in = nullptr;
  int32_t* d_S_in = nullptr;
  float* h_fit_out = nullptr;        // pinned fitness of usaphmp_eval (written by the device through its mapping)
  int in_cap = 0;

  // GA
  Pop ga;
  Pop one;
  int ga_R = 0, ga_P = 0;
  uint32_t* anc = nullptr;
  float* anc_fit = nullptr;
  uint32_t* best = nullptr;
  float* best_fit = nullptr;
  int* gen = nullptr;
  int* done = nullptr;
  uint32_t* mask0 = nullptr;
  Task ga_task{};
  bool ga_ready = false;
  int64_t ga_evals = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t graph_stream = nullptr;
  cudaStream_t copy_stream = nullptr;          // usaphmp_eval: input copies in chunks
  cudaEvent_t chunk_ev[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t prof_ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

namespace {

DevInst inst_of(const usaphmp_s* h) {
  DevInst in;
  in.n = h->n; in.p = h->p; in.ldw = h->ldw; in.ns = h->ns; in.nw = h->nw;
  in.symmetric = h->symmetric;
  in.routing = h->prm.routing;
  in.chi = (float)h->chi; in.alpha = (float)h->alpha; in.delta = (float)h->delta;
  in.chi_d = h->chi; in.alpha_d = h->alpha; in.delta_d = h->delta;
  in.W = h->W; in.C = h->C; in.CT = h->symmetric ? h->C : h->CTbuf;
  in.O = h->O; in.D = h->D; in.Whi = h->Whi; in.Wlo = h->Wlo;
  in.wtri = h->symmetric;
  in.Ufold = h->symmetric ? h->Ufold : nullptr;
  return in;
}

bool use_tc(const usaphmp_s* h) { return h->prm.path == USAPHMP_PATH_SPLIT_BF16; }
bool use_fp64(const usaphmp_s* h) { return h->prm.path == USAPHMP_PATH_FP64_REF; }

// Scratch of the fp64 reference path for B chromosomes (allocated outside any
// stream capture: by the calls that evaluate and by ensure_ga).
int ensure_fp64(usaphmp_s* h, int B) {
  if (!use_fp64(h)) return USAPHMP_OK;
  const bool paths = h->prm.routing != USAPHMP_ROUTE_DIRECT;
  if (h->cap64 >= B && (!paths || h->d_paths64)) return USAPHMP_OK;
  dfree(h->ac, h->d_part64); dfree(h->ac, h->d_cost64); dfree(h->ac, h->d_paths64);
  h->cap64 = 0;
  CK(dalloc(h->ac, &h->d_part64, (size_t)B * rescore_parts(h->n)));
  CK(dalloc(h->ac, &h->d_cost64, (size_t)B));
  if (paths) CK(dalloc(h->ac, &h->d_paths64, (size_t)B * h->p * h->p));
  h->cap64 = B;
  return USAPHMP_OK;
}

// Per-instance inputs of the allocation local search (W transposed, fp64
// flow sums), made on first use.
int ensure_ls(usaphmp_s* h, cudaStream_t s) {
  if (h->d_WT && h->d_OD64) return USAPHMP_OK;
  dfree(h->ac, h->d_WT); dfree(h->ac, h->d_OD64);
  float* wt = nullptr;
  double* od = nullptr;
  CK(dalloc(h->ac, &wt, (size_t)h->n * h->ldw));
  const cudaError_t e = dalloc(h->ac, &od, (size_t)2 * h->n);
  if (e != cudaSuccess) {
    dfree(h->ac, wt);
    return cuda_fail(e, "dalloc(h->ac, &od, 2 * n)");
  }
  CK(cudaMemsetAsync(wt, 0, sizeof(float) * (size_t)h->n * h->ldw, s));
  launch_ls_prepare(h->W, h->n, h->ldw, wt, od, s);
  CK(cudaGetLastError());
  h->d_WT = wt;
  h->d_OD64 = od;
  return USAPHMP_OK;
}

// fp64 reference evaluation of a task whose hubs and slots are set (the
// hub-path tables exist whenever the task routes through hubs).
void launch_fp64_eval(usaphmp_s* h, const Task& task, cudaStream_t s) {
  launch_rescore(task.in, task.pop.B, task.pop.hubs, task.pop.slot, h->d_part64, h->d_cost64, s, h->d_paths64, 1.0);
  launch_fit_from_fp64(h->d_cost64, task.pop.fit, task.pop.B, task.pop.out_scale, s);
}

int part_rows(const usaphmp_s* h, int B) {
  return use_tc(h) ? tc_part_rows(h->n) : plain_rows(h->n, B);
}

size_t part_elems(const usaphmp_s* h, int B) {
  const size_t tc = (size_t)tc_part_rows(h->n) * B;
  const size_t plain = (size_t)plain_rows(h->n, B) * B;
  return std::max(tc, plain);
}

int ensure_pop(usaphmp_s* h, Pop& P, int B, size_t need_part = 0) {
  need_part = std::max(need_part, part_elems(h, B));
  if (P.cap >= B && P.part_cap >= need_part) return USAPHMP_OK;
  P.release(h->ac);
  CK(dalloc(h->ac, &P.mask, (size_t)B * h->nw));
  CK(dalloc(h->ac, &P.hubs, (size_t)B * h->p));
  CK(dalloc(h->ac, &P.slot, (size_t)B * h->ns));
  CK(dalloc(h->ac, &P.t12, (size_t)B));
  CK(dalloc(h->ac, &P.chub, (size_t)B * chub_cstride(h->p)));
  CK(dalloc(h->ac, &P.part, need_part));
  CK(dalloc(h->ac, &P.fit, (size_t)B));
  P.cap = B;
  P.part_cap = need_part;
  return USAPHMP_OK;
}

PopBuf popbuf(const usaphmp_s* h, const Pop& P, int B) {
  PopBuf pb;
  pb.B = B;
  pb.mask = P.mask; pb.hubs = P.hubs; pb.slot = P.slot; pb.t12 = P.t12;
  pb.chub = P.chub; pb.part = P.part; pb.fit = P.fit;
  pb.npart = part_rows(h, B);
  pb.hubs_in = nullptr;
  pb.slot_in = nullptr;
  pb.status = h->d_status;
  pb.out_scale = 1.0f;
  pb.status_host = nullptr;
  pb.bad = h->d_bad;
  return pb;
}

// Factor of §4.3 applied to objective values returned to the caller.
double output_scale(const usaphmp_s* h) {
  switch (h->prm.scale) {
    case USAPHMP_SCALE_MILLI: return 1e-3;
    case USAPHMP_SCALE_PER_FLOW: return 1.0 / h->total_flow;
    default: return 1.0;
  }
}

Task make_task(const usaphmp_s* h, const PopBuf& pb) {
  Task t{};
  t.in = inst_of(h);
  t.pop = pb;
  t.tmap_hi = h->tmaps;
  t.tmap_lo = h->tmaps ? static_cast<const char*>(h->tmaps) + sizeof(CUtensorMap) : nullptr;
  return t;
}

// The error a device status word (and the index of the first invalid
// chromosome) stands for.
int status_error(uint32_t st, int bad, const char* what) {
  if (st & kStatusTimeout) return fail(USAPHMP_ETIMEOUT, std::string(what) + ": a device wait timed out");
  if (st & kStatusBadChromosome)
    return fail(USAPHMP_EINVAL_CHROM, std::string(what) + ": chromosome " + std::to_string(bad) +
                                          " is not a valid single allocation (distinct hubs, S[i] an open hub, S[hub] = hub)");
  if (st & kStatusBadValue) return fail(USAPHMP_EINVAL, std::string(what) + ": W or C has a negative or non-finite entry");
  return USAPHMP_OK;
}

int check_status(usaphmp_s* h, cudaStream_t s, const char* what) {
  CK(cudaMemcpyAsync(h->h_status, h->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h->h_bad, h->d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return status_error(*h->h_status, *h->h_bad, what);
}

int reset_status(usaphmp_s* h, cudaStream_t s) {
  CK(cudaMemsetAsync(h->d_status, 0, sizeof(uint32_t), s));
  CK(cudaMemsetAsync(h->d_bad, 0x7f, sizeof(int), s));
  return USAPHMP_OK;
}

// Transfer term + reduction for a task whose hubs/slots/t12/chub are set.
int run_transfer(usaphmp_s* h, const Task& task, cudaStream_t s) {
  TaskSet ts{nullptr, &task, 1};
  if (use_fp64(h)) {
    RET(ensure_fp64(h, task.pop.B));
    launch_fp64_eval(h, task, s);
    CK(cudaGetLastError());
    return USAPHMP_OK;
  }
  if (use_tc(h))
    launch_eval_tc(ts, h->num_sms, h->d_status, s, h->tile);
  else
    launch_eval_plain(ts, s);
  CK(cudaGetLastError());
  launch_reduce(ts, s);
  CK(cudaGetLastError());
  return USAPHMP_OK;
}

// Allocation (nearest or given), access terms, transfer term, reduction.
int run_eval(usaphmp_s* h, const Task& task, bool nearest, cudaStream_t s) {
  TaskSet ts{nullptr, &task, 1};
  launch_alloc(ts, nearest, use_tc(h), s);
  CK(cudaGetLastError());
  return run_transfer(h, task, s);
}

int encode_tmaps(usaphmp_s* h) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
  if (!fn || q != cudaDriverEntryPointSuccess) return fail(USAPHMP_ECUDA, "cuTensorMapEncodeTiled not available");
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  CUtensorMap maps[2];
  for (int k = 0; k < 2; ++k) {
    const cuuint64_t dims[2] = {(cuuint64_t)h->ldw, (cuuint64_t)h->n};
    const cuuint64_t strides[1] = {(cuuint64_t)h->ldw * 2};
    const cuuint32_t box[2] = {64, 128};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(&maps[k], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, k == 0 ? (void*)h->Whi : (void*)h->Wlo,
                        dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(USAPHMP_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  }
  CK(dalloc(h->ac, &h->tmaps, sizeof(maps)));
  if (h->ac.pool)
    CK(cudaMemcpyAsync(h->tmaps, maps, sizeof(maps), cudaMemcpyHostToDevice, h->ac.stream));   // pageable: staged now
  else
    CK(cudaMemcpy(h->tmaps, maps, sizeof(maps), cudaMemcpyHostToDevice));
  return USAPHMP_OK;
}

int create_common(usaphmp_s* h, const float* W, const float* C, bool dev, cudaStream_t s) {
  const int n = h->n;
  CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
  h->ac.stream = h->stream;
  int dev_id = 0;
  CK(cudaGetDevice(&dev_id));
  CK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev_id));
  int optin = 0;
  CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev_id));
  prepare_eval_plain(optin);
  prepare_eval_tc();
  CK(cudaGetLastError());
  const size_t mat = (size_t)n * h->ldw;
  CK(dalloc(h->ac, &h->W, mat));
  CK(dalloc(h->ac, &h->C, mat));
  CK(dalloc(h->ac, &h->O, h->ns));   // padded to ns: the allocation kernel reads four nodes at a time
  CK(dalloc(h->ac, &h->D, h->ns));
  CK(dalloc(h->ac, &h->Whi, mat));
  CK(dalloc(h->ac, &h->Wlo, mat));
  CK(dalloc(h->ac, &h->d_status, 1));
  CK(dalloc(h->ac, &h->d_bad, 1));
  CK(dalloc(h->ac, &h->d_dscratch, n));
  CK(dalloc(h->ac, &h->d_total, 1));
  if (h->ac.pool) {
    h->h_status = new uint32_t[1];
    h->h_bad = new int[1];
  } else {
    CK(cudaMallocHost(&h->h_status, sizeof(uint32_t)));
    CK(cudaMallocHost(&h->h_bad, sizeof(int)));
  }
  if (!dev) s = h->stream;
  CK(cudaMemsetAsync(h->W, 0, mat * sizeof(float), s));
  CK(cudaMemsetAsync(h->C, 0, mat * sizeof(float), s));
  const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpy2DAsync(h->W, h->ldw * sizeof(float), W, n * sizeof(float), n * sizeof(float), n, kind, s));
  CK(cudaMemcpy2DAsync(h->C, h->ldw * sizeof(float), C, n * sizeof(float), n * sizeof(float), n, kind, s));
  RET(reset_status(h, s));
  launch_check_values(h->W, h->C, n, h->ldw, h->d_status, s);
  CK(cudaMemsetAsync(h->O, 0, sizeof(float) * h->ns, s));
  CK(cudaMemsetAsync(h->D, 0, sizeof(float) * h->ns, s));
  launch_flows(h->W, n, h->ldw, h->O, h->D, s);
  launch_total_flow(h->W, n, h->ldw, h->d_dscratch, h->d_total, s);
  CK(cudaMemcpyAsync(&h->total_flow, h->d_total, sizeof(double), cudaMemcpyDeviceToHost, s));
  uint32_t* d_asym = reinterpret_cast<uint32_t*>(h->d_bad);  // reuse as a flag
  CK(cudaMemsetAsync(d_asym, 0, sizeof(uint32_t), s));
  launch_asymmetry(h->C, n, h->ldw, d_asym, s);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(h->h_bad, d_asym, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h->h_status, h->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (*h->h_status & kStatusBadValue) return fail(USAPHMP_EINVAL, "W or C has a negative or non-finite entry");
  h->symmetric = (*h->h_bad == 0) ? 1 : 0;
  // symmetric C: every hub-to-hub table (direct or hub paths) is symmetric,
  // so the tensor-core evaluator takes the folded, upper-triangular U
  if (h->symmetric) {
    CK(dalloc(h->ac, &h->Ufold, mat));
    launch_split_bf16_upper(h->W, h->Whi, h->Wlo, h->Ufold, n, h->ldw, s);
  } else
    launch_split_bf16(h->W, h->Whi, h->Wlo, (long long)mat, s);
  if (!h->symmetric) {
    CK(dalloc(h->ac, &h->CTbuf, mat));
    CK(cudaMemsetAsync(h->CTbuf, 0, mat * sizeof(float), s));
    launch_transpose(h->C, h->CTbuf, n, h->ldw, s);
    CK(cudaGetLastError());
  }
  RET(encode_tmaps(h));
  CK(cudaStreamSynchronize(s));
  return USAPHMP_OK;
}

int create_impl(int32_t n, int32_t p, const float* W, const float* C, double chi, double alpha, double delta,
                bool dev, void* stream, usaphmp_t* out, cudaMemPool_t pool = nullptr) {
  const NvtxRange nvtx_range("usaphmp_create");
  if (!out) return fail(USAPHMP_EINVAL, "out is NULL");
  *out = nullptr;
  if (!W || !C) return fail(USAPHMP_EINVAL, "W or C is NULL");
  if (n < 2 || n > kMaxN) return fail(USAPHMP_EINVAL, "n must be in [2, 16384]");
  if (p < 1 || p > n || p > kMaxP) return fail(USAPHMP_EINVAL, "p must be in [1, min(n, 255)]");
  if (!(chi >= 0) || !(alpha >= 0) || !(delta >= 0) || chi > 1e30 || alpha > 1e30 || delta > 1e30)
    return fail(USAPHMP_EINVAL, "chi, alpha, delta must be finite and >= 0");
  usaphmp_s* h = new usaphmp_s();
  h->ac.pool = dev ? nullptr : pool;   // pool handles are made from host arrays on their own stream
  h->n = n; h->p = p;
  h->ldw = round_up(n, 8);
  h->ns = round_up(n, 64);
  h->nw = (n + 31) / 32;
  h->chi = chi; h->alpha = alpha; h->delta = delta;
  h->prm.islands = 64;
  h->prm.island_size = 64;
  h->prm.n1 = 10;
  h->prm.path = USAPHMP_PATH_SPLIT_BF16;
  h->prm.elitist = 0;
  h->prm.use_graph = 1;
  h->prm.routing = USAPHMP_ROUTE_DIRECT;
  h->prm.scale = USAPHMP_SCALE_RAW;
  h->prm.local_search = 0;
  h->prm.island_offset = 0;
  const int r = create_common(h, W, C, dev, static_cast<cudaStream_t>(stream));
  if (r != USAPHMP_OK) {
    const std::string msg = g_err;
    usaphmp_destroy(h);
    g_err = msg;
    return r;
  }
  *out = h;
  return USAPHMP_OK;
}

void drop_graph(usaphmp_s* h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->gexec = nullptr;
  h->graph = nullptr;
}

// Chunks of a host-buffer evaluation: about 1024 chromosomes each (at most
// 8), one for smaller calls.  The canonical form and the access terms of a
// chunk run while the later chunks are still being copied; the transfer term
// then runs once over all B (one launch keeps the tensor-core tiles full).
#ifndef USAPHMP_EVAL_CHUNK
#define USAPHMP_EVAL_CHUNK 1024
#endif
int eval_chunks(int B) {
  const int K = B / USAPHMP_EVAL_CHUNK;
  return K < 1 ? 1 : (K > 8 ? 8 : K);
}

// Canonical form, allocation terms, transfer term and reduction of B
// chromosomes given in node ids, enqueued on s (no synchronisation).
int enqueue_eval_canonical(usaphmp_s* h, int B, const int32_t* hubs_in, const int32_t* S, float* fit_out,
                           cudaStream_t s) {
  RET(ensure_pop(h, h->ev, B));
  RET(reset_status(h, s));
  PopBuf pb = popbuf(h, h->ev, B);
  pb.fit = fit_out;
  pb.out_scale = (float)output_scale(h);
  const Task task = make_task(h, pb);
  if (launch_canon_alloc(task, hubs_in, S, h->d_bad, 0, use_tc(h), s)) {
    CK(cudaGetLastError());
    return run_transfer(h, task, s);
  }
  launch_canon(hubs_in, S, B, h->n, h->p, h->ns, h->ev.hubs, h->ev.slot, h->d_status, h->d_bad, s);
  CK(cudaGetLastError());
  return run_eval(h, task, false, s);
}

int eval_canonical(usaphmp_s* h, int B, const int32_t* hubs_in, const int32_t* S, float* fit_out, cudaStream_t s) {
  RET(enqueue_eval_canonical(h, B, hubs_in, S, fit_out, s));
  return check_status(h, s, "usaphmp_eval");
}

// GA state for R islands of P (B = R*P); (re)allocated when the shape changes.
int ensure_ga(usaphmp_s* h) {
  const int R = h->prm.islands, P = h->prm.island_size, B = R * P;
  RET(ensure_pop(h, h->ga, B));
  RET(ensure_pop(h, h->one, 1));
  if (h->ga_R != R || h->ga_P != P || !h->anc) {
    h->ga_R = h->ga_P = 0;  // stays 0 unless every buffer below is allocated
    dfree(h->ac, h->anc); dfree(h->ac, h->anc_fit); dfree(h->ac, h->best); dfree(h->ac, h->best_fit); dfree(h->ac, h->gen); dfree(h->ac, h->mask0);
    dfree(h->ac, h->done);
    CK(dalloc(h->ac, &h->done, 1));
    CK(h->ac.pool ? cudaMemsetAsync(h->done, 0, sizeof(int), h->ac.stream) : cudaMemset(h->done, 0, sizeof(int)));
    CK(dalloc(h->ac, &h->anc, (size_t)R * h->nw));
    CK(dalloc(h->ac, &h->anc_fit, (size_t)R));
    CK(dalloc(h->ac, &h->best, (size_t)h->nw));
    CK(dalloc(h->ac, &h->best_fit, 1));
    CK(dalloc(h->ac, &h->gen, 1));
    CK(dalloc(h->ac, &h->mask0, (size_t)h->nw));
    h->ga_R = R;
    h->ga_P = P;
  }
  const int np = rescore_parts(h->n);
  if (h->rpart_cap < np) {
    dfree(h->ac, h->d_rpart); dfree(h->ac, h->d_cost);
    CK(dalloc(h->ac, &h->d_rpart, (size_t)np * 2));
    CK(dalloc(h->ac, &h->d_cost, 2));
    h->rpart_cap = np;
  }
  if (!h->d_dist64) CK(dalloc(h->ac, &h->d_dist64, (size_t)h->p * h->p));
  if (!h->d_ls) CK(dalloc(h->ac, &h->d_ls, local_search_scratch_doubles(h->n, h->p)));
  if (!h->d_ls_count) CK(dalloc(h->ac, &h->d_ls_count, 2));
  RET(ensure_fp64(h, R * P));
  return USAPHMP_OK;
}

Task ga_task_of(usaphmp_s* h, unsigned long long seed) {
  const int R = h->prm.islands, P = h->prm.island_size;
  Task t = make_task(h, popbuf(h, h->ga, R * P));
  t.ga.R = R; t.ga.P = P; t.ga.N1 = h->prm.n1; t.ga.elitist = h->prm.elitist;
  t.ga.island_offset = h->prm.island_offset;
  t.ga.seed = seed;
  t.ga.gen = h->gen; t.ga.anc = h->anc; t.ga.anc_fit = h->anc_fit;
  t.ga.best = h->best; t.ga.best_fit = h->best_fit;
  t.ga.done = h->done;
  return t;
}

int enqueue_generation(usaphmp_s* h, cudaStream_t s) {
  TaskSet ts{nullptr, &h->ga_task, 1};
  launch_children(ts, s);
  launch_alloc(ts, true, use_tc(h), s);
  if (use_fp64(h)) {
    launch_fp64_eval(h, h->ga_task, s);   // scratch sized by ensure_ga
    launch_select(ts, s);
  } else {
    if (use_tc(h))
      launch_eval_tc(ts, h->num_sms, h->d_status, s, h->tile);
    else
      launch_eval_plain(ts, s);
    launch_reduce_select(ts, s);
  }
  CK(cudaGetLastError());
  return USAPHMP_OK;
}

// Decodes a mask into ascending hubs on the host (tiny; result copy-out only).
std::vector<int32_t> mask_to_hubs(const std::vector<uint32_t>& m, int n) {
  std::vector<int32_t> hubs;
  for (int i = 0; i < n; ++i)
    if (m[i >> 5] & (1u << (i & 31))) hubs.push_back(i);
  return hubs;
}

}  // namespace

int usaphmp::report_error(int code, const std::string& msg) { return fail(code, msg); }

int usaphmp::create_pooled(int32_t n, int32_t p, const float* W, const float* C, double chi, double alpha,
                           double delta, cudaMemPool_t pool, usaphmp_t* out) {
  return create_impl(n, p, W, C, chi, alpha, delta, false, nullptr, out, pool);
}

cudaStream_t usaphmp::handle_stream(const usaphmp_s* h) { return h->stream; }

const Task& usaphmp::handle_ga_task(const usaphmp_s* h) { return h->ga_task; }
bool usaphmp::handle_uses_tc(const usaphmp_s* h) { return use_tc(h); }
void usaphmp::handle_note_generations(usaphmp_s* h, int g) {
  h->ga_evals += (int64_t)g * h->prm.islands * h->prm.island_size;
}

size_t usaphmp::handle_device_bytes(int n, int p, int R, int P) {
  const size_t ldw = round_up(n, 8), ns = round_up(n, 64), nw = (n + 31) / 32;
  const size_t B = (size_t)R * P;
  const size_t mat = (size_t)n * ldw;
  // W, C and either CT (asymmetric C) or the fp32 folded U (symmetric C); Whi, Wlo; O, D (ns each); misc
  size_t bytes = 3 * mat * 4 + 2 * mat * 2 + 2 * ns * 4 + 2 * (size_t)n * 4 + 256;
  const size_t rows = std::max((size_t)tc_part_rows(n), (size_t)plain_rows(n, (int)B));
  const size_t per_chrom = nw * 4 + (size_t)p * 4 + ns + 8 + (size_t)chub_cstride(p) * 4 + rows * 4;
  bytes += (B + 1) * per_chrom + (size_t)R * (nw * 4 + 4) + 3 * nw * 4 + 1024;
  return bytes;
}

extern "C" {

const char* usaphmp_last_error(void) { return g_err.c_str(); }

int usaphmp_create(int32_t n, int32_t p, const float* W, const float* C, double chi, double alpha,
                   double delta, usaphmp_t* out) {
  return create_impl(n, p, W, C, chi, alpha, delta, false, nullptr, out);
}

int usaphmp_create_dev(int32_t n, int32_t p, const float* W, const float* C, double chi, double alpha,
                       double delta, void* stream, usaphmp_t* out) {
  return create_impl(n, p, W, C, chi, alpha, delta, true, stream, out);
}

void usaphmp_destroy(usaphmp_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graph(h);
  if (h->graph_stream) cudaStreamDestroy(h->graph_stream);
  for (cudaEvent_t& ev : h->chunk_ev)
    if (ev) cudaEventDestroy(ev);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  for (int k = 0; k < 6; ++k)
    if (h->prof_ev[k]) cudaEventDestroy(h->prof_ev[k]);
  dfree(h->ac, h->W); dfree(h->ac, h->C); dfree(h->ac, h->CTbuf); dfree(h->ac, h->Ufold); dfree(h->ac, h->O); dfree(h->ac, h->D); dfree(h->ac, h->Whi); dfree(h->ac, h->Wlo);
  dfree(h->ac, h->tmaps);
  dfree(h->ac, h->d_status); dfree(h->ac, h->d_bad); dfree(h->ac, h->d_dscratch); dfree(h->ac, h->d_cost); dfree(h->ac, h->d_rpart);
  dfree(h->ac, h->d_dist64); dfree(h->ac, h->d_total); dfree(h->ac, h->d_ls); dfree(h->ac, h->d_ls_count); dfree(h->ac, h->d_WT); dfree(h->ac, h->d_OD64);
  dfree(h->ac, h->d_ls_batch);
  h->ls_batch_cap = 0;
  dfree(h->ac, h->d_part64); dfree(h->ac, h->d_cost64); dfree(h->ac, h->d_paths64);
  if (h->ac.pool) {
    delete[] h->h_status;
    delete[] h->h_bad;
  } else {
    if (h->h_status) cudaFreeHost(h->h_status);
    if (h->h_bad) cudaFreeHost(h->h_bad);
  }
  h->ev.release(h->ac); h->ga.release(h->ac); h->one.release(h->ac);
  dfree(h->ac, h->d_hubs_in); dfree(h->ac, h->d_S_in);
  if (h->h_fit_out) cudaFreeHost(h->h_fit_out);
  dfree(h->ac, h->anc); dfree(h->ac, h->anc_fit); dfree(h->ac, h->best); dfree(h->ac, h->best_fit); dfree(h->ac, h->gen); dfree(h->ac, h->mask0);
  dfree(h->ac, h->done);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

int usaphmp_set_params(usaphmp_t h, const usaphmp_params* prm) {
  if (!h || !prm) return fail(USAPHMP_EINVAL, "NULL argument");
  if (prm->islands < 1 || prm->island_size < 2 || (prm->island_size & 1))
    return fail(USAPHMP_EINVAL, "islands must be >= 1 and island_size even and >= 2");
  if ((long long)prm->islands * prm->island_size > (1 << 24) ||
      (long long)prm->islands * prm->island_size * h->p >= (1ll << 31))
    return fail(USAPHMP_EINVAL, "population too large");
  if (prm->n1 < 0) return fail(USAPHMP_EINVAL, "n1 must be >= 0");
  if (prm->island_offset < 0 ||
      ((long long)prm->island_offset + prm->islands) * prm->island_size > 0x7fffffffll)
    return fail(USAPHMP_EINVAL, "island_offset must be >= 0 and (island_offset + islands) * island_size < 2^31");
  if (prm->path != USAPHMP_PATH_PLAIN_FP32 && prm->path != USAPHMP_PATH_SPLIT_BF16 &&
      prm->path != USAPHMP_PATH_FP64_REF)
    return fail(USAPHMP_EINVAL, "unknown path");
  if (prm->routing != USAPHMP_ROUTE_DIRECT && prm->routing != USAPHMP_ROUTE_HUB_PATHS)
    return fail(USAPHMP_EINVAL, "unknown routing");
  if (prm->scale != USAPHMP_SCALE_RAW && prm->scale != USAPHMP_SCALE_MILLI && prm->scale != USAPHMP_SCALE_PER_FLOW)
    return fail(USAPHMP_EINVAL, "unknown scale");
  if (prm->scale == USAPHMP_SCALE_PER_FLOW && !(h->total_flow > 0.0))
    return fail(USAPHMP_EINVAL, "scale per unit flow needs a positive total flow");
  if (prm->local_search < 0) return fail(USAPHMP_EINVAL, "local_search must be >= 0");
  h->prm = *prm;
  h->ga_ready = false;
  drop_graph(h);
  return USAPHMP_OK;
}

int usaphmp_set_tile(usaphmp_t h, const usaphmp_tile* tile) {
  if (!h || !tile) return fail(USAPHMP_EINVAL, "NULL argument");
  TcTile t;
  t.ntile = tile->ntile;
  t.stages = tile->stages;
  t.raster = tile->raster;
  t.pair = tile->pair;
  if (!tc_tile_fits(t, h->p))
    return fail(USAPHMP_EINVAL, "tile shape: ntile in {64, 128, 256} and >= p, stages 2..4 within shared memory "
                                "(ntile 256: at most 3, or 4 with pair 1), raster 0 or 1, pair 0 or 1");
  h->tile = t;
  drop_graph(h);
  return USAPHMP_OK;
}

int usaphmp_get_tile(usaphmp_t h, usaphmp_tile* tile) {
  if (!h || !tile) return fail(USAPHMP_EINVAL, "NULL argument");
  tile->ntile = h->tile.ntile;
  tile->stages = h->tile.stages;
  tile->raster = h->tile.raster;
  tile->pair = h->tile.pair;
  return USAPHMP_OK;
}

int usaphmp_autotune(usaphmp_t h, int32_t reps, const char* cache_path, usaphmp_tile* chosen, double* chosen_ms,
                     double* default_ms, int32_t* from_cache) {
  const NvtxRange nvtx_range("usaphmp_autotune");
  if (!h) return fail(USAPHMP_EINVAL, "NULL handle");
  if (reps < 1 || reps > 1000) return fail(USAPHMP_EINVAL, "reps must be in [1, 1000]");
  if (from_cache) *from_cache = 0;
  if (chosen_ms) *chosen_ms = 0;
  if (default_ms) *default_ms = 0;
  auto report = [&]() -> int {
    if (chosen) RET(usaphmp_get_tile(h, chosen));
    return USAPHMP_OK;
  };
  if (!use_tc(h)) return report();
  const int B = h->prm.islands * h->prm.island_size;
  int dev_id = 0;
  CK(cudaGetDevice(&dev_id));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, dev_id));
  // the folded operand runs other K loops than the full W: separate buckets
  const std::string device = std::string(prop.name) + (h->symmetric ? " (folded operand)" : "");
  if (cache_path) {
    usaphmp_tile t{};
    const int r = usaphmp_tile_cache_lookup(cache_path, device.c_str(), h->n, h->p, B, &t, nullptr);
    if (r < 0) return r;
    if (r == 1 && usaphmp_set_tile(h, &t) == USAPHMP_OK) {
      if (from_cache) *from_cache = 1;
      return report();
    }
  }
  // A population to time on: one generation grown from the initial solution.
  cudaStream_t s = h->stream;
  RET(usaphmp_ga_begin(h, 0x74756e65ull, s));
  RET(enqueue_generation(h, s));
  h->ga_ready = false;
  std::vector<TcTile> cands{TcTile{}};
  for (int pr : {0, 1})
    for (int nt : {256, 128, 64})
      for (int st : {2, 3, 4})
        for (int ra : {0, 1}) {
          TcTile t;
          t.ntile = nt; t.stages = st; t.raster = ra; t.pair = pr;
          const TcTile d{};
          const bool is_default = nt == d.ntile && st == d.stages && ra == d.raster && pr == d.pair;
          if (!is_default && tc_tile_fits(t, h->p)) cands.push_back(t);
        }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(ce, "cudaEventCreate"); }
  TaskSet ts{nullptr, &h->ga_task, 1};
  double best_ms = 0, dflt_ms = 0;
  TcTile best{};
  for (size_t k = 0; k < cands.size() && ce == cudaSuccess; ++k) {
    launch_eval_tc(ts, h->num_sms, h->d_status, s, cands[k]);
    ce = cudaEventRecord(e0, s);
    for (int r = 0; r < reps && ce == cudaSuccess; ++r) {
      launch_eval_tc(ts, h->num_sms, h->d_status, s, cands[k]);
      ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    const double per = (double)ms / reps;
    if (k == 0) dflt_ms = per;
    if (k == 0 || per < best_ms) {
      best_ms = per;
      best = cands[k];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(ce);
  RET(check_status(h, s, "usaphmp_autotune"));
  h->tile = best;
  drop_graph(h);
  if (cache_path) {
    const usaphmp_tile t{best.ntile, best.stages, best.raster, best.pair};
    RET(usaphmp_tile_cache_store(cache_path, device.c_str(), h->n, h->p, B, &t, best_ms));
  }
  if (chosen_ms) *chosen_ms = best_ms;
  if (default_ms) *default_ms = dflt_ms;
  return report();
}

int usaphmp_get_params(usaphmp_t h, usaphmp_params* prm) {
  if (!h || !prm) return fail(USAPHMP_EINVAL, "NULL argument");
  *prm = h->prm;
  return USAPHMP_OK;
}

int usaphmp_get_info(usaphmp_t h, usaphmp_info* info) {
  if (!h || !info) return fail(USAPHMP_EINVAL, "NULL argument");
  info->n = h->n;
  info->p = h->p;
  info->ldw = h->ldw;
  info->ns = h->ns;
  info->c_symmetric = h->symmetric;
  info->tc_folded = h->symmetric;
  return USAPHMP_OK;
}

int usaphmp_eval_dev(usaphmp_t h, int32_t B, const int32_t* hubs, const int32_t* S, float* fitness, void* stream) {
  const NvtxRange nvtx_range("usaphmp_eval_dev");
  if (!h) return fail(USAPHMP_EINVAL, "NULL handle");
  if (B < 0) return fail(USAPHMP_EINVAL, "B < 0");
  if (B == 0) return USAPHMP_OK;
  if (!hubs || !S || !fitness) return fail(USAPHMP_EINVAL, "NULL argument");
  return eval_canonical(h, B, hubs, S, fitness, static_cast<cudaStream_t>(stream));
}

int usaphmp_eval(usaphmp_t h, int32_t B, const int32_t* hubs, const int32_t* S, double* fitness) {
  const NvtxRange nvtx_range("usaphmp_eval");
  if (!h) return fail(USAPHMP_EINVAL, "NULL handle");
  if (B < 0) return fail(USAPHMP_EINVAL, "B < 0");
  if (B == 0) return USAPHMP_OK;
  if (!hubs || !S || !fitness) return fail(USAPHMP_EINVAL, "NULL argument");
  cudaStream_t s = h->stream;
  if (h->in_cap < B) {
    dfree(h->ac, h->d_hubs_in); dfree(h->ac, h->d_S_in);
    if (h->h_fit_out) cudaFreeHost(h->h_fit_out);
    h->h_fit_out = nullptr;
    h->in_cap = 0;
    CK(dalloc(h->ac, &h->d_hubs_in, (size_t)B * h->p));
    CK(dalloc(h->ac, &h->d_S_in, (size_t)B * h->n));
    CK(cudaMallocHost(&h->h_fit_out, sizeof(float) * ((size_t)B + 2)));   // + the two status words
    h->in_cap = B;
  }
  // The inputs arrive in K chunks on a copy stream; the canonical form and
  // the allocation kernel (access terms, hub-cost tables) of each chunk run
  // as soon as it has landed, overlapping the copies of the later chunks,
  // and the transfer term and the reduction then run once over all B.  A
  // chromosome's fitness does not depend on the chunk or the batch it is
  // evaluated in (every stage works per chromosome and sums in a fixed order).
  const int K = eval_chunks(B);
  if (K > 1 && !h->copy_stream) {
    CK(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    for (cudaEvent_t& ev : h->chunk_ev) CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  }
  cudaStream_t cs = K > 1 ? h->copy_stream : s;
  // every return below happens after the copies from the caller's memory
  // have finished (both streams are synchronised)
  auto finish = [&](int rc) {
    cudaStreamSynchronize(cs);
    cudaStreamSynchronize(s);
    return rc;
  };
  int rc = ensure_pop(h, h->ev, B);
  if (rc != USAPHMP_OK) return rc;
  if (use_fp64(h) && (rc = ensure_fp64(h, B)) != USAPHMP_OK) return rc;
  // all copies first, back to back on the copy stream (hub ids whole, then S
  // chunk by chunk, an event after each chunk), so the copy engine never
  // waits for the host to enqueue the kernels
  auto chunk = [&](int k, int& c0, int& nb) {
    c0 = (int)((long long)B * k / K);
    nb = (int)((long long)B * (k + 1) / K) - c0;
  };
  cudaError_t e = cudaMemcpyAsync(h->d_hubs_in, hubs, sizeof(int32_t) * (size_t)B * h->p, cudaMemcpyHostToDevice, cs);
  for (int k = 0; k < K && e == cudaSuccess; ++k) {
    int c0, nb;
    chunk(k, c0, nb);
    e = cudaMemcpyAsync(h->d_S_in + (size_t)c0 * h->n, S + (size_t)c0 * h->n, sizeof(int32_t) * nb * h->n,
                        cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && K > 1) e = cudaEventRecord(h->chunk_ev[k], cs);
  }
  if (e != cudaSuccess) return finish(cuda_fail(e, "usaphmp_eval input copies"));
  if ((rc = reset_status(h, s)) != USAPHMP_OK) return finish(rc);
  PopBuf full = popbuf(h, h->ev, B);
  // the reduction writes the fitness, then the status words, straight into
  // the pinned host buffer (mapped into the device's address space): no
  // copy-out (the fp64 reference path reads the status with copies)
  full.fit = h->h_fit_out;
  uint32_t* st_host = reinterpret_cast<uint32_t*>(h->h_fit_out + B);
  if (!use_fp64(h)) full.status_host = st_host;
  full.out_scale = (float)output_scale(h);
  const int cst = chub_cstride(h->p);
  for (int k = 0; k < K; ++k) {
    int c0, nb;
    chunk(k, c0, nb);
    if (K > 1 && (e = cudaStreamWaitEvent(s, h->chunk_ev[k], 0)) != cudaSuccess)
      return finish(cuda_fail(e, "usaphmp_eval input copies"));
    PopBuf pc = full;
    pc.B = nb;
    pc.hubs += (size_t)c0 * h->p;
    pc.slot += (size_t)c0 * h->ns;
    pc.t12 += c0;
    pc.chub += (size_t)c0 * cst;
    const Task tc = make_task(h, pc);
    const int32_t* hin = h->d_hubs_in + (size_t)c0 * h->p;
    const int32_t* sin = h->d_S_in + (size_t)c0 * h->n;
    if (!launch_canon_alloc(tc, hin, sin, h->d_bad, c0, use_tc(h), s)) {
      launch_canon(hin, sin, nb, h->n, h->p, h->ns, pc.hubs, pc.slot, h->d_status, h->d_bad, s, c0);
      TaskSet ts{nullptr, &tc, 1};
      launch_alloc(ts, false, use_tc(h), s);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return finish(cuda_fail(e, "usaphmp_eval allocation"));
  }
  if ((rc = run_transfer(h, make_task(h, full), s)) != USAPHMP_OK) return finish(rc);
  if (full.status_host) {   // one synchronisation, then the words the reduction wrote
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return finish(cuda_fail(e, "usaphmp_eval"));
    if ((rc = status_error(st_host[0], (int)st_host[1], "usaphmp_eval")) != USAPHMP_OK) return rc;
  } else if ((rc = check_status(h, s, "usaphmp_eval")) != USAPHMP_OK) {
    return rc;
  }
  for (int b = 0; b < B; ++b) fitness[b] = h->h_fit_out[b];
  return USAPHMP_OK;
}

int usaphmp_layout(usaphmp_t h, int32_t* ns, int32_t* nw) {
  if (!h) return fail(USAPHMP_EINVAL, "NULL handle");
  if (ns) *ns = h->ns;
  if (nw) *nw = h->nw;
  return USAPHMP_OK;
}

int usaphmp_initial_dev(usaphmp_t h, uint32_t* mask, int32_t* hubs, void* stream) {
  if (!h || !mask || !hubs) return fail(USAPHMP_EINVAL, "NULL argument");
  launch_middle_nodes(h->C, h->n, h->ldw, h->p, h->d_dscratch, mask, hubs, static_cast<cudaStream_t>(stream));
  CK(cudaGetLastError());
  return USAPHMP_OK;
}

int usaphmp_children_dev(usaphmp_t h, int32_t R, int32_t P, const uint32_t* anc, uint64_t seed, int32_t g,
                         uint32_t* mask, int32_t* hubs, void* stream) {
  if (!h || !anc || !mask || !hubs) return fail(USAPHMP_EINVAL, "NULL argument");
  if (R < 1 || P < 2 || (P & 1) || g < 0) return fail(USAPHMP_EINVAL, "bad R, P or g");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  RET(ensure_ga(h));
  Task t{};
  t.in = inst_of(h);
  t.pop.B = R * P;
  t.pop.mask = mask;
  t.pop.hubs = hubs;
  t.ga.R = R; t.ga.P = P; t.ga.seed = seed;
  t.ga.anc = const_cast<uint32_t*>(anc);
  t.ga.gen = h->gen;
  CK(cudaMemcpyAsync(h->gen, &g, sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));  // g lives on the host stack
  TaskSet ts{nullptr, &t, 1};
  launch_children(ts, s);
  CK(cudaGetLastError());
  return USAPHMP_OK;
}

int usaphmp_allocate_dev(usaphmp_t h, int32_t B, const int32_t* hubs, uint8_t* slot, void* stream) {
  if (!h || !hubs || !slot) return fail(USAPHMP_EINVAL, "NULL argument");
  if (reinterpret_cast<uintptr_t>(slot) & 3u) return fail(USAPHMP_EINVAL, "slot must be 4-byte aligned");
  if (B <= 0) return B == 0 ? USAPHMP_OK : fail(USAPHMP_EINVAL, "B < 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  RET(ensure_pop(h, h->ev, B));
  PopBuf pb = popbuf(h, h->ev, B);
  pb.hubs_in = hubs;
  pb.slot = slot;
  const Task t = make_task(h, pb);
  TaskSet ts{nullptr, &t, 1};
  launch_alloc(ts, true, false, s);
  CK(cudaGetLastError());
  return USAPHMP_OK;
}

int usaphmp_eval_slots_dev(usaphmp_t h, int32_t B, const int32_t* hubs, const uint8_t* slot, float* fitness,
                           void* stream) {
  if (!h || !hubs || !slot || !fitness) return fail(USAPHMP_EINVAL, "NULL argument");
  if (reinterpret_cast<uintptr_t>(slot) & 3u) return fail(USAPHMP_EINVAL, "slot must be 4-byte aligned");
  if (B <= 0) return B == 0 ? USAPHMP_OK : fail(USAPHMP_EINVAL, "B < 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  RET(ensure_pop(h, h->ev, B));
  PopBuf pb = popbuf(h, h->ev, B);
  pb.hubs_in = hubs;
  pb.slot_in = slot;
  pb.fit = fitness;
  pb.out_scale = (float)output_scale(h);
  const Task t = make_task(h, pb);
  return run_eval(h, t, false, s);
}

int usaphmp_select_dev(usaphmp_t h, int32_t R, int32_t P, int32_t g, const uint32_t* mask, const float* fitness,
                       uint32_t* anc, float* anc_fit, uint32_t* best, float* best_fit, void* stream) {
  if (!h || !mask || !fitness || !anc || !anc_fit || !best || !best_fit) return fail(USAPHMP_EINVAL, "NULL argument");
  if (R < 1 || P < 1 || g < 0) return fail(USAPHMP_EINVAL, "bad R, P or g");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  RET(ensure_ga(h));
  Task t{};
  t.in = inst_of(h);
  t.pop.B = R * P;
  t.pop.mask = const_cast<uint32_t*>(mask);
  t.pop.fit = const_cast<float*>(fitness);
  t.ga.R = R; t.ga.P = P; t.ga.N1 = h->prm.n1; t.ga.elitist = h->prm.elitist;
  t.ga.anc = anc; t.ga.anc_fit = anc_fit; t.ga.best = best; t.ga.best_fit = best_fit;
  t.ga.gen = h->gen;
  CK(cudaMemcpyAsync(h->gen, &g, sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  TaskSet ts{nullptr, &t, 1};
  launch_select(ts, s);
  CK(cudaGetLastError());
  return USAPHMP_OK;
}

int usaphmp_local_search_dev(usaphmp_t h, int32_t B, const int32_t* hubs, uint8_t* slot, int32_t max_sweeps,
                             int32_t* moves, int32_t* sweeps, void* stream) {
  const NvtxRange nvtx_range("usaphmp_local_search_dev");
  if (!h || !hubs || !slot) return fail(USAPHMP_EINVAL, "NULL argument");
  if (B <= 0) return B == 0 ? USAPHMP_OK : fail(USAPHMP_EINVAL, "B < 0");
  if (max_sweeps < 1) return fail(USAPHMP_EINVAL, "max_sweeps must be >= 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  RET(ensure_ls(h, s));
  const size_t need = (size_t)B * local_search_scratch_doubles(h->n, h->p);
  if (h->ls_batch_cap < need) {
    CK(cudaStreamSynchronize(s));  // a previous call's kernels may still use the old scratch
    dfree(h->ac, h->d_ls_batch);
    h->ls_batch_cap = 0;
    CK(dalloc(h->ac, &h->d_ls_batch, need));
    h->ls_batch_cap = need;
  }
  launch_local_search(inst_of(h), h->d_WT, h->d_OD64, B, hubs, slot, max_sweeps, h->d_ls_batch, moves, sweeps, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return USAPHMP_OK;
}

int usaphmp_rescore_fp64_dev(usaphmp_t h, int32_t B, const int32_t* hubs, const uint8_t* slot, double* cost,
                             void* stream) {
  const NvtxRange nvtx_range("usaphmp_rescore_fp64_dev");
  if (!h || !hubs || !slot || !cost) return fail(USAPHMP_EINVAL, "NULL argument");
  if (B <= 0) return B == 0 ? USAPHMP_OK : fail(USAPHMP_EINVAL, "B < 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* part = nullptr;
  double* dist = nullptr;
  CK(dalloc(h->ac, &part, (size_t)rescore_parts(h->n) * B));
  if (h->prm.routing != USAPHMP_ROUTE_DIRECT) {
    const cudaError_t ea = dalloc(h->ac, &dist, (size_t)B * h->p * h->p);
    if (ea != cudaSuccess) {
      dfree(h->ac, part);
      return cuda_fail(ea, "dalloc(hub-path tables)");
    }
  }
  launch_rescore(inst_of(h), B, hubs, slot, part, cost, s, dist, output_scale(h));
  cudaError_t e = cudaGetLastError();
  cudaError_t e2 = cudaStreamSynchronize(s);
  dfree(h->ac, part);
  dfree(h->ac, dist);
  CK(e);
  CK(e2);
  return USAPHMP_OK;
}

int usaphmp_ga_begin(usaphmp_t h, uint64_t seed, void* stream) {
  const NvtxRange nvtx_range("usaphmp_ga_begin");
  if (!h) return fail(USAPHMP_EINVAL, "NULL handle");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  RET(ensure_ga(h));
  drop_graph(h);
  RET(reset_status(h, s));
  // initial solution (§4.1) and its fitness
  launch_middle_nodes(h->C, h->n, h->ldw, h->p, h->d_dscratch, h->mask0, h->one.hubs, s);
  CK(cudaGetLastError());
  const Task t1 = make_task(h, popbuf(h, h->one, 1));
  RET(run_eval(h, t1, true, s));
  h->ga_task = ga_task_of(h, seed);
  launch_ga_init(h->ga_task, h->mask0, h->one.fit, s);
  CK(cudaGetLastError());
  h->ga_ready = true;
  h->ga_evals = 1;
  return USAPHMP_OK;
}

int usaphmp_ga_run(usaphmp_t h, int32_t generations, void* stream) {
  const NvtxRange nvtx_range("usaphmp_ga_run");
  if (!h) return fail(USAPHMP_EINVAL, "NULL handle");
  if (!h->ga_ready) return fail(USAPHMP_EINVAL, "usaphmp_ga_begin first");
  if (generations < 0) return fail(USAPHMP_EINVAL, "generations < 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int B = h->prm.islands * h->prm.island_size;
  if (h->prm.use_graph) {
    if (!h->gexec) {
      if (!h->graph_stream) CK(cudaStreamCreateWithFlags(&h->graph_stream, cudaStreamNonBlocking));
      CK(cudaStreamBeginCapture(h->graph_stream, cudaStreamCaptureModeThreadLocal));
      const int r = enqueue_generation(h, h->graph_stream);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(h->graph_stream, &g);
      if (r != USAPHMP_OK) { if (g) cudaGraphDestroy(g); return r; }
      CK(e);
      h->graph = g;
      CK(cudaGraphInstantiate(&h->gexec, h->graph, 0));
    }
    for (int i = 0; i < generations; ++i) CK(cudaGraphLaunch(h->gexec, s));
  } else {
    for (int i = 0; i < generations; ++i) RET(enqueue_generation(h, s));
  }
  h->ga_evals += (int64_t)generations * B;
  return USAPHMP_OK;
}

int usaphmp_ga_run_profiled(usaphmp_t h, int32_t generations, void* stream, double* stage_ms) {
  const NvtxRange nvtx_range("usaphmp_ga_run_profiled");
  if (!h || !stage_ms) return fail(USAPHMP_EINVAL, "NULL argument");
  if (!h->ga_ready) return fail(USAPHMP_EINVAL, "usaphmp_ga_begin first");
  if (generations < 0) return fail(USAPHMP_EINVAL, "generations < 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int k = 0; k < 6; ++k)
    if (!h->prof_ev[k]) CK(cudaEventCreate(&h->prof_ev[k]));
  const int B = h->prm.islands * h->prm.island_size;
  TaskSet ts{nullptr, &h->ga_task, 1};
  for (int g = 0; g < generations; ++g) {
    CK(cudaEventRecord(h->prof_ev[0], s));
    launch_children(ts, s);
    CK(cudaEventRecord(h->prof_ev[1], s));
    launch_alloc(ts, true, use_tc(h), s);
    CK(cudaEventRecord(h->prof_ev[2], s));
    if (use_fp64(h))
      launch_fp64_eval(h, h->ga_task, s);
    else if (use_tc(h))
      launch_eval_tc(ts, h->num_sms, h->d_status, s, h->tile);
    else
      launch_eval_plain(ts, s);
    CK(cudaEventRecord(h->prof_ev[3], s));
    if (use_fp64(h))
      launch_select(ts, s);
    else
      launch_reduce_select(ts, s);
    CK(cudaEventRecord(h->prof_ev[4], s));
    CK(cudaEventRecord(h->prof_ev[5], s));
    CK(cudaGetLastError());
    CK(cudaEventSynchronize(h->prof_ev[5]));
    for (int k = 0; k < 5; ++k) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, h->prof_ev[k], h->prof_ev[k + 1]));
      stage_ms[k] += ms;
    }
    float all = 0.f;
    CK(cudaEventElapsedTime(&all, h->prof_ev[0], h->prof_ev[5]));
    stage_ms[5] += all;
    h->ga_evals += B;
  }
  return USAPHMP_OK;
}

namespace {
// Host layout of a saved GA state: this header, then anc [R][nw] u32,
// anc_fit [R] f32, best [nw] u32, best_fit f32, padded to 8 bytes.
struct GaStateHeader {
  uint32_t magic;  // "USGA"
  uint32_t version;
  int32_t n, p, nw, R, P, n1, elitist, island_offset;
  uint64_t seed;
  int32_t gen;
  int32_t reserved;
  int64_t evals;
};
constexpr uint32_t kGaStateMagic = 0x41475355u;
constexpr uint32_t kGaStateVersion = 1;

int64_t ga_state_bytes(const usaphmp_s* h) {
  const int64_t R = h->prm.islands, nw = h->nw;
  const int64_t b = (int64_t)sizeof(GaStateHeader) + 4 * (R * nw + R + nw + 1);
  return (b + 7) / 8 * 8;
}
}  // namespace

int usaphmp_debug_fail_allocations(int32_t after) {
  g_fail_after.store(after < 0 ? -1 : after);
  return USAPHMP_OK;
}

int usaphmp_selftest_wait_timeout(int64_t limit_ns, uint32_t* status, int64_t* elapsed_ns) {
  if (!status || !elapsed_ns) return fail(USAPHMP_EINVAL, "NULL argument");
  if (limit_ns < 1000 || limit_ns > 10000000000ll) return fail(USAPHMP_EINVAL, "limit_ns must be in [1e3, 1e10]");
  unsigned long long el = 0;
  const int rc = selftest_wait_timeout((uint64_t)limit_ns, status, &el);
  if (rc != USAPHMP_OK) return rc;
  *elapsed_ns = (int64_t)el;
  if (*status & 0x80000000u) return fail(USAPHMP_ECUDA, "wait self-test: a wait on an incomplete barrier succeeded");
  if (!(*status & kStatusTimeout)) return fail(USAPHMP_ECUDA, "wait self-test: the waits did not time out");
  return fail(USAPHMP_ETIMEOUT, "wait self-test: the bounded waits gave up as expected");
}

int usaphmp_ga_state_bytes(usaphmp_t h, int64_t* bytes) {
  if (!h || !bytes) return fail(USAPHMP_EINVAL, "NULL argument");
  *bytes = ga_state_bytes(h);
  return USAPHMP_OK;
}

int usaphmp_ga_save(usaphmp_t h, void* buf, int64_t bytes, void* stream) {
  if (!h || !buf) return fail(USAPHMP_EINVAL, "NULL argument");
  if (!h->ga_ready) return fail(USAPHMP_EINVAL, "usaphmp_ga_begin first");
  if (bytes != ga_state_bytes(h)) return fail(USAPHMP_EINVAL, "usaphmp_ga_save: buffer size differs from usaphmp_ga_state_bytes");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Task& t = h->ga_task;
  GaStateHeader hd{};
  hd.magic = kGaStateMagic;
  hd.version = kGaStateVersion;
  hd.n = h->n; hd.p = h->p; hd.nw = h->nw;
  hd.R = t.ga.R; hd.P = t.ga.P; hd.n1 = t.ga.N1; hd.elitist = t.ga.elitist; hd.island_offset = t.ga.island_offset;
  hd.seed = t.ga.seed;
  hd.evals = h->ga_evals;
  char* out = static_cast<char*>(buf);
  std::memset(out, 0, (size_t)bytes);
  uint32_t* anc = reinterpret_cast<uint32_t*>(out + sizeof(GaStateHeader));
  float* anc_fit = reinterpret_cast<float*>(anc + (size_t)hd.R * hd.nw);
  uint32_t* best = reinterpret_cast<uint32_t*>(anc_fit + hd.R);
  float* best_fit = reinterpret_cast<float*>(best + hd.nw);
  CK(cudaMemcpyAsync(anc, h->anc, sizeof(uint32_t) * hd.R * hd.nw, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(anc_fit, h->anc_fit, sizeof(float) * hd.R, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(best, h->best, sizeof(uint32_t) * hd.nw, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(best_fit, h->best_fit, sizeof(float), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&hd.gen, h->gen, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::memcpy(out, &hd, sizeof(hd));
  return USAPHMP_OK;
}

int usaphmp_ga_load(usaphmp_t h, const void* buf, int64_t bytes, void* stream) {
  if (!h || !buf) return fail(USAPHMP_EINVAL, "NULL argument");
  if (bytes != ga_state_bytes(h)) return fail(USAPHMP_EINVAL, "usaphmp_ga_load: buffer size differs from usaphmp_ga_state_bytes");
  GaStateHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  if (hd.magic != kGaStateMagic || hd.version != kGaStateVersion)
    return fail(USAPHMP_EINVAL, "usaphmp_ga_load: not a saved GA state of this layout version");
  if (hd.n != h->n || hd.p != h->p || hd.nw != h->nw || hd.R != h->prm.islands || hd.P != h->prm.island_size ||
      hd.n1 != h->prm.n1 || hd.elitist != h->prm.elitist || hd.island_offset != h->prm.island_offset)
    return fail(USAPHMP_EINVAL, "usaphmp_ga_load: the state was saved with another instance size or GA parameters");
  if (hd.gen < 0) return fail(USAPHMP_EINVAL, "usaphmp_ga_load: negative generation");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  RET(ensure_ga(h));
  drop_graph(h);
  const char* in = static_cast<const char*>(buf);
  const uint32_t* anc = reinterpret_cast<const uint32_t*>(in + sizeof(GaStateHeader));
  const float* anc_fit = reinterpret_cast<const float*>(anc + (size_t)hd.R * hd.nw);
  const uint32_t* best = reinterpret_cast<const uint32_t*>(anc_fit + hd.R);
  const float* best_fit = reinterpret_cast<const float*>(best + hd.nw);
  CK(cudaMemcpyAsync(h->anc, anc, sizeof(uint32_t) * hd.R * hd.nw, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->anc_fit, anc_fit, sizeof(float) * hd.R, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->best, best, sizeof(uint32_t) * hd.nw, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->best_fit, best_fit, sizeof(float), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->gen, &hd.gen, sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(h->done, 0, sizeof(int), s));
  CK(cudaStreamSynchronize(s));
  RET(reset_status(h, s));
  h->ga_task = ga_task_of(h, hd.seed);
  h->ga_evals = hd.evals;
  h->ga_ready = true;
  return USAPHMP_OK;
}

int usaphmp_ga_islands(usaphmp_t h, uint32_t* masks, float* fit, void* stream) {
  if (!h) return fail(USAPHMP_EINVAL, "NULL handle");
  if (!h->ga_ready) return fail(USAPHMP_EINVAL, "usaphmp_ga_begin first");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int R = h->ga_task.ga.R;
  if (masks) CK(cudaMemcpyAsync(masks, h->anc, sizeof(uint32_t) * R * h->nw, cudaMemcpyDeviceToHost, s));
  if (fit) CK(cudaMemcpyAsync(fit, h->anc_fit, sizeof(float) * R, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return USAPHMP_OK;
}

int usaphmp_ga_population(usaphmp_t h, uint32_t* masks, float* fit, void* stream) {
  if (!h) return fail(USAPHMP_EINVAL, "NULL handle");
  if (!h->ga_ready) return fail(USAPHMP_EINVAL, "usaphmp_ga_begin first");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Task& t = h->ga_task;
  const size_t B = (size_t)t.ga.R * t.ga.P;
  if (masks) CK(cudaMemcpyAsync(masks, t.pop.mask, sizeof(uint32_t) * B * h->nw, cudaMemcpyDeviceToHost, s));
  if (fit) CK(cudaMemcpyAsync(fit, t.pop.fit, sizeof(float) * B, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return USAPHMP_OK;
}

int usaphmp_ga_merge(usaphmp_t h, const uint32_t* mask, float fit, void* stream) {
  if (!h || !mask) return fail(USAPHMP_EINVAL, "NULL argument");
  if (!h->ga_ready) return fail(USAPHMP_EINVAL, "usaphmp_ga_begin first");
  int bits = 0;
  for (int x = 0; x < h->nw; ++x) {
    uint32_t v = mask[x];
    if (x == h->nw - 1 && (h->n & 31)) {
      if (v >> (h->n & 31)) return fail(USAPHMP_EINVAL, "usaphmp_ga_merge: mask has bits at nodes >= n");
    }
    bits += __builtin_popcount(v);
  }
  if (bits != h->p) return fail(USAPHMP_EINVAL, "usaphmp_ga_merge: mask does not hold p hubs");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaMemcpyAsync(h->mask0, mask, sizeof(uint32_t) * h->nw, cudaMemcpyHostToDevice, s));
  launch_set_ancestors(h->anc, h->anc_fit, h->ga_task.ga.R, h->nw, h->mask0, fit, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return USAPHMP_OK;
}

int usaphmp_ga_result(usaphmp_t h, usaphmp_result* best, void* stream) {
  const NvtxRange nvtx_range("usaphmp_ga_result");
  if (!h || !best) return fail(USAPHMP_EINVAL, "NULL argument");
  if (!h->ga_ready) return fail(USAPHMP_EINVAL, "usaphmp_ga_begin first");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<uint32_t> m(h->nw);
  float bf = 0.f;
  CK(cudaMemcpyAsync(m.data(), h->best, sizeof(uint32_t) * h->nw, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&bf, h->best_fit, sizeof(float), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  RET(check_status(h, s, "usaphmp_ga"));
  std::vector<int32_t> hubs = mask_to_hubs(m, h->n);
  if ((int)hubs.size() != h->p) return fail(USAPHMP_ECUDA, "internal: best mask does not hold p hubs");
  CK(cudaMemcpyAsync(h->one.hubs, hubs.data(), sizeof(int32_t) * h->p, cudaMemcpyHostToDevice, s));
  const Task t1 = make_task(h, popbuf(h, h->one, 1));
  TaskSet ts{nullptr, &t1, 1};
  launch_alloc(ts, true, false, s);
  CK(cudaGetLastError());
  if (h->prm.local_search > 0) {
    // improve the nearest allocation of the best hubs, then take the fast
    // path's fitness of the improved solution
    RET(ensure_ls(h, s));
    launch_local_search(inst_of(h), h->d_WT, h->d_OD64, 1, h->one.hubs, h->one.slot, h->prm.local_search, h->d_ls,
                        h->d_ls_count, h->d_ls_count + 1, s);
    CK(cudaGetLastError());
    PopBuf pb = popbuf(h, h->one, 1);
    pb.slot_in = h->one.slot;
    RET(run_eval(h, make_task(h, pb), false, s));
    CK(cudaMemcpyAsync(&bf, h->one.fit, sizeof(float), cudaMemcpyDeviceToHost, s));
  }
  launch_rescore(inst_of(h), 1, h->one.hubs, h->one.slot, h->d_rpart, h->d_cost, s, h->d_dist64,
                 output_scale(h));
  CK(cudaGetLastError());
  std::vector<uint8_t> sl(h->ns);
  double cost = 0;
  CK(cudaMemcpyAsync(sl.data(), h->one.slot, h->ns, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&cost, h->d_cost, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (best->hubs) std::memcpy(best->hubs, hubs.data(), sizeof(int32_t) * h->p);
  if (best->S)
    for (int i = 0; i < h->n; ++i) best->S[i] = hubs[sl[i]];
  best->cost_fp64 = cost;
  best->cost_fp32 = (float)(bf * output_scale(h));
  best->evals = h->ga_evals;
  return USAPHMP_OK;
}

int usaphmp_solve(usaphmp_t h, int32_t generations, uint64_t seed, usaphmp_result* best) {
  const NvtxRange nvtx_range("usaphmp_solve");
  if (!h || !best) return fail(USAPHMP_EINVAL, "NULL argument");
  if (generations < 0) return fail(USAPHMP_EINVAL, "generations < 0");
  const auto t0 = std::chrono::steady_clock::now();
  RET(usaphmp_ga_begin(h, seed, h->stream));
  RET(usaphmp_ga_run(h, generations, h->stream));
  RET(usaphmp_ga_result(h, best, h->stream));
  best->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return USAPHMP_OK;
}

}  // extern "C"
