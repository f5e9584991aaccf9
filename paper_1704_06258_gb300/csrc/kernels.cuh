// Host-side launchers of the library's kernels (all stream-ordered, no sync).
#pragma once
#include <utility>
#include <nvtx3/nvToolsExt.h>
#include <string>

#include "common.cuh"

namespace usaphmp {

constexpr int kMaxTasks = 64;

// Launch with programmatic stream serialisation (see pdl_wait in common.cuh).
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// launch_pdl with clusters of `cluster` consecutive blocks (grid a multiple).
template <class... KArgs, class... Args>
inline void launch_pdl_cluster(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                               int cluster, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = (unsigned)cluster;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Block ranges of the tasks of one launch: task t owns global blocks
// [o[t], o[t+1]).  Passed by value so that a captured graph keeps it.
struct BlockOffsets {
  int ntasks;
  int o[kMaxTasks + 1];
};

__device__ inline int task_of(const BlockOffsets& bo, int blk) {
  int t = 0;
  while (t + 1 < bo.ntasks && bo.o[t + 1] <= blk) ++t;
  return t;
}

// The tasks of one launch as the host sees them: `h` (host array, read by
// launchers for sizes) and, for several tasks, the same array in device
// memory `d`.  A single task with d == nullptr travels by value in the
// kernel parameters, so nothing has to stay alive in device memory for it.
struct TaskSet {
  const Task* d;
  const Task* h;
  int count;
};

// What kernels receive (as a __grid_constant__ parameter).
struct TaskParam {
  Task one;
  const Task* many;
  BlockOffsets bo;
};

__device__ __forceinline__ const Task& task_at(const TaskParam& tp, int t) {
  return tp.many ? tp.many[t] : tp.one;
}

inline TaskParam make_param(const TaskSet& ts) {
  TaskParam tp;
  tp.one = ts.h[0];
  tp.many = (ts.count == 1 && ts.d == nullptr) ? nullptr : ts.d;
  tp.bo.ntasks = ts.count;
  tp.bo.o[0] = 0;
  return tp;
}

// NVTX range over a scope of host code (names the library's calls in a
// profiler's timeline; costs a branch when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// setup.cu
void launch_check_values(const float* W, const float* C, int n, int ldw, uint32_t* status, cudaStream_t s);
void launch_split_bf16(const float* W, __nv_bfloat16* Whi, __nv_bfloat16* Wlo, long long total, cudaStream_t s);
void launch_split_bf16_upper(const float* W, __nv_bfloat16* Uhi, __nv_bfloat16* Ulo, float* Uf, int n, int ldw,
                             cudaStream_t s);
void launch_flows(const float* W, int n, int ldw, float* O, float* D, cudaStream_t s);
// *out = sum of all W entries in fp64 (rows: n doubles of scratch).
void launch_total_flow(const float* W, int n, int ldw, double* rows, double* out, cudaStream_t s);
void launch_asymmetry(const float* C, int n, int ldw, uint32_t* flag, cudaStream_t s);
void launch_transpose(const float* C, float* CT, int n, int ldw, cudaStream_t s);
void launch_middle_nodes(const float* C, int n, int ldw, int p, double* dscratch, uint32_t* mask,
                         int32_t* hubs, cudaStream_t s);

// canon.cu: validates (hubs, S) in node ids and writes ascending hubs + slots.
void launch_canon(const int32_t* hubs_in, const int32_t* S, int B, int n, int p, int ns,
                  int32_t* hubs_out, uint8_t* slot, uint32_t* status, int* bad_index, cudaStream_t s,
                  int index_base = 0);

// alloc.cu: nearest allocation (or the given slots), access terms t12 and
// (with_chub) the hub-to-hub cost table chub.
void launch_alloc(const TaskSet& ts, bool nearest, bool with_chub, cudaStream_t s);
// Canonical form of chromosomes given as hub ids + S (validation, sorted hubs,
// slot codes) fused with the given-slot allocation terms and hub-cost tables;
// direct hub arcs only (returns false for hub-path routing, launching nothing).
bool launch_canon_alloc(const Task& task, const int32_t* hubs_in, const int32_t* S, int* bad_index, int index_base,
                        bool with_chub, cudaStream_t s);

// eval_plain.cu: fp32 CUDA-core transfer sums into pop.part[r][b]; the
// number of partial rows per task is plain_rows(n, B).
int plain_rows(int n, int B);
void launch_eval_plain(const TaskSet& ts, cudaStream_t s);
// Raises the dynamic shared-memory limit of the plain kernels (once, outside
// any stream capture).
void prepare_eval_plain(int max_smem);

// eval_tc.cu: split-bf16 tcgen05 transfer sums into pop.part[r][b] with r
// the 32-row group of W (tc_part_rows(n) = 4*ceil(n/128) rows).
// Tile shape of a launch: MMA width ntile (64, 128 or 256 columns; a tile
// holds floor(ntile/p) chromosomes), shared-memory stages (2..4) and the
// raster order of the persistent tile loop (0: column tiles of a row block
// first, 1: row blocks of a column tile first) and the CTA-pair mode (1: a
// cluster of two CTAs runs each M = 256 MMA over two row blocks, each CTA
// holding its row block of U and half of the one-hot columns).  The results
// do not depend on it.
struct TcTile {
  int ntile = 256;
  int stages = 3;
  int raster = 0;
  int pair = 0;
};
// true when the shape's layout fits shared memory and p <= ntile
bool tc_tile_fits(const TcTile& t, int p);
size_t tc_slab_bytes(const TcTile& t);
void launch_eval_tc(const TaskSet& ts, int num_sms, uint32_t* status, cudaStream_t s,
                    const TcTile& tile = TcTile{});
int tc_part_rows(int n);
// Clusters of two CTAs the pair-mode evaluator can run at once on the current
// device (0 before prepare_eval_tc, or when none fits).
int tc_pair_slots();
// Runs k_wait_selftest (see eval_tc.cu); 0 or a USAPHMP_E* code.
int selftest_wait_timeout(uint64_t limit_ns, uint32_t* status, unsigned long long* elapsed_ns);
void prepare_eval_tc();

// reduce.cu: fit[b] = t12[b] + alpha * (sum of partials, fixed order).
void launch_reduce(const TaskSet& ts, cudaStream_t s);

// ga.cu: offspring (exchange, crossover, mutation, correction) and selection.
void launch_children(const TaskSet& ts, cudaStream_t s);
void launch_set_ancestors(uint32_t* anc, float* anc_fit, int R, int nw, const uint32_t* mask, float fit,
                          cudaStream_t s);
void launch_select(const TaskSet& ts, cudaStream_t s);
// ga.cu: fitness reduction fused with selection (GA generations only).
void launch_reduce_select(const TaskSet& ts, cudaStream_t s);

// Start state of a single-task GA: ancestors and best-ever = mask0, fit0.
void launch_ga_init(const Task& task, const uint32_t* mask0, const float* fit0, cudaStream_t s);

// rescore.cu: fp64 pair-form objective of B chromosomes of one instance.
// With in.routing != 0, `dist` (B*p*p doubles of scratch) receives the
// chromosomes' fp64 hub-path tables first; callers must pass it then.
void launch_rescore(const DevInst& in, int B, const int32_t* hubs, const uint8_t* slot,
                    double* part, double* cost, cudaStream_t s, double* dist = nullptr, double scale = 1.0);
int rescore_parts(int n);
// fit[b] = (float)cost[b] * scale (the fitness of the fp64 reference path).
void launch_fit_from_fp64(const double* cost, float* fit, int B, float scale, cudaStream_t s);

// local_search.cu: fp64 single-reallocation sweeps for fixed hubs (slots in
// place); scratch holds local_search_scratch_doubles(n, p) per chromosome.
// WT = W transposed and OD = [O_i; D_i] in fp64 (2n doubles), made once per
// instance by launch_ls_prepare.
size_t local_search_scratch_doubles(int n, int p);
void launch_ls_prepare(const float* W, int n, int ldw, float* WT, double* OD, cudaStream_t s);
void launch_local_search(const DevInst& in, const float* WT, const double* OD, int B, const int32_t* hubs,
                         uint8_t* slot, int max_sweeps, double* scratch, int32_t* moves, int32_t* sweeps,
                         cudaStream_t s);

// capi.cu: records the calling thread's last error message; returns `code`.
int report_error(int code, const std::string& msg);

}  // namespace usaphmp

// capi.cu: what the serving loop needs from a handle (after usaphmp_ga_begin).
struct usaphmp_s;
namespace usaphmp {
const Task& handle_ga_task(const usaphmp_s* h);
// A handle whose device memory comes from `pool` by stream-ordered
// allocations on its own stream (handle_stream), so that making and
// destroying it never synchronises the device (the serving loop's handles).
int create_pooled(int32_t n, int32_t p, const float* W, const float* C, double chi, double alpha, double delta,
                  cudaMemPool_t pool, usaphmp_s** out);
cudaStream_t handle_stream(const usaphmp_s* h);
bool handle_uses_tc(const usaphmp_s* h);
void handle_note_generations(usaphmp_s* h, int generations);
// Device bytes a handle holds for an instance of n nodes and p hubs running
// the GA with population B = R * P (upper bound: counts a transposed C).
size_t handle_device_bytes(int n, int p, int R, int P);

}  // namespace usaphmp
