// Shared device-side definitions of the USApHMP library (sm_103a).
//
// Layouts (row-major throughout):
//   W, C          fp32  [n][ldw]   ldw = n rounded up to 8, zero padding
//   CT            fp32  [n][ldw]   C transposed (aliases C when C is symmetric)
//   Whi, Wlo      bf16  [n][ldw]   W = Whi + Wlo + O(2^-17 |W|); for symmetric C
//                                  the same split of U = W + W^T folded onto j >= i
//   O, D          fp32  [ns]       originating / destined flow (§3), zero past n
//   mask          u32   [B][nw]    hub mask H of §4.1, bit i%32 of word i/32
//   hubs          i32   [B][p]     open hubs in ascending node order
//   slot          u8    [B][ns]    rank in `hubs` of the hub serving node i;
//                                  ns = n rounded up to 64, padding = 0xFF
//   chub          fp32  [B][cstride]  hub-to-hub costs of chromosome b:
//                 chub[b][k * hstride + l] = C[hubs_b[k], hubs_b[l]], rows of
//                 hstride = p | 1 floats (odd, so that 32 different rows fall
//                 on 32 different shared-memory banks); cstride = p * hstride
//                 rounded up to 4 (16-byte aligned tables for bulk copies)
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace usaphmp {

constexpr int kMaxN = 16384;
constexpr int kMaxP = 255;
constexpr uint8_t kSlotPad = 0xFF;

// Bits of the device status word (errors raised inside kernels).
enum : uint32_t {
  kStatusBadChromosome = 1u,
  kStatusTimeout = 2u,
  kStatusBadValue = 4u,
};

__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// One node's access terms chi*O_i*C[i,h(i)] + delta*D_i*C[h(i),i], written
// with explicit roundings so that every kernel computes the same bits.
__device__ __forceinline__ float access_term(float chi, float Oi, float cih, float delta, float Di, float chi_i) {
  return __fmaf_rn(__fmul_rn(delta, Di), chi_i, __fmul_rn(__fmul_rn(chi, Oi), cih));
}
// A chromosome's p x p hub-cost table (chub): row k at k * hstride floats.
// The odd row stride puts 32 different rows on 32 different shared-memory
// banks, so a warp whose lanes read one column of rows s(lane) never
// conflicts; tables start 16 bytes apart (whole bulk copies).
__host__ __device__ inline int chub_hstride(int p) { return p | 1; }
__host__ __device__ inline int chub_cstride(int p) { return round_up(p * chub_hstride(p), 4); }

// The plain evaluator keeps one p x p hub-cost table and the slot codes of a
// chromosome in shared memory; past this budget (p above about 220) it reads
// the chromosome's chub rows from global memory instead, and the allocation
// kernel writes them for every path.
constexpr size_t kPlainSmemBudget = 200 * 1024;
__host__ __device__ inline bool plain_global_table(int p, int ns) {
  return (size_t)round_up(p * p * 4, 16) + (size_t)ns > kPlainSmemBudget;
}

// Immutable per-instance device data.
struct DevInst {
  int n, p, ldw, ns, nw, symmetric;
  int routing;  // 0: direct hub arc, 1: shortest paths over open-hub arcs
  float chi, alpha, delta;                // for the fp32 and split-bf16 paths
  double chi_d, alpha_d, delta_d;         // as given, for the fp64 rescoring
  const float* W;
  const float* C;
  const float* CT;
  const float* O;
  const float* D;
  const __nv_bfloat16* Whi;
  const __nv_bfloat16* Wlo;
  // 1: Whi/Wlo hold the split of U (W + W^T folded above the diagonal, W_ii
  // on it, 0 below), valid when every hub-to-hub table is symmetric; the
  // tensor-core evaluator then skips the K blocks left of the diagonal.
  int wtri;
  const float* Ufold;  // the same U in fp32 [n][ldw] (symmetric C), else nullptr
};

// A population of B chromosomes and its evaluation buffers.
struct PopBuf {
  int B;
  uint32_t* mask;
  int32_t* hubs;
  uint8_t* slot;
  // Optional caller-supplied inputs of the allocation kernel; when set they
  // are range-checked and copied into `hubs` / `slot` (out-of-range entries
  // raise kStatusBadChromosome and are replaced by 0).
  const int32_t* hubs_in;
  const uint8_t* slot_in;
  float* t12;      // access terms chi*O*C + delta*D*C per chromosome
  float* chub;
  float* part;     // partial transfer sums (layout set by the evaluator)
  int npart;       // number of partial rows: part[r][b], r < npart
  float* fit;      // fp32 fitness
  uint32_t* status;  // device status word (kStatus* bits)
  float out_scale;   // factor k_reduce applies to the fitness it writes (1: raw cost)
  // Optional pinned host words k_reduce fills after the evaluation: [0] the
  // status word, [1] the index of the first invalid chromosome (`bad`), so a
  // host call reads them without copies of its own.
  uint32_t* status_host;
  const int* bad;
};

// Island GA state (§5): R islands of P chromosomes.
struct GaState {
  int R, P, N1, elitist;  // N1 = 0: no merge (the caller merges islands across GPUs)
  int island_offset;      // global index of island 0 (random streams of a shard)
  unsigned long long seed;
  int* gen;            // device generation counter
  uint32_t* anc;       // [R][nw]
  float* anc_fit;      // [R]
  uint32_t* best;      // [nw]
  float* best_fit;     // [1]
  int* done;           // blocks finished in the fused selection (self-resetting)
};

struct Task {
  DevInst in;
  PopBuf pop;
  GaState ga;
  const void* tmap_hi;  // CUtensorMap in device memory (split path)
  const void* tmap_lo;
};

// Finds the task owning global block `blk` given per-task block offsets
// (off[0] = 0, off[t+1] = off[t] + blocks of task t).
__device__ inline int find_task(const int* off, int ntasks, int blk) {
  int t = 0;
  while (t + 1 < ntasks && off[t + 1] <= blk) ++t;
  return t;
}

// Programmatic dependent launch: a kernel launched with launch_pdl may start
// while the previous kernel of its stream is finishing; pdl_wait() returns
// once that kernel has completed and its writes are visible (at once when
// the launch has no such dependency), so every kernel calls it before its
// first global access.  pdl_allow_next() lets the next kernel launch once
// every block of this one has started.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_allow_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ inline float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum_{r < rows} x[r * stride], added in ascending r (the fixed order every
// evaluator's partial sums are reduced in), loads issued 32 at a time.
__device__ __forceinline__ float sum_rows_in_order(const float* __restrict__ x, int rows, long long stride) {
  float s = 0.f;
  int r = 0;
  for (; r + 32 <= rows; r += 32) {
    float v[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) v[u] = x[(long long)(r + u) * stride];
#pragma unroll
    for (int u = 0; u < 32; ++u) s += v[u];
  }
  for (; r + 16 <= rows; r += 16) {
    float v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) v[u] = x[(long long)(r + u) * stride];
#pragma unroll
    for (int u = 0; u < 16; ++u) s += v[u];
  }
  for (; r + 8 <= rows; r += 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = x[(long long)(r + u) * stride];
#pragma unroll
    for (int u = 0; u < 8; ++u) s += v[u];
  }
  for (; r < rows; ++r) s += x[(long long)r * stride];
  return s;
}

// Block-wide sum in a fixed order (warp butterflies, then warps in order).
// `red` holds at least blockDim.x/32 floats. Result valid in every thread.
__device__ inline float block_sum(float v, float* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  float s = 0.f;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

__device__ inline double block_sum_f64(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

}  // namespace usaphmp
