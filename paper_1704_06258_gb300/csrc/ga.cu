// Device GA step of the island model of §5 on n-bit hub masks.
//
// Offspring of island r, generation g (one block of two warps per pair of
// members 2m, 2m+1; warp w builds member q = 2m + w):
//   1. parent_q = the island's ancestor after one hub <-> spoke exchange
//      (the move that duplicates the ancestor into a population, §4.1);
//   2. single-point crossover of the pair (§4.2): one cut c in [1, n-1]
//      drawn for the pair; child_q keeps bits [0, c) of parent_q and takes
//      [c, n) from its partner;
//   3. mutation: one more hub <-> spoke exchange (§4.2);
//   4. correction back to exactly p hubs (§4.2): close the k-th open node or
//      open the k-th closed node, k drawn uniformly, until p are open.
// "k-th" counts in ascending node order.  Every draw comes from a
// Philox4x32-10 stream keyed by the seed and addressed by (g, q, operator);
// a value below m is the high word of (32-bit draw) * m.
//
// Selection (§5): each island's ancestor becomes its best child (lowest
// member index on ties, or kept when the elitist flag is set and the child
// is not strictly better); the best-ever solution changes only on a strict
// improvement (islands in ascending order); every N1 generations all
// ancestors are replaced by the best island's ancestor (lowest island on
// ties), and the generation counter advances.
#include "common.cuh"
#include "kernels.cuh"

#include <algorithm>

namespace usaphmp {

namespace {

enum : uint32_t { kOpExchange = 0, kOpCrossover = 1, kOpCorrection = 2, kOpMutation = 3 };

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// The Philox blocks a warp's operators draw from, computed at once, one per
// lane (lane 0: exchange block 0; 1: the pair's crossover block 0; 2:
// mutation block 0; 3..31: correction blocks 0..28).  A stream's later
// blocks, beyond the table, are computed when needed.
constexpr int kTableCorrection = 29;
__device__ __forceinline__ int table_lane(uint32_t op, uint32_t d) {
  if (op == kOpExchange) return d == 0 ? 0 : -1;
  if (op == kOpCrossover) return d == 0 ? 1 : -1;
  if (op == kOpMutation) return d == 0 ? 2 : -1;
  return d < (uint32_t)kTableCorrection ? 3 + (int)d : -1;
}

__device__ __forceinline__ uint32_t word_of(const uint4& b, int i) {
  return i == 0 ? b.x : i == 1 ? b.y : i == 2 ? b.z : b.w;
}

// One operator's stream of 32-bit draws (warp-uniform calls): words of block
// d = 0, 1, ... in order, taken from the warp's table while it holds them.
struct Draws {
  uint4 ctr;
  uint2 key;
  uint4 buf;
  int used;
  int src;               // lane holding the current block, -1: computed into buf
  const uint4* table;    // this lane's table block
  __device__ Draws(unsigned long long seed, uint32_t g, uint32_t q, uint32_t op, const uint4* mine)
      : ctr(make_uint4(g, q, op, 0u)), key(make_uint2((uint32_t)seed, (uint32_t)(seed >> 32))), used(4), src(-1),
        table(mine) {}
  __device__ uint32_t word() {
    if (used == 4) {
      src = table_lane(ctr.z, ctr.w);
      if (src < 0) buf = philox4x32_10(ctr, key);
      ctr.w += 1u;
      used = 0;
    }
    const uint32_t w = src >= 0 ? __shfl_sync(0xffffffffu, word_of(*table, used), src) : word_of(buf, used);
    ++used;
    return w;
  }
  __device__ uint32_t below(uint32_t m) { return __umulhi(word(), m); }
};

__device__ __forceinline__ uint32_t closed_word(uint32_t w, int x, int nw, int n) {
  w = ~w;
  if (x == nw - 1 && (n & 31)) w &= (1u << (n & 31)) - 1u;
  return w;
}

__device__ int popcount_mask(const uint32_t* mw, int nw) {
  int c = 0;
  for (int x = threadIdx.x & 31; x < nw; x += 32) c += __popc(mw[x]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  return c;
}

// Node id of the k-th open (closed = false) or closed node; warp-uniform.
__device__ int kth_node(const uint32_t* mw, int nw, int n, uint32_t k, bool closed) {
  const int lane = threadIdx.x & 31;
  uint32_t base = 0;
  for (int c0 = 0; c0 < nw; c0 += 32) {
    const int x = c0 + lane;
    uint32_t w = 0;
    if (x < nw) w = closed ? closed_word(mw[x], x, nw, n) : mw[x];
    const uint32_t cnt = __popc(w);
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (k < base + total) {
      const uint32_t ball = __ballot_sync(0xffffffffu, base + incl > k);
      const int L = __ffs(ball) - 1;
      const uint32_t ww = __shfl_sync(0xffffffffu, w, L);
      const uint32_t before = __shfl_sync(0xffffffffu, incl - cnt, L);
      // the (k - base - before)-th set bit of ww: lane b holds bit b and
      // counts the set bits below it
      const uint32_t kk = k - base - before;
      const bool hit = ((ww >> lane) & 1u) && (uint32_t)__popc(ww & ((1u << lane) - 1u)) == kk;
      return (c0 + L) * 32 + (__ffs(__ballot_sync(0xffffffffu, hit)) - 1);
    }
    base += total;
  }
  return -1;
}

__device__ void flip(uint32_t* mw, int node) {
  if ((threadIdx.x & 31) == 0 && node >= 0) mw[node >> 5] ^= 1u << (node & 31);
  __syncwarp();
}

// One hub <-> spoke exchange; two draws are taken whatever the mask.
__device__ void exchange(uint32_t* mw, int nw, int n, Draws& d) {
  const int h = popcount_mask(mw, nw);
  const uint32_t i = d.below((uint32_t)h);
  const uint32_t j = d.below((uint32_t)(n - h));
  if (h > 0 && h < n) {
    const int a = kth_node(mw, nw, n, i, false);
    const int b = kth_node(mw, nw, n, j, true);
    flip(mw, a);
    flip(mw, b);
  }
}

__device__ void correct(uint32_t* mw, int nw, int n, int p, Draws& d) {
  int h = popcount_mask(mw, nw);
  while (h > p) {
    flip(mw, kth_node(mw, nw, n, d.below((uint32_t)h), false));
    --h;
  }
  while (h < p) {
    flip(mw, kth_node(mw, nw, n, d.below((uint32_t)(n - h)), true));
    ++h;
  }
}

}  // namespace

__global__ void __launch_bounds__(64) k_children(const __grid_constant__ TaskParam tp) {
  extern __shared__ uint32_t msm[];
  pdl_wait();
  pdl_allow_next();
  const int t = task_of(tp.bo, blockIdx.x);
  const Task& T = task_at(tp, t);
  const int n = T.in.n, p = T.in.p, nw = T.in.nw;
  const int P = T.ga.P;
  const unsigned long long seed = T.ga.seed;
  const uint32_t g = (uint32_t)*T.ga.gen;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q0 = 2 * (blockIdx.x - tp.bo.o[t]);
  const int q = q0 + w;
  const int r = q / P;
  // random streams are addressed by the global chromosome index
  const uint32_t goff = (uint32_t)T.ga.island_offset * (uint32_t)P;
  uint32_t* par = msm + w * nw;
  uint32_t* oth = msm + (1 - w) * nw;
  uint32_t* ch = msm + (2 + w) * nw;
  // the warp's Philox table (see table_lane), all blocks computed side by side
  uint4 mine;
  {
    const uint32_t op = lane == 0 ? kOpExchange : lane == 1 ? kOpCrossover : lane == 2 ? kOpMutation : kOpCorrection;
    const uint32_t qq = goff + (uint32_t)(lane == 1 ? q0 : q);
    const uint32_t d = lane < 3 ? 0u : (uint32_t)(lane - 3);
    mine = philox4x32_10(make_uint4(g, qq, op, d), make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  }

  for (int x = lane; x < nw; x += 32) {
    uint32_t v = T.ga.anc[(long long)r * nw + x];
    if (x == nw - 1 && (n & 31)) v &= (1u << (n & 31)) - 1u;  // nodes >= n are never hubs
    par[x] = v;
  }
  __syncwarp();
  {
    Draws d(seed, g, goff + (uint32_t)q, kOpExchange, &mine);
    exchange(par, nw, n, d);
  }
  __syncthreads();
  {
    Draws d(seed, g, goff + (uint32_t)q0, kOpCrossover, &mine);
    const int c = 1 + (int)d.below((uint32_t)(n - 1));
    for (int x = lane; x < nw; x += 32) {
      const uint32_t own = par[x], other = oth[x];
      const int lo = x * 32;
      uint32_t v;
      if (lo + 32 <= c) v = own;
      else if (lo >= c) v = other;
      else {
        const uint32_t m = (1u << (c - lo)) - 1u;
        v = (own & m) | (other & ~m);
      }
      ch[x] = v;
    }
    __syncwarp();
  }
  {
    Draws d(seed, g, goff + (uint32_t)q, kOpMutation, &mine);
    exchange(ch, nw, n, d);
  }
  {
    Draws d(seed, g, goff + (uint32_t)q, kOpCorrection, &mine);
    correct(ch, nw, n, p, d);
  }
  uint32_t* out = T.pop.mask + (long long)q * nw;
  int32_t* hubs = T.pop.hubs + (long long)q * p;
  int base = 0;
  for (int c0 = 0; c0 < nw; c0 += 32) {
    const int x = c0 + lane;
    uint32_t v = (x < nw) ? ch[x] : 0u;
    if (x < nw) out[x] = v;
    const int cnt = __popc(v);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    int pos = base + incl - cnt;
    while (v) {
      hubs[pos++] = x * 32 + (__ffs(v) - 1);
      v &= v - 1u;
    }
    base += __shfl_sync(0xffffffffu, incl, 31);
  }
}

// Selection key: a NaN fitness ranks after every number (as +inf), so an
// argmin always lands on a member of the island.
__device__ __forceinline__ float rank_key(float x) { return isnan(x) ? INFINITY : x; }

// Per island: best child -> ancestor.
__global__ void k_select_islands(const __grid_constant__ TaskParam tp) {
  const int t = task_of(tp.bo, blockIdx.x);
  const Task& T = task_at(tp, t);
  const int r = blockIdx.x - tp.bo.o[t];
  const int P = T.ga.P, nw = T.in.nw, lane = threadIdx.x;
  const float* f = T.pop.fit + (long long)r * P;
  float v = INFINITY;
  int idx = 0x7fffffff;
  for (int j = lane; j < P; j += 32) {
    const float x = rank_key(f[j]);
    if (x < v || (x == v && j < idx)) { v = x; idx = j; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov < v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  if (T.ga.elitist && !(v < T.ga.anc_fit[r])) return;
  const uint32_t* src = T.pop.mask + (long long)(r * P + idx) * nw;
  uint32_t* dst = T.ga.anc + (long long)r * nw;
  for (int x = lane; x < nw; x += 32) dst[x] = src[x];
  if (lane == 0) T.ga.anc_fit[r] = v;
}

// Per task: best-ever update, merge every N1 generations, generation += 1.
__global__ void k_select_global(const __grid_constant__ TaskParam tp) {
  __shared__ float sv[32];
  __shared__ int si[32];
  __shared__ int s_rb;
  const Task& T = task_at(tp, blockIdx.x);
  const int R = T.ga.R, nw = T.in.nw;
  float v = INFINITY;
  int idx = 0x7fffffff;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    const float x = rank_key(T.ga.anc_fit[r]);
    if (x < v || (x == v && r < idx)) { v = x; idx = r; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov < v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  if ((threadIdx.x & 31) == 0) { sv[threadIdx.x >> 5] = v; si[threadIdx.x >> 5] = idx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (sv[w] < v || (sv[w] == v && si[w] < idx)) { v = sv[w]; idx = si[w]; }
    s_rb = idx;
  }
  __syncthreads();
  const int rb = s_rb;
  const float fb = T.ga.anc_fit[rb];
  const uint32_t* src = T.ga.anc + (long long)rb * nw;
  const bool improve = fb < *T.ga.best_fit;
  __syncthreads();
  if (improve) {
    for (int x = threadIdx.x; x < nw; x += blockDim.x) T.ga.best[x] = src[x];
    if (threadIdx.x == 0) *T.ga.best_fit = fb;
  }
  const int g = *T.ga.gen;
  if (T.ga.N1 > 0 && (g + 1) % T.ga.N1 == 0) {
    for (long long e = threadIdx.x; e < (long long)R * nw; e += blockDim.x) {
      const int r = (int)(e / nw);
      if (r != rb) T.ga.anc[e] = src[e - (long long)r * nw];
    }
    for (int r = threadIdx.x; r < R; r += blockDim.x)
      if (r != rb) T.ga.anc_fit[r] = fb;
  }
  __syncthreads();
  if (threadIdx.x == 0) *T.ga.gen = g + 1;
}

// Fitness reduction fused with selection, one block per island: the block
// assembles its members' fitness (t12 + alpha * partials, fixed order),
// replaces the island ancestor, and the last island block of the task to
// finish (counted with an atomic after a fence) performs the best-ever
// update, the merge every N1 generations and the generation increment -- the
// same steps as k_reduce + k_select_islands + k_select_global.
__global__ void __launch_bounds__(128) k_reduce_select(const __grid_constant__ TaskParam tp) {
  __shared__ float sv[4];
  __shared__ int si[4];
  __shared__ int s_last, s_rb;
  pdl_wait();
  pdl_allow_next();
  const int t = task_of(tp.bo, blockIdx.x);
  const Task& T = task_at(tp, t);
  const int r = blockIdx.x - tp.bo.o[t];
  const int P = T.ga.P, R = T.ga.R, nw = T.in.nw, B = T.pop.B;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float v = INFINITY;
  int idx = 0x7fffffff;
  for (int j = threadIdx.x; j < P; j += blockDim.x) {
    const int q = r * P + j;
    const float s = sum_rows_in_order(T.pop.part + q, T.pop.npart, B);
    const float f = T.pop.t12[q] + T.in.alpha * s;
    T.pop.fit[q] = f;
    const float x = rank_key(f);
    if (x < v || (x == v && j < idx)) { v = x; idx = j; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov < v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  if (lane == 0) { sv[wid] = v; si[wid] = idx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (sv[w] < v || (sv[w] == v && si[w] < idx)) { v = sv[w]; idx = si[w]; }
    sv[0] = v;
    si[0] = idx;
  }
  __syncthreads();
  v = sv[0];
  idx = si[0];
  const bool take = !(T.ga.elitist && !(v < T.ga.anc_fit[r]));
  if (take) {
    const uint32_t* src = T.pop.mask + (long long)(r * P + idx) * nw;
    uint32_t* dst = T.ga.anc + (long long)r * nw;
    for (int x = threadIdx.x; x < nw; x += blockDim.x) dst[x] = src[x];
    if (threadIdx.x == 0) T.ga.anc_fit[r] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(T.ga.done, 1) == R - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // global step (this block saw every island's update)
  v = INFINITY;
  idx = 0x7fffffff;
  for (int rr = threadIdx.x; rr < R; rr += blockDim.x) {
    const float x = rank_key(__ldcg(T.ga.anc_fit + rr));
    if (x < v || (x == v && rr < idx)) { v = x; idx = rr; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov < v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  if (lane == 0) { sv[wid] = v; si[wid] = idx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (sv[w] < v || (sv[w] == v && si[w] < idx)) { v = sv[w]; idx = si[w]; }
    s_rb = idx;
  }
  __syncthreads();
  const int rb = s_rb;
  const float fb = __ldcg(T.ga.anc_fit + rb);
  const uint32_t* src = T.ga.anc + (long long)rb * nw;
  const bool improve = fb < *T.ga.best_fit;
  __syncthreads();
  if (improve) {
    for (int x = threadIdx.x; x < nw; x += blockDim.x) T.ga.best[x] = __ldcg(src + x);
    if (threadIdx.x == 0) *T.ga.best_fit = fb;
  }
  const int g = *T.ga.gen;
  if (T.ga.N1 > 0 && (g + 1) % T.ga.N1 == 0) {
    for (long long e = threadIdx.x; e < (long long)R * nw; e += blockDim.x) {
      const int rr = (int)(e / nw);
      if (rr != rb) T.ga.anc[e] = __ldcg(src + (e - (long long)rr * nw));
    }
    for (int rr = threadIdx.x; rr < R; rr += blockDim.x)
      if (rr != rb) T.ga.anc_fit[rr] = fb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *T.ga.gen = g + 1;
    *T.ga.done = 0;
  }
}

void launch_reduce_select(const TaskSet& ts, cudaStream_t s) {
  TaskParam tp = make_param(ts);
  for (int t = 0; t < ts.count; ++t) tp.bo.o[t + 1] = tp.bo.o[t] + ts.h[t].ga.R;
  const int blocks = tp.bo.o[ts.count];
  if (blocks == 0) return;
  launch_pdl(k_reduce_select, blocks, 128, 0, s, tp);
}

// Start state: every ancestor and the best-ever = the initial solution.
__global__ void k_ga_init(const __grid_constant__ Task T, const uint32_t* __restrict__ mask0,
                          const float* __restrict__ fit0) {
  const int R = T.ga.R, nw = T.in.nw;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)R * nw;
       e += (long long)gridDim.x * blockDim.x)
    T.ga.anc[e] = mask0[e % nw];
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x)
    T.ga.anc_fit[r] = *fit0;
  if (blockIdx.x == 0) {
    for (int x = threadIdx.x; x < nw; x += blockDim.x) T.ga.best[x] = mask0[x];
    if (threadIdx.x == 0) { *T.ga.best_fit = *fit0; *T.ga.gen = 0; *T.ga.done = 0; }
  }
}

void launch_children(const TaskSet& ts, cudaStream_t s) {
  TaskParam tp = make_param(ts);
  int nw = 1;
  for (int t = 0; t < ts.count; ++t) {
    tp.bo.o[t + 1] = tp.bo.o[t] + ts.h[t].pop.B / 2;
    nw = std::max(nw, ts.h[t].in.nw);
  }
  const int blocks = tp.bo.o[ts.count];
  if (blocks == 0) return;
  launch_pdl(k_children, blocks, 64, 4 * nw * sizeof(uint32_t), s, tp);
}

void launch_select(const TaskSet& ts, cudaStream_t s) {
  TaskParam tp = make_param(ts);
  for (int t = 0; t < ts.count; ++t) tp.bo.o[t + 1] = tp.bo.o[t] + ts.h[t].ga.R;
  const int blocks = tp.bo.o[ts.count];
  if (blocks == 0) return;
  k_select_islands<<<blocks, 32, 0, s>>>(tp);
  k_select_global<<<ts.count, 256, 0, s>>>(tp);
}

void launch_ga_init(const Task& task, const uint32_t* mask0, const float* fit0, cudaStream_t s) {
  k_ga_init<<<8, 256, 0, s>>>(task, mask0, fit0);
}

// Every island's ancestor <- mask (nw words), its fitness <- fit: the merge
// step of §5 when the best island lives on another GPU.
__global__ void k_set_ancestors(uint32_t* anc, float* anc_fit, int R, int nw, const uint32_t* mask, float fit) {
  const int r = blockIdx.x;
  for (int x = threadIdx.x; x < nw; x += blockDim.x) anc[(long long)r * nw + x] = mask[x];
  if (threadIdx.x == 0) anc_fit[r] = fit;
}

void launch_set_ancestors(uint32_t* anc, float* anc_fit, int R, int nw, const uint32_t* mask, float fit,
                          cudaStream_t s) {
  if (R > 0) k_set_ancestors<<<R, 128, 0, s>>>(anc, anc_fit, R, nw, mask, fit);
}

}  // namespace usaphmp
