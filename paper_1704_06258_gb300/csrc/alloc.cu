// Nearest-hub allocation (§4.1; checked after every operator in §5) and the
// access terms of objective (1), §3:
//   slot_b(i) = argmin_l C[i, hubs_b[l]]   (lowest node id on ties; a hub
//               serves itself),
//   t12_b     = sum_i chi*O_i*C[i,h(i)] + delta*D_i*C[h(i),i],
// plus, for the tensor-core evaluator, the hub-to-hub cost table
// chub_b[k][l] = C[hubs_b[k], hubs_b[l]] (layout in common.cuh).  With
// hub-path routing (eq. 4) the table holds instead the cheapest path cost
// over arcs between the chromosome's open hubs, zero on the diagonal
// (Floyd-Warshall in place, one pass per intermediate hub).
// C[i, hub] is read as CT[hub][i], so the loads of consecutive nodes are
// coalesced.  With direct hub arcs (the GA's hot path) one warp allocates one
// chromosome (k_alloc_warp): no block barriers, and a whole population's
// warps are resident at once, so the latency of the L2 gathers of one
// chromosome overlaps that of every other.  Hub-path routing keeps one block
// per chromosome (k_alloc), whose threads share the Floyd-Warshall passes.
#include "common.cuh"
#include "kernels.cuh"

#include <algorithm>

namespace usaphmp {

namespace {
// Hub-path tables up to this many entries (p <= 110) are relaxed in shared
// memory; larger ones in place in global memory.
constexpr int kFwSmemEntries = 12288;
// Threads per chromosome block: with four nodes per thread, 128 threads keep
// a block of n = 1000 nodes two groups deep and let more blocks share an SM.
constexpr int kAllocThreads = 128;
// Hub-path table entries each thread keeps in registers (p*p <= kFwOwn * kAllocThreads).
constexpr int kFwOwn = 4;
}

template <bool kNearest>
__global__ void __launch_bounds__(kAllocThreads) k_alloc(const __grid_constant__ TaskParam tp, int with_chub) {
  __shared__ int hs[kMaxP];
  __shared__ float red[32];
  pdl_wait();
  pdl_allow_next();
  const int t = task_of(tp.bo, blockIdx.x);
  const Task& T = task_at(tp, t);
  const int b = blockIdx.x - tp.bo.o[t];
  const int n = T.in.n, p = T.in.p, ldw = T.in.ldw, ns = T.in.ns;
  const float* __restrict__ C = T.in.C;
  const float* __restrict__ CT = T.in.CT;
  const float* __restrict__ O = T.in.O;
  const float* __restrict__ D = T.in.D;
  const float chi = T.in.chi, delta = T.in.delta;
  const bool sym = T.in.symmetric != 0;
  uint8_t* __restrict__ slot = T.pop.slot + (long long)b * ns;
  const uint8_t* __restrict__ slot_in = T.pop.slot_in ? T.pop.slot_in + (long long)b * ns : slot;
  bool bad = false;
  for (int k = threadIdx.x; k < p; k += blockDim.x) {
    int v = T.pop.hubs_in ? T.pop.hubs_in[(long long)b * p + k] : T.pop.hubs[(long long)b * p + k];
    if (v < 0 || v >= n) { bad = true; v = 0; }
    hs[k] = v;
    if (T.pop.hubs_in) T.pop.hubs[(long long)b * p + k] = v;
  }
  __syncthreads();

  float acc = 0.f;
  if (kNearest) {
    // Four consecutive nodes per thread: one 16-byte load of CT[hub][i..i+3]
    // per hub (rows are zero-padded to ldw, a multiple of 8), compares in
    // ascending hub order per node (lowest hub on ties).  Hubs serve
    // themselves: a node that is a hub takes its own slot afterwards.
    __shared__ uint32_t hub_bits[kMaxN / 32];
    for (int w = threadIdx.x; w < (n + 31) / 32; w += blockDim.x) {
      uint32_t bits = 0u;
      for (int k = 0; k < p; ++k)
        if ((hs[k] >> 5) == w) bits |= 1u << (hs[k] & 31);
      hub_bits[w] = bits;
    }
    __syncthreads();
    const int n4 = (n + 3) >> 2;
    for (int g = threadIdx.x; g < n4; g += blockDim.x) {
      const int i0 = g << 2;
      float4 best = __ldg(reinterpret_cast<const float4*>(CT + (long long)hs[0] * ldw) + g);
      int b0 = 0, b1 = 0, b2 = 0, b3 = 0;
      int l = 1;
      for (; l + 4 <= p; l += 4) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = __ldg(reinterpret_cast<const float4*>(CT + (long long)hs[l + u] * ldw) + g);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (v[u].x < best.x) { best.x = v[u].x; b0 = l + u; }
          if (v[u].y < best.y) { best.y = v[u].y; b1 = l + u; }
          if (v[u].z < best.z) { best.z = v[u].z; b2 = l + u; }
          if (v[u].w < best.w) { best.w = v[u].w; b3 = l + u; }
        }
      }
      for (; l < p; ++l) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(CT + (long long)hs[l] * ldw) + g);
        if (v.x < best.x) { best.x = v.x; b0 = l; }
        if (v.y < best.y) { best.y = v.y; b1 = l; }
        if (v.z < best.z) { best.z = v.z; b2 = l; }
        if (v.w < best.w) { best.w = v.w; b3 = l; }
      }
      // one node of the group: own slot for a hub, access terms, slot code
      const float4 o4 = __ldg(reinterpret_cast<const float4*>(O) + g);
      const float4 d4 = __ldg(reinterpret_cast<const float4*>(D) + g);
      const uint32_t hw = hub_bits[i0 >> 5];  // the group's four nodes share one bitmap word
      auto finish = [&](int i, int bl, float cih, float oi, float di) -> uint32_t {
        if (i >= n) return (uint32_t)kSlotPad;
        if ((hw >> (i & 31)) & 1u) {
          for (int q = 0; q < p; ++q)
            if (hs[q] == i) bl = q;
          cih = CT[(long long)i * ldw + i];
        }
        const float chi_i = sym ? cih : C[(long long)hs[bl] * ldw + i];  // C[h(i), i]
        acc += access_term(chi, oi, cih, delta, di, chi_i);
        return (uint32_t)bl;
      };
      const uint32_t s0 = finish(i0, b0, best.x, o4.x, d4.x);
      const uint32_t s1 = finish(i0 + 1, b1, best.y, o4.y, d4.y);
      const uint32_t s2 = finish(i0 + 2, b2, best.z, o4.z, d4.z);
      const uint32_t s3 = finish(i0 + 3, b3, best.w, o4.w, d4.w);
      const uint32_t packed = s0 | (s1 << 8) | (s2 << 16) | (s3 << 24);
      *reinterpret_cast<uint32_t*>(slot + i0) = packed;
    }
    for (int i = (n4 << 2) + threadIdx.x; i < ns; i += blockDim.x) slot[i] = kSlotPad;
  } else {
    // given slots: the same four-node groups and summation order as above,
    // the four gathers of a group issued before their terms are added
    const int n4 = (n + 3) >> 2;
    for (int g = threadIdx.x; g < n4; g += blockDim.x) {
      const int i0 = g << 2;
      const uint32_t codes = *reinterpret_cast<const uint32_t*>(slot_in + i0);
      int bl[4];
      float cih[4], chi_i[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        bl[k] = (int)((codes >> (8 * k)) & 0xFFu);
        if (i0 + k < n && bl[k] >= p) bad = true;
        if (i0 + k >= n || bl[k] >= p) bl[k] = 0;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = min(i0 + k, n - 1);
        cih[k] = CT[(long long)hs[bl[k]] * ldw + i];                       // C[i, h(i)]
        chi_i[k] = sym ? cih[k] : C[(long long)hs[bl[k]] * ldw + i];      // C[h(i), i]
      }
      const float4 o4 = __ldg(reinterpret_cast<const float4*>(O) + g);
      const float4 d4 = __ldg(reinterpret_cast<const float4*>(D) + g);
      const float ok[4] = {o4.x, o4.y, o4.z, o4.w}, dk[4] = {d4.x, d4.y, d4.z, d4.w};
      uint32_t packed = 0u;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = i0 + k;
        if (i < n) {
          acc += access_term(chi, ok[k], cih[k], delta, dk[k], chi_i[k]);
          packed |= (uint32_t)bl[k] << (8 * k);
        } else {
          packed |= (uint32_t)kSlotPad << (8 * k);
        }
      }
      *reinterpret_cast<uint32_t*>(slot + i0) = packed;
    }
    for (int i = (n4 << 2) + threadIdx.x; i < ns; i += blockDim.x) slot[i] = kSlotPad;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(T.pop.status, kStatusBadChromosome);
  const float s = block_sum(acc, red);
  if (threadIdx.x == 0) T.pop.t12[b] = s;
  const bool routed = T.in.routing != 0;
  if (with_chub || routed || plain_global_table(p, T.in.ns)) {
    const int hst = chub_hstride(p), cst = chub_cstride(p);
    float* ch = T.pop.chub + (long long)b * cst;
    for (int e = threadIdx.x; e < cst; e += blockDim.x) {
      const int k = e / hst, l = e - k * hst;
      ch[e] = (k < p && l < p && !(routed && k == l)) ? C[(long long)hs[k] * ldw + hs[l]] : 0.f;
    }
    if (routed) {
      // Pass m relaxes every (a, c) through hub m.  Row m and column m do not
      // change during pass m (their diagonal entry is 0 and costs are >= 0),
      // so the in-place updates of one pass do not race.
      extern __shared__ float fw[];
      const bool in_smem = p * p <= kFwSmemEntries;
      __syncthreads();
      if (in_smem && p * p <= kFwOwn * kAllocThreads) {
        // small p: every thread owns up to kFwOwn entries and keeps them in
        // registers; shared memory holds the table for the others' reads.
        float v[kFwOwn];
        int e4[kFwOwn];
#pragma unroll
        for (int k = 0; k < kFwOwn; ++k) {
          const int e = threadIdx.x + kAllocThreads * k;
          const int a = e / p, c = e - a * p;
          e4[k] = e < p * p ? e : -1;
          v[k] = e < p * p ? ch[a * hst + c] : 0.f;
          if (e < p * p) fw[e] = v[k];
        }
        __syncthreads();
        int ra[kFwOwn], rc[kFwOwn];
#pragma unroll
        for (int k = 0; k < kFwOwn; ++k) {
          ra[k] = e4[k] >= 0 ? e4[k] / p : 0;
          rc[k] = e4[k] >= 0 ? e4[k] - ra[k] * p : 0;
        }
        for (int m = 0; m < p; ++m) {
#pragma unroll
          for (int k = 0; k < kFwOwn; ++k) {
            if (e4[k] >= 0) {
              const float nv = fw[ra[k] * p + m] + fw[m * p + rc[k]];
              if (nv < v[k]) {
                v[k] = nv;
                fw[e4[k]] = nv;
              }
            }
          }
          __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < kFwOwn; ++k)
          if (e4[k] >= 0) ch[ra[k] * hst + rc[k]] = v[k];
      } else {
        // warp w relaxes rows w, w + nwarps, ...; lane l columns l, l + 32, ...
        float* d = in_smem ? fw : ch;
        const int ld = in_smem ? p : hst;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
        if (in_smem) {
          for (int a = wid; a < p; a += nwarp)
            for (int c = lane; c < p; c += 32) fw[a * p + c] = ch[a * hst + c];
          __syncthreads();
        }
        for (int m = 0; m < p; ++m) {
          for (int a = wid; a < p; a += nwarp) {
            const float dam = d[a * ld + m];
            for (int c = lane; c < p; c += 32) {
              const float nv = dam + d[m * ld + c];
              if (nv < d[a * ld + c]) d[a * ld + c] = nv;
            }
          }
          __syncthreads();
        }
        if (in_smem)
          for (int a = wid; a < p; a += nwarp)
            for (int c = lane; c < p; c += 32) ch[a * hst + c] = fw[a * p + c];
      }
    }
  }
}


// Hub-cost table of one chromosome (layout in common.cuh): ch[k * hst + l] =
// C[hs[k]][hs[l]] for k, l < p and 0 in the rest of its cst entries.  Thread
// t of nt takes entries t, t + nt, ..., kBatch at a time with their loads
// issued together; k = e / hst comes from a float product with the
// reciprocal, corrected by one step either way (e < 2^16, so the product is
// off by far less than one).
template <int kBatch>
__device__ inline void fill_chub(float* __restrict__ ch, const float* __restrict__ C, const int* hs, int p, int ldw,
                                 int t, int nt) {
  const int hst = chub_hstride(p), cst = chub_cstride(p);
  const float inv = 1.0f / (float)hst;
  for (int e0 = t; e0 < cst; e0 += kBatch * nt) {
    float v[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int e = e0 + u * nt;
      int k = (int)(((float)e + 0.5f) * inv);
      int l = e - k * hst;
      if (l < 0) { --k; l += hst; } else if (l >= hst) { ++k; l -= hst; }
      v[u] = (e < cst && k < p && l < p) ? C[(long long)hs[k] * ldw + hs[l]] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u)
      if (e0 + u * nt < cst) ch[e0 + u * nt] = v[u];
  }
}

// Direct hub arcs: G warps per chromosome (G = 1, 2 or 4 by n alone), four
// chromosomes' worth of warps per block.  Thread u of a chromosome's 32G
// takes the four-node groups u, u + 32G, ...: one 16-byte load of
// CT[hub][i..i+3] per hub, the compares in ascending hub order (lowest hub on
// ties); hubs serve themselves (the hubs are ascending, so a per-thread
// pointer finds the hubs inside each group).  The access terms are summed
// per thread in group order, over each warp by a fixed butterfly and over the
// G warps in order; the given-slot variant sums in the same order, so both
// give the same t12 for the same slots, and since G depends on n only a
// chromosome's t12 does not depend on the batch it is in.
#ifndef USAPHMP_ALLOC_WARPS
#define USAPHMP_ALLOC_WARPS 4
#endif
constexpr int kAllocWarps = USAPHMP_ALLOC_WARPS;   // warps per block
// Four-node groups a thread searches at once (their loads in flight together).
constexpr int kAllocGroups = 2;
// Four-node groups a thread gathers at once when the slots are given.
constexpr int kGivenGroups = 3;
// Row offsets of hubs 1, 5, 9, ... start on 16-byte boundaries: entry k at
// kHoPad + k of a row of kHoRow ints (a multiple of four, so every warp's
// row starts on a 16-byte boundary too).
constexpr int kHoPad = 3;
constexpr int kHoRow = (kHoPad + kMaxP + 1 + 3) / 4 * 4;
static_assert(kHoRow % 4 == 0 && kHoRow >= kHoPad + kMaxP, "hub offset rows");

__host__ __device__ inline int alloc_warps_per_chrom(int n) { return n <= 2048 ? 1 : (n <= 4096 ? 2 : 4); }

// Block offsets of a launch count blocks: task t owns blocks [o[t], o[t+1]),
// ceil(B_t / (kAllocWarps / G_t)) of them.
template <bool kNearest>
__global__ void __launch_bounds__(32 * kAllocWarps) k_alloc_warp(const __grid_constant__ TaskParam tp, int with_chub) {
  __shared__ int hs_all[kAllocWarps][kMaxP];
  __shared__ __align__(16) int ho_all[kAllocWarps][kHoRow];
  __shared__ float red[kAllocWarps];
  pdl_wait();
  pdl_allow_next();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int t = task_of(tp.bo, blockIdx.x);
  const Task& T = task_at(tp, t);
  const int n = T.in.n, p = T.in.p, ldw = T.in.ldw, ns = T.in.ns;
  const int G = alloc_warps_per_chrom(n);          // block-uniform
  const int cpb = kAllocWarps / G;                 // chromosomes per block
  const int wl = wib % G;                          // warp within its chromosome
  const int b = (blockIdx.x - tp.bo.o[t]) * cpb + wib / G;
  const bool live = b < T.pop.B;
  const float* __restrict__ C = T.in.C;
  const float* __restrict__ CT = T.in.CT;
  const float* __restrict__ O = T.in.O;
  const float* __restrict__ D = T.in.D;
  const float chi = T.in.chi, delta = T.in.delta;
  const bool sym = T.in.symmetric != 0;
  int* hs = hs_all[wib - wl];                      // the chromosome's first warp's row
  int* ho = ho_all[wib - wl];                      // ho[kHoPad + k] = float4 offset of CT row hs[k]
  const int u0 = wl * 32 + lane, stride = 32 * G;  // thread within the chromosome
  bool bad = false;
  float acc = 0.f;
  if (live) {
    uint8_t* __restrict__ slot = T.pop.slot + (long long)b * ns;
    const uint8_t* __restrict__ slot_in = T.pop.slot_in ? T.pop.slot_in + (long long)b * ns : slot;
    for (int k = u0; k < p; k += stride) {
      int v = T.pop.hubs_in ? T.pop.hubs_in[(long long)b * p + k] : T.pop.hubs[(long long)b * p + k];
      if (v < 0 || v >= n) { bad = true; v = 0; }
      hs[k] = v;
      ho[kHoPad + k] = v * (ldw >> 2);
      if (T.pop.hubs_in) T.pop.hubs[(long long)b * p + k] = v;
    }
  }
  if (G == 1) __syncwarp(); else __syncthreads();
  if (live) {
    uint8_t* __restrict__ slot = T.pop.slot + (long long)b * ns;
    const uint8_t* __restrict__ slot_in = T.pop.slot_in ? T.pop.slot_in + (long long)b * ns : slot;
    const int n4 = (n + 3) >> 2;
    if (kNearest) {
      // kAllocGroups of the thread's groups at a time (more loads in flight);
      // the hub rows' float4 offsets come four at a time from shared memory
      const float4* __restrict__ CT4 = reinterpret_cast<const float4*>(CT);
      int kp = 0;   // first hub not below the current group's first node
      for (int g = u0; g < n4; g += kAllocGroups * stride) {
        float4 best[kAllocGroups], o4[kAllocGroups], d4[kAllocGroups];
        int sl[kAllocGroups][4];
        const float4* col[kAllocGroups];   // column group gj of CT (a valid one for a missing group)
#pragma unroll
        for (int j = 0; j < kAllocGroups; ++j) {
          const int gj = g + j * stride;
          col[j] = CT4 + (gj < n4 ? gj : g);
          best[j] = __ldg(col[j] + ho[kHoPad]);
          o4[j] = __ldg(reinterpret_cast<const float4*>(O) + (gj < n4 ? gj : g));
          d4[j] = __ldg(reinterpret_cast<const float4*>(D) + (gj < n4 ? gj : g));
          sl[j][0] = sl[j][1] = sl[j][2] = sl[j][3] = 0;
        }
        int l = 1;
        for (; l + 4 <= p; l += 4) {
          const int4 o = *reinterpret_cast<const int4*>(ho + kHoPad + l);
          const int off[4] = {o.x, o.y, o.z, o.w};
          float4 v[kAllocGroups][4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < kAllocGroups; ++j) v[j][u] = __ldg(col[j] + off[u]);
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < kAllocGroups; ++j) {
              if (v[j][u].x < best[j].x) { best[j].x = v[j][u].x; sl[j][0] = l + u; }
              if (v[j][u].y < best[j].y) { best[j].y = v[j][u].y; sl[j][1] = l + u; }
              if (v[j][u].z < best[j].z) { best[j].z = v[j][u].z; sl[j][2] = l + u; }
              if (v[j][u].w < best[j].w) { best[j].w = v[j][u].w; sl[j][3] = l + u; }
            }
        }
        for (; l < p; ++l) {
          const int off = ho[kHoPad + l];
#pragma unroll
          for (int j = 0; j < kAllocGroups; ++j) {
            const float4 v = __ldg(col[j] + off);
            if (v.x < best[j].x) { best[j].x = v.x; sl[j][0] = l; }
            if (v.y < best[j].y) { best[j].y = v.y; sl[j][1] = l; }
            if (v.z < best[j].z) { best[j].z = v.z; sl[j][2] = l; }
            if (v.w < best[j].w) { best[j].w = v.w; sl[j][3] = l; }
          }
        }
#pragma unroll
        for (int j = 0; j < kAllocGroups; ++j) {
          const int gj = g + j * stride;
          if (gj >= n4) break;
          const int i0 = gj << 2;
          // hubs inside the group serve themselves
          while (kp < p && hs[kp] < i0) ++kp;
          for (int q = kp; q < p && hs[q] < i0 + 4; ++q) {
            const int h = hs[q];
            const float own = CT[(long long)h * ldw + h];
            switch (h - i0) {
              case 0: sl[j][0] = q; best[j].x = own; break;
              case 1: sl[j][1] = q; best[j].y = own; break;
              case 2: sl[j][2] = q; best[j].z = own; break;
              default: sl[j][3] = q; best[j].w = own; break;
            }
          }
          // one node of the group: access terms (in node order) and slot code
          auto node = [&](int k, int sk, float cih, float oi, float di) -> uint32_t {
            const int i = i0 + k;
            if (i >= n) return (uint32_t)kSlotPad << (8 * k);
            const float chi_i = sym ? cih : C[(long long)hs[sk] * ldw + i];   // C[h(i), i]
            acc += access_term(chi, oi, cih, delta, di, chi_i);
            return (uint32_t)sk << (8 * k);
          };
          uint32_t packed = node(0, sl[j][0], best[j].x, o4[j].x, d4[j].x);
          packed |= node(1, sl[j][1], best[j].y, o4[j].y, d4[j].y);
          packed |= node(2, sl[j][2], best[j].z, o4[j].z, d4[j].z);
          packed |= node(3, sl[j][3], best[j].w, o4[j].w, d4[j].w);
          *reinterpret_cast<uint32_t*>(slot + i0) = packed;
        }
      }
    } else {
      // given slots: kGivenGroups of the thread's groups at a time, their
      // slot codes loaded together and then their gathers, so one group's
      // loads do not wait for the previous group's
      for (int g = u0; g < n4; g += kGivenGroups * stride) {
        uint32_t codes[kGivenGroups];
#pragma unroll
        for (int j = 0; j < kGivenGroups; ++j) {
          const int gj = g + j * stride;
          codes[j] = gj < n4 ? *reinterpret_cast<const uint32_t*>(slot_in + (gj << 2)) : 0u;
        }
        int bl[kGivenGroups][4];
        float cih[kGivenGroups][4], chi_i[kGivenGroups][4];
#pragma unroll
        for (int j = 0; j < kGivenGroups; ++j) {
          const int gj = g + j * stride;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int i = (gj << 2) + k;
            const bool valid = gj < n4 && i < n;
            bl[j][k] = (int)((codes[j] >> (8 * k)) & 0xFFu);
            if (valid && bl[j][k] >= p) bad = true;
            if (!valid || bl[j][k] >= p) bl[j][k] = 0;
          }
        }
#pragma unroll
        for (int j = 0; j < kGivenGroups; ++j) {
          const int gj = g + j * stride;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int e = ho[kHoPad + bl[j][k]] * 4 + min((gj << 2) + k, n - 1);   // hub row, node i
            cih[j][k] = CT[e];                       // C[i, h(i)]
            chi_i[j][k] = sym ? cih[j][k] : C[e];    // C[h(i), i]
          }
        }
#pragma unroll
        for (int j = 0; j < kGivenGroups; ++j) {
          const int gj = g + j * stride;
          if (gj >= n4) break;
          const int i0 = gj << 2;
          const float4 o4 = __ldg(reinterpret_cast<const float4*>(O) + gj);
          const float4 d4 = __ldg(reinterpret_cast<const float4*>(D) + gj);
          const float ok[4] = {o4.x, o4.y, o4.z, o4.w}, dk[4] = {d4.x, d4.y, d4.z, d4.w};
          uint32_t packed = 0u;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int i = i0 + k;
            if (i < n) {
              acc += access_term(chi, ok[k], cih[j][k], delta, dk[k], chi_i[j][k]);
              packed |= (uint32_t)bl[j][k] << (8 * k);
            } else {
              packed |= (uint32_t)kSlotPad << (8 * k);
            }
          }
          *reinterpret_cast<uint32_t*>(slot + i0) = packed;
        }
      }
    }
    for (int i = (n4 << 2) + u0; i < ns; i += stride) slot[i] = kSlotPad;
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(T.pop.status, kStatusBadChromosome);
  }
  acc = warp_sum(acc);
  if (G > 1) {
    if (lane == 0) red[wib] = acc;
    __syncthreads();
    if (wl == 0) {
      acc = red[wib];
      for (int w = 1; w < G; ++w) acc += red[wib + w];
    }
  }
  if (live && wl == 0 && lane == 0) T.pop.t12[b] = acc;
  if (live && (with_chub || plain_global_table(p, ns)))
    fill_chub<16>(T.pop.chub + (long long)b * chub_cstride(p), C, hs, p, ldw, u0, stride);
}

// Chromosomes given in the encoding of §4.1 (p hub node ids in any order and
// S[i] = the hub serving node i), direct hub arcs: the validation and
// canonical form (hubs ascending, slot codes = ranks of S[i] among them; the
// checks of eq. 2, 3 and 5 and "a hub serves itself", §4.1) fused with the
// given-slot allocation kernel above, whose groups, warps per chromosome and
// summation order it keeps (the same t12 bits for the same slots).  S of a
// thread's first kCanonGroups groups is loaded before the hub phase, so that
// those loads overlap the hub loads and ranks.
constexpr int kCanonGroups = 4;

__global__ void __launch_bounds__(32 * kAllocWarps)
k_canon_alloc(const __grid_constant__ Task T, const int32_t* __restrict__ hubs_in, const int32_t* __restrict__ S,
              int* bad_index, int index_base, int with_chub) {
  extern __shared__ __align__(16) unsigned char rank_all[];   // per chromosome: rank[n], 0xFF = not a hub
  __shared__ int hs_all[kAllocWarps][kMaxP];
  __shared__ __align__(16) int ho_all[kAllocWarps][kHoRow];
  __shared__ int hraw_all[kAllocWarps][kMaxP];
  __shared__ float red[kAllocWarps];
  __shared__ int cbad[kAllocWarps];
  pdl_wait();
  pdl_allow_next();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int n = T.in.n, p = T.in.p, ldw = T.in.ldw, ns = T.in.ns;
  const int G = alloc_warps_per_chrom(n), cpb = kAllocWarps / G, wl = wib % G, c = wib / G;
  const int b = blockIdx.x * cpb + c;
  const bool live = b < T.pop.B;
  const int n16 = round_up(n, 16), n4 = (n + 3) >> 2;
  uint8_t* rank = rank_all + (size_t)c * n16;
  int* hs = hs_all[wib - wl];
  int* ho = ho_all[wib - wl];
  int* hraw = hraw_all[wib - wl];
  const int u0 = wl * 32 + lane, stride = 32 * G;
  const float* __restrict__ C = T.in.C;
  const float* __restrict__ CT = T.in.CT;
  const float chi = T.in.chi, delta = T.in.delta;
  const bool sym = T.in.symmetric != 0;
  const int32_t* Sb = S + (long long)b * n;
  int sv[kCanonGroups][4];
  auto load_groups = [&](int g0) {
#pragma unroll
    for (int j = 0; j < kCanonGroups; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = ((g0 + j * stride) << 2) + k;
        sv[j][k] = (live && g0 + j * stride < n4 && i < n) ? Sb[i] : 0;
      }
  };
  if (threadIdx.x < kAllocWarps) cbad[threadIdx.x] = 0;
  if (live) {
    for (int q = u0; q < n16 / 16; q += stride) reinterpret_cast<uint4*>(rank)[q] = make_uint4(~0u, ~0u, ~0u, ~0u);
    for (int k = u0; k < p; k += stride) hraw[k] = hubs_in[(long long)b * p + k];
  }
  load_groups(u0);
  __syncthreads();
  bool bad = false;
  if (live) {
    for (int k = u0; k < p; k += stride) {
      const int v = hraw[k];
      if (v < 0 || v >= n) { bad = true; continue; }
      int r = 0;
      bool dup = false;
      for (int l = 0; l < p; ++l) {
        const int u = hraw[l];
        r += u < v;
        dup |= (u == v) & (l != k);
      }
      if (dup) { bad = true; continue; }
      rank[v] = (uint8_t)r;
      hs[r] = v;
      ho[kHoPad + r] = v * (ldw >> 2);
      T.pop.hubs[(long long)b * p + r] = v;
    }
    if (bad) cbad[c] = 1;
  }
  __syncthreads();
  const bool ok = live && cbad[c] == 0;
  float acc = 0.f;
  if (ok) {
    uint8_t* __restrict__ slot = T.pop.slot + (long long)b * ns;
    for (int g0 = u0; g0 < n4; g0 += kCanonGroups * stride) {
      if (g0 != u0) load_groups(g0);
      // slot codes of the thread's groups (four per word), then all their gathers
      uint32_t codes[kCanonGroups];
#pragma unroll
      for (int j = 0; j < kCanonGroups; ++j) {
        codes[j] = 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int i = ((g0 + j * stride) << 2) + k, s = sv[j][k];
          uint32_t code = 0u;
          if (g0 + j * stride < n4 && i < n) {
            if (s < 0 || s >= n || rank[s] == kSlotPad || (rank[i] != kSlotPad && s != i))
              bad = true;
            else
              code = rank[s];
          }
          codes[j] |= code << (8 * k);
        }
      }
      float cih[kCanonGroups][4];
#pragma unroll
      for (int j = 0; j < kCanonGroups; ++j)
#pragma unroll
        for (int k = 0; k < 4; ++k)
          cih[j][k] = CT[ho[kHoPad + ((codes[j] >> (8 * k)) & 0xFFu)] * 4 +
                         min(((g0 + j * stride) << 2) + k, n - 1)];   // C[i, h(i)]
#pragma unroll
      for (int j = 0; j < kCanonGroups; ++j) {
        const int gj = g0 + j * stride;
        if (gj >= n4) break;
        const int i0 = gj << 2;
        const float4 o4 = __ldg(reinterpret_cast<const float4*>(T.in.O) + gj);
        const float4 d4 = __ldg(reinterpret_cast<const float4*>(T.in.D) + gj);
        const float ok4[4] = {o4.x, o4.y, o4.z, o4.w}, dk[4] = {d4.x, d4.y, d4.z, d4.w};
        uint32_t packed = 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int i = i0 + k;
          const uint32_t code = (codes[j] >> (8 * k)) & 0xFFu;
          if (i < n) {
            const float chi_i = sym ? cih[j][k] : C[ho[kHoPad + code] * 4 + i];   // C[h(i), i]
            acc += access_term(chi, ok4[k], cih[j][k], delta, dk[k], chi_i);
            packed |= code << (8 * k);
          } else {
            packed |= (uint32_t)kSlotPad << (8 * k);
          }
        }
        *reinterpret_cast<uint32_t*>(slot + i0) = packed;
      }
    }
    for (int i = (n4 << 2) + u0; i < ns; i += stride) slot[i] = kSlotPad;
    if (bad) cbad[c] = 1;
  }
  acc = warp_sum(acc);
  if (G > 1) {
    if (lane == 0) red[wib] = acc;
    __syncthreads();
    if (wl == 0) {
      acc = red[wib];
      for (int w = 1; w < G; ++w) acc += red[wib + w];
    }
  }
  if (ok && wl == 0 && lane == 0) T.pop.t12[b] = acc;
  if (ok && (with_chub || plain_global_table(p, ns)))
    fill_chub<8>(T.pop.chub + (long long)b * chub_cstride(p), C, hs, p, ldw, u0, stride);
  __syncthreads();
  if (live && wl == 0 && lane == 0 && cbad[c]) {
    atomicOr(T.pop.status, kStatusBadChromosome);
    atomicMin(bad_index, index_base + b);
  }
}

bool launch_canon_alloc(const Task& task, const int32_t* hubs_in, const int32_t* S, int* bad_index, int index_base,
                        bool with_chub, cudaStream_t s) {
  if (task.in.routing != 0) return false;   // hub-path tables come from the block kernel
  if (task.pop.B <= 0) return true;
  const int cpb = kAllocWarps / alloc_warps_per_chrom(task.in.n);
  const size_t smem = (size_t)cpb * round_up(task.in.n, 16);
  launch_pdl(k_canon_alloc, (task.pop.B + cpb - 1) / cpb, 32 * kAllocWarps, smem, s, task, hubs_in, S, bad_index,
             index_base, with_chub ? 1 : 0);
  return true;
}

void launch_alloc(const TaskSet& ts, bool nearest, bool with_chub, cudaStream_t s) {
  TaskParam tp = make_param(ts);
  for (int t = 0; t < ts.count; ++t) tp.bo.o[t + 1] = tp.bo.o[t] + ts.h[t].pop.B;
  const int chrom = tp.bo.o[ts.count];
  if (chrom == 0) return;
  bool routed = false;
  for (int t = 0; t < ts.count; ++t) routed |= ts.h[t].in.routing != 0;
  if (!routed) {
    // blocks per task from the task's own n: its warps per chromosome, and so
    // its summation order, never depend on the other tasks of the launch
    TaskParam tw = make_param(ts);
    for (int t = 0; t < ts.count; ++t) {
      const int cpb = kAllocWarps / alloc_warps_per_chrom(ts.h[t].in.n);
      tw.bo.o[t + 1] = tw.bo.o[t] + (ts.h[t].pop.B + cpb - 1) / cpb;
    }
    const int blocks = tw.bo.o[ts.count];
    if (nearest)
      launch_pdl(k_alloc_warp<true>, blocks, 32 * kAllocWarps, 0, s, tw, with_chub ? 1 : 0);
    else
      launch_pdl(k_alloc_warp<false>, blocks, 32 * kAllocWarps, 0, s, tw, with_chub ? 1 : 0);
    return;
  }
  const int blocks = chrom;
  size_t smem = 0;
  for (int t = 0; t < ts.count; ++t) {
    const int p = ts.h[t].in.p;
    if (ts.h[t].in.routing && p * p <= kFwSmemEntries) smem = std::max(smem, (size_t)p * p * sizeof(float));
  }
  if (nearest)
    launch_pdl(k_alloc<true>, blocks, kAllocThreads, smem, s, tp, with_chub ? 1 : 0);
  else
    launch_pdl(k_alloc<false>, blocks, kAllocThreads, smem, s, tp, with_chub ? 1 : 0);
}

}  // namespace usaphmp
