// Validation and canonical form of chromosomes given in the encoding of
// §4.1: p hub node ids (any order) and S[i] = the hub serving node i.
// A chromosome is valid when its hubs are distinct nodes (eq. 5), every
// S[i] is one of them (eq. 2-3) and every hub serves itself (§4.1).
// Output: hubs in ascending order and slot[i] = rank of S[i] among them.
#include "common.cuh"
#include "kernels.cuh"

namespace usaphmp {

// G warps per chromosome (G = 1, 2 or 4 by n), kCanonWarps / G chromosomes
// per block, so that the dependent phases of one chromosome (hub ranks, then
// the slot codes) overlap those of the block's other chromosomes.
constexpr int kCanonWarps = 8;
// four-node groups whose S entries a thread loads at once
constexpr int kCanonGroups = 8;
__host__ __device__ inline int canon_warps_per_chrom(int n) { return n <= 2048 ? 1 : (n <= 4096 ? 2 : 4); }
// shared memory of one chromosome: rank[n] (padded to 16 bytes), then hs[p]
__host__ __device__ inline int canon_smem_per_chrom(int n, int p) { return round_up(n, 16) + round_up(4 * p, 16); }

__global__ void __launch_bounds__(32 * kCanonWarps)
k_canon(const int32_t* __restrict__ hubs_in, const int32_t* __restrict__ S, int B, int n, int p, int ns,
        int32_t* __restrict__ hubs_out, uint8_t* __restrict__ slot, uint32_t* status, int* bad_index,
        int index_base) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int cbad[kCanonWarps];
  const int G = canon_warps_per_chrom(n), cpb = kCanonWarps / G;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wl = wib % G, c = wib / G;
  const int b = blockIdx.x * cpb + c;
  const bool live = b < B;
  uint8_t* rank = sm + (size_t)c * canon_smem_per_chrom(n, p);   // 0xFF = not a hub
  int* hs = reinterpret_cast<int*>(rank + round_up(n, 16));
  const int u0 = wl * 32 + lane, stride = 32 * G;
  auto sync = [&]() { if (G == 1) __syncwarp(); else __syncthreads(); };
  if (threadIdx.x < kCanonWarps) cbad[threadIdx.x] = 0;
  const int32_t* Sb = S + (long long)b * n;
  const int n4 = ns >> 2;
  // S entries of kCanonGroups four-node groups of this thread: loaded
  // together, the first batch before the hub phase so that its loads overlap
  // the hub loads and ranks
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
  if (live) {
    for (int q = u0; q < round_up(n, 16) / 16; q += stride)
      reinterpret_cast<uint4*>(rank)[q] = make_uint4(~0u, ~0u, ~0u, ~0u);
    for (int k = u0; k < p; k += stride) hs[k] = hubs_in[(long long)b * p + k];
  }
  load_groups(u0);
  __syncthreads();
  bool bad = false;
  if (live) {
    for (int k = u0; k < p; k += stride) {
      const int v = hs[k];
      if (v < 0 || v >= n) { bad = true; continue; }
      int r = 0;
      bool dup = false;
      for (int l = 0; l < p; ++l) {
        const int u = hs[l];
        r += u < v;
        dup |= (u == v) & (l != k);
      }
      if (dup) { bad = true; continue; }
      rank[v] = (uint8_t)r;
      hubs_out[(long long)b * p + r] = v;
    }
    if (bad) cbad[c] = 1;
  }
  sync();
  const bool bad_hubs = live && cbad[c] != 0;
  if (live && !bad_hubs) {
    for (int g0 = u0; g0 < n4; g0 += kCanonGroups * stride) {
      if (g0 != u0) load_groups(g0);
#pragma unroll
      for (int j = 0; j < kCanonGroups; ++j) {
        const int g = g0 + j * stride;
        if (g >= n4) break;
        const int i0 = g << 2;
        uint32_t packed = 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int i = i0 + k, s = sv[j][k];
          uint32_t code = kSlotPad;
          if (i < n) {
            if (s < 0 || s >= n || rank[s] == kSlotPad || (rank[i] != kSlotPad && s != i)) {
              bad = true;
              code = 0;
            } else {
              code = rank[s];
            }
          }
          packed |= code << (8 * k);
        }
        *reinterpret_cast<uint32_t*>(slot + (long long)b * ns + i0) = packed;
      }
    }
    if (bad) cbad[c] = 1;
  }
  __syncthreads();
  if (live && wl == 0 && lane == 0 && cbad[c]) {
    atomicOr(status, kStatusBadChromosome);
    atomicMin(bad_index, index_base + b);
  }
}

void launch_canon(const int32_t* hubs_in, const int32_t* S, int B, int n, int p, int ns,
                  int32_t* hubs_out, uint8_t* slot, uint32_t* status, int* bad_index, cudaStream_t s,
                  int index_base) {
  if (B <= 0) return;
  const int cpb = kCanonWarps / canon_warps_per_chrom(n);
  const size_t smem = (size_t)cpb * canon_smem_per_chrom(n, p);
  k_canon<<<(B + cpb - 1) / cpb, 32 * kCanonWarps, smem, s>>>(hubs_in, S, B, n, p, ns, hubs_out, slot, status,
                                                             bad_index, index_base);
}

}  // namespace usaphmp
