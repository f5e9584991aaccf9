// Validation and canonical form of chromosomes given in the encoding of
// §4.1: p hub node ids (any order) and S[i] = the hub serving node i.
// A chromosome is valid when its hubs are distinct nodes (eq. 5), every
// S[i] is one of them (eq. 2-3) and every hub serves itself (§4.1).
// Output: hubs in ascending order and slot[i] = rank of S[i] among them.
#include "common.cuh"
#include "kernels.cuh"

namespace usaphmp {

__global__ void k_canon(const int32_t* __restrict__ hubs_in, const int32_t* __restrict__ S,
                        int n, int p, int ns, int32_t* __restrict__ hubs_out,
                        uint8_t* __restrict__ slot, uint32_t* status, int* bad_index, int index_base) {
  extern __shared__ __align__(16) unsigned char sm[];
  uint8_t* rank = sm;                                         // [n], 0xFF = not a hub
  int* hs = reinterpret_cast<int*>(sm + round_up(n, 16));     // [p]
  const int b = blockIdx.x;
  bool bad = false;
  for (int i = threadIdx.x; i < n; i += blockDim.x) rank[i] = kSlotPad;
  for (int k = threadIdx.x; k < p; k += blockDim.x) hs[k] = hubs_in[(long long)b * p + k];
  __syncthreads();
  for (int k = threadIdx.x; k < p; k += blockDim.x) {
    const int v = hs[k];
    if (v < 0 || v >= n) { bad = true; continue; }
    int r = 0;
    for (int l = 0; l < p; ++l) {
      const int u = hs[l];
      if (u < v) ++r;
      else if (u == v && l != k) bad = true;
    }
    if (!bad) {
      rank[v] = (uint8_t)r;
      hubs_out[(long long)b * p + r] = v;
    }
  }
  if (__syncthreads_or(bad)) {
    if (threadIdx.x == 0) { atomicOr(status, kStatusBadChromosome); atomicMin(bad_index, index_base + b); }
    return;
  }
  // four nodes per thread: their S entries loaded together, one 32-bit store
  const int32_t* Sb = S + (long long)b * n;
  for (int g = threadIdx.x; g < (ns >> 2); g += blockDim.x) {
    const int i0 = g << 2;
    int sv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) sv[k] = (i0 + k < n) ? Sb[i0 + k] : 0;
    uint32_t packed = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = i0 + k, s = sv[k];
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
  if (__syncthreads_or(bad) && threadIdx.x == 0) {
    atomicOr(status, kStatusBadChromosome);
    atomicMin(bad_index, index_base + b);
  }
}

void launch_canon(const int32_t* hubs_in, const int32_t* S, int B, int n, int p, int ns,
                  int32_t* hubs_out, uint8_t* slot, uint32_t* status, int* bad_index, cudaStream_t s,
                  int index_base) {
  if (B <= 0) return;
  const size_t smem = round_up(n, 16) + sizeof(int) * p;
  k_canon<<<B, 256, smem, s>>>(hubs_in, S, n, p, ns, hubs_out, slot, status, bad_index, index_base);
}

}  // namespace usaphmp
