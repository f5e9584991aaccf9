// Instance set-up kernels: input checks, W split into bf16 hi + lo, the flows
// O and D of §3, the symmetry test and transpose of C, and the middle-node
// initial solution of §4.1.
#include "common.cuh"
#include "kernels.cuh"

namespace usaphmp {

// Flags any W or C entry that is negative or not finite (the objective of
// §3 is defined for non-negative flows and costs).
__global__ void k_check_values(const float* __restrict__ W, const float* __restrict__ C,
                               int n, int ldw, uint32_t* status) {
  const long long total = (long long)n * ldw;
  bool bad = false;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const float w = W[e], c = C[e];
    bad |= !(w >= 0.f) || !(c >= 0.f) || isinf(w) || isinf(c);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, kStatusBadValue);
}

// W = Whi + Wlo: Whi is W rounded to bf16, Wlo the rounded remainder (the
// remainder W - Whi is exact in fp32).
__global__ void k_split_bf16(const float* __restrict__ W, __nv_bfloat16* __restrict__ Whi,
                             __nv_bfloat16* __restrict__ Wlo, long long total) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const float w = W[e];
    const __nv_bfloat16 hi = __float2bfloat16_rn(w);
    Whi[e] = hi;
    Wlo[e] = __float2bfloat16_rn(w - __bfloat162float(hi));
  }
}

// The same split of U, the pairs (i, j) and (j, i) folded onto j > i:
// U[i][j] = W[i][j] + W[j][i] for j > i, U[i][i] = W[i][i], 0 below the
// diagonal and in the padding columns.  When every hub-to-hub cost table is
// symmetric, sum_ij W[i][j] Chub[s(i)][s(j)] = sum_ij U[i][j] Chub[s(i)][s(j)].
// 32 x 32 tiles: tile (bx, by) of W and its mirror tile (by, bx) through
// shared memory, so that both reads are coalesced.
__global__ void k_split_bf16_upper(const float* __restrict__ W, __nv_bfloat16* __restrict__ Uhi,
                                   __nv_bfloat16* __restrict__ Ulo, float* __restrict__ Uf, int n, int ldw) {
  __shared__ float mir[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = bx + r, j = by + threadIdx.x;  // mirror tile: rows bx.., columns by..
    mir[r][threadIdx.x] = (i < n && j < n) ? W[(long long)i * ldw + j] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = by + r, j = bx + threadIdx.x;
    if (i >= n || j >= ldw) continue;
    float u = 0.f;
    if (j < n) {
      const float w = W[(long long)i * ldw + j];
      u = j > i ? w + mir[threadIdx.x][r] : (j == i ? w : 0.f);
    }
    const __nv_bfloat16 hi = __float2bfloat16_rn(u);
    Uhi[(long long)i * ldw + j] = hi;
    Ulo[(long long)i * ldw + j] = __float2bfloat16_rn(u - __bfloat162float(hi));
    Uf[(long long)i * ldw + j] = u;
  }
}

// O_i = sum_j W[i][j] (one block per row), fp64 accumulation, fp32 result.
__global__ void k_row_flows(const float* __restrict__ W, int n, int ldw, float* __restrict__ O) {
  __shared__ double red[32];
  const int i = blockIdx.x;
  double s = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) s += (double)W[(long long)i * ldw + j];
  s = block_sum_f64(s, red);
  if (threadIdx.x == 0) O[i] = (float)s;
}

// Total flow sum_i sum_j W[i][j] in fp64: row sums (one block per row), then
// one block adds the rows; the divisor of the per-unit-flow fitness of §4.3.
__global__ void k_row_sums64(const float* __restrict__ W, int n, int ldw, double* __restrict__ rows) {
  __shared__ double red[32];
  const int i = blockIdx.x;
  double s = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) s += (double)W[(long long)i * ldw + j];
  s = block_sum_f64(s, red);
  if (threadIdx.x == 0) rows[i] = s;
}

__global__ void k_sum64(const double* __restrict__ x, int n, double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
  s = block_sum_f64(s, red);
  if (threadIdx.x == 0) *out = s;
}

// D_j = sum_i W[i][j] (one thread per column, coalesced over j).
__global__ void k_col_flows(const float* __restrict__ W, int n, int ldw, float* __restrict__ D) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += (double)W[(long long)i * ldw + j];
  D[j] = (float)s;
}

// Sets *flag when C differs from its transpose anywhere (bitwise compare).
__global__ void k_asymmetry(const float* __restrict__ C, int n, int ldw, uint32_t* flag) {
  const long long total = (long long)n * n;
  bool diff = false;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    if (j > i) diff |= __float_as_uint(C[(long long)i * ldw + j]) != __float_as_uint(C[(long long)j * ldw + i]);
  }
  if (__syncthreads_or(diff) && threadIdx.x == 0) atomicOr(flag, 1u);
}

__global__ void k_transpose(const float* __restrict__ C, float* __restrict__ CT, int n, int ldw) {
  __shared__ float tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = by + r, j = bx + threadIdx.x;
    tile[r][threadIdx.x] = (i < n && j < n) ? C[(long long)i * ldw + j] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = bx + r, i = by + threadIdx.x;
    if (i < n && j < n) CT[(long long)j * ldw + i] = tile[threadIdx.x][r];
  }
}

// d_i = sum_j C[i][j], the "middle node" score of §4.1, correctly rounded to
// fp64: the entries are non-negative fp32 values, so each one is an integer
// multiple of 2^-149 below 2^128 and the row sum is an exact integer count of
// 2^-149 (under 2^292).  Every thread adds its entries' 24-bit significands,
// shifted to their place, into nine 32-bit-aligned 64-bit digits (no digit
// can overflow: each gets at most 2n addends below 2^32), the digits are
// summed over the block (integer addition: exact in any order) and thread 0
// carries them into a 320-bit integer and rounds it once, to nearest with
// ties to even.  The score therefore does not depend on the order of the
// entries: rows that are permutations of each other, and mathematically
// equal sums, tie exactly, and the lower id wins as §4.1's selection asks.
constexpr int kScoreDigits = 9;   // bit 32*k of the sum scaled by 2^149

__device__ double digits_to_double(const unsigned long long (&acc)[kScoreDigits]) {
  uint32_t limb[kScoreDigits + 1];
  unsigned long long carry = 0;
  for (int q = 0; q < kScoreDigits; ++q) {
    const unsigned long long t = acc[q] + carry;
    limb[q] = (uint32_t)t;
    carry = t >> 32;
  }
  limb[kScoreDigits] = (uint32_t)carry;
  int top = kScoreDigits;
  while (top >= 0 && limb[top] == 0u) --top;
  if (top < 0) return 0.0;
  const int L = 32 * top + 32 - __clz(limb[top]);   // bit length of the integer
  auto bit = [&](int q) -> uint32_t { return q < 0 ? 0u : (limb[q >> 5] >> (q & 31)) & 1u; };
  unsigned long long mant = 0;                      // the leading 53 bits (zeros below bit 0)
  for (int q = L - 1; q >= L - 53; --q) mant = (mant << 1) | bit(q);
  int e2 = L - 1 - 149;                             // binary exponent of the leading bit
  if (L > 53 && bit(L - 54)) {                      // round bit set: round up unless an exact tie to even
    bool sticky = false;
    for (int q = L - 55; q >= 0 && !sticky; --q) sticky = bit(q) != 0u;
    if (sticky || (mant & 1ull)) {
      if ((++mant) >> 53) {
        mant >>= 1;
        ++e2;
      }
    }
  }
  // normal for every sum here: -149 <= e2 <= 170
  return __longlong_as_double((long long)(((unsigned long long)(e2 + 1023) << 52) | (mant & ((1ull << 52) - 1))));
}

__global__ void __launch_bounds__(256) k_middle_score(const float* __restrict__ C, int n, int ldw,
                                                      double* __restrict__ d) {
  __shared__ unsigned long long part[8][kScoreDigits];
  const int i = blockIdx.x;
  unsigned long long acc[kScoreDigits];
#pragma unroll
  for (int q = 0; q < kScoreDigits; ++q) acc[q] = 0ull;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const uint32_t bits = __float_as_uint(C[(long long)i * ldw + j]) & 0x7FFFFFFFu;   // -0.0 counts as 0
    const uint32_t e = bits >> 23;
    const uint32_t m = (bits & 0x7FFFFFu) | (e ? 0x800000u : 0u);
    const uint32_t sh = e ? e - 1u : 0u;            // value = m * 2^(sh - 149)
    const unsigned long long v = (unsigned long long)m << (sh & 31u);
    const uint32_t k = sh >> 5, lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
#pragma unroll
    for (int q = 0; q < kScoreDigits; ++q) {
      acc[q] += (q == (int)k) ? lo : 0u;
      acc[q] += (q == (int)k + 1) ? hi : 0u;
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kScoreDigits; ++q) {
    unsigned long long v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) part[w][q] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot[kScoreDigits];
    for (int q = 0; q < kScoreDigits; ++q) {
      tot[q] = 0ull;
      for (int x = 0; x < (int)(blockDim.x >> 5); ++x) tot[q] += part[x][q];
    }
    d[i] = digits_to_double(tot);
  }
}

// Middle-node hubs (§4.1): node i is a hub when fewer than p nodes precede it
// in the order (d, node id), i.e. its rank among the n scores is below p.
// One thread per node counts the nodes before it (scores staged through
// shared memory); a warp covers 32 consecutive nodes, so its ballot is one
// word of the hub mask.
constexpr int kRankThreads = 128, kRankTile = 2048;

__global__ void __launch_bounds__(kRankThreads) k_middle_rank(const double* __restrict__ d, int n, int p, int nw,
                                                             uint32_t* __restrict__ mask) {
  __shared__ double tile[kRankTile];
  const int i = blockIdx.x * kRankThreads + threadIdx.x;
  const double di = i < n ? d[i] : 0.0;
  int rank = 0;
  for (int j0 = 0; j0 < n; j0 += kRankTile) {
    const int cnt = min(kRankTile, n - j0);
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += kRankThreads) tile[j] = d[j0 + j];
    __syncthreads();
    for (int j = 0; j < cnt; ++j) {
      const double x = tile[j];
      rank += (x < di || (x == di && j0 + j < i)) ? 1 : 0;
    }
  }
  const uint32_t word = __ballot_sync(0xffffffffu, i < n && rank < p);
  const int wi = i >> 5;
  if ((threadIdx.x & 31) == 0 && wi < nw) mask[wi] = word;
}

// Ascending hub list of a mask (one warp; prefix counts of the words).
__global__ void k_mask_hubs(const uint32_t* __restrict__ mask, int nw, int32_t* __restrict__ hubs) {
  const int lane = threadIdx.x;
  int base = 0;
  for (int c0 = 0; c0 < nw; c0 += 32) {
    const int x = c0 + lane;
    uint32_t v = x < nw ? mask[x] : 0u;
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

// ---------------------------------------------------------------- launchers
static int grid_for(long long total, int threads) {
  long long g = (total + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return (int)(g < 1 ? 1 : g);
}

void launch_check_values(const float* W, const float* C, int n, int ldw, uint32_t* status, cudaStream_t s) {
  k_check_values<<<grid_for((long long)n * ldw, 256), 256, 0, s>>>(W, C, n, ldw, status);
}

void launch_split_bf16(const float* W, __nv_bfloat16* Whi, __nv_bfloat16* Wlo, long long total, cudaStream_t s) {
  k_split_bf16<<<grid_for(total, 256), 256, 0, s>>>(W, Whi, Wlo, total);
}

void launch_split_bf16_upper(const float* W, __nv_bfloat16* Uhi, __nv_bfloat16* Ulo, float* Uf, int n, int ldw,
                             cudaStream_t s) {
  dim3 grid((ldw + 31) / 32, (n + 31) / 32), block(32, 8);
  k_split_bf16_upper<<<grid, block, 0, s>>>(W, Uhi, Ulo, Uf, n, ldw);
}

void launch_total_flow(const float* W, int n, int ldw, double* rows, double* out, cudaStream_t s) {
  k_row_sums64<<<n, 256, 0, s>>>(W, n, ldw, rows);
  k_sum64<<<1, 256, 0, s>>>(rows, n, out);
}

void launch_flows(const float* W, int n, int ldw, float* O, float* D, cudaStream_t s) {
  k_row_flows<<<n, 256, 0, s>>>(W, n, ldw, O);
  k_col_flows<<<(n + 127) / 128, 128, 0, s>>>(W, n, ldw, D);
}

void launch_asymmetry(const float* C, int n, int ldw, uint32_t* flag, cudaStream_t s) {
  k_asymmetry<<<grid_for((long long)n * n, 256), 256, 0, s>>>(C, n, ldw, flag);
}

void launch_transpose(const float* C, float* CT, int n, int ldw, cudaStream_t s) {
  dim3 grid((n + 31) / 32, (n + 31) / 32), block(32, 8);
  k_transpose<<<grid, block, 0, s>>>(C, CT, n, ldw);
}

void launch_middle_nodes(const float* C, int n, int ldw, int p, double* dscratch, uint32_t* mask,
                         int32_t* hubs, cudaStream_t s) {
  k_middle_score<<<n, 256, 0, s>>>(C, n, ldw, dscratch);
  const int nw = (n + 31) / 32;
  k_middle_rank<<<(n + kRankThreads - 1) / kRankThreads, kRankThreads, 0, s>>>(dscratch, n, p, nw, mask);
  k_mask_hubs<<<1, 32, 0, s>>>(mask, nw, hubs);
}

}  // namespace usaphmp
