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

// d_i = sum_j C[i][j] in fp64: the "middle node" score of §4.1.
__global__ void k_middle_score(const float* __restrict__ C, int n, int ldw, double* __restrict__ d) {
  __shared__ double red[32];
  const int i = blockIdx.x;
  double s = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) s += (double)C[(long long)i * ldw + j];
  s = block_sum_f64(s, red);
  if (threadIdx.x == 0) d[i] = s;
}

// One block: the p nodes with the smallest d (lower node id on ties) become
// the hubs of the initial solution; writes the mask and the ascending hubs.
__global__ void k_middle_select(const double* __restrict__ d, int n, int p, int nw,
                                uint32_t* __restrict__ mask, int32_t* __restrict__ hubs) {
  extern __shared__ uint32_t taken[];   // nw words
  __shared__ double bv[32];
  __shared__ int bi[32];
  for (int w = threadIdx.x; w < nw; w += blockDim.x) taken[w] = 0u;
  __syncthreads();
  for (int r = 0; r < p; ++r) {
    double v = 1e308;
    int idx = 0x7fffffff;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if (taken[i >> 5] & (1u << (i & 31))) continue;
      const double x = d[i];
      if (x < v || (x == v && i < idx)) { v = x; idx = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (ov < v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = v; bi[threadIdx.x >> 5] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double bestv = bv[0];
      int besti = bi[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (bv[w] < bestv || (bv[w] == bestv && bi[w] < besti)) { bestv = bv[w]; besti = bi[w]; }
      taken[besti >> 5] |= 1u << (besti & 31);
    }
    __syncthreads();
  }
  for (int w = threadIdx.x; w < nw; w += blockDim.x) mask[w] = taken[w];
  if (threadIdx.x == 0) {
    int k = 0;
    for (int i = 0; i < n && k < p; ++i)
      if (taken[i >> 5] & (1u << (i & 31))) hubs[k++] = i;
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
  k_middle_select<<<1, 1024, nw * sizeof(uint32_t), s>>>(dscratch, n, p, nw, mask, hubs);
}

}  // namespace usaphmp
