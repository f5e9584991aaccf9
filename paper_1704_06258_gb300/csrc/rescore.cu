// FP64 rescoring of chromosomes by the pair form of objective (1), §3:
//   cost = sum_i sum_j W[i][j] * (chi*C[i,h(i)] + alpha*C[h(i),h(j)] + delta*C[h(j),j]),
// every product and sum in fp64 from the fp32 instance values.  It shares no
// arithmetic with the fp32 and split-bf16 evaluators and is used for the
// returned objective of a solve and for the error of the fast paths.
#include "common.cuh"
#include "kernels.cuh"

namespace usaphmp {

namespace {
constexpr int kParts = 128;
}

__global__ void __launch_bounds__(256) k_rescore_part(DevInst in, const int32_t* __restrict__ hubs,
                                                     const uint8_t* __restrict__ slot, double* __restrict__ part) {
  __shared__ int hs[256];
  __shared__ double red[8];
  const int b = blockIdx.y, part_idx = blockIdx.x, nparts = gridDim.x;
  const int n = in.n, p = in.p, ldw = in.ldw;
  // Inputs are trusted (canonical form); out-of-range entries are clamped so
  // that a bad caller buffer cannot make the kernel read outside C.
  for (int k = threadIdx.x; k < p; k += blockDim.x) {
    const int v = hubs[(long long)b * p + k];
    hs[k] = (v >= 0 && v < n) ? v : 0;
  }
  for (int k = p + threadIdx.x; k < 256; k += blockDim.x) hs[k] = 0;
  __syncthreads();
  const uint8_t* sl = slot + (long long)b * in.ns;
  const int chunk = (n + nparts - 1) / nparts;
  const int i0 = part_idx * chunk, i1 = min(n, i0 + chunk);
  const double chi = in.chi, alpha = in.alpha, delta = in.delta;
  double s = 0.0;
  for (int i = i0; i < i1; ++i) {
    const int hi = hs[sl[i]];
    const double collect = chi * (double)in.C[(long long)i * ldw + hi];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const int hj = hs[sl[j]];
      const double path = collect + alpha * (double)in.C[(long long)hi * ldw + hj] +
                          delta * (double)in.C[(long long)hj * ldw + j];
      s += (double)in.W[(long long)i * ldw + j] * path;
    }
  }
  s = block_sum_f64(s, red);
  if (threadIdx.x == 0) part[(long long)b * nparts + part_idx] = s;
}

__global__ void k_rescore_final(const double* __restrict__ part, int nparts, int B, double* __restrict__ cost) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double s = 0.0;
  for (int k = 0; k < nparts; ++k) s += part[(long long)b * nparts + k];
  cost[b] = s;
}

int rescore_parts(int n) { return n < kParts ? n : kParts; }

void launch_rescore(const DevInst& in, int B, const int32_t* hubs, const uint8_t* slot,
                    double* part, double* cost, cudaStream_t s) {
  if (B <= 0) return;
  const int np = rescore_parts(in.n);
  k_rescore_part<<<dim3(np, B), 256, 0, s>>>(in, hubs, slot, part);
  k_rescore_final<<<(B + 127) / 128, 128, 0, s>>>(part, np, B, cost);
}

}  // namespace usaphmp
