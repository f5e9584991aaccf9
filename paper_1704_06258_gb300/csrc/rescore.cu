// FP64 rescoring of chromosomes by the pair form of objective (1), §3:
//   cost = sum_i sum_j W[i][j] * (chi*C[i,h(i)] + alpha*T[h(i),h(j)] + delta*C[h(j),j]),
// every product and sum in fp64 from the fp32 instance values and the fp64
// factors chi, alpha, delta as the caller gave them, with T = C
// (direct hub arc) or, for hub-path routing (eq. 4), T = the cheapest path
// over arcs between the chromosome's open hubs (Floyd-Warshall in fp64,
// zero on the diagonal).  It shares no arithmetic with the fp32 and
// split-bf16 evaluators and is used for the returned objective of a solve
// and for the error of the fast paths.
#include "common.cuh"
#include "kernels.cuh"

namespace usaphmp {

namespace {
constexpr int kParts = 128;
}

// dist[b][a][c] = cheapest path from hub a to hub c of chromosome b over its
// hub arcs, fp64; one block per chromosome, one pass per intermediate hub
// (row and column m are fixed during pass m: zero diagonal, costs >= 0).
__global__ void __launch_bounds__(256) k_hub_paths64(DevInst in, const int32_t* __restrict__ hubs,
                                                    double* __restrict__ dist) {
  __shared__ int hs[256];
  const int b = blockIdx.x, n = in.n, p = in.p, ldw = in.ldw;
  for (int k = threadIdx.x; k < p; k += blockDim.x) {
    const int v = hubs[(long long)b * p + k];
    hs[k] = (v >= 0 && v < n) ? v : 0;
  }
  __syncthreads();
  double* d = dist + (long long)b * p * p;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int a = e / p, c = e - a * p;
    d[e] = (a == c) ? 0.0 : (double)in.C[(long long)hs[a] * ldw + hs[c]];
  }
  __syncthreads();
  for (int m = 0; m < p; ++m) {
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
      const int a = e / p, c = e - a * p;
      const double v = d[a * p + m] + d[m * p + c];
      if (v < d[e]) d[e] = v;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_rescore_part(DevInst in, const int32_t* __restrict__ hubs,
                                                     const uint8_t* __restrict__ slot, const double* dist,
                                                     double* __restrict__ part) {
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
  const double chi = in.chi_d, alpha = in.alpha_d, delta = in.delta_d;
  const double* db = dist ? dist + (long long)b * p * p : nullptr;
  double s = 0.0;
  for (int i = i0; i < i1; ++i) {
    const int si = min((int)sl[i], p - 1);
    const int hi = hs[si];
    const double collect = chi * (double)in.C[(long long)i * ldw + hi];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const int sj = min((int)sl[j], p - 1);
      const int hj = hs[sj];
      const double leg = db ? db[si * p + sj] : (double)in.C[(long long)hi * ldw + hj];
      const double path = collect + alpha * leg + delta * (double)in.C[(long long)hj * ldw + j];
      s += (double)in.W[(long long)i * ldw + j] * path;
    }
  }
  s = block_sum_f64(s, red);
  if (threadIdx.x == 0) part[(long long)b * nparts + part_idx] = s;
}

__global__ void k_rescore_final(const double* __restrict__ part, int nparts, int B, double scale,
                                double* __restrict__ cost) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double s = 0.0;
  for (int k = 0; k < nparts; ++k) s += part[(long long)b * nparts + k];
  cost[b] = s * scale;
}

int rescore_parts(int n) { return n < kParts ? n : kParts; }

__global__ void k_fit_from_fp64(const double* __restrict__ cost, float* __restrict__ fit, int B, float scale) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) fit[b] = (float)cost[b] * scale;
}

void launch_fit_from_fp64(const double* cost, float* fit, int B, float scale, cudaStream_t s) {
  if (B > 0) k_fit_from_fp64<<<(B + 255) / 256, 256, 0, s>>>(cost, fit, B, scale);
}

void launch_rescore(const DevInst& in, int B, const int32_t* hubs, const uint8_t* slot,
                    double* part, double* cost, cudaStream_t s, double* dist, double scale) {
  if (B <= 0) return;
  const int np = rescore_parts(in.n);
  const bool routed = in.routing != 0 && dist != nullptr;
  if (routed) k_hub_paths64<<<B, 256, 0, s>>>(in, hubs, dist);
  k_rescore_part<<<dim3(np, B), 256, 0, s>>>(in, hubs, slot, routed ? dist : nullptr, part);
  k_rescore_final<<<(B + 127) / 128, 128, 0, s>>>(part, np, B, scale, cost);
}

}  // namespace usaphmp
