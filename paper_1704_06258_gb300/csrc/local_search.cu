// Allocation local search for fixed hubs, in fp64: sweeps over the spokes in
// ascending node order; spoke i moves from its hub a to the open hub b with
// the most negative change of objective (1), §3 (the lowest hub on equal
// changes), when that change is negative; sweeps repeat until one moves
// nothing or max_sweeps have run.  Hubs keep serving themselves (eq. 3).
//
// With M[u][l] = sum_j W[u][j] [s(j) = l] and N[u][l] = sum_j W[j][u] [s(j) = l]
// (the flows of node u to and from the spokes of hub slot l) and T the
// transfer-leg costs between hub slots (C between hubs, or the hub-path
// table), the change of moving spoke i from slot a to slot b is
//   chi O_i (C[i,h_b] - C[i,h_a]) + delta D_i (C[h_b,i] - C[h_a,i])
//   + alpha sum_l (M'[i][l] (T[b][l] - T[a][l]) + N'[i][l] (T[l][b] - T[l][a]))
//   + alpha W_ii (T[b][b] - T[a][a]),
// M' and N' leaving out the pair (i, i); O_i = sum_l M[i][l] and
// D_i = sum_l N[i][l].  After a move, column i of W moves between columns a
// and b of M and row i of W between those of N.
//
// One block per chromosome; M, N and T live in a per-chromosome fp64 scratch.
#include "common.cuh"
#include "kernels.cuh"

namespace usaphmp {

namespace {
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
}

__host__ __device__ inline size_t scratch_doubles(int n, int p) { return 2 * (size_t)n * p + (size_t)p * p; }

size_t local_search_scratch_doubles(int n, int p) { return scratch_doubles(n, p); }

__global__ void __launch_bounds__(kThreads) k_local_search(DevInst in, const int32_t* __restrict__ hubs,
                                                           uint8_t* __restrict__ slot, int max_sweeps,
                                                           double* __restrict__ scratch, int32_t* moves_out,
                                                           int32_t* sweeps_out) {
  __shared__ int hs[256];
  __shared__ double dlt[256];
  __shared__ int decision;
  const int b = blockIdx.x, n = in.n, p = in.p, ldw = in.ldw;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* __restrict__ W = in.W;
  const float* __restrict__ C = in.C;
  for (int k = tid; k < p; k += kThreads) {
    const int v = hubs[(long long)b * p + k];
    hs[k] = (v >= 0 && v < n) ? v : 0;
  }
  uint8_t* sl = slot + (long long)b * in.ns;
  double* M = scratch + (long long)b * scratch_doubles(n, p);
  double* N = M + (size_t)n * p;
  double* T = N + (size_t)n * p;
  __syncthreads();

  // T: hub-to-hub leg costs; the hub-path table (Floyd-Warshall, zero
  // diagonal) under hub-path routing.
  for (int e = tid; e < p * p; e += kThreads) {
    const int a = e / p, c = e - a * p;
    T[e] = (in.routing && a == c) ? 0.0 : (double)C[(long long)hs[a] * ldw + hs[c]];
  }
  __syncthreads();
  if (in.routing) {
    for (int m = 0; m < p; ++m) {
      for (int e = tid; e < p * p; e += kThreads) {
        const int a = e / p, c = e - a * p;
        const double v = T[a * p + m] + T[m * p + c];
        if (v < T[e]) T[e] = v;
      }
      __syncthreads();
    }
  }

  // M and N in fixed order: thread u owns rows M[u][.] and N[u][.].
  for (int u = tid; u < n; u += kThreads) {
    double* mu = M + (size_t)u * p;
    double* nu = N + (size_t)u * p;
    for (int l = 0; l < p; ++l) {
      mu[l] = 0.0;
      nu[l] = 0.0;
    }
    for (int j = 0; j < n; ++j) {
      const int s = min((int)sl[j], p - 1);
      mu[s] += (double)W[(long long)u * ldw + j];
      nu[s] += (double)W[(long long)j * ldw + u];
    }
  }
  __syncthreads();

  const double chi = in.chi_d, alpha = in.alpha_d, delta = in.delta_d;
  int moves = 0, sweeps = 0;
  for (int sw = 0; sw < max_sweeps; ++sw) {
    ++sweeps;
    bool moved = false;
    for (int i = 0; i < n; ++i) {
      const int a = min((int)sl[i], p - 1);
      if (hs[a] == i) continue;  // a hub serves itself (same answer in every thread)
      const double* mi = M + (size_t)i * p;
      const double* ni = N + (size_t)i * p;
      const double wii = (double)W[(long long)i * ldw + i];
      // change for every candidate slot c: warp w takes c = w, w + 8, ...
      for (int c = warp; c < p; c += kWarps) {
        double t = 0.0;
        if (c != a) {
          for (int l = lane; l < p; l += 32) {
            const double ml = mi[l] - (l == a ? wii : 0.0), nl = ni[l] - (l == a ? wii : 0.0);
            t += ml * (T[c * p + l] - T[a * p + l]) + nl * (T[l * p + c] - T[l * p + a]);
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) {
          double oi = 0.0, di = 0.0;
          for (int l = 0; l < p; ++l) {
            oi += mi[l];
            di += ni[l];
          }
          const int hc = hs[c], ha = hs[a];
          const double acc = chi * oi * ((double)C[(long long)i * ldw + hc] - (double)C[(long long)i * ldw + ha]) +
                             delta * di * ((double)C[(long long)hc * ldw + i] - (double)C[(long long)ha * ldw + i]);
          dlt[c] = (c == a) ? 0.0 : acc + alpha * (t + wii * (T[c * p + c] - T[a * p + a]));
        }
      }
      __syncthreads();
      if (tid == 0) {
        int best = -1;
        double bd = 0.0;
        for (int c = 0; c < p; ++c)
          if (c != a && dlt[c] < bd) {
            bd = dlt[c];
            best = c;
          }
        decision = best;
        if (best >= 0) sl[i] = (uint8_t)best;
      }
      __syncthreads();
      const int nb = decision;
      if (nb >= 0) {
        for (int u = tid; u < n; u += kThreads) {
          const double wui = (double)W[(long long)u * ldw + i], wiu = (double)W[(long long)i * ldw + u];
          M[(size_t)u * p + a] -= wui;
          M[(size_t)u * p + nb] += wui;
          N[(size_t)u * p + a] -= wiu;
          N[(size_t)u * p + nb] += wiu;
        }
        ++moves;
        moved = true;
        __syncthreads();
      }
    }
    if (!moved) break;
  }
  if (tid == 0) {
    if (moves_out) moves_out[b] = moves;
    if (sweeps_out) sweeps_out[b] = sweeps;
  }
}

void launch_local_search(const DevInst& in, int B, const int32_t* hubs, uint8_t* slot, int max_sweeps,
                         double* scratch, int32_t* moves, int32_t* sweeps, cudaStream_t s) {
  if (B <= 0) return;
  k_local_search<<<B, kThreads, 0, s>>>(in, hubs, slot, max_sweeps, scratch, moves, sweeps);
}

}  // namespace usaphmp
