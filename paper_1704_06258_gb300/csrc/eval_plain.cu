// Plain FP32 CUDA-core evaluator of the transfer term of objective (1), §3:
//   T3_b = sum_i sum_j W[i][j] * C[h_b(i), h_b(j)]
//        = sum_i sum_j W[i][j] * Chub_b[s_b(i)][s_b(j)],
// with Chub_b[k][l] = C[hubs_b[k], hubs_b[l]] (p x p, in shared memory) and
// s_b the slot codes.  A block takes KB chromosomes and a range of rows; each
// thread owns 4 consecutive columns, keeps their slot codes (as table
// offsets) in registers and streams the rows of W once for all KB
// chromosomes: per (pair, chromosome) one shared-memory gather and one FMA.
// For symmetric C the rows of W are those of the folded U = W + W^T on and
// above the diagonal (0 below): each pair (i, j), (j, i) costs one gather,
// and a thread's column chunk stops at its diagonal row.
// Partial sums go to part[row_split][b]; the reduction kernel adds them in a
// fixed order.  Rows are summed in chunks of 32 before joining the running
// sum, which keeps the fp32 error near (32 + n/32) ulp instead of n ulp.
#include "common.cuh"
#include "kernels.cuh"

#include <algorithm>

namespace usaphmp {

namespace {

constexpr int kThreads = 256;

__host__ __device__ inline int plain_tpr(int need) {
  // threads per row: enough to cover `need` column chunks, power of two
  int t = 32;
  while (t < need && t < kThreads) t <<= 1;
  return t;
}

inline int plain_kb(int p, int ns) {
  // chromosomes per block: as many as the shared memory comfortably holds
  for (int kb : {8, 4, 2, 1}) {
    const size_t bytes = (size_t)kb * p * p * 4 + (size_t)kb * ns;
    if (bytes <= 96 * 1024) return kb;
  }
  return 1;
}

inline size_t plain_smem(int kb, int p, int ns) {
  if (plain_global_table(p, ns)) return (size_t)ns;  // kb is 1 then
  return (size_t)round_up(kb * p * p * 4, 16) + (size_t)kb * ns;
}

// One chromosome whose hub-cost table is too large for shared memory: the
// same sums, gathering Chub_b[s_b(i)][s_b(j)] from its chub rows in global
// memory (L2-resident, row stride hst).
__device__ __forceinline__ float plain_global_sum(const float* __restrict__ W, const float* __restrict__ chub,
                                                  const uint8_t* sl, int n, int ldw, int hst, int r0, int r1,
                                                  int tpr, int G, int grp, int c4) {
  float acc = 0.f;
  for (int cb = c4; cb < ldw / 4; cb += tpr) {
    const int j0 = cb * 4;
    int cj[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) cj[c] = (j0 + c < n) ? (int)sl[j0 + c] : 0;
    for (int i = r0 + grp; i < r1; i += 32 * G) {
      float part = 0.f;
      const int iend = min(r1, i + 32 * G);
      for (int ii = i; ii < iend; ii += G) {
        const float4 w = __ldg(reinterpret_cast<const float4*>(W + (long long)ii * ldw + j0));
        const float* row = chub + (int)sl[ii] * hst;
        part = fmaf(w.x, __ldg(row + cj[0]), part);
        part = fmaf(w.y, __ldg(row + cj[1]), part);
        part = fmaf(w.z, __ldg(row + cj[2]), part);
        part = fmaf(w.w, __ldg(row + cj[3]), part);
      }
      acc += part;
    }
  }
  return acc;
}

// The KB slot codes of one node (node-major layout, KB-byte aligned).
template <int KB>
__device__ __forceinline__ unsigned long long node_codes(const uint8_t* q) {
  if constexpr (KB == 8) return *reinterpret_cast<const unsigned long long*>(q);
  else if constexpr (KB == 4) return *reinterpret_cast<const uint32_t*>(q);
  else if constexpr (KB == 2) return *reinterpret_cast<const uint16_t*>(q);
  else return *q;
}

}  // namespace

template <int KB>
__global__ void __launch_bounds__(kThreads, 2) k_eval_plain(const __grid_constant__ TaskParam tp) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ float red[kThreads / 32];
  pdl_wait();
  pdl_allow_next();
  const int t = task_of(tp.bo, blockIdx.x);
  const Task& T = task_at(tp, t);
  const int n = T.in.n, p = T.in.p, ldw = T.in.ldw, ns = T.in.ns, B = T.pop.B;
  const int nrs = T.pop.npart;
  const int local = blockIdx.x - tp.bo.o[t];
  const int group = local / nrs, rs = local - group * nrs;
  const int b0 = group * KB;
  const int nb = min(KB, B - b0);
  const int pp = p * p;
  const bool gtab = KB == 1 && plain_global_table(p, ns);
  float* tab = reinterpret_cast<float*>(sm);
  uint8_t* sl = gtab ? sm : sm + round_up(KB * pp * 4, 16);
  const float* __restrict__ C = T.in.C;
  const float* __restrict__ W = T.in.W;
  const int32_t* __restrict__ hubs = T.pop.hubs;

  // hub-path routing: the allocation kernel left the routed table in chub
  const bool routed = T.in.routing != 0;
  const int hst = chub_hstride(p), cst = chub_cstride(p);
  for (int e = threadIdx.x; !gtab && e < KB * pp; e += kThreads) {
    const int bb = e / pp, r = e - bb * pp, k = r / p, l = r - k * p;
    float v = 0.f;
    if (bb < nb) {
      const int32_t* hb = hubs + (long long)(b0 + bb) * p;
      v = routed ? T.pop.chub[(long long)(b0 + bb) * cst + k * hst + l] : C[(long long)hb[k] * ldw + hb[l]];
    }
    tab[e] = v;
  }
  // slot codes node-major: sl[j * KB + bb], the KB codes of one node in one
  // KB-byte word (one shared load per row for all chromosomes of the block)
  {
    const uint8_t* __restrict__ src = T.pop.slot + (long long)b0 * ns;
    for (int e = threadIdx.x; e < KB * ns; e += kThreads) {
      const int j = e / KB, bb = e - j * KB;
      sl[e] = (bb < nb) ? src[(long long)bb * ns + j] : (uint8_t)0;
    }
  }
  __syncthreads();

  const int chunk = (n + nrs - 1) / nrs;
  const int r0 = rs * chunk, r1 = min(n, r0 + chunk);
  // Folded operand (symmetric C): U is zero below the diagonal, so column
  // chunk j0..j0+3 needs rows up to j0+3 only; a thread takes a chunk and its
  // mirror (cols4 - 1 - chunk), which together span n rows.
  const bool fold = !gtab && T.in.Ufold != nullptr;
  const float* __restrict__ Wm = fold ? T.in.Ufold : W;
  const int cols4 = ldw / 4;
  const int nchunk = fold ? (cols4 + 1) / 2 : cols4;
  const int tpr = plain_tpr(nchunk);
  const int G = kThreads / tpr;
  const int grp = threadIdx.x / tpr, c4 = threadIdx.x - grp * tpr;

  float acc[KB];
#pragma unroll
  for (int bb = 0; bb < KB; ++bb) acc[bb] = 0.f;
  if (gtab)
    acc[0] = plain_global_sum(W, T.pop.chub + (long long)b0 * chub_cstride(p), sl, n, ldw, chub_hstride(p), r0, r1,
                              tpr, G, grp, c4);

  for (int cp = c4; !gtab && cp < nchunk; cp += tpr)
  for (int side = 0; side < (fold ? 2 : 1); ++side) {
    const int cb = side == 0 ? cp : cols4 - 1 - cp;
    if (side == 1 && cb <= cp) break;  // the middle chunk of an odd count: once
    const int j0 = cb * 4;
    const int rend = fold ? min(r1, j0 + 4) : r1;
    int coff[KB][4];
#pragma unroll
    for (int bb = 0; bb < KB; ++bb)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = j0 + c;
        coff[bb][c] = bb * pp + ((j < n) ? (int)sl[j * KB + bb] : 0);
      }
    for (int i = r0 + grp; i < rend; i += 32 * G) {
      float part[KB];
#pragma unroll
      for (int bb = 0; bb < KB; ++bb) part[bb] = 0.f;
      const int iend = min(rend, i + 32 * G);
      // rows ascending; the W loads of four rows are issued before their sums
      auto row_sum = [&](const float4& w, int ii) {
        const unsigned long long codes = node_codes<KB>(sl + ii * KB);
#pragma unroll
        for (int bb = 0; bb < KB; ++bb) {
          const float* row = tab + (int)((codes >> (8 * bb)) & 0xFFu) * p;
          float s = part[bb];
          s = fmaf(w.x, row[coff[bb][0]], s);
          s = fmaf(w.y, row[coff[bb][1]], s);
          s = fmaf(w.z, row[coff[bb][2]], s);
          s = fmaf(w.w, row[coff[bb][3]], s);
          part[bb] = s;
        }
      };
      int ii = i;
      for (; ii + 3 * G < iend; ii += 4 * G) {
        float4 w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) w[u] = __ldg(reinterpret_cast<const float4*>(Wm + (long long)(ii + u * G) * ldw + j0));
#pragma unroll
        for (int u = 0; u < 4; ++u) row_sum(w[u], ii + u * G);
      }
      for (; ii < iend; ii += G) row_sum(__ldg(reinterpret_cast<const float4*>(Wm + (long long)ii * ldw + j0)), ii);
#pragma unroll
      for (int bb = 0; bb < KB; ++bb) acc[bb] += part[bb];
    }
  }

#pragma unroll
  for (int bb = 0; bb < KB; ++bb) {
    const float s = block_sum(acc[bb], red);
    if (threadIdx.x == 0 && bb < nb) T.pop.part[(long long)rs * B + b0 + bb] = s;
  }
}

int plain_rows(int n, int /*B*/) {
  // Row splits (blocks per chromosome group, partial sums per chromosome)
  // grow with n only -- one per 512 rows, a power of two, at most 8 -- so a
  // chromosome's partial sums, and so its fitness bits, do not depend on the
  // size of the batch it is evaluated in.
  int rs = 1;
  while (rs < 8 && rs * 2 * 512 <= n) rs <<= 1;
  return rs;
}

void launch_eval_plain(const TaskSet& ts, cudaStream_t s) {
  // Tasks of one launch share the block shape; KB is chosen for the largest.
  int kb = 8;
  size_t smem = 0;
  for (int t = 0; t < ts.count; ++t) kb = std::min(kb, plain_kb(ts.h[t].in.p, ts.h[t].in.ns));
  TaskParam tp = make_param(ts);
  for (int t = 0; t < ts.count; ++t) {
    const Task& T = ts.h[t];
    const int groups = (T.pop.B + kb - 1) / kb;
    tp.bo.o[t + 1] = tp.bo.o[t] + groups * T.pop.npart;
    smem = std::max(smem, plain_smem(kb, T.in.p, T.in.ns));
  }
  const int blocks = tp.bo.o[ts.count];
  if (blocks == 0) return;
  switch (kb) {
#define USAPHMP_PLAIN_CASE(K)                                 \
  case K:                                                     \
    launch_pdl(k_eval_plain<K>, blocks, kThreads, smem, s, tp); \
    break;
    USAPHMP_PLAIN_CASE(8)
    USAPHMP_PLAIN_CASE(4)
    USAPHMP_PLAIN_CASE(2)
    USAPHMP_PLAIN_CASE(1)
#undef USAPHMP_PLAIN_CASE
  }
}

template <class K>
static void raise_smem_limit(K kernel, int max_smem) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - (int)fa.sharedSizeBytes);
}

void prepare_eval_plain(int max_smem) {
  raise_smem_limit(k_eval_plain<8>, max_smem);
  raise_smem_limit(k_eval_plain<4>, max_smem);
  raise_smem_limit(k_eval_plain<2>, max_smem);
  raise_smem_limit(k_eval_plain<1>, max_smem);
}

}  // namespace usaphmp
