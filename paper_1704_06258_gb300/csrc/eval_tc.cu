// Split-bf16 tensor-core evaluator of the transfer term of objective (1), §3.
//
// For chromosome b with slot codes s_b and one-hot allocation matrix
// A_b[j][l] = [s_b(j) == l] (n x p), the transfer term is
//   T3_b = sum_i sum_l M_b[i][l] * Chub_b[s_b(i)][l],   M_b = W A_b,
// i.e. the inner sum over j of objective (1) grouped by the hub serving j.
// All chromosomes of a launch are packed side by side as the columns
// (b, l) -> b*p + l of one GEMM  D = W [A_1 .. A_B]  (n x n times n x B*p):
//   * W enters as two bf16 operands, W = Whi + Wlo + O(2^-17 |W|), loaded by
//     TMA with the 128-byte swizzle; both are multiplied by the same one-hot
//     operand and accumulated into one fp32 TMEM tile (tcgen05.mma, kind::f16);
//   * the one-hot operand is never stored in global memory: producer warps
//     expand it from the u8 slot codes straight into shared memory, in the
//     same swizzled K-major layout;
//   * the epilogue reads the accumulator from TMEM, multiplies each element
//     D[i][(b,l)] by Chub_b[s_b(i)][l] = chubT[b][l][s_b(i)] and sums the 32
//     rows held by each warp with a fixed butterfly, writing one partial per
//     (32-row group, column); D itself never leaves the SM.
// Persistent kernel, one CTA per SM, warp roles: 0 TMA, 1 MMA (+ TMEM
// allocation), 4-7 epilogue (TMEM lane quarters 0-3), 8-15 one-hot
// producers.  Tiles are 128 rows x 256 columns x 64-deep K blocks, three
// shared-memory stages, two TMEM accumulators (512 columns) so the epilogue of
// one tile overlaps the MMAs of the next.  Every wait is bounded: after
// kTimeoutNs the kernel raises kStatusTimeout, drains its own copies and
// MMAs, frees TMEM and returns.
#include "common.cuh"
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace usaphmp {

namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 3;
constexpr int kThreads = 512;
constexpr uint32_t A_BYTES = BM * BK * 2;                 // 16 KB
constexpr uint32_t B_BYTES = BN * BK * 2;                 // 32 KB
constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + B_BYTES;   // 64 KB
constexpr uint32_t TMEM_COLS = 2 * BN;
constexpr int kTblChrom = 96;                              // chromosomes per tile kept in the epilogue table
constexpr uint32_t kTblOffset = STAGES * STAGE_BYTES;      // u8 [4 warps][kTblChrom][32 rows]
constexpr uint32_t kTblBytes = 4 * kTblChrom * 32;
constexpr uint32_t kBarOffset = kTblOffset + kTblBytes;
constexpr int kNumBars = 3 * STAGES + 5;
constexpr size_t kSmemBytes = 1024 + kBarOffset + 8 * kNumBars + 16;
constexpr uint64_t kTimeoutNs = 2000000000ull;
constexpr uint32_t IDESC = ptx::idesc_bf16_f32(BM, BN);

struct Bars {
  uint32_t base;
  __device__ uint32_t full_tma(int s) const { return base + 8 * s; }
  __device__ uint32_t full_oh(int s) const { return base + 8 * (STAGES + s); }
  __device__ uint32_t empty(int s) const { return base + 8 * (2 * STAGES + s); }
  __device__ uint32_t tfull(int b) const { return base + 8 * (3 * STAGES + b); }
  __device__ uint32_t tempty(int b) const { return base + 8 * (3 * STAGES + 2 + b); }
  __device__ uint32_t drain() const { return base + 8 * (3 * STAGES + 4); }
};

// Single-thread bounded wait.  Returns false on timeout or when another role
// has already aborted.
__device__ bool wait_one(uint32_t bar, uint32_t parity, volatile int* abort_flag, uint32_t* status) {
  if (ptx::mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = ptx::globaltimer();
  for (uint32_t i = 1;; ++i) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 0) {
      if (*abort_flag) return false;
      if (ptx::globaltimer() - t0 > kTimeoutNs) {
        *abort_flag = 1;
        atomicOr(status, kStatusTimeout);
        return false;
      }
    }
  }
}

// Bounded wait that ignores the abort flag (used only while draining).
__device__ void wait_drain(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = ptx::globaltimer();
  while (!ptx::mbar_try_wait(bar, parity))
    if (ptx::globaltimer() - t0 > kTimeoutNs) return;
}

// Warp-collective bounded wait: every lane returns the same answer.
__device__ bool wait_warp(uint32_t bar, uint32_t parity, volatile int* abort_flag, uint32_t* status) {
  const uint64_t t0 = ptx::globaltimer();
  for (uint32_t i = 0;; ++i) {
    const bool ok = ptx::mbar_try_wait(bar, parity);
    if (__all_sync(0xffffffffu, ok)) return true;
    if ((i & 255u) == 255u) {
      int stop = 0;
      if ((threadIdx.x & 31) == 0) {
        stop = *abort_flag;
        if (!stop && ptx::globaltimer() - t0 > kTimeoutNs) {
          *abort_flag = 1;
          atomicOr(status, kStatusTimeout);
          stop = 1;
        }
      }
      if (__shfl_sync(0xffffffffu, stop, 0)) return false;
    }
  }
}

struct TileRef {
  int task, m, nb;
};

__device__ __forceinline__ TileRef decode_tile(const TaskParam& tp, int g) {
  TileRef r;
  r.task = task_of(tp.bo, g);
  const Task& T = task_at(tp, r.task);
  const int local = g - tp.bo.o[r.task];
  const int Bp = T.pop.B * T.in.p;
  const int nt = (Bp + BN - 1) / BN;
  r.m = local / nt;
  r.nb = local - r.m * nt;
  return r;
}

// 8 slot codes (two words) -> 8 bf16 values, 1.0 where the code equals l.
__device__ __forceinline__ uint4 onehot8(uint32_t w0, uint32_t w1, uint32_t lrep) {
  const uint32_t m0 = __vcmpeq4(w0, lrep), m1 = __vcmpeq4(w1, lrep);
  uint4 o;
  o.x = __byte_perm(m0, 0u, 0x1100) & 0x3F803F80u;
  o.y = __byte_perm(m0, 0u, 0x3322) & 0x3F803F80u;
  o.z = __byte_perm(m1, 0u, 0x1100) & 0x3F803F80u;
  o.w = __byte_perm(m1, 0u, 0x3322) & 0x3F803F80u;
  return o;
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}

// Lane L ends with the sum over the 32 lanes of v[L] (fixed butterfly order).
__device__ __forceinline__ float transpose_sum32(float* v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    const bool upper = (lane & step) != 0;
#pragma unroll
    for (int c = 0; c < step; ++c) {
      const float send = upper ? v[c] : v[c + step];
      const float keep = upper ? v[c + step] : v[c];
      v[c] = keep + __shfl_xor_sync(0xffffffffu, send, step);
    }
  }
  return v[0];
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 1)
    k_eval_tc(const __grid_constant__ TaskParam tp, int total_tiles, uint32_t* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw = ptx::smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sm = smem_raw + (base - raw);
  const Bars bars{base + kBarOffset};
  volatile uint32_t* tmem_holder = reinterpret_cast<volatile uint32_t*>(sm + kBarOffset + 8 * kNumBars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + kBarOffset + 8 * kNumBars + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(bars.full_tma(s), 1);
      ptx::mbar_init(bars.full_oh(s), 256);
      ptx::mbar_init(bars.empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(bars.tfull(b), 1);
      ptx::mbar_init(bars.tempty(b), 128);
    }
    ptx::mbar_init(bars.drain(), 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(ptx::smem_u32(const_cast<uint32_t*>(tmem_holder)), TMEM_COLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ TMA producer
    int it = 0;
    bool ok = true;
    for (int g = blockIdx.x; g < total_tiles && ok; g += gridDim.x) {
      const TileRef tr = decode_tile(tp, g);
      const Task& T = task_at(tp, tr.task);
      const int nk = (T.in.n + BK - 1) / BK;
      for (int kb = 0; kb < nk; ++kb, ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
        if (!(ok = wait_one(bars.empty(s), ph ^ 1u, abort_flag, status))) break;
        const uint32_t a_hi = base + s * STAGE_BYTES;
        ptx::mbar_arrive_expect_tx(bars.full_tma(s), 2 * A_BYTES);
        ptx::tma_load_2d(a_hi, T.tmap_hi, kb * BK, tr.m * BM, bars.full_tma(s));
        ptx::tma_load_2d(a_hi + A_BYTES, T.tmap_lo, kb * BK, tr.m * BM, bars.full_tma(s));
      }
    }
    for (int j = it - STAGES < 0 ? 0 : it - STAGES; j < it; ++j)
      wait_drain(bars.full_tma(j % STAGES), (uint32_t)(j / STAGES) & 1u);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------- MMA issuer
    int it = 0, tl = 0;
    bool ok = true;
    for (int g = blockIdx.x; g < total_tiles && ok; g += gridDim.x, ++tl) {
      const TileRef tr = decode_tile(tp, g);
      const int nk = (task_at(tp, tr.task).in.n + BK - 1) / BK;
      const int buf = tl & 1;
      const uint32_t use = (uint32_t)(tl >> 1);
      if (!(ok = wait_one(bars.tempty(buf), (use & 1u) ^ 1u, abort_flag, status))) break;
      ptx::tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(buf * BN);
      for (int kb = 0; kb < nk; ++kb, ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
        if (!(ok = wait_one(bars.full_tma(s), ph, abort_flag, status))) break;
        if (!(ok = wait_one(bars.full_oh(s), ph, abort_flag, status))) break;
        ptx::tc_fence_after();
        const uint32_t a_hi = base + s * STAGE_BYTES, a_lo = a_hi + A_BYTES, bt = a_lo + A_BYTES;
#pragma unroll
        for (int k = 0; k < BK / 16; ++k) {
          const uint64_t bdesc = ptx::sw128_desc(bt + 32 * k);
          ptx::mma_bf16(d, ptx::sw128_desc(a_hi + 32 * k), bdesc, IDESC, (kb | k) != 0);
          ptx::mma_bf16(d, ptx::sw128_desc(a_lo + 32 * k), bdesc, IDESC, 1u);
        }
        ptx::tc_commit(bars.empty(s));
      }
      if (ok) ptx::tc_commit(bars.tfull(buf));
    }
    ptx::tc_commit(bars.drain());
    wait_drain(bars.drain(), 0);
  } else if (warp >= 4 && warp < 8) {
    // --------------------------------------------------------------- epilogue
    const int quarter = warp & 3;
    uint8_t* tbl = sm + kTblOffset + quarter * (kTblChrom * 32);
    int tl = 0;
    for (int g = blockIdx.x; g < total_tiles; g += gridDim.x, ++tl) {
      const TileRef tr = decode_tile(tp, g);
      const Task& T = task_at(tp, tr.task);
      const int n = T.in.n, p = T.in.p, ns = T.in.ns;
      const int Bp = T.pop.B * p;
      const uint8_t* __restrict__ slot = T.pop.slot;
      const float* __restrict__ chubT = T.pop.chubT;
      float* __restrict__ out = T.pop.part + (long long)(tr.m * 4 + quarter) * Bp;
      const int row = tr.m * BM + quarter * 32 + lane;
      const bool rvalid = row < n;
      const int col0 = tr.nb * BN;
      const int b_first = col0 / p;
      const int b_last = (min(col0 + BN, Bp) - 1) / p;
      const int nch = b_last - b_first + 1;
      const bool use_tbl = nch <= kTblChrom;
      // Slot codes of this warp's 32 rows for every chromosome of the tile
      // (u8 table [chromosome][lane]), gathered while the tile's MMAs run.
      if (use_tbl) {
        __syncwarp();
        for (int c0 = 0; c0 < nch; c0 += 8) {
          uint8_t sv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            sv[u] = (rvalid && c0 + u < nch) ? __ldg(slot + (long long)(b_first + c0 + u) * ns + row) : (uint8_t)0;
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (c0 + u < nch) tbl[(c0 + u) * 32 + lane] = sv[u];
        }
        __syncwarp();
      }
      const int buf = tl & 1;
      const uint32_t use = (uint32_t)(tl >> 1);
      if (!wait_warp(bars.tfull(buf), use & 1u, abort_flag, status)) break;
      ptx::tc_fence_after();
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * BN);
      int b = b_first, l = col0 - b_first * p;
      for (int c0 = 0; c0 < BN; c0 += 32) {
        // factors chubT[b][l][s_b(row)] of the 32 columns: every index is
        // clamped to a valid entry so that all loads issue back to back; the
        // columns past B*p and the rows past n are zeroed afterwards.
        float f[32];
        if (use_tbl) {
          int bb = b - b_first, ll = l;
#pragma unroll
          for (int cc = 0; cc < 32; ++cc) {
            const int col = min(col0 + c0 + cc, Bp - 1);
            const int sr = tbl[min(bb, nch - 1) * 32 + lane];
            f[cc] = __ldg(chubT + (long long)col * p + sr);
            if (++ll == p) { ll = 0; ++bb; }
          }
        } else {
          int bb = b, ll = l;
#pragma unroll
          for (int cc = 0; cc < 32; ++cc) {
            const int col = min(col0 + c0 + cc, Bp - 1);
            const int sr = __ldg(slot + (long long)min(bb, b_last) * ns + (rvalid ? row : 0));
            f[cc] = __ldg(chubT + (long long)col * p + min(sr, p - 1));
            if (++ll == p) { ll = 0; ++bb; }
          }
        }
#pragma unroll
        for (int cc = 0; cc < 32; ++cc) {
          if (++l == p) { l = 0; ++b; }
          if (!rvalid || col0 + c0 + cc >= Bp) f[cc] = 0.f;
        }
        float v[32];
        ptx::tmem_ld_32x32(taddr + (uint32_t)c0, v);
        if (c0 + 32 == BN) {
          ptx::tc_fence_before();
          ptx::mbar_arrive(bars.tempty(buf));
        }
#pragma unroll
        for (int cc = 0; cc < 32; ++cc) v[cc] *= f[cc];
        const float sum = transpose_sum32(v);
        const int col = col0 + c0 + lane;
        if (col < Bp) out[col] = sum;
      }
    }
  } else if (warp >= 8) {
    // -------------------------------------------------------- one-hot producers
    const int r = threadIdx.x - 256;
    int it = 0;
    bool ok = true;
    for (int g = blockIdx.x; g < total_tiles && ok; g += gridDim.x) {
      const TileRef tr = decode_tile(tp, g);
      const Task& T = task_at(tp, tr.task);
      const int n = T.in.n, p = T.in.p, ns = T.in.ns;
      const int Bp = T.pop.B * p;
      const int nk = (n + BK - 1) / BK;
      const int col = tr.nb * BN + r;
      const bool valid = col < Bp;
      const int b = valid ? col / p : 0;
      const uint32_t lrep = (uint32_t)(valid ? col - b * p : 0) * 0x01010101u;
      const uint8_t* srow = T.pop.slot + (long long)b * ns;
      const uint32_t swz = (uint32_t)(r & 7);
      const uint4* src = reinterpret_cast<const uint4*>(srow);
      const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
      // slot codes of the next K block are loaded one block ahead
      uint4 n0 = zero4, n1 = zero4, n2 = zero4, n3 = zero4;
      if (valid) { n0 = __ldg(src); n1 = __ldg(src + 1); n2 = __ldg(src + 2); n3 = __ldg(src + 3); }
      for (int kb = 0; kb < nk; ++kb, ++it) {
        const uint4 q0 = n0, q1 = n1, q2 = n2, q3 = n3;
        if (valid && kb + 1 < nk) {
          const uint4* nx = src + (kb + 1) * (BK / 16);
          n0 = __ldg(nx); n1 = __ldg(nx + 1); n2 = __ldg(nx + 2); n3 = __ldg(nx + 3);
        }
        const int s = it % STAGES;
        const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
        if (!(ok = wait_warp(bars.empty(s), ph ^ 1u, abort_flag, status))) break;
        const uint32_t dst = base + s * STAGE_BYTES + 2 * A_BYTES + (uint32_t)r * 128u;
        if (valid) {
          st_shared_v4(dst + ((0u ^ swz) << 4), onehot8(q0.x, q0.y, lrep));
          st_shared_v4(dst + ((1u ^ swz) << 4), onehot8(q0.z, q0.w, lrep));
          st_shared_v4(dst + ((2u ^ swz) << 4), onehot8(q1.x, q1.y, lrep));
          st_shared_v4(dst + ((3u ^ swz) << 4), onehot8(q1.z, q1.w, lrep));
          st_shared_v4(dst + ((4u ^ swz) << 4), onehot8(q2.x, q2.y, lrep));
          st_shared_v4(dst + ((5u ^ swz) << 4), onehot8(q2.z, q2.w, lrep));
          st_shared_v4(dst + ((6u ^ swz) << 4), onehot8(q3.x, q3.y, lrep));
          st_shared_v4(dst + ((7u ^ swz) << 4), onehot8(q3.z, q3.w, lrep));
        } else {
          const uint4 z = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
          for (uint32_t c = 0; c < 8; ++c) st_shared_v4(dst + (c << 4), z);
        }
        ptx::fence_proxy_async_smem();
        ptx::mbar_arrive(bars.full_oh(s));
      }
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, TMEM_COLS);
  }
}

int tc_part_rows(int n) { return 4 * ((n + BM - 1) / BM); }

void prepare_eval_tc() {
  cudaFuncSetAttribute(k_eval_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
}

void launch_eval_tc(const TaskSet& ts, int num_sms, uint32_t* status, cudaStream_t s) {
  TaskParam tp = make_param(ts);
  for (int t = 0; t < ts.count; ++t) {
    const Task& T = ts.h[t];
    const int mt = (T.in.n + BM - 1) / BM;
    const int nt = (T.pop.B * T.in.p + BN - 1) / BN;
    tp.bo.o[t + 1] = tp.bo.o[t] + mt * nt;
  }
  const int total = tp.bo.o[ts.count];
  if (total == 0) return;
  const int grid = total < num_sms ? total : num_sms;
  k_eval_tc<<<grid, kThreads, kSmemBytes, s>>>(tp, total, status);
}

}  // namespace usaphmp
