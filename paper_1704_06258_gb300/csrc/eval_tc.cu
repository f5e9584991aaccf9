// Split-bf16 tensor-core evaluator of the transfer term of objective (1), §3.
//
// For chromosome b with slot codes s_b and one-hot allocation matrix
// A_b[j][l] = [s_b(j) == l] (n x p), the transfer term is
//   T3_b = sum_i sum_l M_b[i][l] * Chub_b[s_b(i)][l],   M_b = W A_b,
// i.e. the inner sum over j of objective (1) grouped by the hub serving j.
// The chromosomes of a launch are packed side by side as the columns
// (b, l) -> b*p + l of one GEMM  D = W [A_1 .. A_B]  (n x n times n x B*p):
//   * W enters as two bf16 operands, W = Whi + Wlo + O(2^-17 |W|), loaded by
//     TMA with the 128-byte swizzle; both are multiplied by the same one-hot
//     operand and accumulated into one fp32 TMEM tile (tcgen05.mma, kind::f16);
//   * when C is symmetric every Chub_b is symmetric, the pairs (i, j) and
//     (j, i) share one factor, and W is replaced by U (W + W^T folded onto
//     j > i, W_ii on the diagonal, 0 below): row block m then needs only the
//     K blocks from column 128 m on, about half of the MMAs;
//   * the one-hot operand is never stored in global memory: producer warps
//     expand it from the u8 slot codes straight into shared memory, in the
//     same swizzled K-major layout;
//   * a column tile holds whole chromosomes only (CPT = floor(ntile/p) of
//     them, MMA width N = CPT*p rounded up to 16), so the epilogue can finish
//     each chromosome inside the tile: every thread (one row i of W) forms
//     sum_l D[i][(b,l)] * Chub_b[s_b(i)][l] with the Chub tables of the
//     tile's chromosomes bulk-copied into shared memory, and a warp
//     butterfly adds the 32 rows; one partial per (32-row group, chromosome)
//     is written, D itself never leaves the SM.
// Persistent kernel, one CTA per SM, warp roles: 0 TMA, 1 MMA (+ TMEM
// allocation), 2-9 epilogue (warp w reads TMEM lane quarter w%4 and one half
// of the tile's chromosomes), 10-17 one-hot producers.  Tiles are 128 rows x
// N columns x 64-deep K blocks; the tile shape of a launch (TcTile: ntile
// 64/128/256, 2-4 shared-memory stages, raster order) sets the layout of
// shared memory, and two TMEM accumulators of ntile columns let the epilogue
// of one tile overlap the MMAs of the next.  Every wait is bounded: after
// kTimeoutNs the kernel raises kStatusTimeout, drains its own copies and
// MMAs, frees TMEM and returns.
#include <type_traits>

#include "usaphmp.h"

#include "common.cuh"
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace usaphmp {

namespace {

constexpr int BM = 128, BK = 64;
constexpr int kEpiWarp0 = 2, kEpiWarps = 8;
constexpr int kProdWarp0 = kEpiWarp0 + kEpiWarps;
constexpr int kThreads = 32 * (kProdWarp0 + 8);
constexpr uint32_t A_BYTES = BM * BK * 2;                 // 16 KB
constexpr int kMaxStages = 4;
constexpr int kTblChrom = 86;                              // chromosomes of a tile whose slot codes are tabled
constexpr int kTblWarpChrom = kTblChrom / 2;               // per epilogue warp: u8 [8 warps][43][32 rows]
constexpr uint32_t kTblBytes = kEpiWarps * kTblWarpChrom * 32;
constexpr int kNumBars = 3 * kMaxStages + 7;
// top of shared memory: the barriers, the TMEM address and abort flag, then
// (16-byte aligned) the pair mode's signal slots: one 16-byte landing slot
// per stage and one source slot
constexpr uint32_t kSigOff = (8 * kNumBars + 8 + 15) & ~15u;
constexpr uint32_t kTopBytes = kSigOff + 16 * (kMaxStages + 1);
constexpr uint32_t kSmemBytes = 232448;                    // dynamic shared memory of one CTA (227 KB)
constexpr uint32_t kUsable = kSmemBytes - 1024;            // after aligning the base to 1024
constexpr uint64_t kTimeoutNs = 2000000000ull;

// Shared-memory layout of a tile shape: `stages` stages of [A_hi | A_lo | B]
// (B = ntile rows x 128 bytes; in pair mode this CTA's half, ntile / 2
// rows), then the slab for the tile's Chub tables (whatever room is left),
// the slot-code table and the barriers at the top.
struct Lay {
  int ntile, stages, raster, pair;
  uint32_t stage_bytes, slab_off, slab_bytes, tbl_off, bar_off;
  bool ok;
};

__host__ __device__ inline Lay lay_of(const TcTile& t) {
  Lay L;
  L.ntile = t.ntile;
  L.stages = t.stages;
  L.raster = t.raster;
  L.pair = t.pair;
  L.stage_bytes = 2 * A_BYTES + (uint32_t)(t.pair ? t.ntile / 2 : t.ntile) * BK * 2;
  L.bar_off = (kUsable - kTopBytes) & ~15u;
  L.tbl_off = (L.bar_off - kTblBytes) & ~15u;
  L.slab_off = (uint32_t)t.stages * L.stage_bytes;
  L.ok = (t.ntile == 64 || t.ntile == 128 || t.ntile == 256) && t.stages >= 2 && t.stages <= kMaxStages &&
         (t.raster == 0 || t.raster == 1) && (t.pair == 0 || (t.pair == 1 && t.ntile >= 64)) &&
         L.slab_off <= L.tbl_off;
  L.slab_bytes = L.ok ? (L.tbl_off - L.slab_off) & ~15u : 0;
  return L;
}

struct Bars {
  uint32_t base;
  __device__ uint32_t full_tma(int s) const { return base + 8 * s; }
  __device__ uint32_t full_oh(int s) const { return base + 8 * (kMaxStages + s); }
  __device__ uint32_t empty(int s) const { return base + 8 * (2 * kMaxStages + s); }
  __device__ uint32_t tfull(int b) const { return base + 8 * (3 * kMaxStages + b); }
  __device__ uint32_t tempty(int b) const { return base + 8 * (3 * kMaxStages + 2 + b); }
  __device__ uint32_t drain() const { return base + 8 * (3 * kMaxStages + 4); }
  __device__ uint32_t slab_full() const { return base + 8 * (3 * kMaxStages + 5); }
  __device__ uint32_t slab_empty() const { return base + 8 * (3 * kMaxStages + 6); }
  __device__ uint32_t sig(int s) const { return base + kSigOff + 16 * s; }
  __device__ uint32_t sig_src() const { return base + kSigOff + 16 * kMaxStages; }
};

// Single-thread bounded wait.  Returns false on timeout or when another role
// has already aborted.
// kCluster: acquire at cluster scope (barriers the other CTA of a pair
// arrives on).
template <bool kCluster = false>
__device__ __forceinline__ bool try_wait(uint32_t bar, uint32_t parity) {
  if constexpr (kCluster)
    return ptx::mbar_try_wait_cluster(bar, parity);
  else
    return ptx::mbar_try_wait(bar, parity);
}

template <bool kCluster = false>
__device__ __forceinline__ bool wait_one(uint32_t bar, uint32_t parity, volatile int* abort_flag, uint32_t* status,
                                         uint64_t limit_ns = kTimeoutNs) {
  if (try_wait<kCluster>(bar, parity)) return true;
  const uint64_t t0 = ptx::globaltimer();
  for (uint32_t i = 1;; ++i) {
    if (try_wait<kCluster>(bar, parity)) return true;
    if ((i & 255u) == 0) {
      if (*abort_flag) return false;
      if (ptx::globaltimer() - t0 > limit_ns) {
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
template <bool kCluster = false>
__device__ __forceinline__ bool wait_warp(uint32_t bar, uint32_t parity, volatile int* abort_flag, uint32_t* status,
                                          uint64_t limit_ns = kTimeoutNs) {
  const uint64_t t0 = ptx::globaltimer();
  for (uint32_t i = 0;; ++i) {
    const bool ok = try_wait<kCluster>(bar, parity);
    if (__all_sync(0xffffffffu, ok)) return true;
    if ((i & 255u) == 255u) {
      int stop = 0;
      if ((threadIdx.x & 31) == 0) {
        stop = *abort_flag;
        if (!stop && ptx::globaltimer() - t0 > limit_ns) {
          *abort_flag = 1;
          atomicOr(status, kStatusTimeout);
          stop = 1;
        }
      }
      if (__shfl_sync(0xffffffffu, stop, 0)) return false;
    }
  }
}

// Column geometry of a task: whole chromosomes per tile.
struct Geo {
  int cpt;    // chromosomes per column tile
  int nt;     // column tiles
  bool slab;  // Chub tables of a full tile fit in the shared slab
};

__host__ __device__ __forceinline__ Geo geo_of(int p, int B, const Lay& L) {
  Geo g;
  g.cpt = L.ntile / p;
  g.nt = (B + g.cpt - 1) / g.cpt;
  g.slab = (size_t)g.cpt * chub_cstride(p) * 4 <= L.slab_bytes;
  return g;
}

// Position in the ring of shared-memory stages: stage index and the parity
// of its current use, advanced without a division per K block.
struct Ring {
  int s = 0, n;
  uint32_t ph = 0;
  __device__ explicit Ring(int stages) : n(stages) {}
  __device__ void next() {
    if (++s == n) {
      s = 0;
      ph ^= 1u;
    }
  }
};

struct TileRef {
  int task, m0, m, nb;   // m0: first row block of the unit; m: this CTA's row block
};

// Tile g of the launch -> (task, row unit, column tile nb).  A row unit is
// one row block, or two (2u, 2u + 1) in pair mode, where CTA rank r of the
// pair takes row block 2u + r.  Raster 0 walks the column tiles of one row
// unit first (CTAs running side by side share the W stripe), raster 1 the
// row units of one column tile first (they share the chromosomes' slot codes
// and hub tables).
__device__ __forceinline__ TileRef decode_tile(const TaskParam& tp, int g, const Lay& L, int rank) {
  TileRef r;
  r.task = task_of(tp.bo, g);
  const Task& T = task_at(tp, r.task);
  const int local = g - tp.bo.o[r.task];
  int u;
  if (L.raster == 0) {
    const int nt = geo_of(T.in.p, T.pop.B, L).nt;
    u = local / nt;
    r.nb = local - u * nt;
  } else {
    const int mt = (T.in.n + BM - 1) / BM;
    const int mu = L.pair ? (mt + 1) >> 1 : mt;
    r.nb = local / mu;
    u = local - r.nb * mu;
  }
  r.m0 = L.pair ? 2 * u : u;
  r.m = r.m0 + rank;
  return r;
}

// The tile a CTA (a pair of CTAs in pair mode) takes in round r of the
// persistent loop: tiles rG .. rG+G-1 go to slots 0 .. G-1, and with `snake`
// to slots G-1 .. 0 in odd rounds, so that over the rounds every slot gets
// an even share of tiles sorted by cost (row-unit-major tiles of a folded W,
// whose K loops shorten with the row).
__device__ __forceinline__ int tile_of_round(int r, bool snake, int pair) {
  const int G = (int)gridDim.x >> pair, c = (int)blockIdx.x >> pair;
  return r * G + ((snake && (r & 1)) ? G - 1 - c : c);
}

// First K block of row block m: with the folded U (zero left of the
// diagonal) the blocks left of column 128 m add nothing.
__device__ __forceinline__ int k_begin(const Task& T, int m) { return T.in.wtri ? (m * BM) / BK : 0; }

// 8 slot codes (two words) -> 8 bf16 values, 1.0 where the code equals the
// row's slot l, 0 elsewhere, element k in the k-th 16-bit lane: each code c
// becomes the bf16 bit pattern 0x4000 | c (a finite normal number, distinct
// for every byte c; prmt with 0x40 bytes), and one bf16x2 compare against
// lpair = the same pattern of l in both halves gives 1.0 or 0.0 per half.
__device__ __forceinline__ uint32_t bf16x2_eq(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("set.eq.bf16x2.bf16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t codes_to_bf16x2(uint32_t w, uint32_t sel) {
  uint32_t r;
  asm("prmt.b32 %0, %1, 0x40404040, %2;" : "=r"(r) : "r"(w), "r"(sel));
  return r;
}
__device__ __forceinline__ uint4 onehot8_set(uint32_t w0, uint32_t w1, uint32_t lpair) {
  uint4 o;
  o.x = bf16x2_eq(codes_to_bf16x2(w0, 0x5140u), lpair);
  o.y = bf16x2_eq(codes_to_bf16x2(w0, 0x5342u), lpair);
  o.z = bf16x2_eq(codes_to_bf16x2(w1, 0x5140u), lpair);
  o.w = bf16x2_eq(codes_to_bf16x2(w1, 0x5342u), lpair);
  return o;
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}

struct EpiArgs {
  uint32_t taddr;
  int cb, ce, p, hst, cst, ns, row, lane;
  bool rvalid, use_tbl;
  const uint8_t* tbl;
  const uint8_t* slot;
  const float* fbase;
  float* out;
};

// The sums over the warp's 32 rows of 8 chromosomes at a time, taken as the
// chromosomes' values arrive (a transposed butterfly).  Chromosomes 2i and
// 2i + 1 meet at the step over lane bit 16: each lane keeps one of the two
// and adds its partner's copy of it; the pairs (0,1), (2,3) of those meet at
// bit 8, the two halves at bit 4, then bits 2 and 1 as usual.  Every
// chromosome's total is the same tree of pairwise sums as the one-value
// butterfly (lanes l, l^16, then l^8, ...), so it has the same bits, in 9
// shuffles instead of 40, with at most four partial sums live.  Lane l ends
// with the total of chromosome 4 b4 + 2 b8 + b16 (b the bits of l); lanes
// with l % 4 == 0 store it.
struct Tree8 {
  float prev, w0, x0, x1;
};

__device__ __forceinline__ float tree_pair(float lo, float hi, bool b, int m) {
  const float send = b ? lo : hi;
  return (b ? hi : lo) + __shfl_xor_sync(0xffffffffu, send, m);
}

// Feeds chromosome bs + jj's per-lane value (0 past the warp's range).
template <int JJ>
__device__ __forceinline__ void tree_add(Tree8& t, int lane, float v) {
  if constexpr ((JJ & 1) == 0) {
    t.prev = v;
  } else {
    const float w = tree_pair(t.prev, v, lane & 16, 16);
    if constexpr ((JJ & 2) == 0) {
      t.w0 = w;
    } else {
      const float x = tree_pair(t.w0, w, lane & 8, 8);
      if constexpr (JJ < 4) t.x0 = x; else t.x1 = x;
    }
  }
}

__device__ __forceinline__ void tree_store(const EpiArgs& a, int bs, const Tree8& t) {
  const int lane = a.lane;
  float y = tree_pair(t.x0, t.x1, lane & 4, 4);
  y += __shfl_xor_sync(0xffffffffu, y, 2);
  y += __shfl_xor_sync(0xffffffffu, y, 1);
  const int j = ((lane & 4) ? 4 : 0) + ((lane & 8) ? 2 : 0) + ((lane & 16) ? 1 : 0);
  if ((lane & 3) == 0 && bs + j < a.ce) a.out[bs + j] = y;
}

// Unrolls f(integral_constant<jj>) for jj = 0..7.
template <int JJ = 0, class F>
__device__ __forceinline__ void unroll8(F&& f) {
  if constexpr (JJ < 8) {
    f(std::integral_constant<int, JJ>{});
    unroll8<JJ + 1>(f);
  }
}

// The row's slot in chromosome c and its factors Chub_c[s_c(row)][0..p).
__device__ __forceinline__ const float* epi_factors(const EpiArgs& a, int c) {
  const int p = a.p;
  const int sr = !a.rvalid ? 0
                 : a.use_tbl ? min((int)a.tbl[(c - a.cb) * 32 + a.lane], p - 1)
                             : min((int)__ldg(a.slot + (long long)c * a.ns + a.row), p - 1);
  return a.fbase + c * a.cst + sr * a.hst;
}

// Epilogue of one warp over its chromosomes [cb, ce), 8 at a time: per
// chromosome the p accumulator columns (TMEM loads of WID columns), the row's
// p factors (one load each, free of bank conflicts by the odd row stride)
// and one fma chain, fed to a Tree8.  Rows past n hold zeros (the TMA fills
// them), so they add nothing.
template <int WID>
__device__ __forceinline__ void epi_chromosomes(const EpiArgs& a) {
  constexpr int LMAX = 32;
  const int p = a.p;
  for (int bs = a.cb; bs < a.ce; bs += 8) {
    Tree8 t;
    unroll8([&](auto J) {
      constexpr int jj = decltype(J)::value;
      const int c = bs + jj;
      float acc = 0.f;
      if (c < a.ce) {
        const float* frow = epi_factors(a, c);
        for (int l0 = 0; l0 < p; l0 += LMAX) {
          const int nl = min(LMAX, p - l0);
          uint32_t v[LMAX];
#pragma unroll
          for (int l = 0; l < LMAX; ++l) v[l] = 0u;
          const uint32_t ta = a.taddr + (uint32_t)(c * p + l0);
#pragma unroll
          for (int l = 0; l < LMAX; l += WID) {
            if (l < nl) {
              if constexpr (WID == 4)
                ptx::tmem_ld_32x4(ta + l, v[l], v[l + 1], v[l + 2], v[l + 3]);
              else if constexpr (WID == 2)
                ptx::tmem_ld_32x2(ta + l, v[l], v[l + 1]);
              else
                ptx::tmem_ld_32x1(ta + l, v[l]);
            }
          }
          ptx::tmem_ld_wait32(v);
#pragma unroll
          for (int l = 0; l < LMAX; ++l)
            if (l < nl) acc = fmaf(__uint_as_float(v[l]), frow[l0 + l], acc);
        }
      }
      tree_add<jj>(t, a.lane, acc);
    });
    tree_store(a, bs, t);
  }
}

// epi_chromosomes for p <= LM (16, 24 or 32), software-pipelined over the
// chromosomes: the TMEM loads of chromosome c + 1 are in flight while
// chromosome c is summed (two register buffers of LM columns; every wait::ld
// finds only the loads it waits for outstanding).  Same arithmetic, same
// order.
template <int WID, int LM>
__device__ __forceinline__ void epi_issue(const EpiArgs& a, int c, uint32_t (&v)[LM]) {
  const uint32_t ta = a.taddr + (uint32_t)(c * a.p);
#pragma unroll
  for (int l = 0; l < LM; l += WID) {
    if (l < a.p) {
      if constexpr (WID == 4)
        ptx::tmem_ld_32x4(ta + l, v[l], v[l + 1], v[l + 2], v[l + 3]);
      else if constexpr (WID == 2)
        ptx::tmem_ld_32x2(ta + l, v[l], v[l + 1]);
      else
        ptx::tmem_ld_32x1(ta + l, v[l]);
    }
  }
}

template <int LM>
__device__ __forceinline__ float epi_dot(const EpiArgs& a, int c, const uint32_t (&v)[LM]) {
  const int p = a.p;
  const float* frow = epi_factors(a, c);
  float acc = 0.f;
#pragma unroll
  for (int l = 0; l < LM; ++l)
    if (l < p) acc = fmaf(__uint_as_float(v[l]), frow[l], acc);
  return acc;
}

template <int WID, int LM>
__device__ __forceinline__ void epi_chromosomes_pipe(const EpiArgs& a) {
  if (a.cb >= a.ce) return;
  uint32_t va[LM], vb[LM];
#pragma unroll
  for (int l = 0; l < LM; ++l) va[l] = vb[l] = 0u;
  epi_issue<WID, LM>(a, a.cb, va);
  // batches start at cb + 8k, so an even offset in a batch is always in va
  for (int bs = a.cb; bs < a.ce; bs += 8) {
    Tree8 t;
    unroll8([&](auto J) {
      constexpr int jj = decltype(J)::value;
      const int c = bs + jj;
      float d = 0.f;
      if (c < a.ce) {
        if constexpr ((jj & 1) == 0) {
          ptx::tmem_ld_wait_n<LM>(va);
          if (c + 1 < a.ce) epi_issue<WID, LM>(a, c + 1, vb);
          d = epi_dot<LM>(a, c, va);
        } else {
          ptx::tmem_ld_wait_n<LM>(vb);
          if (c + 1 < a.ce) epi_issue<WID, LM>(a, c + 1, va);
          d = epi_dot<LM>(a, c, vb);
        }
      }
      tree_add<jj>(t, a.lane, d);
    });
    tree_store(a, bs, t);
  }
}

template <int LM>
__device__ __forceinline__ void epi_pipe_width(const EpiArgs& a) {
  if ((a.p & 3) == 0)
    epi_chromosomes_pipe<4, LM>(a);
  else if ((a.p & 1) == 0)
    epi_chromosomes_pipe<2, LM>(a);
  else
    epi_chromosomes_pipe<1, LM>(a);
}

}  // namespace

// kPair: a cluster of two CTAs per MMA (cta_group::2, M = 256).  Rank 0
// issues every MMA and commit; the barriers it waits on (stage full, one-hot
// full, accumulator empty) live in its shared memory and count the arrivals
// of both CTAs (TMA bytes of both; its 8 producer warps and the signal copy
// of rank 1's forwarder; 2 x 8 epilogue warps); its commits arrive on the
// stage-empty and accumulator-full barriers of both CTAs.
template <bool kPair>
__global__ void __launch_bounds__(kThreads, 1)
    k_eval_tc(const __grid_constant__ TaskParam tp, int total_tiles, uint32_t* status, const Lay L, int snake) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw = ptx::smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sm = smem_raw + (base - raw);
  const Bars bars{base + L.bar_off};
  volatile uint32_t* tmem_holder = reinterpret_cast<volatile uint32_t*>(sm + L.bar_off + 8 * kNumBars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + L.bar_off + 8 * kNumBars + 4);
  const int STAGES = L.stages;
  const uint32_t STAGE_BYTES = L.stage_bytes;
  const uint32_t tmem_cols = 2u * (uint32_t)L.ntile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = kPair ? (int)ptx::cluster_ctarank() : 0;
  const int pshift = kPair ? 1 : 0;
  constexpr int kPeers = kPair ? 2 : 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kMaxStages; ++s) {
      ptx::mbar_init(bars.full_tma(s), 1);
      // one arrival per producer warp (in pair mode rank 0's barrier also
      // waits for the 16 bytes rank 1's forwarder copies in, see below)
      ptx::mbar_init(bars.full_oh(s), 8);
      ptx::mbar_init(bars.empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(bars.tfull(b), 1);
      ptx::mbar_init(bars.tempty(b), kEpiWarps * kPeers); // one arrival per epilogue warp
    }
    ptx::mbar_init(bars.drain(), 1);
    ptx::mbar_init(bars.slab_full(), 1);
    ptx::mbar_init(bars.slab_empty(), kEpiWarps);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    if constexpr (kPair) {
      ptx::tmem_alloc_pair(ptx::smem_u32(const_cast<uint32_t*>(tmem_holder)), tmem_cols);
      ptx::tmem_relinquish_pair();
    } else {
      ptx::tmem_alloc(ptx::smem_u32(const_cast<uint32_t*>(tmem_holder)), tmem_cols);
      ptx::tmem_relinquish();
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  // both CTAs' barriers are initialised before either arrives on the other's
  if constexpr (kPair) ptx::cluster_sync();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  // barriers and TMEM are set up: now wait for the allocation kernel's output
  pdl_wait();
  pdl_allow_next();

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ TMA producer
    // Both CTAs load their own row block of U_hi / U_lo; in pair mode the
    // completions count on rank 0's stage barrier, whose single arrival
    // (rank 0's) expects the bytes of both.
    int it = 0;
    Ring ring(STAGES);
    bool ok = true;
    for (int rd = 0, g = tile_of_round(0, snake, pshift); g < total_tiles && ok;
         g = tile_of_round(++rd, snake, pshift)) {
      const TileRef tr = decode_tile(tp, g, L, rank);
      const Task& T = task_at(tp, tr.task);
      const int nk = (T.in.n + BK - 1) / BK;
      for (int kb = k_begin(T, tr.m0); kb < nk; ++kb, ++it, ring.next()) {
        const int s = ring.s;
        if (!(ok = wait_one(bars.empty(s), ring.ph ^ 1u, abort_flag, status))) break;
        const uint32_t a_hi = base + s * STAGE_BYTES;
        if constexpr (kPair) {
          if (rank == 0) ptx::mbar_arrive_expect_tx(bars.full_tma(s), 4 * A_BYTES);
          const uint32_t fb = ptx::mapa(bars.full_tma(s), 0);
          ptx::tma_load_2d_pair(a_hi, T.tmap_hi, kb * BK, tr.m * BM, fb);
          ptx::tma_load_2d_pair(a_hi + A_BYTES, T.tmap_lo, kb * BK, tr.m * BM, fb);
        } else {
          ptx::mbar_arrive_expect_tx(bars.full_tma(s), 2 * A_BYTES);
          ptx::tma_load_2d(a_hi, T.tmap_hi, kb * BK, tr.m * BM, bars.full_tma(s));
          ptx::tma_load_2d(a_hi + A_BYTES, T.tmap_lo, kb * BK, tr.m * BM, bars.full_tma(s));
        }
      }
    }
    // the copies still in flight land before the CTA exits (in pair mode
    // rank 0's barrier counts both CTAs' copies; rank 1 is held by the
    // final cluster barrier until rank 0 has seen them land)
    if (rank == 0)
      for (int j = it - STAGES < 0 ? 0 : it - STAGES; j < it; ++j)
        wait_drain(bars.full_tma(j % STAGES), (uint32_t)(j / STAGES) & 1u);
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ------------------------------------------------------------- MMA issuer
    int tl = 0;
    Ring ring(STAGES);
    bool ok = true;
    const uint32_t peer = kPair ? 1u : 0u;
    for (int rd = 0, g = tile_of_round(0, snake, pshift); g < total_tiles && ok;
         g = tile_of_round(++rd, snake, pshift), ++tl) {
      const TileRef tr = decode_tile(tp, g, L, rank);
      const Task& T = task_at(tp, tr.task);
      const int p = T.in.p;
      const Geo geo = geo_of(p, T.pop.B, L);
      const int nchrom = min(geo.cpt, T.pop.B - tr.nb * geo.cpt);
      const uint32_t idesc = ptx::idesc_bf16_f32(kPeers * BM, round_up(nchrom * p, 16 * kPeers));
      const int nk = (T.in.n + BK - 1) / BK;
      const int kb0 = k_begin(T, tr.m0);
      const int buf = tl & 1;
      const uint32_t use = (uint32_t)(tl >> 1);
      if (!(ok = wait_one<kPair>(bars.tempty(buf), (use & 1u) ^ 1u, abort_flag, status))) break;
      ptx::tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(buf * L.ntile);
      for (int kb = kb0; kb < nk; ++kb, ring.next()) {
        const int s = ring.s;
        if (!(ok = wait_one(bars.full_tma(s), ring.ph, abort_flag, status))) break;
        if (!(ok = wait_one<kPair>(bars.full_oh(s), ring.ph, abort_flag, status))) break;
        ptx::tc_fence_after();
        const uint32_t a_hi = base + s * STAGE_BYTES, a_lo = a_hi + A_BYTES, bt = a_lo + A_BYTES;
#pragma unroll
        for (int k = 0; k < BK / 16; ++k) {
          const uint64_t bdesc = ptx::sw128_desc(bt + 32 * k);
          const uint32_t acc = (kb != kb0 || k != 0) ? 1u : 0u;
          if constexpr (kPair) {
            ptx::mma_bf16_pair(d, ptx::sw128_desc(a_hi + 32 * k), bdesc, idesc, acc);
            ptx::mma_bf16_pair(d, ptx::sw128_desc(a_lo + 32 * k), bdesc, idesc, 1u);
          } else {
            ptx::mma_bf16(d, ptx::sw128_desc(a_hi + 32 * k), bdesc, idesc, acc);
            ptx::mma_bf16(d, ptx::sw128_desc(a_lo + 32 * k), bdesc, idesc, 1u);
          }
        }
        if constexpr (kPair) {
          ptx::tc_commit_pair(bars.empty(s));
          ptx::tc_commit_pair(ptx::mapa(bars.empty(s), peer));
        } else {
          ptx::tc_commit(bars.empty(s));
        }
      }
      if (ok) {
        if constexpr (kPair) {
          ptx::tc_commit_pair(bars.tfull(buf));
          ptx::tc_commit_pair(ptx::mapa(bars.tfull(buf), peer));
        } else {
          ptx::tc_commit(bars.tfull(buf));
        }
      }
    }
    if constexpr (kPair)
      ptx::tc_commit_pair(bars.drain());
    else
      ptx::tc_commit(bars.drain());
    wait_drain(bars.drain(), 0);
  } else if (kPair && warp == 1 && lane == 0) {
    // ------------------------------------------- one-hot forwarder (rank 1)
    // Rank 1's producer warps arrive on their own CTA's barrier; this thread
    // passes each completed stage on to rank 0's barrier as the completion
    // of a 16-byte copy into rank 0's shared memory (an async-proxy signal,
    // which costs the thread nothing; a cluster-scope release arrive stalls
    // its thread for about a K block's MMA time).  Rank 0's first producer
    // warp adds the 16 bytes to the barrier's expected count.
    Ring ring(STAGES);
    bool ok = true;
    for (int rd = 0, g = tile_of_round(0, snake, pshift); g < total_tiles && ok;
         g = tile_of_round(++rd, snake, pshift)) {
      const TileRef tr = decode_tile(tp, g, L, rank);
      const Task& T = task_at(tp, tr.task);
      const int nk = (T.in.n + BK - 1) / BK;
      for (int kb = k_begin(T, tr.m0); kb < nk; ++kb, ring.next()) {
        const int s = ring.s;
        if (!(ok = wait_one(bars.full_oh(s), ring.ph, abort_flag, status))) break;
        ptx::fence_proxy_async_smem();
        ptx::bulk_copy_cluster(ptx::mapa(bars.sig(s), 0), bars.sig_src(), 16, ptx::mapa(bars.full_oh(s), 0));
      }
    }
  } else if (warp >= kEpiWarp0 && warp < kEpiWarp0 + kEpiWarps) {
    // --------------------------------------------------------------- epilogue
    const int quarter = warp & 3, half = (warp - kEpiWarp0) >> 2;
    // this warp's own slot-code table: rows of its chromosomes [cb, ce) of the
    // current tile (private, so refilling it for the next tile cannot race
    // with the other warps still reading theirs, whatever the next tile's
    // chromosome split)
    uint8_t* tbl = sm + L.tbl_off + (warp - kEpiWarp0) * (kTblWarpChrom * 32);
    const float* slab = reinterpret_cast<const float*>(sm + L.slab_off);
    int tl = 0;
    for (int rd = 0, g = tile_of_round(0, snake, pshift); g < total_tiles;
         g = tile_of_round(++rd, snake, pshift), ++tl) {
      const TileRef tr = decode_tile(tp, g, L, rank);
      const Task& T = task_at(tp, tr.task);
      const int n = T.in.n, p = T.in.p, ns = T.in.ns, B = T.pop.B;
      const Geo geo = geo_of(p, B, L);
      const int b0 = tr.nb * geo.cpt;
      const int nchrom = min(geo.cpt, B - b0);
      const int hst = chub_hstride(p), cst = chub_cstride(p);
      const float* __restrict__ chub = T.pop.chub + (long long)b0 * cst;
      const uint8_t* __restrict__ slot = T.pop.slot + (long long)b0 * ns;
      const int row = tr.m * BM + quarter * 32 + lane;
      const bool rvalid = row < n;
      // in pair mode the second row block of the last unit can lie past n:
      // its CTA keeps step with the barriers but has no rows to sum
      const bool live = !kPair || tr.m * BM < n;
      const bool use_tbl = nchrom <= kTblChrom;
      // this warp's chromosomes: [cb, ce)
      const int split = (nchrom + 1) >> 1;
      const int cb = half ? split : 0, ce = half ? nchrom : split;
      // Chub tables of the tile's chromosomes -> slab (single buffer, one
      // bulk copy issued once every epilogue warp has released the slab).
      if (warp == kEpiWarp0 && lane == 0) {
        if (wait_one(bars.slab_empty(), (uint32_t)(tl & 1) ^ 1u, abort_flag, status)) {
          if (geo.slab) {
            const uint32_t bytes = (uint32_t)(nchrom * cst * 4);
            ptx::mbar_arrive_expect_tx(bars.slab_full(), bytes);
            ptx::bulk_load(base + L.slab_off, chub, bytes, bars.slab_full());
          } else {
            ptx::mbar_arrive(bars.slab_full());
          }
        }
      }
      // slot codes of this warp's 32 rows for its chromosomes
      if (use_tbl && live) {
        __syncwarp();
        for (int c0 = cb; c0 < ce; c0 += 8) {
          uint8_t sv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            sv[u] = (rvalid && c0 + u < ce) ? __ldg(slot + (long long)(c0 + u) * ns + row) : (uint8_t)0;
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (c0 + u < ce) tbl[(c0 + u - cb) * 32 + lane] = sv[u];
        }
        __syncwarp();
      }
      const int buf = tl & 1;
      const uint32_t use = (uint32_t)(tl >> 1);
      if (!wait_warp(bars.tfull(buf), use & 1u, abort_flag, status)) break;
      if (!wait_warp(bars.slab_full(), (uint32_t)(tl & 1), abort_flag, status)) break;
      ptx::tc_fence_after();
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * L.ntile);
      float* __restrict__ out = T.pop.part + (long long)(tr.m * 4 + quarter) * B + b0;
      const float* fbase = geo.slab ? slab : chub;
      // one code path per TMEM load width (the widest that keeps every
      // column offset c*p + l aligned)
      const EpiArgs ea{taddr, cb, ce, p, hst, cst, ns, row, lane, rvalid, use_tbl, tbl, slot, fbase, out};
      if (!live) {
      } else if (p <= 16) {
        epi_pipe_width<16>(ea);
      } else if (p <= 24) {
        epi_pipe_width<24>(ea);
      } else if ((p & 3) == 0) {
        epi_chromosomes<4>(ea);
      } else if ((p & 1) == 0) {
        epi_chromosomes<2>(ea);
      } else {
        epi_chromosomes<1>(ea);
      }
      // every accumulator read of this warp has completed (each lane waited
      // for its loads): release the buffer, one arrival for the warp
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (rank == 0)
          ptx::mbar_arrive(bars.tempty(buf));
        else
          ptx::mbar_arrive_cluster(ptx::mapa(bars.tempty(buf), 0));
        ptx::mbar_arrive(bars.slab_empty());
      }
    }
  } else if (kPair && warp >= kProdWarp0) {
    // ------------------------------------------- one-hot producers, pair mode
    // This CTA holds B columns [rank N/2, (rank + 1) N/2) (N = the tile's MMA
    // width, a multiple of 32): thread t makes K half t / 128 (32 codes) of
    // local row t % 128.  The warps arrive on their own CTA's barrier.
    const int t = threadIdx.x - 32 * kProdWarp0;
    const int rl = t & 127, kh = t >> 7;
    const uint32_t swz = (uint32_t)(rl & 7);
    const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
    Ring ring(STAGES);
    bool ok = true;
    for (int rd = 0, g = tile_of_round(0, snake, pshift); g < total_tiles && ok;
         g = tile_of_round(++rd, snake, pshift)) {
      const TileRef tr = decode_tile(tp, g, L, rank);
      const Task& T = task_at(tp, tr.task);
      const int n = T.in.n, p = T.in.p, ns = T.in.ns, B = T.pop.B;
      const Geo geo = geo_of(p, B, L);
      const int b0 = tr.nb * geo.cpt;
      const int nchrom = min(geo.cpt, B - b0);
      const int half = round_up(nchrom * p, 32) >> 1;
      const int r = rank * half + rl;                  // column of B
      const int nk = (n + BK - 1) / BK;
      const int kb0 = k_begin(T, tr.m0);
      const bool write = rl < half;
      const bool valid = write && r < nchrom * p;    // columns in [nchrom*p, N) are zero
      const int c = valid ? r / p : 0;
      const uint32_t lpair = (0x4000u | (uint32_t)(valid ? r - c * p : 0)) * 0x00010001u;
      const uint4* src = reinterpret_cast<const uint4*>(T.pop.slot + (long long)(b0 + c) * ns) + 2 * kh;
      // slot codes of the next K block are loaded one block ahead
      uint4 n0 = zero4, n1 = zero4;
      if (valid) {
        const uint4* f = src + kb0 * (BK / 16);
        n0 = __ldg(f); n1 = __ldg(f + 1);
      }
      for (int kb = kb0; kb < nk; ++kb, ring.next()) {
        const uint4 q0 = n0, q1 = n1;
        if (valid && kb + 1 < nk) {
          const uint4* nx = src + (kb + 1) * (BK / 16);
          n0 = __ldg(nx); n1 = __ldg(nx + 1);
        }
        const int s = ring.s;
        if (!(ok = wait_warp(bars.empty(s), ring.ph ^ 1u, abort_flag, status))) break;
        const uint32_t dst = base + s * STAGE_BYTES + 2 * A_BYTES + (uint32_t)rl * 128u;
        const uint32_t q = 4u * (uint32_t)kh;
        if (valid) {
          st_shared_v4(dst + (((q + 0u) ^ swz) << 4), onehot8_set(q0.x, q0.y, lpair));
          st_shared_v4(dst + (((q + 1u) ^ swz) << 4), onehot8_set(q0.z, q0.w, lpair));
          st_shared_v4(dst + (((q + 2u) ^ swz) << 4), onehot8_set(q1.x, q1.y, lpair));
          st_shared_v4(dst + (((q + 3u) ^ swz) << 4), onehot8_set(q1.z, q1.w, lpair));
        } else if (write) {
#pragma unroll
          for (uint32_t u = 0; u < 4; ++u) st_shared_v4(dst + (((q + u) ^ swz) << 4), zero4);
        }
        ptx::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          if (rank == 0 && warp == kProdWarp0)
            ptx::mbar_arrive_expect_tx(bars.full_oh(s), 16);
          else
            ptx::mbar_arrive(bars.full_oh(s));
        }
      }
    }
  } else if (!kPair && warp >= kProdWarp0) {
    // -------------------------------------------------------- one-hot producers
    const int r = threadIdx.x - 32 * kProdWarp0;
    Ring ring(STAGES);
    bool ok = true;
    for (int rd = 0, g = tile_of_round(0, snake, 0); g < total_tiles && ok; g = tile_of_round(++rd, snake, 0)) {
      const TileRef tr = decode_tile(tp, g, L, 0);
      const Task& T = task_at(tp, tr.task);
      const int n = T.in.n, p = T.in.p, ns = T.in.ns, B = T.pop.B;
      const Geo geo = geo_of(p, B, L);
      const int b0 = tr.nb * geo.cpt;
      const int nchrom = min(geo.cpt, B - b0);
      const int nmma = round_up(nchrom * p, 16);
      const int nk = (n + BK - 1) / BK;
      const int kb0 = k_begin(T, tr.m);
      const bool valid = r < nchrom * p;   // rows in [nchrom*p, nmma) are zero
      const bool write = r < nmma;
      const int c = valid ? r / p : 0;
      const uint32_t lpair = (0x4000u | (uint32_t)(valid ? r - c * p : 0)) * 0x00010001u;
      const uint8_t* srow = T.pop.slot + (long long)(b0 + c) * ns;
      const uint32_t swz = (uint32_t)(r & 7);
      const uint4* src = reinterpret_cast<const uint4*>(srow);
      const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
      // slot codes of the next K block are loaded one block ahead
      uint4 n0 = zero4, n1 = zero4, n2 = zero4, n3 = zero4;
      if (valid) {
        const uint4* f = src + kb0 * (BK / 16);
        n0 = __ldg(f); n1 = __ldg(f + 1); n2 = __ldg(f + 2); n3 = __ldg(f + 3);
      }
      for (int kb = kb0; kb < nk; ++kb, ring.next()) {
        const uint4 q0 = n0, q1 = n1, q2 = n2, q3 = n3;
        if (valid && kb + 1 < nk) {
          const uint4* nx = src + (kb + 1) * (BK / 16);
          n0 = __ldg(nx); n1 = __ldg(nx + 1); n2 = __ldg(nx + 2); n3 = __ldg(nx + 3);
        }
        const int s = ring.s;
        if (!(ok = wait_warp(bars.empty(s), ring.ph ^ 1u, abort_flag, status))) break;
        const uint32_t dst = base + s * STAGE_BYTES + 2 * A_BYTES + (uint32_t)r * 128u;
        if (valid) {
          st_shared_v4(dst + ((0u ^ swz) << 4), onehot8_set(q0.x, q0.y, lpair));
          st_shared_v4(dst + ((1u ^ swz) << 4), onehot8_set(q0.z, q0.w, lpair));
          st_shared_v4(dst + ((2u ^ swz) << 4), onehot8_set(q1.x, q1.y, lpair));
          st_shared_v4(dst + ((3u ^ swz) << 4), onehot8_set(q1.z, q1.w, lpair));
          st_shared_v4(dst + ((4u ^ swz) << 4), onehot8_set(q2.x, q2.y, lpair));
          st_shared_v4(dst + ((5u ^ swz) << 4), onehot8_set(q2.z, q2.w, lpair));
          st_shared_v4(dst + ((6u ^ swz) << 4), onehot8_set(q3.x, q3.y, lpair));
          st_shared_v4(dst + ((7u ^ swz) << 4), onehot8_set(q3.z, q3.w, lpair));
        } else if (write) {
#pragma unroll
          for (uint32_t q = 0; q < 8; ++q) st_shared_v4(dst + ((q ^ swz) << 4), zero4);
        }
        // each lane makes its stores visible to the tensor core, then the warp
        // arrives once
        ptx::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(bars.full_oh(s));
      }
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  // in pair mode neither CTA frees its TMEM or exits while rank 0's MMAs may
  // still use the other's shared memory and TMEM (rank 0 has drained them
  // before it reaches this barrier)
  if constexpr (kPair) ptx::cluster_sync();
  if (warp == 1) {
    ptx::tc_fence_after();
    if constexpr (kPair)
      ptx::tmem_dealloc_pair(tmem, tmem_cols);
    else
      ptx::tmem_dealloc(tmem, tmem_cols);
  }
}

int tc_part_rows(int n) { return 4 * ((n + BM - 1) / BM); }

// Clusters of two that can run at once on each device (pair mode's grid),
// found once per device when its handles are set up.
static int g_pair_slots[64];

void prepare_eval_tc() {
  cudaFuncSetAttribute(k_eval_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  cudaFuncSetAttribute(k_eval_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || g_pair_slots[dev] > 0) return;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kSmemBytes;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, k_eval_tc<true>, &cfg) == cudaSuccess && clusters > 0)
    g_pair_slots[dev] = clusters;
  else
    cudaGetLastError();
}

int tc_pair_slots() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  return g_pair_slots[dev];
}

bool tc_tile_fits(const TcTile& t, int p) { return lay_of(t).ok && p <= t.ntile; }

size_t tc_slab_bytes(const TcTile& t) { return lay_of(t).slab_bytes; }

void launch_eval_tc(const TaskSet& ts, int num_sms, uint32_t* status, cudaStream_t s, const TcTile& tile) {
  // a shape that does not fit every task of the launch falls back to the default
  TcTile t = tile;
  for (int k = 0; k < ts.count; ++k)
    if (!tc_tile_fits(t, ts.h[k].in.p)) t = TcTile{};
  // pair mode needs its cluster slots counted (prepare_eval_tc)
  const int slots = tc_pair_slots();
  if (t.pair && slots <= 0) t.pair = 0;
  const Lay L = lay_of(t);
  TaskParam tp = make_param(ts);
  for (int k = 0; k < ts.count; ++k) {
    const Task& T = ts.h[k];
    const int mt = (T.in.n + BM - 1) / BM;
    const int mu = L.pair ? (mt + 1) / 2 : mt;   // row units
    tp.bo.o[k + 1] = tp.bo.o[k] + (T.pop.B > 0 ? mu * geo_of(T.in.p, T.pop.B, L).nt : 0);
  }
  const int total = tp.bo.o[ts.count];
  if (total == 0) return;
  int snake = 0;
  for (int k = 0; k < ts.count; ++k) snake |= ts.h[k].in.wtri;
  if (L.pair) {
    const int pairs = total < slots ? total : slots;
    launch_pdl_cluster(k_eval_tc<true>, 2 * pairs, kThreads, kSmemBytes, s, 2, tp, total, status, L, snake);
  } else {
    const int grid = total < num_sms ? total : num_sms;
    launch_pdl(k_eval_tc<false>, grid, kThreads, kSmemBytes, s, tp, total, status, L, snake);
  }
}

// Self-test of the bounded waits: the warps of one block wait on an mbarrier
// that nothing completes, one thread with wait_one and one warp with
// wait_warp, under a short limit.  Both must give up: the first records
// kStatusTimeout and raises the abort flag, the second stops on the flag
// (or on its own limit); bit 31 of *status marks a wait that wrongly
// succeeded.  The kernel then returns normally.
__global__ void k_wait_selftest(uint64_t limit_ns, uint32_t* status, unsigned long long* elapsed_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  const uint32_t b = ptx::smem_u32(&bar);
  if (threadIdx.x == 0) {
    ptx::mbar_init(b, 1);
    abort_flag = 0;
    ptx::fence_mbar_init();
  }
  __syncthreads();
  const uint64_t t0 = ptx::globaltimer();
  bool ok = false;
  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) ok = wait_one(b, 0, &abort_flag, status, limit_ns);
  } else {
    ok = wait_warp(b, 0, &abort_flag, status, limit_ns);
  }
  if (ok) atomicOr(status, 0x80000000u);
  __syncthreads();
  if (threadIdx.x == 0) *elapsed_ns = ptx::globaltimer() - t0;
}

int selftest_wait_timeout(uint64_t limit_ns, uint32_t* status, unsigned long long* elapsed_ns) {
  uint32_t* d_status = nullptr;
  unsigned long long* d_el = nullptr;
  cudaError_t e = cudaMalloc(&d_status, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&d_el, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(d_status, 0, sizeof(uint32_t));
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 64>>>(limit_ns, d_status, d_el);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(status, d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(elapsed_ns, d_el, sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  cudaFree(d_status);
  cudaFree(d_el);
  return e == cudaSuccess ? 0 : report_error(USAPHMP_ECUDA, std::string("wait self-test: ") + cudaGetErrorString(e));
}

}  // namespace usaphmp
