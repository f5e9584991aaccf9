// Allocation local search for fixed hubs, in fp64: sweeps over the spokes in
// ascending node order; spoke i moves from its hub a to the open hub b with
// the most negative change of objective (1), §3 (the lowest hub on equal
// changes), when that change is negative; sweeps repeat until one moves
// nothing or max_sweeps have run.  Hubs keep serving themselves (eq. 3).
//
// With M[l][u] = sum_j W[u][j] [s(j) = l] and N[l][u] = sum_j W[j][u] [s(j) = l]
// (the flows of node u to and from the spokes of hub slot l) and T the
// transfer-leg costs between hub slots (C between hubs, or the hub-path
// table), the cost of spoke i served by slot c, up to terms that do not
// depend on c, is
//   F(c) = chi O_i C[i,h_c] + delta D_i C[h_c,i]
//        + alpha (sum_l M[l][i] T[c][l] + N[l][i] T[l][c]
//                 + W_ii (T[c][c] - T[c][a] - T[a][c])),
// the W_ii terms replacing the pair (i, i) that M and N count under slot a
// (O_i, D_i: row and column sums of W).  The change of moving i from a to c
// is F(c) - F(a).  After a move, column i of W moves between rows a and b of
// M, and row i of W between those of N.
//
// One block per chromosome.  M and N live slot-major in a per-chromosome
// fp64 scratch (moves update two coalesced rows of each), each entry summed
// in ascending j as a pair of fp32 numbers (Knuth's TwoSum: the rounding
// error of every addition is carried in the low word; relative error about
// 2^-46) and stored as their fp64 sum.  The spokes are visited in windows of
// K whose M/N columns, C entries and flow sums are staged in shared memory;
// T stays in shared memory when it fits.  One thread per candidate slot
// evaluates F.
//
// fp64 arithmetic runs at a small fraction of the fp32 rate on this GPU, so
// every spoke is screened in fp32 first: each F(c) is computed in fp32 with
// the bound e(c) = (2p + 16) 2^-23 Fabs(c) on its error (Fabs: the same sum
// over absolute values; the rounding analysis of a (p + 8)-term sum with
// fp32 inputs gives (p + 8) 2^-24 Fabs, and the fp64 result is within a
// 2^-29 fraction of that).  When F(c) - e(c) > F(a) + e(a) for every c != a,
// the fp64 rule moves nothing and the spoke is done; otherwise F is
// evaluated in fp64 and decides.  A screened spoke costs one block barrier,
// an fp64 evaluation one more, a move one more.
#include "common.cuh"
#include "kernels.cuh"

namespace usaphmp {

namespace {
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr size_t kSmemBudget = 200 * 1024;

__host__ __device__ inline int t_stride(int p) { return p | 1; }  // odd: conflict-free fp64 rows
__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

// hi + lo += x with the rounding error of the addition kept in lo (TwoSum).
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bp = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  hi = s;
  lo = __fadd_rn(lo, e);
}

// Shared-memory layout of one block (byte offsets), T last so that it can be
// left out when it does not fit.
struct LsLayout {
  size_t mw, nw, cw, ctw, ow, dw, ww, f64, cl, scan, hs, start, pos, perm, sl, t, bytes;
  size_t mw32, nw32, oc32, dd32, ww32, g, ga, lo, t32;
  int K, t_smem, screen;
};

__host__ __device__ inline LsLayout ls_layout(int n, int p, int ns) {
  LsLayout L;
  L.K = p <= 64 ? 32 : (p <= 128 ? 16 : 8);
  size_t o = 0;
  L.mw = o; o = al16(o + sizeof(double) * L.K * p);
  L.nw = o; o = al16(o + sizeof(double) * L.K * p);
  L.cw = o; o = al16(o + sizeof(float) * L.K * p);
  L.ctw = o; o = al16(o + sizeof(float) * L.K * p);
  L.ow = o; o = al16(o + sizeof(double) * L.K);
  L.dw = o; o = al16(o + sizeof(double) * L.K);
  L.ww = o; o = al16(o + sizeof(double) * L.K);
  L.f64 = o; o = al16(o + sizeof(double) * 2 * (p + 1));  // two buffers each (alternate scans)
  L.cl = o; o = al16(o + sizeof(int) * 2 * (p + 1));
  L.scan = o; o = al16(o + sizeof(int) * 4);
  L.hs = o; o = al16(o + sizeof(int) * p);
  L.start = o; o = al16(o + sizeof(int) * (p + 1));
  L.pos = o; o = al16(o + sizeof(int) * p);
  L.perm = o; o = al16(o + sizeof(uint16_t) * n);
  L.sl = o; o = al16(o + (size_t)ns);
  L.mw32 = o; o = al16(o + sizeof(float) * L.K * p);
  L.nw32 = o; o = al16(o + sizeof(float) * L.K * p);
  L.oc32 = o; o = al16(o + sizeof(float) * L.K);
  L.dd32 = o; o = al16(o + sizeof(float) * L.K);
  L.ww32 = o; o = al16(o + sizeof(float) * L.K);
  L.g = o; o = al16(o + sizeof(float) * L.K * p);
  L.ga = o; o = al16(o + sizeof(float) * L.K * p);
  L.lo = o; o = al16(o + sizeof(float) * p);
  const size_t t32b = al16(sizeof(float) * p * t_stride(p));
  L.screen = (o + t32b <= kSmemBudget) ? 1 : 0;
  L.t32 = o;
  if (L.screen) o += t32b;
  L.t = o;
  const size_t tb = sizeof(double) * p * t_stride(p);
  L.t_smem = (o + tb <= kSmemBudget) ? 1 : 0;
  L.bytes = L.t_smem ? o + tb : o;
  return L;
}
}  // namespace

__host__ __device__ inline size_t scratch_doubles(int n, int p) {
  return 2 * (size_t)n * p + (size_t)p * t_stride(p);
}

size_t local_search_scratch_doubles(int n, int p) { return scratch_doubles(n, p); }

// O_i = sum_j W[i][j] and D_i = sum_j W[j][i] in fp64, ascending j (one
// thread per node; WT is W transposed, so both reads are coalesced).
__global__ void k_ls_flows64(const float* __restrict__ W, const float* __restrict__ WT, int n, int ldw,
                             double* __restrict__ OD) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double o = 0.0, d = 0.0;
  for (int j = 0; j < n; ++j) {
    o += (double)WT[(long long)j * ldw + i];
    d += (double)W[(long long)j * ldw + i];
  }
  OD[i] = o;
  OD[n + i] = d;
}

void launch_ls_prepare(const float* W, int n, int ldw, float* WT, double* OD, cudaStream_t s) {
  launch_transpose(W, WT, n, ldw, s);
  k_ls_flows64<<<(n + 127) / 128, 128, 0, s>>>(W, WT, n, ldw, OD);
}

// fp32 dot products of the staged spokes k0 <= k < k1 with every slot c:
// G[k][c] = sum_l M[l][i] T[c][l] + N[l][i] T[l][c] and Ga the same over
// |M|, |N| (all threads of the block).
__device__ __forceinline__ void window_dots(const float* Mw32, const float* Nw32, const float* T32, float* G,
                                            float* Ga, int k0, int k1, int p, int tp) {
  for (int e = threadIdx.x + k0 * p; e < k1 * p; e += kThreads) {
    const int k = e / p, c = e - k * p;
    const float* mw = Mw32 + k * p;
    const float* nw = Nw32 + k * p;
    const float* Tc = T32 + c * tp;
    float gm = 0.f, gn = 0.f, am = 0.f, an = 0.f;
#pragma unroll 4
    for (int l = 0; l < p; ++l) {
      const float tcl = Tc[l], tlc = T32[l * tp + c], ml = mw[l], nl = nw[l];
      gm = __fmaf_rn(ml, tcl, gm);
      gn = __fmaf_rn(nl, tlc, gn);
      am = __fmaf_rn(fabsf(ml), tcl, am);
      an = __fmaf_rn(fabsf(nl), tlc, an);
    }
    G[e] = gm + gn;
    Ga[e] = am + an;
  }
}

__global__ void __launch_bounds__(kThreads) k_local_search(DevInst in, const float* __restrict__ WT,
                                                           const double* __restrict__ OD,
                                                           const int32_t* __restrict__ hubs,
                                                           uint8_t* __restrict__ slot, int max_sweeps,
                                                           double* __restrict__ scratch, int32_t* moves_out,
                                                           int32_t* sweeps_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int b = blockIdx.x, n = in.n, p = in.p, ldw = in.ldw, tp = t_stride(p);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const LsLayout L = ls_layout(n, p, in.ns);
  const int K = L.K;
  double* Mw = reinterpret_cast<double*>(smem + L.mw);
  double* Nw = reinterpret_cast<double*>(smem + L.nw);
  float* Cw = reinterpret_cast<float*>(smem + L.cw);
  float* CTw = reinterpret_cast<float*>(smem + L.ctw);
  double* Ow = reinterpret_cast<double*>(smem + L.ow);
  double* Dw = reinterpret_cast<double*>(smem + L.dw);
  double* Ww = reinterpret_cast<double*>(smem + L.ww);
  double* F64 = reinterpret_cast<double*>(smem + L.f64);
  int* cl = reinterpret_cast<int*>(smem + L.cl);
  int* scan = reinterpret_cast<int*>(smem + L.scan);
  int* hs = reinterpret_cast<int*>(smem + L.hs);
  int* start = reinterpret_cast<int*>(smem + L.start);
  int* pos = reinterpret_cast<int*>(smem + L.pos);
  uint16_t* perm = reinterpret_cast<uint16_t*>(smem + L.perm);
  uint8_t* sl = smem + L.sl;
  float* Mw32 = reinterpret_cast<float*>(smem + L.mw32);
  float* Nw32 = reinterpret_cast<float*>(smem + L.nw32);
  float* Oc32 = reinterpret_cast<float*>(smem + L.oc32);
  float* Dd32 = reinterpret_cast<float*>(smem + L.dd32);
  float* Ww32 = reinterpret_cast<float*>(smem + L.ww32);
  float* G = reinterpret_cast<float*>(smem + L.g);
  float* Ga = reinterpret_cast<float*>(smem + L.ga);
  float* lo_s = reinterpret_cast<float*>(smem + L.lo);
  float* T32 = reinterpret_cast<float*>(smem + L.t32);

  const float* __restrict__ W = in.W;
  const float* __restrict__ C = in.C;
  const float* __restrict__ CT = in.CT;
  double* M = scratch + (long long)b * scratch_doubles(n, p);
  double* N = M + (size_t)n * p;
  double* T = L.t_smem ? reinterpret_cast<double*>(smem + L.t) : N + (size_t)n * p;
  uint8_t* gsl = slot + (long long)b * in.ns;

  for (int k = tid; k < p; k += kThreads) {
    const int v = hubs[(long long)b * p + k];
    hs[k] = (v >= 0 && v < n) ? v : 0;
  }
  for (int l = tid; l <= p; l += kThreads) start[l] = 0;
  __syncthreads();
  for (int i = tid; i < n; i += kThreads) {
    const int s = min((int)gsl[i], p - 1);
    sl[i] = (uint8_t)s;
    atomicAdd(&start[s + 1], 1);
  }
  // T: hub-to-hub leg costs; the hub-path table (Floyd-Warshall, zero
  // diagonal) under hub-path routing.
  for (int e = tid; e < p * p; e += kThreads) {
    const int a = e / p, c = e - a * p;
    T[a * tp + c] = (in.routing && a == c) ? 0.0 : (double)C[(long long)hs[a] * ldw + hs[c]];
  }
  __syncthreads();
  if (tid == 0)
    for (int l = 0; l < p; ++l) start[l + 1] += start[l];
  if (in.routing) {
    for (int m = 0; m < p; ++m) {
      for (int e = tid; e < p * p; e += kThreads) {
        const int a = e / p, c = e - a * p;
        const double v = T[a * tp + m] + T[m * tp + c];
        if (v < T[a * tp + c]) T[a * tp + c] = v;
      }
      __syncthreads();
    }
  }
  __syncthreads();
  if (L.screen)
    for (int e = tid; e < p * p; e += kThreads) {
      const int a = e / p, c = e - a * p;
      T32[a * tp + c] = (float)T[a * tp + c];
    }
  // nodes grouped by slot, ascending node order within a slot (stable
  // counting sort, one warp, 32 nodes per step)
  if (warp == 0) {
    for (int l = lane; l < p; l += 32) pos[l] = start[l];
    __syncwarp();
    for (int j0 = 0; j0 < n; j0 += 32) {
      const int j = j0 + lane;
      const int s = j < n ? (int)sl[j] : 256 + lane;
      const unsigned grp = __match_any_sync(0xffffffffu, s);
      if (j < n) perm[pos[s] + __popc(grp & ((1u << lane) - 1u))] = (uint16_t)j;
      __syncwarp();
      if (j < n && lane == 31 - __clz(grp)) pos[s] += __popc(grp);
      __syncwarp();
    }
  }
  __syncthreads();
  // M and N, each entry summed in ascending j (coalesced over u)
  for (int u = tid; u < n; u += kThreads) {
    for (int l = 0; l < p; ++l) {
      float mh = 0.f, ml = 0.f, qh = 0.f, ql = 0.f;
      const int e = start[l + 1];
      for (int t = start[l]; t < e; ++t) {
        const long long j = perm[t];
        two_sum_acc(mh, ml, WT[j * ldw + u]);
        two_sum_acc(qh, ql, W[j * ldw + u]);
      }
      M[(size_t)l * n + u] = (double)mh + (double)ml;
      N[(size_t)l * n + u] = (double)qh + (double)ql;
    }
  }
  __syncthreads();

  const double chi = in.chi_d, alpha = in.alpha_d, delta = in.delta_d;
  const float alpha32 = (float)alpha;
  const float eps = (float)(2 * p + 16) * 1.1920929e-7f;  // (2p + 16) 2^-23
  int moves = 0, sweeps = 0, q = 0;
  for (int sw = 0; sw < max_sweeps; ++sw) {
    ++sweeps;
    bool moved = false;
    for (int i0 = 0; i0 < n; i0 += K) {
      const int kk = min(K, n - i0);
      // (loads of four entries issued before their stores: one L2 round
      // trip per four)
      for (int e0 = tid; e0 < kk * p; e0 += 4 * kThreads) {
        double m[4], r[4];
        float cv[4], ctv[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const int e = min(e0 + x * kThreads, kk * p - 1);
          const int l = e / kk, i = i0 + e - l * kk;
          m[x] = M[(size_t)l * n + i];
          r[x] = N[(size_t)l * n + i];
          cv[x] = C[(long long)i * ldw + hs[l]];
          ctv[x] = CT[(long long)i * ldw + hs[l]];
        }
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const int e = e0 + x * kThreads;
          if (e < kk * p) {
            const int l = e / kk, k = e - l * kk;
            Mw[k * p + l] = m[x];
            Nw[k * p + l] = r[x];
            Mw32[k * p + l] = (float)m[x];
            Nw32[k * p + l] = (float)r[x];
            Cw[k * p + l] = cv[x];
            CTw[k * p + l] = ctv[x];
          }
        }
      }
      for (int k = tid; k < kk; k += kThreads) {
        const int i = i0 + k;
        const float wii = W[(long long)i * ldw + i];
        Ow[k] = OD[i];
        Dw[k] = OD[n + i];
        Ww[k] = (double)wii;
        Oc32[k] = (float)(chi * OD[i]);
        Dd32[k] = (float)(delta * OD[n + i]);
        Ww32[k] = wii;
      }
      __syncthreads();
      if (L.screen) {
        window_dots(Mw32, Nw32, T32, G, Ga, 0, kk, p, tp);
        __syncthreads();
      }
      int k = 0;
      while (true) {
        // warp 0 walks the spokes from k until one that the fp32 screen
        // cannot settle, and lists the slots to evaluate in fp64 there:
        // cl[0] = its own slot a, then every c != a with F(c) - e(c) not
        // above F(a) + e(a), ascending.  scan, cl and F64 alternate between
        // two buffers, so that the next scan never overwrites what a slower
        // warp still reads.
        int* clq = cl + q * (p + 1);
        int* scq = scan + 2 * q;
        double* Fq = F64 + q * (p + 1);
        q ^= 1;
        if (warp == 0) {
          int kx = k;
          for (; kx < kk; ++kx) {
            const int i = i0 + kx;
            const int a = sl[i];
            if (hs[a] == i) continue;  // a hub serves itself
            float hia = __int_as_float(0x7f800000);
            if (L.screen) {
              float lo = __int_as_float(0x7f800000);
              const float oc = Oc32[kx], dd = Dd32[kx], wi = Ww32[kx];
              for (int c = lane; c < p; c += 32) {
                const float* Tc = T32 + c * tp;
                const float cp = wi * Tc[c], cn = wi * (Tc[a] + T32[a * tp + c]);
                const float acc = oc * Cw[kx * p + c] + dd * CTw[kx * p + c];
                const float F = acc + alpha32 * (G[kx * p + c] + cp - cn);
                const float Fabs = acc + alpha32 * (Ga[kx * p + c] + cp + cn);
                const float e = eps * Fabs;
                if (c == a) {
                  hia = F + e;
                } else {
                  float v = F - e;
                  if (!(v == v)) v = __int_as_float(0xff800000);  // NaN: undecided (-inf)
                  lo_s[c] = v;
                  lo = fminf(lo, v);
                }
              }
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
              hia = __shfl_sync(0xffffffffu, hia, a & 31);
              if (lo > hia) continue;  // the fp64 rule moves nothing here
            }
            int cnt = 1;
            for (int c0 = 0; c0 < p; c0 += 32) {
              const int c = c0 + lane;
              const bool take = c < p && c != a && (!L.screen || !(lo_s[c] > hia));
              const unsigned bal = __ballot_sync(0xffffffffu, take);
              if (take) clq[cnt + __popc(bal & ((1u << lane) - 1u))] = c;
              cnt += __popc(bal);
            }
            if (lane == 0) {
              clq[0] = a;
              scq[1] = cnt;
            }
            break;
          }
          if (lane == 0) scq[0] = kx;
        }
        __syncthreads();
        const int kx = scq[0];
        if (kx >= kk) break;
        const int cnt = scq[1];
        const int i = i0 + kx;
        const int a = clq[0];
        // fp64 F of the listed slots: one warp per slot, lanes over l
        for (int idx = warp; idx < cnt; idx += kWarps) {
          const int c = clq[idx];
          const double* mw = Mw + kx * p;
          const double* nw = Nw + kx * p;
          double t = 0.0;
          for (int l = lane; l < p; l += 32) t = fma(mw[l], T[c * tp + l], fma(nw[l], T[l * tp + c], t));
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
          if (lane == 0) {
            const double g = t + Ww[kx] * (T[c * tp + c] - T[c * tp + a] - T[a * tp + c]);
            Fq[idx] = chi * Ow[kx] * (double)Cw[kx * p + c] + delta * Dw[kx] * (double)CTw[kx * p + c] + alpha * g;
          }
        }
        __syncthreads();
        const double fa = Fq[0];
        double best = __longlong_as_double(0x7ff0000000000000ll);
        int nb = p;
        for (int idx = 1; idx < cnt; ++idx) {
          const double F = Fq[idx];
          const int c = clq[idx];
          if (F < best || (F == best && c < nb)) {
            best = F;
            nb = c;
          }
        }
        k = kx + 1;
        if (!(nb < p && best < fa)) continue;  // no move
        if (tid == 0) {
          sl[i] = (uint8_t)nb;
          gsl[i] = (uint8_t)nb;
        }
        for (int u0 = tid; u0 < n; u0 += 4 * kThreads) {
          double wui[4], wiu[4], ma[4], mb[4], qa[4], qb[4];
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            const int u = min(u0 + x * kThreads, n - 1);
            wui[x] = (double)WT[(long long)i * ldw + u];
            wiu[x] = (double)W[(long long)i * ldw + u];
            ma[x] = M[(size_t)a * n + u];
            mb[x] = M[(size_t)nb * n + u];
            qa[x] = N[(size_t)a * n + u];
            qb[x] = N[(size_t)nb * n + u];
          }
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            const int u = u0 + x * kThreads;
            if (u < n) {
              M[(size_t)a * n + u] = ma[x] - wui[x];
              M[(size_t)nb * n + u] = mb[x] + wui[x];
              N[(size_t)a * n + u] = qa[x] - wiu[x];
              N[(size_t)nb * n + u] = qb[x] + wiu[x];
              const int k2 = u - i0;
              if (k2 > kx && k2 < kk) {  // the staged copies of the spokes still to visit
                const double sa = Mw[k2 * p + a] - wui[x], sb = Mw[k2 * p + nb] + wui[x];
                const double ta = Nw[k2 * p + a] - wiu[x], tb = Nw[k2 * p + nb] + wiu[x];
                Mw[k2 * p + a] = sa;
                Mw[k2 * p + nb] = sb;
                Nw[k2 * p + a] = ta;
                Nw[k2 * p + nb] = tb;
                Mw32[k2 * p + a] = (float)sa;
                Mw32[k2 * p + nb] = (float)sb;
                Nw32[k2 * p + a] = (float)ta;
                Nw32[k2 * p + nb] = (float)tb;
              }
            }
          }
        }
        ++moves;
        moved = true;
        __syncthreads();
        if (L.screen && k < kk) {
          window_dots(Mw32, Nw32, T32, G, Ga, k, kk, p, tp);
          __syncthreads();
        }
      }
    }
    if (!moved) break;
  }
  if (tid == 0) {
    if (moves_out) moves_out[b] = moves;
    if (sweeps_out) sweeps_out[b] = sweeps;
  }
}

void launch_local_search(const DevInst& in, const float* WT, const double* OD, int B, const int32_t* hubs,
                         uint8_t* slot, int max_sweeps, double* scratch, int32_t* moves, int32_t* sweeps,
                         cudaStream_t s) {
  if (B <= 0) return;
  const LsLayout L = ls_layout(in.n, in.p, in.ns);
  if (L.bytes > 48 * 1024)
    cudaFuncSetAttribute(k_local_search, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
  k_local_search<<<B, kThreads, L.bytes, s>>>(in, WT, OD, hubs, slot, max_sweeps, scratch, moves, sweeps);
}

}  // namespace usaphmp
