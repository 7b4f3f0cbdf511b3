// The one-CTA NNS-EMD solver: every step of a round of Alg. 1 (Sec. III-A)
// for active sets of at most CAP points per side, with all per-point state in
// one CTA's shared memory.  Used for the tail rounds of a large solve, for
// batches of small pairs (one pair per CTA) and by the allocation-free entry
// point.
//
// The coordinates are a policy:
//   GeoSmem   (d <= 8)  coordinates of the active points live in shared
//                       memory and move with the compaction;
//   GeoGlobal (d > 8)   coordinates stay in global memory (L2) and are read
//                       by original index; the NNS step runs 64 x 64 tiles
//                       staged in shared memory by 256-thread groups;
//   GeoSmemCluster      GeoSmem on every CTA of a thread-block cluster: each
//                       CTA holds the whole state, finds the nearest
//                       supplier of its slice of the consumers and sends the
//                       keys to every CTA through distributed shared memory;
//                       the rest of the round runs, identically, in every
//                       CTA (one of them writes the results).
// Grouping, greedy order, flow and compaction are the same for both.
#pragma once

#include <cooperative_groups.h>
#include <math_constants.h>

#include "common.cuh"
#include "kernels.h"

namespace nnsemd {

constexpr int FIN_THREADS = 1024;

// Exclusive prefix sum over the block; `total` receives the block sum.
NNS_DEV int block_scan_excl(int v, int* wt, int& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) wt[w] = x;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    int t = lane < nw ? wt[lane] : 0;
    int y = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += u;
    }
    wt[lane] = y - t;
    if (lane == 31) wt[32] = y;
  }
  __syncthreads();
  total = wt[32];
  const int r = wt[w] + x - v;
  __syncthreads();
  return r;
}

// Per-point state of a pair solved in one CTA (no coordinates).
template <int CAP>
struct CtaCore {
  double sres[CAP];
  double cres[CAP];
  int iidx[CAP];
  int jidx[CAP];
  unsigned long long nnk[CAP];
  unsigned long long mem[CAP];
  unsigned long long mem2[CAP];
  int cnt[CAP + 1];
  int off[CAP + 1];
  unsigned long long acc[XS_LIMBS];
  int wt[33];
  int mt, nt;
  unsigned nflow;
  double total;
  // running totals handed back by the one-warp rounds (warp_rounds)
  unsigned long long w_nnz;
  long long w_rounds, w_pe;
};

struct CtaOut {
  unsigned long long* acc;       // exact accumulator for R (shared, nullable)
  int32_t* plan_i;               // plan (nullable)
  int32_t* plan_j;
  double* plan_f;
  long long plan_cap;
  double* s_glob;                // residual write-back by original index (nullable)
  double* c_glob;
  unsigned* err;
  // Deferred costing (fl_i nullable): every flow's original (i, j, f) is
  // recorded in fl_* (global, slot = running flow count) during the rounds,
  // and the cost terms and plan entries of all of them are computed in one
  // pass after the last round from the original coordinates x, y (row
  // stride d).  The FP64 distance chain then costs its latency once per
  // solve instead of once per round.
  int32_t* fl_i;
  int32_t* fl_j;
  double* fl_f;
  const float* x;
  const float* y;
  int d;
  // serving order: greedy (0) or random (1) with the seed and the global
  // index of the loop's first round (the random protocol's keys)
  int protocol;
  unsigned long long seed;
  long long round_base;
  // nonzero: run the rounds without writing any flow, plan entry, cost term
  // or residual out (a CTA of a cluster whose results another CTA writes)
  int quiet;
  long long fl_cap;  // > 0: capacity of fl_* (a flow beyond it raises EF_CAPACITY)
};

// --------------------------------------------------------------------------
// coordinate policies
// --------------------------------------------------------------------------

template <int D, int DP, bool L1, int CAP>
struct GeoSmem {
  static constexpr int kDP = DP;
  static constexpr int kD = D;
  static constexpr int kThreads = FIN_THREADS;  // threads of the CTA
  float xs[CAP * DP];
  float ys[CAP * DP];
  struct PX { float v[DP]; };

  // FP32 decision key of supplier coordinates xv against consumer
  // coordinates yv (the metric of this policy)
  static NNS_DEV float key_pair(const float* xv, const float* yv) {
    return L1 ? key32<METRIC_L1>(xv, yv, D) : key32<METRIC_SQL2>(xv, yv, D);
  }

  NNS_DEV void load_x(int p, PX& r) const {
#pragma unroll
    for (int k = 0; k < DP; ++k) r.v[k] = xs[p * DP + k];
  }
  NNS_DEV void store_x(int p, const PX& r) {
#pragma unroll
    for (int k = 0; k < DP; ++k) xs[p * DP + k] = r.v[k];
  }
  NNS_DEV void load_y(int q, PX& r) const {
#pragma unroll
    for (int k = 0; k < DP; ++k) r.v[k] = ys[q * DP + k];
  }
  NNS_DEV void store_y(int q, const PX& r) {
#pragma unroll
    for (int k = 0; k < DP; ++k) ys[q * DP + k] = r.v[k];
  }
  template <int C>
  NNS_DEV double dist64(const CtaCore<C>& S, int p, int q, int metric) const {
    return cost_dist64(xs + p * DP, ys + q * DP, D, metric);
  }
  // S.nnk[q] = (key32 bits << 32 | p) of the nearest active supplier;
  // returns S.nnk (every NNS policy returns the array holding the keys)
  template <int C>
  NNS_DEV const unsigned long long* nns(CtaCore<C>& S, int mt, int nt, long long = 0) const {
    const int tid = threadIdx.x, T = blockDim.x;
    int split = 1;
    while (split < 32 && nt * split * 2 <= T) split <<= 1;
    for (int base = 0; base < nt; base += T / split) {
      const int q = base + tid / split, part = tid & (split - 1);
      unsigned long long bk = ~0ULL;
      if (q < nt) {
        float yv[D];
#pragma unroll
        for (int k = 0; k < D; ++k) yv[k] = ys[q * DP + k];
        float best = CUDART_INF_F;
        int bp = -1;
        for (int p = part; p < mt; p += split) {
          const float v = L1 ? key32<METRIC_L1>(xs + p * DP, yv, D) : key32<METRIC_SQL2>(xs + p * DP, yv, D);
          if (bp < 0 || v < best) { best = v; bp = p; }
        }
        if (bp >= 0) bk = pack_key(best, (unsigned)bp);
      }
      for (int o = 1; o < split; o <<= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, bk, o);
        bk = other < bk ? other : bk;
      }
      if (q < nt && part == 0) S.nnk[q] = bk;
    }
    __syncthreads();
    return S.nnk;
  }
};

// The NNS step of GeoSmem spread over the CTAs of a cluster.  CTA r of R
// (R >= 8) scans the consumers [r nt / R, (r+1) nt / R) against every active
// supplier and stores each key into the receive buffer of every CTA of the
// cluster; one cluster barrier (release / acquire) then makes all nt keys
// visible in every CTA, and the round's later steps read them there.  The
// receive buffer alternates between two halves by round parity: a CTA can
// write round t + 1's keys into a peer while the peer still reads round t's,
// never round t + 2's (that needs the peer at the barrier of round t + 1,
// after its round t).  Every CTA holds identical state, so every later step
// gives identical results in all of them.
//
// Inside a CTA a warp takes 64 consumers of the slice (two per lane, packed
// in FP32x2 registers) and a contiguous chunk of the suppliers; all lanes
// read the same supplier (a shared-memory broadcast), so one load feeds 64
// pairs.  Each lane keeps the first minimum of its chunk (ascending
// positions); the chunks merge through a 64-bit atomicMin on (key bits,
// position), which keeps the lowest-index tie-break.
template <int D, int DP, bool L1, int CAP, int NT>
struct GeoSmemCluster : GeoSmem<D, DP, L1, CAP> {
  static constexpr int kThreads = NT;     // threads of each CTA
  static constexpr int kSlice = CAP / 8;  // consumers per CTA at most (R >= 8)
  unsigned long long xk[2][CAP];          // receive buffers (round parity)
  unsigned long long red[kSlice];         // the slice's keys merged over chunks; all ones between rounds

  NNS_DEV float key_one(const float* xv, const float* yv) const {
    return L1 ? key32<METRIC_L1>(xv, yv, D) : key32<METRIC_SQL2>(xv, yv, D);
  }
  // keys of supplier p against the two consumers packed in y2
  NNS_DEV unsigned long long key_two(int p, const unsigned long long* y2, const float* ya, const float* yb) const {
    float xv[D];
#pragma unroll
    for (int k = 0; k < D; ++k) xv[k] = this->xs[p * DP + k];
    if (L1) return f2_pack(key_one(xv, ya), key_one(xv, yb));
    unsigned long long t = f2_sub(f2_pack(xv[0], xv[0]), y2[0]);
    unsigned long long acc = f2_mul(t, t);
#pragma unroll
    for (int k = 1; k < D; ++k) {
      t = f2_sub(f2_pack(xv[k], xv[k]), y2[k]);
      acc = f2_fma(t, t, acc);
    }
    return acc;
  }

  // Set red to all ones (before the first round; each round restores it).
  NNS_DEV void init() {
    for (int i = threadIdx.x; i < kSlice; i += blockDim.x) red[i] = ~0ULL;
  }

  template <int C>
  NNS_DEV const unsigned long long* nns(CtaCore<C>&, int mt, int nt, long long round) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const unsigned rank = cl.block_rank(), ncl = cl.num_blocks();
    const int h = (int)(round & 1);
    // (32-bit arithmetic: nt, mt <= CAP and R, chunks <= 32)
    const int q0 = (int)((unsigned)nt * rank / ncl), q1 = (int)((unsigned)nt * (rank + 1) / ncl);
    const int tid = threadIdx.x, T = blockDim.x, ns = q1 - q0;
    const int cgroups = (ns + 63) >> 6, nw = T >> 5, w = tid >> 5, lane = tid & 31;
    if (cgroups > 0 && w < nw / cgroups * cgroups) {
      const int chunks = nw / cgroups, ch = w / cgroups;
      const int qa = 64 * (w % cgroups) + lane, qb = qa + 32;  // slice positions
      float ya[D], yb[D];
      unsigned long long y2[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        ya[k] = qa < ns ? this->ys[(q0 + qa) * DP + k] : 0.f;
        yb[k] = qb < ns ? this->ys[(q0 + qb) * DP + k] : 0.f;
        y2[k] = f2_pack(ya[k], yb[k]);
      }
      const int s0 = (int)((unsigned)(mt * ch) / (unsigned)chunks);
      const int s1 = (int)((unsigned)(mt * (ch + 1)) / (unsigned)chunks);
      if (s0 < s1) {
        unsigned long long kk = key_two(s0, y2, ya, yb);
        float ba = f2_lo(kk), bb = f2_hi(kk);
        int pa = s0, pb = s0;
        for (int p = s0 + 1; p < s1; ++p) {
          kk = key_two(p, y2, ya, yb);
          const float ka = f2_lo(kk), kb = f2_hi(kk);
          if (ka < ba) { ba = ka; pa = p; }
          if (kb < bb) { bb = kb; pb = p; }
        }
        if (qa < ns) atomicMin(&red[qa], pack_key(ba, (unsigned)pa));
        if (qb < ns) atomicMin(&red[qb], pack_key(bb, (unsigned)pb));
      }
    }
    __syncthreads();
    for (int i = tid; i < ns * (int)ncl; i += T) {
      const int r = i / ns, q = i - r * ns;
      cl.map_shared_rank(&xk[h][0], r)[q0 + q] = red[q];
    }
    cl.sync();
    // restore red for the next round (whose atomics follow this round's
    // barriers)
    for (int i = tid; i < ns; i += T) red[i] = ~0ULL;
    return xk[h];
  }
};

// ---- tiled FP32 NNS for d > 8 ---------------------------------------------

constexpr int TG_M = 64;        // consumers per tile
constexpr int TG_N = 64;        // suppliers per tile
constexpr int TG_K = 32;        // coordinates per staged chunk
constexpr int TG_THREADS = 256; // threads per group (4 x 4 pairs each)
constexpr int TG_PAD = 68;

struct __align__(16) TileSmem {
  float Xs[TG_K][TG_PAD];
  float Ys[TG_K][TG_PAD];
};

NNS_DEV void group_sync(int bar) {
  if (bar == 0) __syncthreads();
  else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(TG_THREADS) : "memory");
}

// One 256-thread group: for the consumers cons[c0 .. c0+nc) (positions in the
// active consumer list, or c0.. directly when cons is null) and the suppliers
// at positions [p0, p1), the lowest (key32 bits << 32 | position).  Each
// thread owns 4 consumers x 4 suppliers of a tile; the key of every pair is
// accumulated over k = 0..d-1 in order (fma from +0, which equals the
// definition's first product), so it is bit-identical to key32.  Returns, in
// the threads with tx == 0, the keys of their 4 consumers (others: ~0).
template <bool L1>
NNS_DEV void group_nns_tile(const float* __restrict__ x, const int* __restrict__ ia, int p0, int p1,
                            const float* __restrict__ y, const int* __restrict__ ja, const int* __restrict__ cons,
                            int c0, int nc, int d, TileSmem& T, int gt, int bar, unsigned long long out[4]) {
  const int tx = gt & 15, ty = gt >> 4;
  float best[4];
  int bpos[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) { best[i] = CUDART_INF_F; bpos[i] = -1; }
  // loader mapping: row r of the tile, 8 consecutive coordinates
  const int lr = gt & 63, lk = (gt >> 6) * 8;
  const int cq = c0 + lr;
  const float* yrow = nullptr;
  if (lr < nc) yrow = y + (size_t)ja[cons ? cons[cq] : cq] * d;
  for (int pt = p0; pt < p1; pt += TG_N) {
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    const int sp = pt + lr;
    const float* xrow = sp < p1 ? x + (size_t)ia[sp] * d : nullptr;
    for (int k0 = 0; k0 < d; k0 += TG_K) {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = k0 + lk + e;
        T.Ys[lk + e][lr] = (yrow && k < d) ? yrow[k] : 0.f;
        T.Xs[lk + e][lr] = xrow ? (k < d ? xrow[k] : 0.f) : CUDART_NAN_F;
      }
      group_sync(bar);
#pragma unroll 8
      for (int k = 0; k < TG_K; ++k) {
        const float4 xv = *reinterpret_cast<const float4*>(&T.Xs[k][tx * 4]);
        const float4 yv = *reinterpret_cast<const float4*>(&T.Ys[k][ty * 4]);
        const float xa[4] = {xv.x, xv.y, xv.z, xv.w};
        const float ya[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float t = __fsub_rn(xa[j], ya[i]);
            acc[i][j] = L1 ? __fadd_rn(acc[i][j], fabsf(t)) : __fmaf_rn(t, t, acc[i][j]);
          }
      }
      group_sync(bar);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (acc[i][j] < best[i]) { best[i] = acc[i][j]; bpos[i] = pt + tx * 4 + j; }
  }
  // reduce over the 16 threads sharing each consumer (adjacent lanes)
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    unsigned long long k = bpos[i] >= 0 ? pack_key(best[i], (unsigned)bpos[i]) : ~0ULL;
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
      const unsigned long long other = __shfl_xor_sync(0xffffffffu, k, o);
      k = other < k ? other : k;
    }
    out[i] = k;
  }
}

template <bool L1, int CAP, int NT = FIN_THREADS>
struct GeoGlobal {
  static constexpr int kDP = 0;
  static constexpr int kThreads = NT;  // threads of the CTA (a multiple of TG_THREADS)
  const float* x;  // [m][d] original coordinates (global)
  const float* y;  // [n][d]
  int d;
  TileSmem tiles[NT / TG_THREADS];
  struct PX {};
  NNS_DEV void load_x(int, PX&) const {}
  NNS_DEV void store_x(int, const PX&) {}
  NNS_DEV void load_y(int, PX&) const {}
  NNS_DEV void store_y(int, const PX&) {}
  template <int C>
  NNS_DEV double dist64(const CtaCore<C>& S, int p, int q, int metric) const {
    return cost_dist64(x + (size_t)S.iidx[p] * d, y + (size_t)S.jidx[q] * d, d, metric);
  }
  template <int C>
  NNS_DEV const unsigned long long* nns(CtaCore<C>& S, int mt, int nt, long long = 0) {
    const int g = threadIdx.x / TG_THREADS, gt = threadIdx.x % TG_THREADS;
    const int ngroups = blockDim.x / TG_THREADS;
    for (int c0 = g * TG_M; c0 < nt; c0 += ngroups * TG_M) {
      unsigned long long out[4];
      group_nns_tile<L1>(x, S.iidx, 0, mt, y, S.jidx, nullptr, c0, min(TG_M, nt - c0), d, tiles[g], gt, 1 + g,
                         out);
      const int tx = gt & 15, ty = gt >> 4;
      if (tx == 0)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int q = c0 + ty * 4 + i;
          if (q < nt) S.nnk[q] = out[i];
        }
    }
    __syncthreads();
    return S.nnk;
  }
};

// Note: GeoGlobal passes the CTA's own index arrays (iidx, jidx) as the
// "position -> original index" maps, so positions are CTA-local.

// --------------------------------------------------------------------------
// compaction and rounds
// --------------------------------------------------------------------------

// Stable compaction of both active lists to the points with weight left.
// Warp w owns positions [32 IT w, 32 IT (w + 1)), lane l the positions
// 32 IT w + 32 k + l (coalesced shared-memory accesses); ballots give each
// kept point its rank inside the warp and one block scan the warps' offsets.
// Every kept value is loaded before the scan's barriers and stored after
// them, so the in-place moves never overwrite a value not yet read.
template <int CAP, class Geo>
NNS_DEV void cta_compact(CtaCore<CAP>& S, Geo& G) {
  constexpr int IT = (CAP + Geo::kThreads - 1) / Geo::kThreads;
  const int tid = threadIdx.x, lane = tid & 31;
  const int base = (tid >> 5) * 32 * IT;
  const unsigned lt = (1u << lane) - 1u;
  const int mt = S.mt, nt = S.nt;
  unsigned bs[IT], bc[IT];
  double sv[IT], cv[IT];
  int iv[IT], jv[IT];
  typename Geo::PX px[IT], py[IT];
  int ns = 0, nc = 0;
#pragma unroll
  for (int k = 0; k < IT; ++k) {
    const int p = base + 32 * k + lane;
    bool ks = false, kc = false;
    if (p < mt) {
      sv[k] = S.sres[p];
      ks = residual_positive(sv[k]);
      if (ks) { iv[k] = S.iidx[p]; G.load_x(p, px[k]); }
    }
    if (p < nt) {
      cv[k] = S.cres[p];
      kc = residual_positive(cv[k]);
      if (kc) { jv[k] = S.jidx[p]; G.load_y(p, py[k]); }
    }
    bs[k] = __ballot_sync(0xffffffffu, ks);
    bc[k] = __ballot_sync(0xffffffffu, kc);
    ns += __popc(bs[k]);
    nc += __popc(bc[k]);
  }
  int tot;
  const int ex = __shfl_sync(0xffffffffu, block_scan_excl(lane == 0 ? (ns | (nc << 16)) : 0, S.wt, tot), 0);
  int ps = ex & 0xffff, pc = ex >> 16;
#pragma unroll
  for (int k = 0; k < IT; ++k) {
    if ((bs[k] >> lane) & 1u) {
      const int d = ps + __popc(bs[k] & lt);
      S.sres[d] = sv[k];
      S.iidx[d] = iv[k];
      G.store_x(d, px[k]);
    }
    if ((bc[k] >> lane) & 1u) {
      const int d = pc + __popc(bc[k] & lt);
      S.cres[d] = cv[k];
      S.jidx[d] = jv[k];
      G.store_y(d, py[k]);
    }
    ps += __popc(bs[k]);
    pc += __popc(bc[k]);
  }
  // every thread read the old counts before the scan's barriers
  if (tid == 0) {
    S.mt = tot & 0xffff;
    S.nt = tot >> 16;
  }
  __syncthreads();
}

// Exclusive scan of in[0..n) into out[0..n) (n <= CAP, NT threads), returns
// the total.
template <int CAP, int NT>
NNS_DEV int block_scan_array(const int* in, int* out, int n, int* wt) {
  constexpr int IT = (CAP + NT - 1) / NT;
  int v[IT];
  int s = 0;
#pragma unroll
  for (int k = 0; k < IT; ++k) {
    const int i = threadIdx.x * IT + k;
    v[k] = i < n ? in[i] : 0;
    s += v[k];
  }
  int tot;
  int ex = block_scan_excl(s, wt, tot);
#pragma unroll
  for (int k = 0; k < IT; ++k) {
    const int i = threadIdx.x * IT + k;
    if (i < n) out[i] = ex;
    ex += v[k];
  }
  return tot;
}

// Active sets both at most warp_cap<Geo>() points go to warp_rounds (two
// per lane).  128 (four per lane) was measured slower on the colour-transfer
// tail than the 16-CTA cluster rounds for sets of 65..128 points (483 against
// 517 pairs/s for the whole solve).
template <class Geo>
NNS_DEV constexpr int warp_cap() { return 64; }

// The remaining rounds of a pair whose active sets both hold at most
// warp_cap<Geo>() points, run by the calling warp alone (shared-memory
// coordinates, kDP > 0): with a few dozen points left, a round of the
// block-wide steps below is mostly barrier latency, and one warp needs none.
// The same steps in the same arithmetic as cta_rounds, so every result is
// identical:
//   NNS     lane = consumer (q = lane, lane + 32, ...), a scan of every
//           active supplier in ascending position, first minimum kept;
//   order   every consumer's rank by (supplier position, serving key,
//           position), counted against all consumers; the members of a
//           group then lie in serving order, groups in supplier order;
//   flow    lane = supplier, the FP64 residual chain over its group;
//   compact ballots keep the points with residual left, in order.
template <int CAP, class Geo>
NNS_DEV void warp_rounds(CtaCore<CAP>& S, Geo& G, int metric, const CtaOut& O, unsigned long long& nnz,
                         long long& rounds, long long& pair_evals, long long round_limit) {
  constexpr int D = Geo::kD;
  constexpr int WH = warp_cap<Geo>() / 32;  // points per lane
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const bool deferred = O.fl_i != nullptr;
  for (;;) {
    const int mt = S.mt, nt = S.nt;
    if (mt == 0 || nt == 0) break;
    if (rounds >= round_limit) {
      if (lane == 0) atomicOr(O.err, EF_ITER);
      break;
    }
    if (lane == 0) S.nflow = 0;
    // ---- NNS: one pass over the suppliers (each read once, a broadcast)
    // for all WH consumers of the lane
    {
      float yv[WH][D], best[WH];
      int bp[WH];
#pragma unroll
      for (int h = 0; h < WH; ++h) {
        const int q = lane + 32 * h;
#pragma unroll
        for (int k = 0; k < D; ++k) yv[h][k] = q < nt ? G.ys[q * Geo::kDP + k] : 0.f;
        best[h] = CUDART_INF_F;
        bp[h] = -1;
      }
      for (int p = 0; p < mt; ++p) {
        float xv[D];
#pragma unroll
        for (int k = 0; k < D; ++k) xv[k] = G.xs[p * Geo::kDP + k];
#pragma unroll
        for (int h = 0; h < WH; ++h) {
          const float v = Geo::key_pair(xv, yv[h]);
          if (bp[h] < 0 || v < best[h]) { best[h] = v; bp[h] = p; }
        }
      }
#pragma unroll
      for (int h = 0; h < WH; ++h) {
        const int q = lane + 32 * h;
        if (q < nt) S.nnk[q] = pack_key(best[h], (unsigned)bp[h]);
      }
    }
    __syncwarp();
    // ---- order: the serving key of every consumer, then its rank
#pragma unroll
    for (int h = 0; h < WH; ++h) {
      const int q = lane + 32 * h;
      if (q < nt) {
        const unsigned long long key = S.nnk[q];
        const unsigned ord = O.protocol == 1 ? rp_key32(O.seed, O.round_base + rounds, S.jidx[q])
                                             : (unsigned)(key >> 32);
        S.mem[q] = ((key & 0xffffffffULL) << 32) | ord;
      }
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < WH; ++h) {
      const int q = lane + 32 * h;
      if (q < nt) {
        const unsigned long long mine = S.mem[q];
        int rank = 0;
        for (int u = 0; u < nt; ++u) {
          const unsigned long long o = S.mem[u];
          rank += (o < mine) | ((o == mine) & (u < q));
        }
        S.mem2[rank] = (unsigned long long)(unsigned)q;
      }
    }
    // group bounds of every supplier: members of lower suppliers, its own
#pragma unroll
    for (int h = 0; h < WH; ++h) {
      const int p = lane + 32 * h;
      if (p < mt) {
        int lo = 0, len = 0;
        for (int u = 0; u < nt; ++u) {
          const int pp = (int)(S.mem[u] >> 32);
          lo += pp < p;
          len += pp == p;
        }
        S.off[p] = lo;
        S.cnt[p] = len;
      }
    }
    __syncwarp();
    // ---- flow, one supplier per lane
#pragma unroll
    for (int h = 0; h < WH; ++h) {
      const int p = lane + 32 * h;
      if (p < mt && S.cnt[p] > 0) {
        const int b = S.off[p], en = b + S.cnt[p];
        double s = S.sres[p];
        for (int r = b; r < en; ++r) {
          if (!residual_positive(s)) break;
          const int q = (int)(S.mem2[r] & 0xffffffffULL);
          double c = S.cres[q];
          const double f = greedy_step(s, c);
          S.cres[q] = c;
          const unsigned k = atomicAdd(&S.nflow, 1u);
          if (O.quiet) {
          } else if (deferred) {
            const unsigned long long slot = nnz + k;
            if (O.fl_cap && (long long)slot >= O.fl_cap) {
              atomicOr(O.err, EF_CAPACITY);
              continue;
            }
            O.fl_i[slot] = S.iidx[p];
            O.fl_j[slot] = S.jidx[q];
            O.fl_f[slot] = f;
            if (O.c_glob) O.c_glob[S.jidx[q]] = c;
          } else {
            // (mem and nnk are free again: the order is in mem2)
            S.mem[k] = ((unsigned long long)p << 32) | (unsigned)q;
            S.nnk[k] = (unsigned long long)__double_as_longlong(f);
          }
        }
        S.sres[p] = s;
        if (O.s_glob) O.s_glob[S.iidx[p]] = s;
      }
    }
    __syncwarp();
    const unsigned nflow = S.nflow;
    if (!(deferred || O.quiet)) {
      for (unsigned base = 0; base < nflow; base += 32) {  // the whole warp (xs_add_warp)
        const unsigned k = base + lane;
        double term = 0.0;
        if (k < nflow) {
          const unsigned long long pq = S.mem[k];
          const int p = (int)(pq >> 32), q = (int)(pq & 0xffffffffULL);
          const double f = __longlong_as_double((long long)S.nnk[k]);
          term = __dmul_rn(f, G.dist64(S, p, q, metric));
          const unsigned long long slot = nnz + k;
          if (O.plan_i) {
            if ((long long)slot < O.plan_cap) {
              O.plan_i[slot] = S.iidx[p];
              O.plan_j[slot] = S.jidx[q];
              O.plan_f[slot] = f;
            } else {
              atomicOr(O.err, EF_CAPACITY);
            }
          }
          if (O.c_glob) O.c_glob[S.jidx[q]] = S.cres[q];
        }
        if (O.acc) xs_add_warp(O.acc, term);  // one call site for the whole warp
      }
      __syncwarp();
    }
    nnz += nflow;
    rounds += 1;
    pair_evals += (long long)mt * nt;
    // ---- compaction: every kept value is read before any is written
    double sv[WH], cv[WH];
    int iv[WH], jv[WH];
    typename Geo::PX px[WH], py[WH];
    unsigned bs[WH], bc[WH];
#pragma unroll
    for (int h = 0; h < WH; ++h) {
      const int i = lane + 32 * h;
      bool ks = false, kc = false;
      if (i < mt) {
        sv[h] = S.sres[i];
        ks = residual_positive(sv[h]);
        if (ks) { iv[h] = S.iidx[i]; G.load_x(i, px[h]); }
      }
      if (i < nt) {
        cv[h] = S.cres[i];
        kc = residual_positive(cv[h]);
        if (kc) { jv[h] = S.jidx[i]; G.load_y(i, py[h]); }
      }
      bs[h] = __ballot_sync(0xffffffffu, ks);
      bc[h] = __ballot_sync(0xffffffffu, kc);
    }
    __syncwarp();
    int ps = 0, pc = 0;
#pragma unroll
    for (int h = 0; h < WH; ++h) {
      if ((bs[h] >> lane) & 1u) {
        const int dd = ps + __popc(bs[h] & lt);
        S.sres[dd] = sv[h];
        S.iidx[dd] = iv[h];
        G.store_x(dd, px[h]);
      }
      if ((bc[h] >> lane) & 1u) {
        const int dd = pc + __popc(bc[h] & lt);
        S.cres[dd] = cv[h];
        S.jidx[dd] = jv[h];
        G.store_y(dd, py[h]);
      }
      ps += __popc(bs[h]);
      pc += __popc(bc[h]);
    }
    __syncwarp();
    if (lane == 0) {
      S.mt = ps;
      S.nt = pc;
    }
    __syncwarp();
  }
}

// Rounds of Alg. 1 until one active side is empty.  nnz, rounds and
// pair_evals are running totals (identical in every thread on return).
// With shared-memory coordinates, the rounds after both active sets fit
// warp_cap<Geo>() run in warp 0 alone (warp_rounds) while the other warps
// wait.
template <int CAP, class Geo>
NNS_DEV void cta_rounds(CtaCore<CAP>& S, Geo& G, int metric, const CtaOut& O, unsigned long long& nnz,
                        long long& rounds, long long& pair_evals, long long round_limit) {
  const int tid = threadIdx.x;
  const int T = blockDim.x;
  const unsigned long long nnz0 = nnz;
  for (;;) {
    const int mt = S.mt, nt = S.nt;
    if (mt == 0 || nt == 0) break;
    if (rounds >= round_limit) {
      if (tid == 0) atomicOr(O.err, EF_ITER);
      break;
    }
    if constexpr (Geo::kDP > 0) {
      if (mt <= warp_cap<Geo>() && nt <= warp_cap<Geo>()) {
        if (tid < 32) {
          warp_rounds(S, G, metric, O, nnz, rounds, pair_evals, round_limit);
          if (tid == 0) {
            S.w_nnz = nnz;
            S.w_rounds = rounds;
            S.w_pe = pair_evals;
          }
        }
        __syncthreads();
        nnz = S.w_nnz;
        rounds = S.w_rounds;
        pair_evals = S.w_pe;
        break;
      }
    }
    // group counters of this round (the NNS step ends with a barrier)
    for (int p = tid; p < mt; p += T) S.cnt[p] = 0;
    if (tid == 0) S.nflow = 0;
    // ---- NNS: nearest active supplier of every active consumer
    const unsigned long long* nk = G.nns(S, mt, nt, rounds);
    // ---- group the consumers by their supplier
    for (int q = tid; q < nt; q += T) atomicAdd(&S.cnt[(int)(nk[q] & 0xffffffffULL)], 1);
    __syncthreads();
    {
      const int tot = block_scan_array<CAP, Geo::kThreads>(S.cnt, S.off, mt, S.wt);
      if (tid == 0) S.off[mt] = tot;
    }
    __syncthreads();
    for (int q = tid; q < nt; q += T) {
      const unsigned long long key = nk[q];
      const int p = (int)(key & 0xffffffffULL);
      const int slot = S.off[p] + atomicSub(&S.cnt[p], 1) - 1;
      const unsigned long long order =
          O.protocol == 1 ? ((unsigned long long)rp_key32(O.seed, O.round_base + rounds, S.jidx[q]) << 32)
                          : (key & 0xffffffff00000000ULL);
      S.mem[slot] = order | (unsigned)q;
    }
    __syncthreads();
    // ---- greedy order: rank of each member inside its group
    for (int r = tid; r < nt; r += T) {
      const unsigned long long e = S.mem[r];
      const int q = (int)(e & 0xffffffffULL);
      const int p = (int)(nk[q] & 0xffffffffULL);
      const int b = S.off[p], en = S.off[p + 1];
      int rank = 0;
      for (int u = b; u < en; ++u) rank += S.mem[u] < e;
      S.mem2[b + rank] = e;
    }
    __syncthreads();
    // ---- flow (greedy protocol), one supplier per thread: the residual
    // chain only; each flow is recorded (deferred costing: its original
    // indices and f in O.fl_*; otherwise (p, q) and f in mem / nnk, which are
    // free after the ordering step; every consumer flows at most once)
    const bool deferred = O.fl_i != nullptr;
    for (int p = tid; p < mt; p += T) {
      const int b = S.off[p], en = S.off[p + 1];
      if (b == en) continue;
      double s = S.sres[p];
      for (int r = b; r < en; ++r) {
        if (!residual_positive(s)) break;
        const int q = (int)(S.mem2[r] & 0xffffffffULL);
        double c = S.cres[q];
        const double f = greedy_step(s, c);
        S.cres[q] = c;
        const unsigned k = atomicAdd(&S.nflow, 1u);
        if (O.quiet) {
        } else if (deferred) {
          const unsigned long long slot = nnz + k;
          if (O.fl_cap && (long long)slot >= O.fl_cap) {
            atomicOr(O.err, EF_CAPACITY);
            continue;
          }
          O.fl_i[slot] = S.iidx[p];
          O.fl_j[slot] = S.jidx[q];
          O.fl_f[slot] = f;
          if (O.c_glob) O.c_glob[S.jidx[q]] = c;
        } else {
          S.mem[k] = ((unsigned long long)p << 32) | (unsigned)q;
          S.nnk[k] = (unsigned long long)__double_as_longlong(f);
        }
      }
      S.sres[p] = s;
      if (O.s_glob) O.s_glob[S.iidx[p]] = s;
    }
    __syncthreads();
    // ---- cost terms and plan entries of the round's flows, one per thread
    const unsigned nflow = S.nflow;
    for (unsigned base = (deferred || O.quiet) ? nflow : 0; base < nflow; base += T) {  // whole warps
      const unsigned k = base + tid;
      double term = 0.0;
      if (k < nflow) {
        const unsigned long long pq = S.mem[k];
        const int p = (int)(pq >> 32), q = (int)(pq & 0xffffffffULL);
        const double f = __longlong_as_double((long long)S.nnk[k]);
        term = __dmul_rn(f, G.dist64(S, p, q, metric));
        const unsigned long long slot = nnz + k;
        if (O.plan_i) {
          if ((long long)slot < O.plan_cap) {
            O.plan_i[slot] = S.iidx[p];
            O.plan_j[slot] = S.jidx[q];
            O.plan_f[slot] = f;
          } else {
            atomicOr(O.err, EF_CAPACITY);
          }
        }
        if (O.c_glob) O.c_glob[S.jidx[q]] = S.cres[q];
      }
      if (O.acc) xs_add_warp(O.acc, term);  // one call site for the whole warp
    }
    // (the compaction rewrites what this loop reads; with the loop empty
    // the flow step's barrier suffices)
    if (!(deferred || O.quiet)) __syncthreads();
    nnz += nflow;
    rounds += 1;
    pair_evals += (long long)mt * nt;
    // ---- weights update: retire spent points, compact
    cta_compact(S, G);
  }
  if (O.fl_i && (O.acc || O.plan_i)) {
    // deferred costing: the terms and plan entries of every flow of the loop
    // (a solve whose later pass costs all its flows records them only)
    for (unsigned long long base = nnz0; base < nnz; base += T) {  // whole warps (xs_add_warp)
      const unsigned long long k = base + tid;
      double term = 0.0;
      if (k < nnz) {
        const int i = O.fl_i[k], j = O.fl_j[k];
        const double f = O.fl_f[k];
        term = __dmul_rn(f, cost_dist64(O.x + (size_t)i * O.d, O.y + (size_t)j * O.d, O.d, metric));
        if (O.plan_i) {
          if ((long long)k < O.plan_cap) {
            O.plan_i[k] = i;
            O.plan_j[k] = j;
            O.plan_f[k] = f;
          } else {
            atomicOr(O.err, EF_CAPACITY);
          }
        }
      }
      if (O.acc) xs_add_warp(O.acc, term);  // one call site for the whole warp
    }
    __syncthreads();
  }
}

// Load one side of a pair (raw rows, weights) into the CTA state, check it,
// and normalise its weights by their correctly rounded total.  With DP > 0
// the coordinates are copied (zero-padded to DP) into dst.
template <int DP, int CAP>
NNS_DEV bool cta_load_side(const float* pts, const double* w, int cnt, int d, float* dst, double* res, int* idx,
                           CtaCore<CAP>& S, unsigned* err) {
  const int tid = threadIdx.x;
  for (int i = tid; i < XS_LIMBS; i += blockDim.x) S.acc[i] = 0ULL;
  __syncthreads();
  bool nonfinite = false, negative = false;
  for (int base = 0; base < cnt; base += blockDim.x) {  // whole warps (xs_add_warp)
    const int p = base + tid;
    double add = 0.0;
    if (p < cnt) {
    if (DP > 0) {
#pragma unroll
      for (int k = 0; k < (DP > 0 ? DP : 1); ++k) {
        const float v = k < d ? pts[(size_t)p * d + k] : 0.f;
        if (!isfinite(v)) nonfinite = true;
        dst[p * DP + k] = v;
      }
    } else {
      for (int k = 0; k < d; ++k)
        if (!isfinite(pts[(size_t)p * d + k])) nonfinite = true;
    }
    const double wv = w[p];
    if (!isfinite(wv)) nonfinite = true;
    else if (wv < 0.0) negative = true;
    res[p] = wv;
    idx[p] = p;
    add = isfinite(wv) && wv > 0.0 ? wv : 0.0;
    }
    xs_add_warp(S.acc, add);  // one call site for the whole warp
  }
  nonfinite = __syncthreads_or(nonfinite);
  negative = __syncthreads_or(negative);
  if (tid == 0) S.total = xs_round(S.acc);
  __syncthreads();
  const double total = S.total;
  if (nonfinite || negative || !(total > 0.0)) {
    if (tid == 0) atomicOr(err, nonfinite ? EF_NONFINITE : (negative ? EF_NEGATIVE : EF_ZERO_MASS));
    __syncthreads();
    return false;
  }
  for (int p = tid; p < cnt; p += blockDim.x) res[p] = __ddiv_rn(res[p], total);
  __syncthreads();
  return true;
}

// Shared memory of a one-CTA solver for d <= 8 (coordinates included).
template <int D, int DP, bool L1>
struct LowdSmem {
  CtaCore<FIN_MAX> S;
  GeoSmem<D, DP, L1, FIN_MAX> G;
};

// Whole pair in one CTA: load both sides, drop zero weights, run all rounds,
// return R (correctly rounded) in thread 0.  Returns false on invalid input.
template <int CAP, class Geo>
NNS_DEV bool cta_solve_pair(CtaCore<CAP>& S, Geo& G, float* xs, float* ys, const float* x, const double* a, int m,
                            const float* y, const double* b, int n, int d, int metric, unsigned* err, double& cost,
                            long long& rounds, long long& pe, int protocol = 0, unsigned long long seed = 0,
                            int32_t* fl_i = nullptr, int32_t* fl_j = nullptr, double* fl_f = nullptr,
                            long long fl_cap = 0) {
  bool ok = cta_load_side<Geo::kDP, CAP>(x, a, m, d, xs, S.sres, S.iidx, S, err);
  if (ok) ok = cta_load_side<Geo::kDP, CAP>(y, b, n, d, ys, S.cres, S.jidx, S, err);
  if (!ok) return false;
  if (threadIdx.x == 0) {
    S.mt = m;
    S.nt = n;
  }
  for (int i = threadIdx.x; i < XS_LIMBS; i += blockDim.x) S.acc[i] = 0ULL;
  __syncthreads();
  cta_compact(S, G);  // drop zero weights
  CtaOut O{S.acc, nullptr, nullptr, nullptr, 0, nullptr, nullptr, err};
  O.protocol = protocol;
  O.seed = seed;
  if (fl_i) {
    // record the flows and cost them all after the last round (the FP64
    // distance is then computed once per flow with the lanes in parallel,
    // not on every round's critical path)
    O.fl_i = fl_i;
    O.fl_j = fl_j;
    O.fl_f = fl_f;
    O.fl_cap = fl_cap;
    O.x = x;
    O.y = y;
    O.d = d;
  }
  unsigned long long nnz = 0;
  rounds = 0;
  pe = 0;
  cta_rounds(S, G, metric, O, nnz, rounds, pe, (long long)m + n);
  __syncthreads();
  if (threadIdx.x == 0) cost = xs_round(S.acc);
  return true;
}

}  // namespace nnsemd
