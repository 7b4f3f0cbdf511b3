// Batched reduced-precision NNS-EMD (d > 8): one persistent launch, one pair
// per CTA, all rounds of Alg. 1 (Sec. III-A) on chip (Sec. III-D batch
// processing), with the NNS operation of every round on the tensor cores.
//
// Per round the CTA
//   1. packs its pair's active points (BF16 / FP16 / FP8 with per-row scale)
//      into its own slot of a global scratch area, in the K-major no-swizzle
//      core-matrix layout, with FP32 norms and the certificate's maxima;
//   2. runs a tcgen05 pipeline over (consumer tile of 128) x (supplier tile
//      of BN): warp 0 issues the bulk copies (TMA), warp 1 owns tensor memory
//      and issues the MMAs into two FP32 accumulators, warps 2..5 keep the
//      top-8 approximate suppliers of each consumer; the pipeline's phase
//      counters live for the whole launch;
//   3. re-ranks the 8 candidates of every consumer with the exact FP32 key
//      (all 32 warps) and certifies the best (tc_common.cuh); consumers that
//      cannot be certified are scanned again in FP32 (64 x 64 tiles);
//   4. groups, serves, retires and compacts exactly as the other one-CTA
//      solvers (cta.cuh).
// The result equals the FP32 path's.  All waits are bounded (EF_TIMEOUT).
#include <math_constants.h>

#include "common.cuh"
#include "cta.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace nnsemd {

// Candidates per consumer in the batched kernel (its 1,024 threads have 64
// registers each; the multi-CTA kernel keeps TC_K = 16).
constexpr int BTC_K = 8;

// Per-CTA scratch in global memory.
struct BtcScratch {
  uint8_t* A;       // consumer tiles
  uint8_t* B;       // supplier tiles
  float* nrm_x;
  float* nrm_sx;    // |x| rounded up (0 on padding)
  float* scale_x;
  float* nrm_y;
  float* scale_y;
  float* cand_v;    // [cap][BTC_K]
  int* cand_p;
  // distance cache of a pair with m * n <= kc_cap (see GeoTC::nns_cached),
  // indexed [original consumer][original supplier]
  float* vcache;    // approximate ranking values v' of the tensor-core pass
  float* kcache;    // exact FP32 keys, NaN until computed
  float* ny_o;      // per original consumer: FP32 squared norm, scale, FP64 norms
  float* sy_o;
  double* yl2_o;
  double* yl1_o;
  double* e_o;      // per original consumer: E of the certificate (certify_E)
};

__host__ __device__ inline size_t btc_slot_layout(uint8_t* base, int cap, int kb, int bn, BtcScratch* out,
                                                  long long kc_cap = 0) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    uint8_t* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  };
  const int qrows = (cap + TC_BM - 1) / TC_BM * TC_BM;
  const int srows = (cap + bn - 1) / bn * bn;
  BtcScratch s;
  s.A = take((size_t)qrows * kb);
  s.B = take((size_t)srows * kb);
  s.nrm_x = (float*)take(srows * sizeof(float));
  s.nrm_sx = (float*)take(srows * sizeof(float));
  s.scale_x = (float*)take(srows * sizeof(float));
  s.nrm_y = (float*)take(qrows * sizeof(float));
  s.scale_y = (float*)take(qrows * sizeof(float));
  s.cand_v = (float*)take((size_t)cap * BTC_K * sizeof(float));
  s.cand_p = (int*)take((size_t)cap * BTC_K * sizeof(int));
  s.vcache = (float*)take((size_t)kc_cap * sizeof(float));
  s.kcache = (float*)take((size_t)kc_cap * sizeof(float));
  s.ny_o = (float*)take(kc_cap ? (size_t)cap * sizeof(float) : 0);
  s.sy_o = (float*)take(kc_cap ? (size_t)cap * sizeof(float) : 0);
  s.yl2_o = (double*)take(kc_cap ? (size_t)cap * sizeof(double) : 0);
  s.yl1_o = (double*)take(kc_cap ? (size_t)cap * sizeof(double) : 0);
  s.e_o = (double*)take(kc_cap ? (size_t)cap * sizeof(double) : 0);
  if (out) *out = s;
  return (off + 255) & ~(size_t)255;
}

size_t batched_tc_slot_bytes(int cap, int kb, int bn, long long kc_cap) {
  return btc_slot_layout(nullptr, cap, kb, bn, nullptr, kc_cap);
}

struct BtcArgs {
  BatchArgs base;
  uint8_t* scratch;          // grid x slot_bytes
  size_t slot_bytes;
  int kb, bn, nstage, fmt;
  unsigned long long* certified;
  unsigned long long* fallbacks;
  unsigned long long* near_ties;
  int rk;                    // candidates re-ranked per consumer (1 .. BTC_K)
  long long kc_cap;          // distance-cache entries per CTA (0: no cache)
};

// The NNS policy of the batched tensor-core solver (coordinates in global
// memory, index-only active lists, like GeoGlobal).
template <bool KIND8, int CAP>
struct GeoTC {
  static constexpr int kDP = 0;
  static constexpr int kThreads = FIN_THREADS;
  struct PX {};
  const float* x;  // this pair's coordinates
  const float* y;
  int d;
  BtcScratch scr;
  int kb, bn, nstage, fmt, rk;
  uint32_t tmem_base;
  unsigned* err;
  uint64_t bar_full[8];
  uint64_t bar_empty[8];
  uint64_t bar_acc_full[2];
  uint64_t bar_acc_empty[2];
  uint64_t bar_a_full;
  uint64_t bar_a_empty;
  // pipeline counters: prod_* only by the producer thread, mma_* only by the
  // MMA thread; epi_acc is read by the epilogue threads at the start of a
  // phase and advanced by one thread after it
  unsigned prod_a, prod_b, mma_a, mma_b, mma_acc, epi_acc;
  unsigned stat_rx, stat_rx1, stat_sx;  // certificate maxima of this round (float bits)
  int nfb;
  unsigned long long ncert, nfall, nnear;
  // distance cache of the current pair: on (m * n fits), filled (after the
  // pair's first round), the pair's supplier and consumer counts (the row
  // length and the number of rows)
  int kc_on, kc_ready, kc_m, kc_n;
  double kc_gam;  // gamma_d of the certificate
  int fb[CAP];
  // staging: tensor-core operand tiles or FP32 fallback tiles (never both at
  // once); the launch reserves max(sizeof(tiles), A + stages * B) bytes
  union __align__(128) Stage {
    TileSmem tiles[FIN_THREADS / TG_THREADS];
    uint8_t bytes[16];
  } U;

  NNS_DEV void load_x(int, PX&) const {}
  NNS_DEV void store_x(int, const PX&) {}
  NNS_DEV void load_y(int, PX&) const {}
  NNS_DEV void store_y(int, const PX&) {}
  template <int C>
  NNS_DEV double dist64(const CtaCore<C>& S, int p, int q, int metric) const {
    return cost_dist64(x + (size_t)S.iidx[p] * d, y + (size_t)S.jidx[q] * d, d, metric);
  }

  // The NNS step of a round from the pair's distance cache (the tensor-core
  // pass of its first round filled every v'): one warp per active consumer.
  //   1. the rk active suppliers with the smallest v' (each lane keeps the
  //      best rk of its share of the suppliers, then rk warp-wide minima
  //      merge the lists; ties by position);
  //   2. their exact FP32 keys, from the key cache or computed (and cached)
  //      by one lane each, in the definition's sequential order;
  //   3. the certificate of the best of them against tau, the rk-th v'
  //      (every other active supplier has v' >= tau; with no other active
  //      supplier every one was a candidate and the best is the answer);
  //   4. otherwise the exact key of every active supplier (cached or
  //      computed), the smallest with its position.
  // The per-supplier maxima of the certificate are those of the first
  // round's active suppliers, a superset of every later round's, so the
  // bound only gets more conservative.  Exact keys are written and read by
  // the warp that owns the consumer in that round; a barrier separates
  // rounds, so a key cached by one warp is seen by the next.
  template <int C>
  NNS_DEV const unsigned long long* nns_cached(CtaCore<C>& S, int mt, int nt) {
    const int tid = threadIdx.x, T = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int K = rk < mt ? rk : mt;
    for (int q = warp; q < nt; q += T / 32) {
      const int j = S.jidx[q];
      const float* vrow = scr.vcache + (size_t)j * kc_m;
      float* krow = scr.kcache + (size_t)j * kc_m;
      const float* yrow = y + (size_t)j * d;
      // 1. candidates: this lane's best BTC_K, then the warp's best K
      float tv[BTC_K];
      int tp[BTC_K];
#pragma unroll
      for (int k = 0; k < BTC_K; ++k) { tv[k] = CUDART_INF_F; tp[k] = -1; }
      // four loads in flight per lane before the insertions that use them
      for (int p0 = lane; p0 < mt; p0 += 128) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int p = p0 + 32 * u;
          v[u] = p < mt ? vrow[S.iidx[p]] : CUDART_INF_F;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (p0 + 32 * u < mt) topk_insert(tv, tp, v[u], p0 + 32 * u);
      }
      unsigned long long sel = ~0ULL, first = ~0ULL, kth = ~0ULL;
      for (int k = 0; k < K; ++k) {
        const unsigned long long mine =
            tp[0] >= 0 ? ((unsigned long long)ordered_bits(tv[0]) << 32) | (unsigned)tp[0] : ~0ULL;
        unsigned long long w = mine;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const unsigned long long other = __shfl_xor_sync(0xffffffffu, w, o);
          w = other < w ? other : w;
        }
        if (mine == w && w != ~0ULL) {  // the winning lane drops its head
#pragma unroll
          for (int i = 0; i + 1 < BTC_K; ++i) {
            tv[i] = tv[i + 1];
            tp[i] = tp[i + 1];
          }
          tv[BTC_K - 1] = CUDART_INF_F;
          tp[BTC_K - 1] = -1;
        }
        if (lane == k) sel = w;
        if (k == 0) first = w;
        kth = w;
      }
      // 2. exact keys of the candidates
      unsigned long long best = ~0ULL;
      if (lane < K && sel != ~0ULL) {
        const int p = (int)(unsigned)sel;
        const int i = S.iidx[p];
        float key = krow[i];
        if (key != key) {
          key = key32<METRIC_SQL2>(x + (size_t)i * d, yrow, d);
          krow[i] = key;
        }
        best = pack_key(key, (unsigned)p);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
        best = other < best ? other : best;
      }
      // 3. the certificate (tau = +inf: no other active supplier)
      bool cert = false;
      if (lane == 0) {
        const unsigned tb = (unsigned)(kth >> 32);
        // (E of this consumer was computed once, when the cache was filled)
        const float tau = mt > K ? __uint_as_float((tb & 0x80000000u) ? (tb & 0x7fffffffu) : ~tb) : CUDART_INF_F;
        cert = best != ~0ULL &&
               (mt <= K || (double)__uint_as_float((unsigned)(best >> 32)) <
                               certify_floor_from_E(scr.ny_o[j], tau, scr.e_o[j], kc_gam));
      }
      cert = __shfl_sync(0xffffffffu, cert, 0);
      if (cert) {
        if (lane == 0) {
          S.nnk[q] = best;
          atomicAdd(&ncert, 1ULL);
          if ((unsigned)best != (unsigned)first) atomicAdd(&nnear, 1ULL);
        }
        continue;
      }
      // 4. the exact scan
      unsigned long long m2 = ~0ULL;
      for (int p = lane; p < mt; p += 32) {
        const int i = S.iidx[p];
        float key = krow[i];
        if (key != key) {
          key = key32<METRIC_SQL2>(x + (size_t)i * d, yrow, d);
          krow[i] = key;
        }
        const unsigned long long kk = pack_key(key, (unsigned)p);
        m2 = kk < m2 ? kk : m2;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, m2, o);
        m2 = other < m2 ? other : m2;
      }
      if (lane == 0) {
        S.nnk[q] = m2;
        atomicAdd(&nfall, 1ULL);
        if ((unsigned)m2 != (unsigned)first) atomicAdd(&nnear, 1ULL);
      }
    }
    __syncthreads();
    return S.nnk;
  }

  template <int C>
  NNS_DEV const unsigned long long* nns(CtaCore<C>& S, int mt, int nt, long long = 0) {
    if (kc_on && kc_ready) return nns_cached(S, mt, nt);
    // with the cache on, this is the pair's first round: the tensor-core
    // pass fills the cache (every v' of the pair) instead of keeping top-K
    const bool fill = kc_on != 0;
    const int tid = threadIdx.x, T = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int qtiles = (nt + TC_BM - 1) / TC_BM;
    const int stiles = (mt + bn - 1) / bn;
    const int nblk = kb / 16;
    // ---- 1. pack both sides
    if (tid == 0) {
      stat_rx = stat_rx1 = stat_sx = 0u;
      nfb = 0;
    }
    if (fill) {
      // no exact key of the pair is known yet
      const long long total = (long long)kc_m * (long long)kc_n;
      for (long long e = tid; e < total; e += T) scr.kcache[e] = CUDART_NAN_F;
    }
    __syncthreads();
    {
      // one warp per row: the lanes take the row's coordinates and 16-byte
      // blocks (coalesced loads, all in flight at once), and the scale and
      // norms are warp reductions.  Any summation order keeps the FP32
      // squared norm within gamma_d |v|^2, the bound the certificate uses.
      const int srows = stiles * bn, qrows = qtiles * TC_BM;
      const int total = srows + qrows;
      for (int row_id = warp; row_id < total; row_id += T / 32) {
        const bool sup = row_id < srows;
        const int p = sup ? row_id : row_id - srows;
        const int cnt = sup ? mt : nt;
        const float* row = p < cnt ? (sup ? x + (size_t)S.iidx[p] * d : y + (size_t)S.jidx[p] * d) : nullptr;
        float mx = 0.f, a2f = 0.f, a1f = 0.f;
        double a2 = 0.0, a1 = 0.0;
        const bool want64 = row && !sup && fill;
        if (row)
          for (int k = lane; k < d; k += 32) {
            const float v = row[k];
            mx = fmaxf(mx, fabsf(v));
            a2f = __fmaf_rn(v, v, a2f);
            a1f = __fadd_rn(a1f, fabsf(v));
            if (want64) {
              a2 += (double)v * v;
              a1 += fabs((double)v);
            }
          }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
          a2f = __fadd_rn(a2f, __shfl_xor_sync(0xffffffffu, a2f, o));
          a1f = __fadd_rn(a1f, __shfl_xor_sync(0xffffffffu, a1f, o));
          if (want64) {
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
          }
        }
        float s = 1.f;  // the row scale of FP16 / FP8 (as row_scale), from the warp's maximum
        if (row && !fmt_is_bf16(fmt) && mx > 0.f) {
          int e;
          frexpf(mx, &e);
          s = ldexpf(1.f, e - 8);
        }
        const int rows = sup ? bn : TC_BM;
        uint8_t* tile = (sup ? scr.B : scr.A) + (size_t)(p / rows) * rows * kb;
        for (int c = lane; c < nblk; c += 32) pack_block(row, d, c, s, fmt, tile, rows, p % rows, sup);
        if (lane == 0) {
          float* nrm = sup ? scr.nrm_x : scr.nrm_y;
          float* scl = sup ? scr.scale_x : scr.scale_y;
          if (row) {
            const float l2sq = a2f, l1 = a1f;
            nrm[p] = l2sq;
            scl[p] = s;
            if (sup) {
              scr.nrm_sx[p] = norm_up(l2sq);
              atomicMax(&stat_rx, __float_as_uint(norm_up(l2sq)));
              atomicMax(&stat_rx1, __float_as_uint(l1 * (1.f + 1e-4f)));
              atomicMax(&stat_sx, __float_as_uint(s));
            } else if (fill) {
              // what the certificate needs of this consumer in every round
              const int j = S.jidx[p];
              scr.ny_o[j] = l2sq;
              scr.sy_o[j] = s;
              scr.yl2_o[j] = sqrt(a2) * (1 + 1e-12);
              scr.yl1_o[j] = a1;
            }
          } else {
            nrm[p] = CUDART_INF_F;
            scl[p] = 1.f;
            if (sup) scr.nrm_sx[p] = 0.f;
          }
        }
      }
    }
    fence_proxy_async_global();                                   // packed tiles -> later bulk copies
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // last round's FP32 tiles -> bulk writes
    __syncthreads();
    // ---- 2. tensor-core pipeline
    const uint32_t a_bytes = TC_BM * kb, b_bytes = bn * kb;
    uint8_t* sA = U.bytes;
    uint8_t* sB = U.bytes + a_bytes;
    bool ok = true;
    if (warp == 0) {
      if (lane == 0) {
        for (int qt = 0; qt < qtiles && ok; ++qt) {
          ok = mbar_wait_bounded(&bar_a_empty, (prod_a & 1) ^ 1);
          if (!ok) break;
          mbar_expect_tx(&bar_a_full, a_bytes);
          tma_load_1d(sA, scr.A + (size_t)qt * a_bytes, a_bytes, &bar_a_full);
          ++prod_a;
          for (int st = 0; st < stiles && ok; ++st) {
            const unsigned s = prod_b % nstage, u = prod_b / nstage;
            ok = mbar_wait_bounded(&bar_empty[s], (u & 1) ^ 1);
            if (!ok) break;
            mbar_expect_tx(&bar_full[s], b_bytes);
            tma_load_1d(sB + (size_t)s * b_bytes, scr.B + (size_t)st * b_bytes, b_bytes, &bar_full[s]);
            ++prod_b;
          }
        }
      }
    } else if (warp == 1) {
      if (lane == 0) {
        const uint32_t idesc = make_idesc(fmt_is_bf16(fmt) ? 1 : 0, TC_BM, bn);
        const int ksteps = kb / 32;
        const uint32_t a0 = smem_u32(sA);
        for (int qt = 0; qt < qtiles && ok; ++qt) {
          ok = mbar_wait_bounded(&bar_a_full, mma_a & 1);
          if (!ok) break;
          for (int st = 0; st < stiles && ok; ++st) {
            const unsigned s = mma_b % nstage, u = mma_b / nstage;
            const unsigned b = mma_acc & 1, v = mma_acc >> 1;
            ok = mbar_wait_bounded(&bar_full[s], u & 1);
            if (ok) ok = mbar_wait_bounded(&bar_acc_empty[b], (v & 1) ^ 1);
            if (!ok) break;
            tc_fence_after();
            const uint32_t b0 = smem_u32(sB + (size_t)s * b_bytes);
            const uint32_t tmem_d = tmem_base + b * (uint32_t)bn;
            for (int k = 0; k < ksteps; ++k) {
              const uint64_t ad = make_desc(a0 + k * 2 * TC_BM * 16, TC_BM * 16, 128);
              const uint64_t bd = make_desc(b0 + k * 2 * bn * 16, bn * 16, 128);
              mma_issue<KIND8 ? FMT_E4M3 : FMT_BF16>(tmem_d, ad, bd, idesc, k > 0 ? 1u : 0u);
            }
            mma_commit(&bar_empty[s]);
            mma_commit(&bar_acc_full[b]);
            ++mma_b;
            ++mma_acc;
          }
          mma_commit(&bar_a_empty);  // A may be overwritten once these MMAs are done
          ++mma_a;
        }
      }
    } else if (warp < 6) {
      const int quarter = warp & 3;
      const int row = quarter * 32 + lane;
      unsigned ea = epi_acc;
      for (int qt = 0; qt < qtiles; ++qt) {
        const int q = qt * TC_BM + row;
        const float sy = q < nt ? scr.scale_y[q] : 1.f;
        const float cy = quant_coeff(fmt, q < nt ? scr.nrm_y[q] : 0.f);
        float tv[BTC_K];
        int tp[BTC_K];
#pragma unroll
        for (int k = 0; k < BTC_K; ++k) { tv[k] = CUDART_INF_F; tp[k] = -1; }
        for (int st = 0; st < stiles; ++st, ++ea) {
          const unsigned b = ea & 1, v = ea >> 1;
          if (ok) ok = mbar_wait_bounded(&bar_acc_full[b], v & 1);
          ok = __all_sync(0xffffffffu, ok);  // warp-uniform: the fill below synchronises the warp
          tc_fence_after();
          if (ok) {
            const float* nx = scr.nrm_x + (size_t)st * bn;
            const float* ns = scr.nrm_sx + (size_t)st * bn;
            const float* sx = scr.scale_x + (size_t)st * bn;
            // fill: this consumer's row of the cache, by original supplier index
            float* vrow = (fill && q < nt) ? scr.vcache + (size_t)S.jidx[q] * kc_m : nullptr;
            for (int c0 = 0; c0 < bn; c0 += 16) {
              uint32_t r[16];
              tmem_ld16(tmem_base + ((uint32_t)(quarter * 32) << 16) + b * (uint32_t)bn + (uint32_t)c0, r);
              float val[16];
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                const float acc = __uint_as_float(r[e]);
                const float w = fmt_is_bf16(fmt) ? -2.f : -2.f * sy * sx[c0 + e];
                val[e] = __fmaf_rn(-cy, ns[c0 + e], __fmaf_rn(w, acc, nx[c0 + e]));
              }
              if (!fill) {
#pragma unroll
                for (int e = 0; e < 16; ++e) topk_insert(tv, tp, val[e], st * bn + c0 + e);
              } else if constexpr (CAP >= 2048) {
                // transpose the warp's 32 rows x 16 columns through the
                // fallback list's buffer (unused while the cache fills), so
                // that each store instruction writes 16 consecutive columns of
                // two rows instead of one column of 32 rows (XOR-swizzled:
                // no bank conflicts either way)
                float* tb = reinterpret_cast<float*>(fb) + (warp - 2) * 512;
#pragma unroll
                for (int e = 0; e < 16; ++e) tb[e * 32 + (lane ^ e)] = val[e];
                __syncwarp();
                const int e = lane & 15;
                const int col = st * bn + c0 + e;
                const int icol = col < mt ? S.iidx[col] : 0;
#pragma unroll 4
                for (int it = 0; it < 16; ++it) {
                  const int rr = 2 * it + (lane >> 4);
                  const int qq = qt * TC_BM + quarter * 32 + rr;
                  if (qq < nt && col < mt) scr.vcache[(size_t)S.jidx[qq] * kc_m + icol] = tb[e * 32 + (rr ^ e)];
                }
                __syncwarp();
              } else {
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                  const int col = st * bn + c0 + e;
                  if (vrow && col < mt) vrow[S.iidx[col]] = val[e];
                }
              }
            }
          }
          tc_fence_before();
          mbar_arrive(&bar_acc_empty[b]);
        }
        if (q < nt && !fill) {
#pragma unroll
          for (int k = 0; k < BTC_K; ++k) {
            scr.cand_v[(size_t)q * BTC_K + k] = tv[k];
            scr.cand_p[(size_t)q * BTC_K + k] = tp[k];
          }
        }
      }
    }
    if (!ok) atomicOr(err, EF_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 64) epi_acc += (unsigned)(qtiles * stiles);
    if (fill) {
      // the cache holds every v' of the pair; this and every later round
      // are answered from it.  The certificate's E of every consumer, once:
      // the supplier maxima of this first round bound every later round's.
      const double rx = __uint_as_float(stat_rx), rx1 = __uint_as_float(stat_rx1);
      const double sxm = __uint_as_float(stat_sx);
      for (int q = tid; q < nt; q += T) {
        const int j = S.jidx[q];
        scr.e_o[j] = certify_E(fmt, d, scr.ny_o[j], scr.yl2_o[j], scr.yl1_o[j], scr.sy_o[j], rx, rx1, sxm);
      }
      if (tid == 0) {
        kc_gam = certify_gamma(d);
        kc_ready = 1;
      }
      __syncthreads();
      return nns_cached(S, mt, nt);
    }
    // ---- 3. exact re-rank + certificate (a warp per consumer)
    const double rx = __uint_as_float(stat_rx), rx1 = __uint_as_float(stat_rx1), sxm = __uint_as_float(stat_sx);
    for (int q = warp; q < nt; q += T / 32) {
      const float* yrow = y + (size_t)S.jidx[q] * d;
      unsigned long long best = ~0ULL;
      if (lane < rk) {
        const int p = scr.cand_p[(size_t)q * BTC_K + lane];
        if (p >= 0) best = pack_key(key32<METRIC_SQL2>(x + (size_t)S.iidx[p] * d, yrow, d), (unsigned)p);
      }
      double yl2 = 0.0, yl1 = 0.0;
      for (int k = lane; k < d; k += 32) {
        yl2 += (double)yrow[k] * yrow[k];
        yl1 += fabs((double)yrow[k]);
      }
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        best = ob < best ? ob : best;
        yl2 += __shfl_xor_sync(0xffffffffu, yl2, o);
        yl1 += __shfl_xor_sync(0xffffffffu, yl1, o);
      }
      if (lane == 0) {
        // tau: the rk-th approximate value; the first candidate is the
        // approximate best, and an exact best elsewhere is a near-tie
        const float tau = scr.cand_v[(size_t)q * BTC_K + rk - 1];
        if (best != ~0ULL && (int)(unsigned)best != scr.cand_p[(size_t)q * BTC_K]) atomicAdd(&nnear, 1ULL);
        const bool cert = best != ~0ULL && certify(fmt, d, scr.nrm_y[q], sqrt(yl2) * (1 + 1e-12), yl1,
                                                    scr.scale_y[q], rx, rx1, sxm, tau,
                                                    __uint_as_float((unsigned)(best >> 32)));
        if (cert) {
          S.nnk[q] = best;
          atomicAdd(&ncert, 1ULL);
        } else {
          fb[atomicAdd(&nfb, 1)] = q;
          atomicAdd(&nfall, 1ULL);
        }
      }
    }
    __syncthreads();
    // ---- 4. FP32 rescan of the consumers that were not certified
    const int nf = nfb;
    if (nf > 0) {
      const int g = tid / TG_THREADS, gt = tid % TG_THREADS;
      const int ngroups = T / TG_THREADS;
      for (int c0 = g * TG_M; c0 < nf; c0 += ngroups * TG_M) {
        unsigned long long out[4];
        group_nns_tile<false>(x, S.iidx, 0, mt, y, S.jidx, fb, c0, min(TG_M, nf - c0), d, U.tiles[g], gt, 1 + g,
                              out);
        const int tx = gt & 15, ty = gt >> 4;
        if (tx == 0)
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int lq = c0 + ty * 4 + i;
            if (lq < nf) S.nnk[fb[lq]] = out[i];
          }
      }
    }
    __syncthreads();
    return S.nnk;
  }
};

template <bool KIND8, int CAP>
struct BtcSmem {
  CtaCore<CAP> S;
  GeoTC<KIND8, CAP> G;  // its staging union is last and may extend past sizeof()
};

template <bool KIND8, int CAP>
size_t btc_smem_bytes(int kb, int bn, int nstage) {
  using M = BtcSmem<KIND8, CAP>;
  const size_t stage = (size_t)TC_BM * kb + (size_t)nstage * bn * kb;
  const size_t have = sizeof(typename GeoTC<KIND8, CAP>::Stage);
  return sizeof(M) + (stage > have ? stage - have : 0);
}

template <bool KIND8, int CAP>
__global__ void __launch_bounds__(FIN_THREADS, 1) k_batched_tc(BtcArgs A) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  BtcSmem<KIND8, CAP>& M = *reinterpret_cast<BtcSmem<KIND8, CAP>*>(smem_raw);
  CtaCore<CAP>& S = M.S;
  GeoTC<KIND8, CAP>& G = M.G;
  __shared__ int s_item;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t ncols = 2u * (uint32_t)A.bn;
  if (tid == 0) {
    for (int s = 0; s < A.nstage; ++s) {
      mbar_init(&G.bar_full[s], 1);
      mbar_init(&G.bar_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&G.bar_acc_full[b], 1);
      mbar_init(&G.bar_acc_empty[b], 4 * 32);
    }
    mbar_init(&G.bar_a_full, 1);
    mbar_init(&G.bar_a_empty, 1);
    mbar_fence_init();
    G.prod_a = G.prod_b = G.mma_a = G.mma_b = G.mma_acc = G.epi_acc = 0u;
    G.ncert = G.nfall = G.nnear = 0ULL;
    G.rk = A.rk;
    G.kb = A.kb;
    G.bn = A.bn;
    G.nstage = A.nstage;
    G.fmt = A.fmt;
    G.err = A.base.err;
    btc_slot_layout(A.scratch + (size_t)blockIdx.x * A.slot_bytes, CAP, A.kb, A.bn, &G.scr, A.kc_cap);
  }
  if (warp == 1) tmem_alloc(&tmem_slot, ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0) G.tmem_base = tmem_slot;
  __syncthreads();
  const BatchArgs& B = A.base;
  for (;;) {
    if (tid == 0) s_item = (int)atomicAdd(B.queue, 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= B.num) break;
    const int pr = B.pair_ids[item];
    const int64_t xo = B.x_off[pr], yo = B.n_shared ? 0 : B.y_off[pr];
    const int m = (int)(B.x_off[pr + 1] - xo), n = B.n_shared ? B.n_shared : (int)(B.y_off[pr + 1] - yo);
    if (tid == 0) {
      G.x = B.x + xo * B.d;
      G.y = B.y + yo * B.d;
      G.d = B.d;
      G.kc_on = (long long)m * n <= A.kc_cap ? 1 : 0;
      G.kc_ready = 0;
      G.kc_m = m;
      G.kc_n = n;
    }
    __syncthreads();
    double cost = 0.0;
    long long rounds = 0, pe = 0;
    const size_t fo = (size_t)blockIdx.x * B.fl_cap;
    const bool ok = cta_solve_pair(S, G, nullptr, nullptr, B.x + xo * B.d, B.a + xo, m, B.y + yo * B.d, B.b + yo, n,
                                   B.d, B.metric, B.err, cost, rounds, pe, B.protocol, B.seed,
                                   B.fl_i ? B.fl_i + fo : nullptr, B.fl_i ? B.fl_j + fo : nullptr,
                                   B.fl_i ? B.fl_f + fo : nullptr, B.fl_cap);
    if (tid == 0) {
      B.costs[pr] = ok ? cost : CUDART_NAN;
      if (B.rounds) B.rounds[pr] = rounds;
      if (B.pair_evals) B.pair_evals[pr] = pe;
    }
    __syncthreads();
  }
  if (tid == 0) {
    atomicAdd(A.certified, G.ncert);
    atomicAdd(A.fallbacks, G.nfall);
    atomicAdd(A.near_ties, G.nnear);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(G.tmem_base, ncols);
}

template <bool KIND8, int CAP>
static int batched_tc_t(const BtcArgs& A, int grid, cudaStream_t st) {
  const size_t smem = btc_smem_bytes<KIND8, CAP>(A.kb, A.bn, A.nstage);
  if (smem > 227 * 1024) return -2;
  cudaError_t e = cudaFuncSetAttribute(k_batched_tc<KIND8, CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return -1;
  k_batched_tc<KIND8, CAP><<<grid, FIN_THREADS, smem, st>>>(A);
  return 0;
}

// Largest number of pipeline stages that fits the shared-memory budget.
int batched_tc_max_stages(int cap, int kb, int bn, int precision) {
  for (int ns = 4; ns >= 1; --ns) {
    size_t b;
    if (precision == 3) b = cap <= 512 ? btc_smem_bytes<true, 512>(kb, bn, ns) : btc_smem_bytes<true, 2048>(kb, bn, ns);
    else b = cap <= 512 ? btc_smem_bytes<false, 512>(kb, bn, ns) : btc_smem_bytes<false, 2048>(kb, bn, ns);
    if (b <= 227 * 1024) return ns;
  }
  return 0;
}

int launch_batched_tc(const BatchArgs& base, int precision, int cap, int kb, int bn, int nstage, uint8_t* scratch,
                      size_t slot_bytes, unsigned long long* certified, unsigned long long* fallbacks,
                      unsigned long long* near_ties, int rerank_k, long long kc_cap, int grid, cudaStream_t st) {
  const int rk = rerank_k >= 1 && rerank_k <= BTC_K ? rerank_k : BTC_K;
  BtcArgs A{base, scratch, slot_bytes, kb, bn, nstage, fmt_of_precision(precision), certified, fallbacks,
            near_ties, rk, kc_cap};
  const bool k8 = precision == 3;
  if (cap <= 512) return k8 ? batched_tc_t<true, 512>(A, grid, st) : batched_tc_t<false, 512>(A, grid, st);
  return k8 ? batched_tc_t<true, 2048>(A, grid, st) : batched_tc_t<false, 2048>(A, grid, st);
}

}  // namespace nnsemd
