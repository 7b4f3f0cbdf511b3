// Reduced-precision NNS for d > 8 on the 5th-generation tensor cores
// (tcgen05, sm_103a), followed by an exact FP32 re-rank with a certificate.
//
//   approx(i, j) = |y_j|^2 + |x_i|^2 - 2 <x~_i, y~_j>
//
// where x~, y~ are BF16 / FP16 / FP8-E4M3 copies of the points (FP16 and FP8
// with a per-row power-of-two scale) and the dot products accumulate in FP32
// in tensor memory.  For every active consumer the kernel keeps the K
// suppliers with the smallest approximate distance.  The re-rank then
// computes the exact FP32 key (the same definition as every other path) of
// those candidates, takes the smallest (lowest position on ties), and
// certifies it (tc_common.cuh): no supplier outside the candidates can reach
// or beat it.  Consumers that cannot be certified are scanned again in FP32
// (k_nns_f32_tiled).  The result is therefore identical to the FP32 path.
//
// K2 k_nns_tc: a CTA owns 128 consumers (the MMA's M) and streams supplier
// tiles of BN rows.  Warp 0 issues 1-D bulk copies (TMA) of the packed tiles
// into a ring of shared-memory stages; warp 1 allocates tensor memory and
// one elected thread issues tcgen05.mma for each tile into a ring of
// TC_NACC FP32 accumulators (BN columns each); warp 2 copies each tile's
// column norms into a ring of its own; the warps from 3 on read each
// accumulator row back with tcgen05.ld (one consumer per thread, two or four
// warps per row, a share of the columns each) and update its top-K.  Every
// wait on an mbarrier is bounded and raises EF_TIMEOUT instead of hanging.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace nnsemd {

// warp 0 operand copies, warp 1 MMA, warp 2 column-norm copies, then the
// epilogue warps (EW / 4 per TMEM lane quarter, each a share of the columns).
// Sixteen epilogue warps (more latency hidden) where their registers fit:
// BF16 operands (no per-column scale) and lists of 8.
__host__ __device__ constexpr int tc_epi_warps(int fmt, int kl) { return fmt_is_bf16(fmt) && kl <= 8 ? 16 : 8; }
__host__ __device__ constexpr int tc_threads(int fmt, int kl) { return 32 * (3 + tc_epi_warps(fmt, kl)); }
// A tile + one B stage must fit in this much dynamic shared memory (what
// every instantiation has left beside its static arrays); more stages use
// what the instantiation actually has left.
constexpr int TC_SMEM_BUDGET = 150 * 1024;
constexpr int TC_SMEM_MAX = 227 * 1024;  // per block, static + dynamic
constexpr int TC_NACC = 4;                  // FP32 accumulators in tensor memory (a ring of tiles in flight)
constexpr int TC_NNRM = 4;                  // column-norm slots (a ring of its own, loaded ahead)

// One thread per point (consecutive threads write consecutive 16-byte rows
// of each column block).  Also writes, per point, the FP32 squared norm, the
// per-row scale and, in `stats`, the maxima of |v|_2, |v|_1 and the scale
// over the points (as float bits; all values >= 0).  Row p holds the point
// idx[sel ? sel[p] : p] for p < cnt (cnt read from cnt_dev when given; the
// rest is padding).
__global__ void k_pack_tc(const float* __restrict__ pts, const int* __restrict__ idx, const int* __restrict__ sel,
                          const int* __restrict__ cnt_dev, int cnt, int rows_pad, int d, int kb, int fmt,
                          int tile_rows, uint8_t* __restrict__ out, float* __restrict__ nrm, float* __restrict__ nrm_s,
                          float* __restrict__ scale, unsigned* __restrict__ stats) {
  const int nblk = kb / 16;
  const int count = cnt_dev ? min(*cnt_dev, cnt) : cnt;
  unsigned m0 = 0u, m1 = 0u, m2 = 0u;  // this thread's maxima (float bits of values >= 0)
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < rows_pad; p += gridDim.x * blockDim.x) {
    const float* row = p < count ? pts + (size_t)idx[sel ? sel[p] : p] * d : nullptr;
    const float s = row_scale(row, d, fmt);
    const int t = p / tile_rows, r = p % tile_rows;
    for (int c = 0; c < nblk; ++c)
      pack_block(row, d, c, s, fmt, out + (size_t)t * tile_rows * kb, tile_rows, r, nrm_s != nullptr);
    {
      if (row) {
        float l2sq, l1;
        row_norms(row, d, l2sq, l1);
        nrm[p] = l2sq;
        if (nrm_s) nrm_s[p] = norm_up(l2sq);
        scale[p] = s;
        m0 = max(m0, __float_as_uint(norm_up(l2sq)));
        m1 = max(m1, __float_as_uint(l1 * (1.f + 1e-4f)));
        m2 = max(m2, __float_as_uint(s));
      } else {
        nrm[p] = CUDART_INF_F;
        if (nrm_s) nrm_s[p] = 0.f;
        scale[p] = 1.f;
      }
    }
  }
  // the maxima: over the warp first, then one atomic per warp (every
  // thread of the block reaches this point: the loop above has no exit)
  m0 = __reduce_max_sync(0xffffffffu, m0);
  m1 = __reduce_max_sync(0xffffffffu, m1);
  m2 = __reduce_max_sync(0xffffffffu, m2);
  if ((threadIdx.x & 31) == 0 && (m0 | m1 | m2)) {
    atomicMax(stats + 0, m0);
    atomicMax(stats + 1, m1);
    atomicMax(stats + 2, m2);
  }
}

// --------------------------------------------------------------------------
// K2
// --------------------------------------------------------------------------

struct TcArgs {
  const uint8_t* A;        // packed consumer tiles (TC_BM rows each)
  const uint8_t* B;        // packed supplier tiles (bn rows each)
  const float* nrm_x;      // [supplier tiles * bn] squared norms (+inf on padding)
  const float* nrm_sx;     // [supplier tiles * bn] norms rounded up (0 on padding)
  const float* nrm_y;      // per-consumer squared norm
  const float* scale_x;    // per-supplier scale
  const float* scale_y;    // per-consumer scale
  int nt;                  // active consumers
  int mt;                  // active suppliers
  int kb;                  // bytes per packed row
  int bn;                  // suppliers per tile
  int nstage;
  int tiles_per_chunk;
  int num_tiles;           // supplier tiles in total
  int nt_pad;              // consumer count rounded up to TC_BM
  float* cand_v;           // [chunks][nt_pad][KL] approximate values (v = |x|^2 - 2 <x~,y~>)
  int* cand_p;             // [chunks][nt_pad][KL] supplier positions
  unsigned* err;
  const int* nq_dev;       // packed consumer rows in use (nullable: nt); tiles past it exit
};

// KL: the length of each consumer's list (TC_K, or TC_K / 2 when at most
// that many candidates are re-ranked: half the insertion work)
template <int FMT, int BN, int KL>
__global__ void __launch_bounds__(tc_threads(FMT, KL), 1) k_nns_tc(TcArgs P) {
  constexpr int EW = tc_epi_warps(FMT, KL);
  constexpr int PARTS = EW / 4;      // epilogue warps per TMEM lane quarter
  constexpr int CPART = BN / PARTS;  // columns of a tile per epilogue warp
  static_assert(CPART % 16 == 0, "whole 16-column blocks per epilogue warp");
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bar_full[8];
  __shared__ __align__(8) uint64_t bar_empty[8];
  __shared__ __align__(8) uint64_t bar_acc_full[TC_NACC];
  __shared__ __align__(8) uint64_t bar_acc_empty[TC_NACC];
  __shared__ __align__(8) uint64_t bar_nrm_full[TC_NNRM];
  __shared__ __align__(8) uint64_t bar_nrm_empty[TC_NNRM];
  __shared__ __align__(8) uint64_t bar_a;
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(16) float nrm_buf[TC_NNRM][3][BN];  // per tile in flight: |x|^2, |x| rounded up, scale
  // per epilogue thread: one 16-column block (at the end: the lists of
  // parts 1.. of each row, merged into part 0's)
  __shared__ __align__(16) float stage[16][EW * 32];
  __shared__ int tag_pos[TagList<KL>::NTAG][EW * 32];  // per epilogue thread: tag -> position
  static_assert(2 * (PARTS - 1) * KL * TC_BM <= 16 * EW * 32, "the merge lists fit in the staging area");
  float* const merge_v = &stage[0][0];                                              // [PARTS-1][KL][TC_BM]
  int* const merge_p = reinterpret_cast<int*>(&stage[0][0]) + (PARTS - 1) * KL * TC_BM;  // same shape

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int qtile = blockIdx.x;
  const int t0 = blockIdx.y * P.tiles_per_chunk;
  const int t1 = min(t0 + P.tiles_per_chunk, P.num_tiles);
  const int ntiles = t1 - t0;
  if (ntiles <= 0) return;
  if (P.nq_dev && qtile * TC_BM >= *P.nq_dev) return;  // the whole CTA leaves before any set-up
  const int kb = P.kb;
  const uint32_t a_bytes = TC_BM * kb;
  const uint32_t b_bytes = BN * kb;
  uint8_t* sA = smem;
  uint8_t* sB = smem + a_bytes;
  const int NST = P.nstage;
  constexpr uint32_t NCOLS = TC_NACC * BN;  // the accumulator ring
  constexpr uint32_t TMEM_ALLOC = NCOLS < 32 ? 32 : NCOLS;
  static_assert(NCOLS <= 512 && (NCOLS & (NCOLS - 1)) == 0, "tensor memory holds 512 columns");
  constexpr uint32_t NRM_BYTES = 3 * BN * sizeof(float);

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&bar_full[s], 1);
      mbar_init(&bar_empty[s], 1);
    }
    for (int b = 0; b < TC_NACC; ++b) {
      mbar_init(&bar_acc_full[b], 1);
      mbar_init(&bar_acc_empty[b], EW);  // one arrival per epilogue warp
    }
    for (int n = 0; n < TC_NNRM; ++n) {
      mbar_init(&bar_nrm_full[n], 1);
      mbar_init(&bar_nrm_empty[n], EW);
    }
    mbar_init(&bar_a, 1);
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(&tmem_slot, TMEM_ALLOC);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_slot;
  bool ok = true;

  if (warp == 0) {
    // ---------------- producer: TMA bulk copies of the operand tiles ----------------
    if (lane == 0) {
      mbar_expect_tx(&bar_a, a_bytes);
      tma_load_1d(sA, P.A + (size_t)qtile * a_bytes, a_bytes, &bar_a);
      for (int t = 0; t < ntiles && ok; ++t) {
        const int s = t % NST, u = t / NST;
        ok = mbar_wait_sleep(&bar_empty[s], (u & 1) ^ 1);
        if (!ok) break;
        mbar_expect_tx(&bar_full[s], b_bytes);
        tma_load_1d(sB + (size_t)s * b_bytes, P.B + (size_t)(t0 + t) * b_bytes, b_bytes, &bar_full[s]);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr int AB = fmt_is_bf16(FMT) ? 1 : 0;
      const uint32_t idesc = make_idesc(AB, TC_BM, BN);
      const int ksteps = kb / 32;
      ok = mbar_wait_bounded(&bar_a, 0);
      const uint32_t a0 = smem_u32(sA);
      for (int t = 0; t < ntiles && ok; ++t) {
        const int s = t % NST, u = t / NST;
        const int b = t % TC_NACC, v = t / TC_NACC;
        ok = mbar_wait_sleep(&bar_full[s], u & 1);
        if (ok) ok = mbar_wait_sleep(&bar_acc_empty[b], (v & 1) ^ 1);
        if (!ok) break;
        tc_fence_after();
        const uint32_t b0 = smem_u32(sB + (size_t)s * b_bytes);
        const uint32_t tmem_d = tmem_base + (uint32_t)(b * BN);
        for (int k = 0; k < ksteps; ++k) {
          const uint64_t ad = make_desc(a0 + k * 2 * TC_BM * 16, TC_BM * 16, 128);
          const uint64_t bd = make_desc(b0 + k * 2 * BN * 16, BN * 16, 128);
          mma_issue<FMT>(tmem_d, ad, bd, idesc, k > 0 ? 1u : 0u);
        }
        mma_commit(&bar_empty[s]);
        mma_commit(&bar_acc_full[b]);
      }
    }
  } else if (warp == 2) {
    // ---------------- producer: the column norms of each tile, a ring of their own ----------------
    if (lane == 0) {
      for (int t = 0; t < ntiles && ok; ++t) {
        const int n = t % TC_NNRM, w = t / TC_NNRM;
        ok = mbar_wait_sleep(&bar_nrm_empty[n], (w & 1) ^ 1);
        if (!ok) break;
        const size_t col = (size_t)(t0 + t) * BN;
        mbar_expect_tx(&bar_nrm_full[n], NRM_BYTES);
        tma_load_1d(nrm_buf[n][0], P.nrm_x + col, BN * sizeof(float), &bar_nrm_full[n]);
        tma_load_1d(nrm_buf[n][1], P.nrm_sx + col, BN * sizeof(float), &bar_nrm_full[n]);
        tma_load_1d(nrm_buf[n][2], P.scale_x + col, BN * sizeof(float), &bar_nrm_full[n]);
      }
    }
  } else {
    // ---------------- epilogue: TMEM -> top-K per consumer ----------------
    // PARTS warps per TMEM lane quarter; each takes CPART of the tile's
    // columns and keeps its own top-K, and the parts merge at the end.
    const int e = warp - 3;
    const int etid = e * 32 + lane;
    const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
    const int part = e >> 2;
    const int row = quarter * 32 + lane;
    const int q = qtile * TC_BM + row;
    const float sy = (q < P.nt) ? P.scale_y[q] : 1.f;
    const float cy = quant_coeff(FMT, (q < P.nt) ? P.nrm_y[q] : 0.f);
    // the list: tagged values (tc_common.cuh), ascending, +inf while not full
    float tv[KL];
    unsigned used = 0u;  // tags held by entries of the list
#pragma unroll
    for (int k = 0; k < KL; ++k) tv[k] = CUDART_INF_F;
    int* const table = &tag_pos[0][etid];
    constexpr int TSTRIDE = EW * 32;
    for (int t = 0; t < ntiles; ++t) {
      const int b = t % TC_NACC, v = t / TC_NACC;
      const int n = t % TC_NNRM, w = t / TC_NNRM;
      if (ok) ok = mbar_wait_sleep(&bar_acc_full[b], v & 1, 200u);
      if (ok) ok = mbar_wait_sleep(&bar_nrm_full[n], w & 1, 200u);
      tc_fence_after();
      if (ok) {
        const int tile = t0 + t;
        const float* nx = nrm_buf[n][0];
        const float* ns = nrm_buf[n][1];
        const float* sx = nrm_buf[n][2];
        // all of this warp's columns of the accumulator at once (one wait
        // for NB loads in flight), then two columns per packed FP32x2 step
        constexpr int NB = CPART / 16;
        uint32_t rr[NB][16];
#pragma unroll
        for (int bb = 0; bb < NB; ++bb)
          tmem_ld16_async(tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * BN + part * CPART + 16 * bb),
                          rr[bb]);
        tmem_ld_wait(rr);
        const unsigned long long mcy2 = f2_pack(-cy, -cy);
        const unsigned long long w2c = f2_pack(-2.f, -2.f);
        const unsigned long long wsy2 = f2_pack(-2.f * sy, -2.f * sy);
#pragma unroll
        for (int bb = 0; bb < NB; ++bb) {
          const int c0 = part * CPART + 16 * bb;
          const uint32_t(&r)[16] = rr[bb];
          float val[16];
#pragma unroll
          for (int k = 0; k < 16; k += 4) {
            const float4 vx = *reinterpret_cast<const float4*>(nx + c0 + k);
            const float4 vs = *reinterpret_cast<const float4*>(ns + c0 + k);
            unsigned long long w01 = w2c, w23 = w2c;
            if (!fmt_is_bf16(FMT)) {
              // w = (-2 sy) sx: both powers of two, so the product is exact
              const float4 vc = *reinterpret_cast<const float4*>(sx + c0 + k);
              w01 = f2_mul(wsy2, f2_pack(vc.x, vc.y));
              w23 = f2_mul(wsy2, f2_pack(vc.z, vc.w));
            }
            const unsigned long long a01 = f2_pack(__uint_as_float(r[k]), __uint_as_float(r[k + 1]));
            const unsigned long long a23 = f2_pack(__uint_as_float(r[k + 2]), __uint_as_float(r[k + 3]));
            const unsigned long long v01 = f2_fma(mcy2, f2_pack(vs.x, vs.y), f2_fma(w01, a01, f2_pack(vx.x, vx.y)));
            const unsigned long long v23 = f2_fma(mcy2, f2_pack(vs.z, vs.w), f2_fma(w23, a23, f2_pack(vx.z, vx.w)));
            val[k] = f2_lo(v01);
            val[k + 1] = f2_hi(v01);
            val[k + 2] = f2_lo(v23);
            val[k + 3] = f2_hi(v23);
          }
          // the block's minimum as a tree of three-input minima (8 for 16)
          const float mn =
              fminf(fmin3(fmin3(val[0], val[1], val[2]), fmin3(val[3], val[4], val[5]), fmin3(val[6], val[7], val[8])),
                    fmin3(fmin3(val[9], val[10], val[11]), fmin3(val[12], val[13], val[14]), val[15]));
          if (mn < tv[KL - 1]) {
            // the few columns that beat the current K-th entry: park the
            // block's values, then one (rolled) insertion per such column
            // that still beats it
            const float thr = tv[KL - 1];
            unsigned msk = 0;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              msk |= (val[k] < thr ? 1u : 0u) << k;
              stage[k][etid] = val[k];
            }
#pragma unroll 1
            while (msk) {
              const int k = __ffs(msk) - 1;
              msk &= msk - 1;
              const float vk = stage[k][etid];
              if (vk < tv[KL - 1]) tag_insert<KL>(tv, used, table, TSTRIDE, vk, tile * BN + c0 + k);
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&bar_acc_empty[b]);
        mbar_arrive(&bar_nrm_empty[n]);
      }
    }
    // untag: positions from the table, values floored to lower bounds of
    // the exact approximate values (every bound taken from a list is then
    // at most the value it stands for)
    int tp[KL];
#pragma unroll
    for (int k = 0; k < KL; ++k) {
      const bool real = tv[k] != CUDART_INF_F;
      tp[k] = real ? table[(__float_as_uint(tv[k]) & TagList<KL>::MASK) * TSTRIDE] : -1;
      if (real) tv[k] = tag_floor(tv[k], TagList<KL>::MASK);
    }
    // merge: parts 1.. hand their lists to part 0 (through the staging
    // area, once every epilogue warp has left it)
    asm volatile("bar.sync 1, %0;" ::"r"(EW * 32) : "memory");
    if (part > 0) {
      const int o = (part - 1) * KL * TC_BM;
#pragma unroll
      for (int k = 0; k < KL; ++k) {
        merge_v[o + k * TC_BM + row] = tv[k];
        merge_p[o + k * TC_BM + row] = tp[k];
      }
    }
    asm volatile("bar.sync 1, %0;" ::"r"(EW * 32) : "memory");
    if (part == 0) {
      for (int pp = 0; pp < PARTS - 1; ++pp) {
        const int o = pp * KL * TC_BM;
#pragma unroll
        for (int k = 0; k < KL; ++k) topk_insert(tv, tp, merge_v[o + k * TC_BM + row], merge_p[o + k * TC_BM + row]);
      }
      if (q < P.nt) {
        const size_t o = ((size_t)blockIdx.y * P.nt_pad + q) * KL;
#pragma unroll
        for (int k = 0; k < KL; ++k) {
          P.cand_v[o + k] = tv[k];
          P.cand_p[o + k] = tp[k];
        }
      }
    }
  }
  if (!ok) atomicOr(P.err, EF_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem_base, TMEM_ALLOC);
}

// --------------------------------------------------------------------------
// exact re-rank + certificate
// --------------------------------------------------------------------------

struct RerankArgs {
  const float* x;       // original coordinates
  const float* y;
  const int* ia;        // active supplier position -> original index
  const int* ja;
  int d, nt, nt_pad, chunks, fmt;
  const float* cand_v;
  const int* cand_p;
  const float* nrm_y;   // FP32 squared norm of each active consumer
  const float* scale_y;
  const unsigned* stats_x;  // max |x|_2, max |x|_1, max scale over active suppliers (float bits)
  unsigned long long* nnkey;
  int* fallback;        // consumer positions to rescan in FP32
  int* nfallback;
  unsigned long long* ncertified;
  unsigned long long* nfallback_total;
  unsigned long long* nnear;  // consumers whose exact best differs from the approximate best
  const int* sel;       // packed row -> consumer position (nullable: identity)
  const int* nq_dev;    // rows in use (nullable: nt)
  int rk;               // candidates of each chunk re-ranked (1 .. kl)
  int kl;               // list length of each chunk (the stride of cand_v / cand_p)
};

// One warp per packed consumer row.  The first rk candidates of every chunk
// are re-ranked; tau is the smallest rk-th approximate value over the chunks
// (every supplier outside them lies at or above it).  A consumer whose exact
// best differs from the candidate the approximate values ranked first (over
// all chunks, lowest position on ties) is counted as a near-tie of the
// operand precision.
__global__ void k_rerank_certify(RerankArgs R) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= (R.nq_dev ? min(*R.nq_dev, R.nt) : R.nt)) return;
  const int q = R.sel ? R.sel[r] : r;
  const float* yrow = R.y + (size_t)R.ja[q] * R.d;
  const int rk = R.rk;
  const int ncand = R.chunks * rk;
  // rows read 16 bytes at a time where d and both bases allow it
  const bool vec = (R.d & 3) == 0 && ((reinterpret_cast<uintptr_t>(R.x) | reinterpret_cast<uintptr_t>(R.y)) & 15) == 0;
  unsigned long long best = ~0ULL, abest = ~0ULL;
  float tau = CUDART_INF_F;  // smallest chunk threshold (rk-th value of each chunk)
  for (int c = lane; c < ncand; c += 32) {
    const int chunk = c / rk, k = c % rk;
    const size_t o = ((size_t)chunk * R.nt_pad + r) * R.kl + k;
    const int p = R.cand_p[o];
    if (k == rk - 1) tau = fminf(tau, R.cand_v[o]);
    if (p < 0) continue;
    if (k == 0) {
      const unsigned long long ak = ((unsigned long long)ordered_bits(R.cand_v[o]) << 32) | (unsigned)p;
      abest = ak < abest ? ak : abest;
    }
    // squared-Euclidean FP32 key (the contraction has no L1 form)
    const float* xr = R.x + (size_t)R.ia[p] * R.d;
    const float acc = vec ? key32_sql2_v4(xr, yrow, R.d) : key32<METRIC_SQL2>(xr, yrow, R.d);
    const unsigned long long key = pack_key(acc, (unsigned)p);
    best = key < best ? key : best;
  }
  // |y|_2^2 and |y|_1 in FP64, split over the lanes
  double yl2 = 0.0, yl1 = 0.0;
  for (int k = lane; k < R.d; k += 32) {
    yl2 += (double)yrow[k] * yrow[k];
    yl1 += fabs((double)yrow[k]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
    best = ob < best ? ob : best;
    const unsigned long long oa = __shfl_xor_sync(0xffffffffu, abest, o);
    abest = oa < abest ? oa : abest;
    tau = fminf(tau, __shfl_xor_sync(0xffffffffu, tau, o));
    yl2 += __shfl_xor_sync(0xffffffffu, yl2, o);
    yl1 += __shfl_xor_sync(0xffffffffu, yl1, o);
  }
  if (lane != 0) return;
  if (best != ~0ULL && (unsigned)best != (unsigned)abest) atomicAdd(R.nnear, 1ULL);
  yl2 = sqrt(yl2) * (1 + 1e-12);
  const bool certified =
      best != ~0ULL && certify(R.fmt, R.d, R.nrm_y[r], yl2, yl1, R.scale_y[r], __uint_as_float(R.stats_x[0]),
                               __uint_as_float(R.stats_x[1]), __uint_as_float(R.stats_x[2]), tau,
                               __uint_as_float((unsigned)(best >> 32)));
  if (certified) {
    R.nnkey[q] = best;
    atomicAdd(R.ncertified, 1ULL);
  } else {
    R.fallback[atomicAdd(R.nfallback, 1)] = q;
    atomicAdd(R.nfallback_total, 1ULL);
  }
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------

size_t tc_kb(int d, int precision) {
  const int esize = precision == 3 ? 1 : 2;
  const int64_t values = (int64_t)d * fmt_parts(fmt_of_precision(precision));
  return (size_t)((values * esize + 31) / 32 * 32);
}

int tc_bn(size_t kb) { return kb <= 384 ? 128 : 64; }

bool tc_supported(int d, int precision) {
  const size_t kb = tc_kb(d, precision);
  const size_t a_bytes = (size_t)TC_BM * kb, b_bytes = (size_t)tc_bn(kb) * kb;
  return a_bytes + b_bytes <= (size_t)TC_SMEM_BUDGET;
}

// B stages (up to 4) in what the instantiation leaves beside its static
// shared memory; the first launch of each instantiation sets the attribute.
template <int FMT, int BN, int KL>
static int launch_tc_t(TcArgs P, dim3 grid, size_t a_bytes, size_t b_bytes, cudaStream_t st) {
  static const int static_smem = [] {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, k_nns_tc<FMT, BN, KL>) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(k_nns_tc<FMT, BN, KL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TC_SMEM_MAX - 1024 - (int)fa.sharedSizeBytes) != cudaSuccess)
      return -1;
    return (int)fa.sharedSizeBytes;
  }();
  if (static_smem < 0) return -1;
  const size_t avail = (size_t)(TC_SMEM_MAX - 1024 - static_smem);
  if (a_bytes + b_bytes > avail) return -2;
  P.nstage = (int)std::min<size_t>(4, (avail - a_bytes) / b_bytes);
  const size_t smem = a_bytes + (size_t)P.nstage * b_bytes;
  k_nns_tc<FMT, BN, KL><<<grid, tc_threads(FMT, KL), smem, st>>>(P);
  return 0;
}

template <int FMT>
static int launch_tc_f(const TcArgs& P, int bn, int kl, dim3 grid, size_t a, size_t b, cudaStream_t st) {
  if (bn == 128) return kl == TC_K ? launch_tc_t<FMT, 128, TC_K>(P, grid, a, b, st)
                                   : launch_tc_t<FMT, 128, TC_K / 2>(P, grid, a, b, st);
  return kl == TC_K ? launch_tc_t<FMT, 64, TC_K>(P, grid, a, b, st) : launch_tc_t<FMT, 64, TC_K / 2>(P, grid, a, b, st);
}

// With sel / nsel_dev the consumers are the positions sel[0 .. *nsel_dev)
// (at most nt of them), e.g. those a learned proposal could not certify.
int launch_nns_tc(const SolveBufs& B, const TcBufs& T, int mt, int nt, int precision, cudaStream_t st,
                  const int* sel, const int* nsel_dev) {
  const int fmt = fmt_of_precision(precision);
  const int kb = (int)tc_kb(B.d, precision);
  const int bn = tc_bn(kb);
  const int qtiles = (nt + TC_BM - 1) / TC_BM;
  const int stiles = (mt + bn - 1) / bn;
  // pack both sides
  if (cudaMemsetAsync(T.stats, 0, 8 * sizeof(unsigned), st) != cudaSuccess) return -1;
  {
    const int64_t work = (int64_t)qtiles * TC_BM;
    int g = (int)std::min<int64_t>((work + 255) / 256, num_sms() * 16);
    k_pack_tc<<<g, 256, 0, st>>>(B.y, B.ja[B.cur], sel, nsel_dev, nt, qtiles * TC_BM, B.d, kb, fmt, TC_BM, T.A,
                                 T.nrm_y, nullptr, T.scale_y, T.stats + 4);
  }
  {
    const int64_t work = (int64_t)stiles * bn;
    int g = (int)std::min<int64_t>((work + 255) / 256, num_sms() * 16);
    k_pack_tc<<<g, 256, 0, st>>>(B.x, B.ia[B.cur], nullptr, nullptr, mt, stiles * bn, B.d, kb, fmt, bn, T.B,
                                 T.nrm_x, T.nrm_sx, T.scale_x, T.stats);
  }
  // chunks of supplier tiles so that the grid covers the GPU several times
  int chunks = (tc_target_ctas() + qtiles - 1) / qtiles;
  if (chunks > stiles) chunks = stiles;
  if (chunks > T.max_chunks) chunks = T.max_chunks;
  const int per = (stiles + chunks - 1) / chunks;
  chunks = (stiles + per - 1) / per;
  const size_t a_bytes = (size_t)TC_BM * kb, b_bytes = (size_t)bn * kb;
  const int nt_pad = qtiles * TC_BM;
  // candidates re-ranked per chunk; the scan keeps half the lists when that suffices
  const int rk = T.rerank_k >= 1 && T.rerank_k <= TC_K ? T.rerank_k : TC_K;
  const int kl = rk <= TC_K / 2 ? TC_K / 2 : TC_K;
  TcArgs P{T.A,      T.B,      T.nrm_x,    T.nrm_sx, T.nrm_y,  T.scale_x,  T.scale_y, nt, mt,
           kb,       bn,       0,          per,      stiles,   nt_pad,     T.cand_v,  T.cand_p, &B.st->err,
           nsel_dev};
  dim3 grid(qtiles, chunks);
  int rc;
  if (T.ev0) cudaEventRecord(T.ev0, st);
  if (fmt == FMT_BF16)
    rc = launch_tc_f<FMT_BF16>(P, bn, kl, grid, a_bytes, b_bytes, st);
  else if (fmt == FMT_BF16X3)
    rc = launch_tc_f<FMT_BF16X3>(P, bn, kl, grid, a_bytes, b_bytes, st);
  else if (fmt == FMT_F16)
    rc = launch_tc_f<FMT_F16>(P, bn, kl, grid, a_bytes, b_bytes, st);
  else
    rc = launch_tc_f<FMT_E4M3>(P, bn, kl, grid, a_bytes, b_bytes, st);
  if (rc) return rc;
  if (T.ev1) cudaEventRecord(T.ev1, st);
  // exact re-rank and certificate
  if (cudaMemsetAsync(T.nfallback, 0, sizeof(int), st) != cudaSuccess) return -1;
  RerankArgs R{B.x,      B.y,        B.ia[B.cur], B.ja[B.cur], B.d,       nt,          nt_pad,
               chunks,   fmt,        T.cand_v,    T.cand_p,    T.nrm_y,   T.scale_y,   T.stats,
               B.nnkey,  T.fallback, T.nfallback, &B.st->certified, &B.st->fallbacks, &B.st->near_ties,
               sel,      nsel_dev,   rk,          kl};
  k_rerank_certify<<<(nt + 7) / 8, 256, 0, st>>>(R);
  // FP32 scan of the consumers that were not certified
  launch_nns_f32(B, mt, nt, T.fallback, T.nfallback, st);
  return 0;
}

// --------------------------------------------------------------------------
// A plain BF16 contraction on the tensor cores, S = X W^T with FP32
// accumulation (rows of X against rows of W), for the learned proposal's
// per-solve passes.  Both operands are packed like K2's (K-major, no
// swizzle, tiles of 128 rows).  The epilogue either stores S + b (a linear
// layer), keeps each row's largest S + b (an assignment), or turns S into a
// lower bound of a squared distance (below).
// --------------------------------------------------------------------------

constexpr int LIN_TILE = 128;  // rows of X and of W per tile
constexpr int LIN_MAX_K = 256; // packed values per row

enum LinMode : int { LIN_STORE = 0, LIN_ARGMAX = 1, LIN_LOWER = 2, LIN_PACK_RELU = 3 };

struct LinArgs {
  const uint8_t* X;
  const uint8_t* W;
  int K;                     // packed values per row
  int rows, N;
  const float* bias;         // STORE / ARGMAX: [N]
  float* Z;                  // STORE / LOWER: [rows][N]
  uint8_t* P;                // PACK_RELU: relu(S + b) packed in BF16 as the next layer's X (N values a row)
  unsigned long long* part;  // ARGMAX: [rows][ceil(N / 128)]
  // LOWER: the rows and columns as points; X and W hold BF16X3 copies
  const float* row_sq_lo;    // [rows] |y|^2 rounded down
  const float* row_nrm_up;   // [rows] |y| rounded up
  const float* col_sq_lo;    // [N] |mu|^2 rounded down
  const float* col_nrm_up;   // [N] |mu| rounded up
  const float* col_radius;   // [N] r_c (rounded up when formed)
  float err_coeff;           // |S - <y, mu>| <= err_coeff |y| |mu| + 1e-30
  unsigned* err;
};

// Rows [0, rows) of src [rows][d] packed in tiles of LIN_TILE rows (padding
// rows zero): BF16 copies (fmt FMT_BF16), or BF16X3 splits (FMT_BF16X3;
// `supplier` picks the segment order) of 3d values per row.  One thread per
// 16-byte block of a row; consecutive threads write consecutive rows of one
// block column.
__global__ void k_pack_rows(const float* __restrict__ src, int rows, int rows_pad, int d, int fmt, bool supplier,
                            uint8_t* __restrict__ out) {
  const int kb = 2 * d * fmt_parts(fmt);
  const int64_t total = (int64_t)rows_pad * (kb / 16);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / rows_pad), p = (int)(i % rows_pad);
    const float* row = p < rows ? src + (size_t)p * d : nullptr;
    const int t = p / LIN_TILE, r = p % LIN_TILE;
    pack_block(row, d, c, 1.f, fmt, out + (size_t)t * LIN_TILE * kb, LIN_TILE, r, supplier);
  }
}

// One CTA per 128 x 128 block of S: both tiles by one bulk copy each, K / 16
// MMAs into a 128-column accumulator, then every thread takes its row's 128
// values through the mode's epilogue (columns >= N and rows >= rows are
// skipped; ARGMAX keeps the largest S + b, lowest column on ties, as a
// packed key in part[row][column tile]).
//
// LOWER: with S~ the computed <y~, mu~> of the BF16X3 copies, |S~ - <y, mu>|
// <= err_coeff |y| |mu| (+ 1e-30 for the subnormal floors), so
//   |y - mu|^2 >= |y|^2_lo + |mu|^2_lo - 2 (S~ + err_coeff |y|_up |mu|_up),
// and the bound on the squared distance to any point of cell `col` is
// max(0, sqrt(that) - r_col)^2, every step rounded toward the bound.
template <int MODE>
__global__ void __launch_bounds__(128, 1) k_linear_tc(LinArgs A) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bar_ld;
  __shared__ __align__(8) uint64_t bar_mma;
  __shared__ uint32_t tslot;
  __shared__ float col_a[LIN_TILE], col_b[LIN_TILE], col_c[LIN_TILE];  // the tile's per-column terms
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t tile_bytes = LIN_TILE * 2 * A.K;
  {
    const int n = blockIdx.x * LIN_TILE + threadIdx.x;
    const bool in = n < A.N;
    if (MODE == LIN_LOWER) {
      col_a[threadIdx.x] = in ? A.col_sq_lo[n] : 0.f;
      col_b[threadIdx.x] = in ? A.col_nrm_up[n] : 0.f;
      col_c[threadIdx.x] = in ? A.col_radius[n] : 0.f;
    } else {
      col_a[threadIdx.x] = in ? A.bias[n] : 0.f;
    }
  }
  uint8_t* sX = smem;
  uint8_t* sW = smem + tile_bytes;
  if (threadIdx.x == 0) {
    mbar_init(&bar_ld, 1);
    mbar_init(&bar_mma, 1);
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(&tslot, LIN_TILE);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar_ld, 2 * tile_bytes);
    tma_load_1d(sX, A.X + (size_t)blockIdx.y * tile_bytes, tile_bytes, &bar_ld);
    tma_load_1d(sW, A.W + (size_t)blockIdx.x * tile_bytes, tile_bytes, &bar_ld);
    if (mbar_wait_bounded(&bar_ld, 0)) {
      tc_fence_after();
      const uint32_t idesc = make_idesc(1, LIN_TILE, LIN_TILE);
      const uint32_t x0 = smem_u32(sX), w0 = smem_u32(sW);
      for (int k = 0; k < A.K / 16; ++k)
        mma_issue<FMT_BF16>(tmem, make_desc(x0 + k * 2 * LIN_TILE * 16, LIN_TILE * 16, 128),
                            make_desc(w0 + k * 2 * LIN_TILE * 16, LIN_TILE * 16, 128), idesc, k > 0 ? 1u : 0u);
      mma_commit(&bar_mma);
    }
  }
  // the accumulator (every lane of a warp agrees before the aligned loads)
  const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar_mma, 0));
  tc_fence_after();
  if (ok) {
    const int row = blockIdx.y * LIN_TILE + warp * 32 + lane;
    const int n0 = blockIdx.x * LIN_TILE;
    const bool live = row < A.rows;
    float ysq = 0.f, ynr = 0.f;
    if (MODE == LIN_LOWER && live) {
      ysq = A.row_sq_lo[row];
      ynr = A.row_nrm_up[row];
    }
    unsigned long long best = 0ULL;
#pragma unroll 1
    for (int cb = 0; cb < LIN_TILE; cb += 64) {
      uint32_t rr[4][16];
#pragma unroll
      for (int b = 0; b < 4; ++b) tmem_ld16_async(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb + 16 * b), rr[b]);
      tmem_ld_wait(rr);
      if (MODE == LIN_PACK_RELU) {
        // 16 columns = two 16-byte blocks of the next layer's packed row
        // (zeros for padding rows, so the next tile holds no garbage)
        const int kb = 2 * A.N;
        uint8_t* base = A.P + (size_t)(row / LIN_TILE) * LIN_TILE * kb + (size_t)(row % LIN_TILE) * 16;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int nb = n0 + cb + 16 * b;
          if (nb >= A.N) continue;
          uint32_t w[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const float lo = live ? fmaxf(__uint_as_float(rr[b][2 * e]) + col_a[nb - n0 + 2 * e], 0.f) : 0.f;
            const float hi = live ? fmaxf(__uint_as_float(rr[b][2 * e + 1]) + col_a[nb - n0 + 2 * e + 1], 0.f) : 0.f;
            w[e] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
                   ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
          }
          *reinterpret_cast<uint4*>(base + (size_t)(nb / 8) * LIN_TILE * 16) = make_uint4(w[0], w[1], w[2], w[3]);
          *reinterpret_cast<uint4*>(base + (size_t)(nb / 8 + 1) * LIN_TILE * 16) = make_uint4(w[4], w[5], w[6], w[7]);
        }
        continue;
      }
      if (!live) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int e = 0; e < 16; e += 4) {
          const int nq = n0 + cb + 16 * b + e;
          float out[4];
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            const int n = nq + f;
            const float sv = __uint_as_float(rr[b][e + f]);
            out[f] = 0.f;
            if (n >= A.N) continue;
            const int cl = n - n0;
            if (MODE == LIN_ARGMAX) {
              const unsigned long long key =
                  ((unsigned long long)ordered_bits(sv + col_a[cl]) << 32) | (0xffffffffu - (unsigned)n);
              best = key > best ? key : best;
            } else if (MODE == LIN_STORE) {
              out[f] = sv + col_a[cl];
            } else {
              const float eb = __fmaf_ru(A.err_coeff, __fmul_ru(ynr, col_b[cl]), 1e-30f);
              const float d2 = __fsub_rd(__fadd_rd(ysq, col_a[cl]), __fmul_ru(2.f, __fadd_ru(sv, eb)));
              // sqrt from below: x * rsqrtf(x) is within 2^-22 of sqrt(x)
              // (rsqrtf is documented to 2 ulp), and the factor 1 - 2^-20
              // takes it under; tiny or non-positive x gives 0
              const float dist = d2 > 1e-30f ? __fmul_rd(__fmul_rd(d2, rsqrtf(d2)), 0.99999905f) : 0.f;
              const float gap = __fsub_rd(dist, col_c[cl]);
              out[f] = gap > 0.f ? __fmul_rd(gap, gap) : 0.f;
            }
          }
          if (MODE != LIN_ARGMAX) {
            float* zr = A.Z + (size_t)row * A.N;
            if ((A.N & 3) == 0 && nq + 3 < A.N) {
              *reinterpret_cast<float4*>(zr + nq) = make_float4(out[0], out[1], out[2], out[3]);
            } else {
#pragma unroll
              for (int f = 0; f < 4; ++f)
                if (nq + f < A.N) zr[nq + f] = out[f];
            }
          }
        }
    }
    if (MODE == LIN_ARGMAX && live) A.part[(size_t)row * gridDim.x + blockIdx.x] = best;
  } else if (threadIdx.x == 0) {
    atomicOr(A.err, EF_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, LIN_TILE);
}

// out[row] = the column of the row's largest partial key
__global__ void k_argmax_parts(const unsigned long long* __restrict__ part, int rows, int tiles, int* __restrict__ out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  unsigned long long best = 0ULL;
  for (int t = 0; t < tiles; ++t) best = max(best, part[(size_t)r * tiles + t]);
  out[r] = (int)(0xffffffffu - (unsigned)(best & 0xffffffffu));
}

// Per point: |p|^2 (sequential fma, relative error <= gamma_d) rounded down
// and |p| rounded up.
__global__ void k_point_norms(const float* __restrict__ pts, int n, int d, float* __restrict__ sq_lo,
                              float* __restrict__ nrm_up) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int k = 0; k < d; ++k) s = __fmaf_rn(pts[(size_t)i * d + k], pts[(size_t)i * d + k], s);
  const double g = certify_gamma(d);
  sq_lo[i] = __fmul_rd(s, __double2float_rd(1.0 - g));
  nrm_up[i] = __fsqrt_ru(__fmul_ru(s, __double2float_ru(1.0 + g / (1.0 - g))));
}

bool linear_tc_supported(int K) { return K >= 16 && K <= LIN_MAX_K && K % 16 == 0; }

size_t linear_tc_packed_bytes(int rows, int K) {
  return (size_t)(rows + LIN_TILE - 1) / LIN_TILE * LIN_TILE * 2 * K;
}

static int pack_rows(const float* src, int rows, int d, int fmt, bool supplier, uint8_t* out, cudaStream_t st) {
  const int rows_pad = (rows + LIN_TILE - 1) / LIN_TILE * LIN_TILE;
  const int64_t work = (int64_t)rows_pad * (2 * d * fmt_parts(fmt) / 16);
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, num_sms() * 16));
  k_pack_rows<<<g, 256, 0, st>>>(src, rows, rows_pad, d, fmt, supplier, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int pack_rows_bf16(const float* src, int rows, int K, uint8_t* out, cudaStream_t st) {
  return pack_rows(src, rows, K, FMT_BF16, false, out, st);
}

template <int MODE>
static int launch_linear_tc(const LinArgs& A, cudaStream_t st) {
  if (!linear_tc_supported(A.K) || A.rows <= 0 || A.N <= 0) return -2;
  const int smem = 2 * LIN_TILE * 2 * LIN_MAX_K;
  static const bool attr =
      cudaFuncSetAttribute(k_linear_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess;
  if (!attr) return -1;
  dim3 grid((A.N + LIN_TILE - 1) / LIN_TILE, (A.rows + LIN_TILE - 1) / LIN_TILE);
  k_linear_tc<MODE><<<grid, 128, 2 * LIN_TILE * 2 * A.K, st>>>(A);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int linear_tc(const uint8_t* X, int rows, int K, const uint8_t* W, const float* bias, int N, float* Z, unsigned* err,
              cudaStream_t st) {
  LinArgs A{};
  A.X = X, A.W = W, A.K = K, A.rows = rows, A.N = N, A.bias = bias, A.Z = Z, A.err = err;
  return launch_linear_tc<LIN_STORE>(A, st);
}

int linear_tc_pack_relu(const uint8_t* X, int rows, int K, const uint8_t* W, const float* bias, int N, uint8_t* out,
                        unsigned* err, cudaStream_t st) {
  if (N % 16) return -2;
  LinArgs A{};
  A.X = X, A.W = W, A.K = K, A.rows = rows, A.N = N, A.bias = bias, A.P = out, A.err = err;
  return launch_linear_tc<LIN_PACK_RELU>(A, st);
}

int linear_tc_argmax(const uint8_t* X, int rows, int K, const uint8_t* W, const float* bias, int N,
                     unsigned long long* part, int* out, unsigned* err, cudaStream_t st) {
  LinArgs A{};
  A.X = X, A.W = W, A.K = K, A.rows = rows, A.N = N, A.bias = bias, A.part = part, A.err = err;
  const int rc = launch_linear_tc<LIN_ARGMAX>(A, st);
  if (rc) return rc;
  k_argmax_parts<<<(rows + 255) / 256, 256, 0, st>>>(part, rows, (N + LIN_TILE - 1) / LIN_TILE, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

bool cell_bounds_tc_supported(int d) { return d % 16 == 0 && linear_tc_supported(3 * d); }

int cell_bounds_tc_cells(const float* mu, int cells, int d, uint8_t* packed, float* sq_lo, float* nrm_up,
                         cudaStream_t st) {
  k_point_norms<<<(cells + 255) / 256, 256, 0, st>>>(mu, cells, d, sq_lo, nrm_up);
  return pack_rows(mu, cells, d, FMT_BF16X3, true, packed, st);
}

int cell_bounds_tc(const float* y, int rows, int d, uint8_t* packed_y, float* y_sq_lo, float* y_nrm_up,
                   const uint8_t* packed_mu, const float* mu_sq_lo, const float* mu_nrm_up, const float* radius,
                   int cells, float* out, unsigned* err, cudaStream_t st) {
  k_point_norms<<<(rows + 255) / 256, 256, 0, st>>>(y, rows, d, y_sq_lo, y_nrm_up);
  if (pack_rows(y, rows, d, FMT_BF16X3, false, packed_y, st)) return -1;
  // |<y~, mu~> - <y, mu>| <= (Q + K 2^-22 nf^2) |y| |mu| for the BF16X3
  // copies (the certificate's quantisation and accumulation terms, K = 3d
  // packed values), with a little slack for this single-precision use
  const int K = 3 * d;
  const double nf = quant_norm_factor(FMT_BF16X3);
  const double c = (quant_err(FMT_BF16X3) + K * 0x1p-22 * nf * nf) * (1.0 + 1e-3);
  LinArgs A{};
  A.X = packed_y, A.W = packed_mu, A.K = K, A.rows = rows, A.N = cells, A.Z = out, A.err = err;
  A.row_sq_lo = y_sq_lo, A.row_nrm_up = y_nrm_up, A.col_sq_lo = mu_sq_lo, A.col_nrm_up = mu_nrm_up;
  A.col_radius = radius;
  float cf = (float)c;
  if ((double)cf < c) cf = std::nextafter(cf, 2.f * cf);  // rounded up
  A.err_coeff = cf;
  return launch_linear_tc<LIN_LOWER>(A, st);
}

}  // namespace nnsemd
