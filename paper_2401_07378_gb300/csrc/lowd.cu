// Low-dimension (d <= 8) NNS-EMD kernels for sm_103a.
//
// K1  k_nns_lowd   -- the NNS operation of Alg. 1 (Sec. III-A) over the
//                     active sets, fused distance + argmin.  Supplier tiles
//                     are staged in shared memory by 1-D TMA bulk copies
//                     (double-buffered on mbarriers); each thread keeps P
//                     consumers in registers and evaluates two of them per
//                     packed FP32x2 instruction.  The argmin runs on groups
//                     of 8 suppliers (3-input min), and the winning group is
//                     re-scanned once at the end to recover the lowest index
//                     attaining the minimum.  Partial results of different
//                     supplier chunks merge through a 64-bit atomicMin on
//                     (key bits, position), which keeps the lowest-index
//                     tie-break.
// cta_rounds       -- all steps of a round (NNS, grouping, greedy flow,
//                     weights update, compaction) for active sets of at most
//                     FIN_MAX points per side, entirely in one CTA's shared
//                     memory.  Used for the tail rounds of a large solve and,
//                     one pair per CTA, for batches of small pairs (Sec. III-D
//                     batch processing).
// k_finish_cl      -- the tail rounds on a thread-block cluster: the NNS step
//                     split over the cluster's CTAs (keys exchanged through
//                     distributed shared memory), up to 2048 points per side.
#include <math_constants.h>

#include <atomic>

#include "common.cuh"
#include "cta.cuh"
#include "kernels.h"

namespace nnsemd {

// --------------------------------------------------------------------------
// K1: fused FP32 distance + argmin, d <= 8
// --------------------------------------------------------------------------

constexpr int K1_THREADS = 256;
// consumers per thread (two per packed register): fewer at larger d so that
// the consumer coordinates stay in registers
__host__ __device__ constexpr int k1_p(int D) { return D <= 3 ? 8 : (D <= 6 ? 4 : 2); }
// resident CTAs per SM the register budget allows (128 or 64 registers)
__host__ __device__ constexpr int k1_min_blocks(int D, int P) { return (P == 2 && D <= 6) ? 4 : 2; }

// K1_P consumers per thread: k1_p(D) for large rounds, 2 for small ones
// (more CTAs, shorter per-thread loops).  A chunk is a multiple of 64
// suppliers; each tile copy stops at the chunk's end rounded up to a whole
// group of 8 (inside the NaN padding of the active list).
template <int D, int DP, bool L1, int K1_P>
__global__ void __launch_bounds__(K1_THREADS, k1_min_blocks(D, K1_P))
    k_nns_lowd(const float* __restrict__ xa, int mt, int chunk, const float* __restrict__ ya, int nt,
               unsigned long long* __restrict__ nnkey, unsigned* __restrict__ err) {
  static_assert(K1_TS % 8 == 0, "tile must hold whole groups");
  static_assert(K1_P % 2 == 0, "consumers are packed in pairs");
  __shared__ __align__(128) float tile[2][K1_TS * DP];
  __shared__ __align__(8) uint64_t bar[2];

  const int tid = threadIdx.x;
  const int q0 = blockIdx.x * (K1_THREADS * K1_P);
  const int p0 = blockIdx.y * chunk;
  const int p1 = min(p0 + chunk, mt);
  if (p0 >= p1) return;

  // this thread's consumers, packed two per 64-bit register
  unsigned long long yy[K1_P / 2][D];
#pragma unroll
  for (int c = 0; c < K1_P / 2; ++c) {
    const int qa = q0 + (2 * c) * K1_THREADS + tid;
    const int qb = q0 + (2 * c + 1) * K1_THREADS + tid;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      float va = qa < nt ? ya[(size_t)qa * DP + k] : 0.f;
      float vb = qb < nt ? ya[(size_t)qb * DP + k] : 0.f;
      yy[c][k] = f2_pack(va, vb);
    }
  }
  float best[K1_P];
  int bestg[K1_P];
#pragma unroll
  for (int c = 0; c < K1_P; ++c) { best[c] = CUDART_INF_F; bestg[c] = -1; }

  const int ntile = (p1 - p0 + K1_TS - 1) / K1_TS;
  // bytes of tile t: its points up to p1 rounded up to 8 (a multiple of 64 B)
  auto tile_bytes = [&](int t) -> unsigned {
    const int base = p0 + t * K1_TS;
    return (unsigned)(min(K1_TS, (p1 - base + 7) & ~7) * DP * sizeof(float));
  };
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0) {
    const unsigned b0 = tile_bytes(0);
    mbar_expect_tx(&bar[0], b0);
    tma_load_1d(tile[0], xa + (size_t)p0 * DP, b0, &bar[0]);
  }
  bool ok = true;
  for (int t = 0; t < ntile; ++t) {
    const int buf = t & 1;
    if (tid == 0 && t + 1 < ntile) {
      const unsigned bn = tile_bytes(t + 1);
      mbar_expect_tx(&bar[buf ^ 1], bn);
      tma_load_1d(tile[buf ^ 1], xa + (size_t)(p0 + (t + 1) * K1_TS) * DP, bn, &bar[buf ^ 1]);
    }
    if (ok) ok = mbar_wait_bounded(&bar[buf], (t >> 1) & 1);
    if (ok) {
      const int base = p0 + t * K1_TS;
      const int ng = (min(p1, base + K1_TS) - base + 7) >> 3;
      const float* xt = tile[buf];
      for (int g = 0; g < ng; ++g) {
        float gmin[K1_P];
#pragma unroll
        for (int c = 0; c < K1_P; ++c) gmin[c] = CUDART_INF_F;
#pragma unroll
        for (int s = 0; s < 8; s += 2) {
          float xv0[DP], xv1[DP];
#pragma unroll
          for (int k = 0; k < DP; ++k) {
            xv0[k] = xt[(g * 8 + s) * DP + k];
            xv1[k] = xt[(g * 8 + s + 1) * DP + k];
          }
#pragma unroll
          for (int c = 0; c < K1_P / 2; ++c) {
            float da0, db0, da1, db1;
            if (L1) {
              unsigned long long t0 = f2_sub(f2_pack(xv0[0], xv0[0]), yy[c][0]);
              unsigned long long u0 = f2_sub(f2_pack(xv1[0], xv1[0]), yy[c][0]);
              da0 = fabsf(f2_lo(t0)); db0 = fabsf(f2_hi(t0));
              da1 = fabsf(f2_lo(u0)); db1 = fabsf(f2_hi(u0));
#pragma unroll
              for (int k = 1; k < D; ++k) {
                unsigned long long tk = f2_sub(f2_pack(xv0[k], xv0[k]), yy[c][k]);
                unsigned long long uk = f2_sub(f2_pack(xv1[k], xv1[k]), yy[c][k]);
                da0 = __fadd_rn(da0, fabsf(f2_lo(tk))); db0 = __fadd_rn(db0, fabsf(f2_hi(tk)));
                da1 = __fadd_rn(da1, fabsf(f2_lo(uk))); db1 = __fadd_rn(db1, fabsf(f2_hi(uk)));
              }
            } else {
              unsigned long long t0 = f2_sub(f2_pack(xv0[0], xv0[0]), yy[c][0]);
              unsigned long long u0 = f2_sub(f2_pack(xv1[0], xv1[0]), yy[c][0]);
              unsigned long long acc0 = f2_mul(t0, t0);
              unsigned long long acc1 = f2_mul(u0, u0);
#pragma unroll
              for (int k = 1; k < D; ++k) {
                unsigned long long tk = f2_sub(f2_pack(xv0[k], xv0[k]), yy[c][k]);
                unsigned long long uk = f2_sub(f2_pack(xv1[k], xv1[k]), yy[c][k]);
                acc0 = f2_fma(tk, tk, acc0);
                acc1 = f2_fma(uk, uk, acc1);
              }
              da0 = f2_lo(acc0); db0 = f2_hi(acc0);
              da1 = f2_lo(acc1); db1 = f2_hi(acc1);
            }
            gmin[2 * c] = fmin3(gmin[2 * c], da0, da1);
            gmin[2 * c + 1] = fmin3(gmin[2 * c + 1], db0, db1);
          }
        }
        const int G = (base >> 3) + g;
#pragma unroll
        for (int c = 0; c < K1_P; ++c) {
          if (gmin[c] < best[c]) { best[c] = gmin[c]; bestg[c] = G; }
        }
      }
    }
    __syncthreads();
  }
  if (__syncthreads_or(!ok)) {
    // a copy never landed: give the last copy of each buffer a bounded
    // chance to complete before the CTA exits, then report
    if (tid == 0) {
      for (int b = 0; b < 2 && b < ntile; ++b) {
        const int uses = (ntile - b + 1) / 2;
        mbar_wait_bounded(&bar[b], (unsigned)(uses - 1) & 1);
      }
      atomicOr(err, EF_TIMEOUT);
    }
    return;
  }

  // resolve the lowest position inside the winning group and merge
#pragma unroll
  for (int c = 0; c < K1_P; ++c) {
    const int q = q0 + c * K1_THREADS + tid;
    if (q >= nt) continue;
    float yv[D];
#pragma unroll
    for (int k = 0; k < D; ++k) yv[k] = (c & 1) ? f2_hi(yy[c >> 1][k]) : f2_lo(yy[c >> 1][k]);
    unsigned long long key;
    if (bestg[c] >= 0) {
      const float* xg = xa + (size_t)bestg[c] * 8 * DP;
      int kk = 0;
      for (int s = 0; s < 8; ++s) {
        float v = L1 ? key32<METRIC_L1>(xg + s * DP, yv, D) : key32<METRIC_SQL2>(xg + s * DP, yv, D);
        if (v == best[c]) { kk = s; break; }
      }
      key = pack_key(best[c], (unsigned)(bestg[c] * 8 + kk));
    } else {
      key = pack_key(CUDART_INF_F, (unsigned)p0);
    }
    atomicMin(nnkey + q, key);
  }
}

// Launch shape of K1 for one round: consumers per thread P and the supplier
// chunk of a CTA, from a cost model of the kernel.  A wave of CTAs costs a
// fixed amount plus P x chunk pairs per thread at a per-pair time that grows
// with the CTAs sharing an SM (the FP32 pipe is shared): at d = 3, 7.9 ns
// per pair per thread alone on an SM for P = k1_p (15.8 ns with the 2
// resident CTAs of the full-size rounds), about 30 % more for P = 2 (the
// supplier loads are shared by fewer consumers), which fits 4 CTAs per SM
// for d <= 6; scaled by (d + 1) / 4 for other d.
struct K1Shape {
  int P, chunk, gx, gy;
};

static K1Shape k1_shape(int D, int mt, int nt) {
  const int PB = k1_p(D);
  const int nsm = num_sms();
  constexpr double kWaveNs = 2000.0;
  constexpr double kAloneFactor = 1.67;
  K1Shape best{PB, 64, 1, 1};
  double best_t = 1e30;
  const int Ps[2] = {PB, 2};
  for (int k = 0; k < 2; ++k) {
    const int P = Ps[k];
    const int per_sm = k1_min_blocks(D, P);
    const double pair_ns = (P == 2 ? 10.2 : 7.9) * (D + 1) / 4.0;  // measured at d = 3
    const long long resident = (long long)nsm * per_sm;
    const int gx = (nt + K1_THREADS * P - 1) / (K1_THREADS * P);
    const int max_gy = (mt + 63) / 64;
    int last_chunk = -1;
    for (int gy0 = 1; gy0 <= max_gy; gy0 += (gy0 < 64 ? 1 : gy0 / 16)) {
      const int chunk = ((mt + gy0 - 1) / gy0 + 63) / 64 * 64;
      if (chunk == last_chunk) continue;
      last_chunk = chunk;
      const int gy = (mt + chunk - 1) / chunk;
      const long long ctas = (long long)gx * gy;
      if (gy > 65535) continue;
      const double per_cta_ns = (double)P * chunk * pair_ns;
      const long long full = ctas / resident, rem = ctas % resident;
      double t = (double)full * (kWaveNs + per_cta_ns * per_sm);
      // a CTA alone on its SM leaves the FP32 pipe partly idle: it runs at
      // about 60 % of two co-resident CTAs' combined rate (measured on the
      // colour-transfer rounds)
      const long long k = (rem + nsm - 1) / nsm;
      if (rem) t += kWaveNs + per_cta_ns * (k > 1 ? (double)k : kAloneFactor);
      if (t < best_t) {
        best_t = t;
        best = K1Shape{P, chunk, gx, gy};
      }
    }
  }
  return best;
}

template <int D, int DP, bool L1>
static void nns_lowd_t(const SolveBufs& B, int mt, int nt, cudaStream_t st) {
  const K1Shape sh = k1_shape(D, mt, nt);
  dim3 grid(sh.gx, sh.gy);
  if (sh.P == 2)
    k_nns_lowd<D, DP, L1, 2><<<grid, K1_THREADS, 0, st>>>(B.xa[B.cur], mt, sh.chunk, B.ya[B.cur], nt, B.nnkey,
                                                          &B.st->err);
  else
    k_nns_lowd<D, DP, L1, k1_p(D)><<<grid, K1_THREADS, 0, st>>>(B.xa[B.cur], mt, sh.chunk, B.ya[B.cur], nt,
                                                                B.nnkey, &B.st->err);
}

int launch_nns_lowd(const SolveBufs& B, int mt, int nt, cudaStream_t st) {
  const bool l1 = B.metric == METRIC_L1;
#define NNS_CASE(DD, DPP)                                             \
  case DD:                                                            \
    if (l1) nns_lowd_t<DD, DPP, true>(B, mt, nt, st);                 \
    else nns_lowd_t<DD, DPP, false>(B, mt, nt, st);                   \
    break;
  switch (B.d) {
    NNS_CASE(1, 2) NNS_CASE(2, 2) NNS_CASE(3, 4) NNS_CASE(4, 4)
    NNS_CASE(5, 8) NNS_CASE(6, 8) NNS_CASE(7, 8) NNS_CASE(8, 8)
    default: return -1;
  }
#undef NNS_CASE
  return 0;
}

// --------------------------------------------------------------------------
// one-CTA solver, d <= 8 (coordinates in shared memory)
// --------------------------------------------------------------------------

// Tail of a single large solve: load the current active lists and finish.
template <int D, int DP, bool L1>
__global__ void __launch_bounds__(FIN_THREADS, 1) k_finish(SolveBufs B, long long round_limit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LowdSmem<D, DP, L1>& L = *reinterpret_cast<LowdSmem<D, DP, L1>*>(smem_raw);
  CtaCore<FIN_MAX>& S = L.S;
  const int tid = threadIdx.x;
  const int mt = B.st->mt, nt = B.st->nt;
  if (mt > FIN_MAX || nt > FIN_MAX) {
    if (tid == 0) atomicOr(&B.st->err, EF_INTERNAL);
    return;
  }
  const float* xa = B.xa[B.cur];
  const float* ya = B.ya[B.cur];
  for (int p = tid; p < mt; p += blockDim.x) {
#pragma unroll
    for (int k = 0; k < DP; ++k) L.G.xs[p * DP + k] = xa[(size_t)p * DP + k];
    S.iidx[p] = B.ia[B.cur][p];
    S.sres[p] = B.s[S.iidx[p]];
  }
  for (int q = tid; q < nt; q += blockDim.x) {
#pragma unroll
    for (int k = 0; k < DP; ++k) L.G.ys[q * DP + k] = ya[(size_t)q * DP + k];
    S.jidx[q] = B.ja[B.cur][q];
    S.cres[q] = B.c[S.jidx[q]];
  }
  if (tid == 0) {
    S.mt = mt;
    S.nt = nt;
  }
  __syncthreads();
  CtaOut O{nullptr, nullptr, nullptr, nullptr, 0, B.s, B.c, &B.st->err,
           B.fl_i, B.fl_j, B.fl_f, B.x, B.y, B.d, B.protocol, B.seed, B.round0};
  unsigned long long nnz = B.st->nnz;
  long long rounds = B.st->rounds, pe = B.st->pair_evals;
  cta_rounds(S, L.G, B.metric, O, nnz, rounds, pe, round_limit);
  if (tid == 0) {
    B.st->nnz = nnz;
    B.st->rounds = rounds;
    B.st->pair_evals = pe;
    B.st->mt = S.mt;
    B.st->nt = S.nt;
  }
}

template <int D, int DP, bool L1>
static int finish_t(const SolveBufs& B, long long round_limit, cudaStream_t st) {
  const size_t smem = sizeof(LowdSmem<D, DP, L1>);
  cudaError_t e = cudaFuncSetAttribute(k_finish<D, DP, L1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return -1;
  k_finish<D, DP, L1><<<1, FIN_THREADS, smem, st>>>(B, round_limit);
  return 0;
}

int launch_finish(const SolveBufs& B, int64_t round_limit, cudaStream_t st) {
  const bool l1 = B.metric == METRIC_L1;
#define FIN_CASE(DD, DPP) \
  case DD:                \
    return l1 ? finish_t<DD, DPP, true>(B, round_limit, st) : finish_t<DD, DPP, false>(B, round_limit, st);
  switch (B.d) {
    FIN_CASE(1, 2) FIN_CASE(2, 2) FIN_CASE(3, 4) FIN_CASE(4, 4)
    FIN_CASE(5, 8) FIN_CASE(6, 8) FIN_CASE(7, 8) FIN_CASE(8, 8)
    default: return -1;
  }
#undef FIN_CASE
}

// --------------------------------------------------------------------------
// the tail on a thread-block cluster (d <= 8)
// --------------------------------------------------------------------------

#ifndef NNSEMD_TAIL_CLUSTER
#define NNSEMD_TAIL_CLUSTER 16  // preferred cluster size (8 where 16 cannot be co-scheduled)
#endif
#ifndef NNSEMD_TAIL_THREADS
#define NNSEMD_TAIL_THREADS 512  // threads per CTA of the cluster tail
#endif
constexpr int FIN_CL_THREADS = NNSEMD_TAIL_THREADS;

template <int D, int DP, bool L1>
struct LowdClusterSmem {
  static constexpr int CAP = fin_cl_cap(DP);
  CtaCore<CAP> S;
  GeoSmemCluster<D, DP, L1, CAP, FIN_CL_THREADS> G;
};

// Every CTA of the cluster loads the current active lists and runs every
// remaining round; the NNS step is split over the cluster (GeoSmemCluster),
// the other steps run redundantly on identical state, and CTA 0 alone writes
// flows, residuals and the solve state.
template <int D, int DP, bool L1>
__global__ void __launch_bounds__(FIN_CL_THREADS, 1) k_finish_cl(SolveBufs B, long long round_limit) {
  namespace cg = cooperative_groups;
  using Sm = LowdClusterSmem<D, DP, L1>;
  constexpr int CAP = Sm::CAP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Sm& L = *reinterpret_cast<Sm*>(smem_raw);
  CtaCore<CAP>& S = L.S;
  cg::cluster_group cl = cg::this_cluster();
  const bool leader = cl.block_rank() == 0;
  const int tid = threadIdx.x;
  const int mt = B.st->mt, nt = B.st->nt;
  if (mt > CAP || nt > CAP || cl.num_blocks() < 8) {  // the same decision in every CTA
    if (tid == 0 && leader) atomicOr(&B.st->err, EF_INTERNAL);
    return;
  }
  const float* xa = B.xa[B.cur];
  const float* ya = B.ya[B.cur];
  for (int p = tid; p < mt; p += blockDim.x) {
#pragma unroll
    for (int k = 0; k < DP; ++k) L.G.xs[p * DP + k] = xa[(size_t)p * DP + k];
    S.iidx[p] = B.ia[B.cur][p];
    S.sres[p] = B.s[S.iidx[p]];
  }
  for (int q = tid; q < nt; q += blockDim.x) {
#pragma unroll
    for (int k = 0; k < DP; ++k) L.G.ys[q * DP + k] = ya[(size_t)q * DP + k];
    S.jidx[q] = B.ja[B.cur][q];
    S.cres[q] = B.c[S.jidx[q]];
  }
  if (tid == 0) {
    S.mt = mt;
    S.nt = nt;
  }
  L.G.init();
  // every CTA of the cluster is running before any writes a peer's memory
  cl.sync();
  CtaOut O{nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr, &B.st->err,
           nullptr, nullptr, nullptr, B.x, B.y, B.d, B.protocol, B.seed, B.round0, 1};
  if (leader)
    O = CtaOut{nullptr, nullptr, nullptr, nullptr, 0, B.s, B.c, &B.st->err,
               B.fl_i, B.fl_j, B.fl_f, B.x, B.y, B.d, B.protocol, B.seed, B.round0, 0};
  unsigned long long nnz = B.st->nnz;
  long long rounds = B.st->rounds, pe = B.st->pair_evals;
  cta_rounds(S, L.G, B.metric, O, nnz, rounds, pe, round_limit);
  if (tid == 0 && leader) {
    B.st->nnz = nnz;
    B.st->rounds = rounds;
    B.st->pair_evals = pe;
    B.st->mt = S.mt;
    B.st->nt = S.nt;
  }
  // no CTA leaves while a peer may still address its shared memory
  cl.sync();
}

// Cluster size usable for k_finish_cl<D, DP, L1> on `dev` (cached): the
// preferred size if the device can co-schedule one such cluster, else 8,
// else 0.
template <int D, int DP, bool L1>
static int finish_cl_size(int dev) {
  static std::atomic<int> cache[64];
  if (dev < 0 || dev >= 64) return 0;
  const int c = cache[dev].load();
  if (c) return c > 0 ? c : 0;
  const size_t smem = sizeof(LowdClusterSmem<D, DP, L1>);
  int found = -1;
  if (cudaFuncSetAttribute(k_finish_cl<D, DP, L1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
          cudaSuccess &&
      cudaFuncSetAttribute(k_finish_cl<D, DP, L1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
          cudaSuccess) {
    for (int cs : {NNSEMD_TAIL_CLUSTER, 8}) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cs;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(cs);
      cfg.blockDim = dim3(FIN_CL_THREADS);
      cfg.dynamicSmemBytes = smem;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, k_finish_cl<D, DP, L1>, &cfg) == cudaSuccess && n > 0) {
        found = cs;
        break;
      }
    }
  }
  cudaGetLastError();  // a refused size is an answer, not an error of the solve
  cache[dev].store(found);
  return found > 0 ? found : 0;
}

template <int D, int DP, bool L1>
static int finish_cl_t(const SolveBufs& B, long long round_limit, cudaStream_t st) {
  static_assert(sizeof(LowdClusterSmem<D, DP, L1>) <= 227 * 1024, "cluster tail state exceeds shared memory");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  const int cs = finish_cl_size<D, DP, L1>(dev);
  if (cs == 0) return -1;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(FIN_CL_THREADS);
  cfg.dynamicSmemBytes = sizeof(LowdClusterSmem<D, DP, L1>);
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_finish_cl<D, DP, L1>, B, round_limit) == cudaSuccess ? 0 : -1;
}

int finish_cluster_cap(int d, int metric) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  const bool l1 = metric == METRIC_L1;
#define FCL_CASE(DD, DPP) \
  case DD:                \
    return (l1 ? finish_cl_size<DD, DPP, true>(dev) : finish_cl_size<DD, DPP, false>(dev)) ? fin_cl_cap(DPP) : 0;
  switch (d) {
    FCL_CASE(1, 2) FCL_CASE(2, 2) FCL_CASE(3, 4) FCL_CASE(4, 4)
    FCL_CASE(5, 8) FCL_CASE(6, 8) FCL_CASE(7, 8) FCL_CASE(8, 8)
    default: return 0;
  }
#undef FCL_CASE
}

int launch_finish_cluster(const SolveBufs& B, int64_t round_limit, cudaStream_t st) {
  const bool l1 = B.metric == METRIC_L1;
#define FCL_CASE(DD, DPP) \
  case DD:                \
    return l1 ? finish_cl_t<DD, DPP, true>(B, round_limit, st) : finish_cl_t<DD, DPP, false>(B, round_limit, st);
  switch (B.d) {
    FCL_CASE(1, 2) FCL_CASE(2, 2) FCL_CASE(3, 4) FCL_CASE(4, 4)
    FCL_CASE(5, 8) FCL_CASE(6, 8) FCL_CASE(7, 8) FCL_CASE(8, 8)
    default: return -1;
  }
#undef FCL_CASE
}

}  // namespace nnsemd
