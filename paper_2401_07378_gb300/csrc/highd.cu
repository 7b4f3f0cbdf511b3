// High-dimension (d > 8) NNS-EMD kernels for sm_103a, FP32 decisions.
//
// k_nns_f32_tiled -- the NNS operation (Alg. 1, Sec. III-A) for d > 8 on CUDA
//                    cores: each CTA is one 256-thread group that runs 64 x 64
//                    (consumer x supplier) tiles, staging 32 coordinates of
//                    each side at a time in shared memory; every thread
//                    accumulates 4 x 4 pairs over k in order, which reproduces
//                    the FP32 key bit for bit.  CTAs split the suppliers into
//                    chunks and merge through atomicMin on (key, position).
//                    With a consumer list it scans only those consumers (the
//                    fallback of the reduced-precision path).
// k_finish_hd      -- the tail rounds of a large solve in one CTA, coordinates
//                    read from L2 by original index.
// k_batched_hd     -- batches of pairs with up to 2,048 points per side, one
//                    pair per CTA, all rounds on chip (Sec. III-D batching).
#include <math_constants.h>

#include "common.cuh"
#include "cta.cuh"
#include "kernels.h"

namespace nnsemd {

template <bool L1>
__global__ void __launch_bounds__(TG_THREADS)
    k_nns_f32_tiled(const float* __restrict__ x, const int* __restrict__ ia, int mt, int chunk,
                    const float* __restrict__ y, const int* __restrict__ ja, const int* __restrict__ cons,
                    const int* __restrict__ ncons_dev, int ncons, int d, unsigned long long* __restrict__ nnkey) {
  __shared__ TileSmem T;
  const int nc_all = ncons_dev ? *ncons_dev : ncons;
  const int c0 = blockIdx.x * TG_M;
  if (c0 >= nc_all) return;
  const int p0 = blockIdx.y * chunk;
  const int p1 = min(p0 + chunk, mt);
  if (p0 >= p1) return;
  unsigned long long out[4];
  group_nns_tile<L1>(x, ia, p0, p1, y, ja, cons, c0, min(TG_M, nc_all - c0), d, T, threadIdx.x, 0, out);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  if (tx == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int lq = c0 + ty * 4 + i;
      if (lq < nc_all) atomicMin(nnkey + (cons ? cons[lq] : lq), out[i]);
    }
  }
}

int launch_nns_f32(const SolveBufs& B, int mt, int ncons, const int* cons, const int* ncons_dev, cudaStream_t st) {
  const int gx = (ncons + TG_M - 1) / TG_M;
  const int target = num_sms() * 6;
  int gy = (target + gx - 1) / gx;
  const int tiles = (mt + TG_N - 1) / TG_N;
  if (gy > tiles) gy = tiles;
  const int chunk = ((tiles + gy - 1) / gy) * TG_N;
  gy = (mt + chunk - 1) / chunk;
  dim3 grid(gx, gy);
  const int cur = B.cur;
  if (B.metric == METRIC_L1)
    k_nns_f32_tiled<true><<<grid, TG_THREADS, 0, st>>>(B.x, B.ia[cur], mt, chunk, B.y, B.ja[cur], cons, ncons_dev,
                                                      ncons, B.d, B.nnkey);
  else
    k_nns_f32_tiled<false><<<grid, TG_THREADS, 0, st>>>(B.x, B.ia[cur], mt, chunk, B.y, B.ja[cur], cons, ncons_dev,
                                                       ncons, B.d, B.nnkey);
  return 0;
}

// --------------------------------------------------------------------------
// one-CTA solver, d > 8
// --------------------------------------------------------------------------

template <bool L1>
struct HighdSmem {
  CtaCore<FIN_MAX_HD> S;
  GeoGlobal<L1, FIN_MAX_HD> G;
};

template <bool L1>
__global__ void __launch_bounds__(FIN_THREADS, 1) k_finish_hd(SolveBufs B, long long round_limit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  HighdSmem<L1>& H = *reinterpret_cast<HighdSmem<L1>*>(smem_raw);
  CtaCore<FIN_MAX_HD>& S = H.S;
  const int tid = threadIdx.x;
  const int mt = B.st->mt, nt = B.st->nt;
  if (mt > FIN_MAX_HD || nt > FIN_MAX_HD) {
    if (tid == 0) atomicOr(&B.st->err, EF_INTERNAL);
    return;
  }
  if (tid == 0) {
    H.G.x = B.x;
    H.G.y = B.y;
    H.G.d = B.d;
    S.mt = mt;
    S.nt = nt;
  }
  for (int p = tid; p < mt; p += blockDim.x) {
    S.iidx[p] = B.ia[B.cur][p];
    S.sres[p] = B.s[S.iidx[p]];
  }
  for (int q = tid; q < nt; q += blockDim.x) {
    S.jidx[q] = B.ja[B.cur][q];
    S.cres[q] = B.c[S.jidx[q]];
  }
  __syncthreads();
  CtaOut O{nullptr, nullptr, nullptr, nullptr, 0, B.s, B.c, &B.st->err,
           B.fl_i, B.fl_j, B.fl_f, B.x, B.y, B.d, B.protocol, B.seed, B.round0};
  unsigned long long nnz = B.st->nnz;
  long long rounds = B.st->rounds, pe = B.st->pair_evals;
  cta_rounds(S, H.G, B.metric, O, nnz, rounds, pe, round_limit);
  if (tid == 0) {
    B.st->nnz = nnz;
    B.st->rounds = rounds;
    B.st->pair_evals = pe;
    B.st->mt = S.mt;
    B.st->nt = S.nt;
  }
}

template <bool L1>
static int finish_hd_t(const SolveBufs& B, long long round_limit, cudaStream_t st) {
  const size_t smem = sizeof(HighdSmem<L1>);
  cudaError_t e = cudaFuncSetAttribute(k_finish_hd<L1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return -1;
  k_finish_hd<L1><<<1, FIN_THREADS, smem, st>>>(B, round_limit);
  return 0;
}

int launch_finish_hd(const SolveBufs& B, int64_t round_limit, cudaStream_t st) {
  return B.metric == METRIC_L1 ? finish_hd_t<true>(B, round_limit, st) : finish_hd_t<false>(B, round_limit, st);
}

template <bool L1>
__global__ void __launch_bounds__(FIN_THREADS, 1) k_batched_hd(BatchArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  HighdSmem<L1>& H = *reinterpret_cast<HighdSmem<L1>*>(smem_raw);
  __shared__ int s_item;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) s_item = (int)atomicAdd(A.queue, 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= A.num) break;
    const int pr = A.pair_ids[item];
    const int64_t xo = A.x_off[pr], yo = A.n_shared ? 0 : A.y_off[pr];
    const int m = (int)(A.x_off[pr + 1] - xo), n = A.n_shared ? A.n_shared : (int)(A.y_off[pr + 1] - yo);
    if (tid == 0) {
      H.G.x = A.x + xo * A.d;
      H.G.y = A.y + yo * A.d;
      H.G.d = A.d;
    }
    __syncthreads();
    double cost = 0.0;
    long long rounds = 0, pe = 0;
    const size_t fo = (size_t)blockIdx.x * A.fl_cap;
    const bool ok = cta_solve_pair(H.S, H.G, nullptr, nullptr, A.x + xo * A.d, A.a + xo, m, A.y + yo * A.d,
                                   A.b + yo, n, A.d, A.metric, A.err, cost, rounds, pe, A.protocol, A.seed,
                                   A.fl_i ? A.fl_i + fo : nullptr, A.fl_i ? A.fl_j + fo : nullptr,
                                   A.fl_i ? A.fl_f + fo : nullptr, A.fl_cap);
    if (tid == 0) {
      A.costs[pr] = ok ? cost : CUDART_NAN;
      if (A.rounds) A.rounds[pr] = rounds;
      if (A.pair_evals) A.pair_evals[pr] = pe;
    }
    __syncthreads();
  }
}

template <bool L1>
static int batched_hd_t(const BatchArgs& A, int grid, cudaStream_t st) {
  const size_t smem = sizeof(HighdSmem<L1>);
  cudaError_t e = cudaFuncSetAttribute(k_batched_hd<L1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return -1;
  k_batched_hd<L1><<<grid, FIN_THREADS, smem, st>>>(A);
  return 0;
}

int launch_batched_hd(const BatchArgs& A, int grid, cudaStream_t st) {
  return A.metric == METRIC_L1 ? batched_hd_t<true>(A, grid, st) : batched_hd_t<false>(A, grid, st);
}

// Pairs of at most HD_SMALL_CAP points per side: a 256-thread CTA each, four
// resident per SM, so that four pairs' latency-bound round loops overlap on
// every SM (a 1,024-thread CTA spends most of a small pair's round in its
// barriers: its NNS tile has one 256-thread group's worth of consumers).
template <bool L1>
struct HighdSmallSmem {
  CtaCore<HD_SMALL_CAP> S;
  GeoGlobal<L1, HD_SMALL_CAP, HD_SMALL_THREADS> G;
};

template <bool L1>
__global__ void __launch_bounds__(HD_SMALL_THREADS, 4) k_batched_hd_small(BatchArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  HighdSmallSmem<L1>& H = *reinterpret_cast<HighdSmallSmem<L1>*>(smem_raw);
  __shared__ int s_item;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) s_item = (int)atomicAdd(A.queue, 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= A.num) break;
    const int pr = A.pair_ids[item];
    const int64_t xo = A.x_off[pr], yo = A.n_shared ? 0 : A.y_off[pr];
    const int m = (int)(A.x_off[pr + 1] - xo), n = A.n_shared ? A.n_shared : (int)(A.y_off[pr + 1] - yo);
    if (m > HD_SMALL_CAP || n > HD_SMALL_CAP) {  // the host routes only small pairs here
      if (tid == 0) atomicOr(A.err, EF_INTERNAL);
      break;
    }
    if (tid == 0) {
      H.G.x = A.x + xo * A.d;
      H.G.y = A.y + yo * A.d;
      H.G.d = A.d;
    }
    __syncthreads();
    double cost = 0.0;
    long long rounds = 0, pe = 0;
    const size_t fo = (size_t)blockIdx.x * A.fl_cap;
    const bool ok = cta_solve_pair(H.S, H.G, nullptr, nullptr, A.x + xo * A.d, A.a + xo, m, A.y + yo * A.d,
                                   A.b + yo, n, A.d, A.metric, A.err, cost, rounds, pe, A.protocol, A.seed,
                                   A.fl_i ? A.fl_i + fo : nullptr, A.fl_i ? A.fl_j + fo : nullptr,
                                   A.fl_i ? A.fl_f + fo : nullptr, A.fl_cap);
    if (tid == 0) {
      A.costs[pr] = ok ? cost : CUDART_NAN;
      if (A.rounds) A.rounds[pr] = rounds;
      if (A.pair_evals) A.pair_evals[pr] = pe;
    }
    __syncthreads();
  }
}

template <bool L1>
static int batched_hd_small_t(const BatchArgs& A, int grid, cudaStream_t st) {
  const size_t smem = sizeof(HighdSmallSmem<L1>);
  cudaError_t e =
      cudaFuncSetAttribute(k_batched_hd_small<L1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return -1;
  k_batched_hd_small<L1><<<grid, HD_SMALL_THREADS, smem, st>>>(A);
  return 0;
}

int launch_batched_hd_small(const BatchArgs& A, int grid, cudaStream_t st) {
  return A.metric == METRIC_L1 ? batched_hd_small_t<true>(A, grid, st) : batched_hd_small_t<false>(A, grid, st);
}

}  // namespace nnsemd
