// One-CTA NNS-EMD solves of whole small pairs, d <= 8 (the rounds of
// cta_rounds with the coordinates in shared memory): a single pair in one
// launch, batches of small pairs in one persistent launch (Sec. III-D batch
// processing), and the allocation-free entry point.
#include <math_constants.h>

#include <atomic>

#include "common.cuh"
#include "cta.cuh"
#include "kernels.h"

namespace nnsemd {

// --------------------------------------------------------------------------
// a whole small pair in one launch: load, normalise, every round, the plan,
// R and the leftover mass (no host round trip between rounds)
// --------------------------------------------------------------------------

template <int D, int DP, bool L1>
__global__ void __launch_bounds__(FIN_THREADS, 1) k_solve_small(SolveBufs B, const double* a, const double* b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LowdSmem<D, DP, L1>& L = *reinterpret_cast<LowdSmem<D, DP, L1>*>(smem_raw);
  CtaCore<FIN_MAX>& S = L.S;
  const int tid = threadIdx.x;
  const int m = (int)B.m, n = (int)B.n;
  bool ok = cta_load_side<DP, FIN_MAX>(B.x, a, m, B.d, L.G.xs, S.sres, S.iidx, S, &B.st->err);
  if (ok) ok = cta_load_side<DP, FIN_MAX>(B.y, b, n, B.d, L.G.ys, S.cres, S.jidx, S, &B.st->err);
  if (!ok) return;
  if (tid == 0) {
    S.mt = m;
    S.nt = n;
  }
  for (int i = tid; i < XS_LIMBS; i += blockDim.x) S.acc[i] = 0ULL;
  __syncthreads();
  cta_compact(S, L.G);  // drop zero weights
  CtaOut O{S.acc, B.plan_i, B.plan_j, B.plan_f, (long long)B.plan_cap, nullptr, nullptr, &B.st->err,
           B.fl_i, B.fl_j, B.fl_f, B.x, B.y, B.d, B.protocol, B.seed, 0};
  unsigned long long nnz = 0;
  long long rounds = 0, pe = 0;
  cta_rounds(S, L.G, B.metric, O, nnz, rounds, pe, (long long)m + n);
  __syncthreads();
  if (tid == 0) B.st->cost = xs_round(S.acc);
  __syncthreads();
  for (int i = tid; i < XS_LIMBS; i += blockDim.x) S.acc[i] = 0ULL;
  __syncthreads();
  for (int base = 0; base < S.mt; base += blockDim.x)  // whole warps (xs_add_warp)
    xs_add_warp(S.acc, base + tid < S.mt ? S.sres[base + tid] : 0.0);
  for (int base = 0; base < S.nt; base += blockDim.x)
    xs_add_warp(S.acc, base + tid < S.nt ? S.cres[base + tid] : 0.0);
  __syncthreads();
  if (tid == 0) {
    B.st->leftover = xs_round(S.acc);
    B.st->nnz = nnz;
    B.st->rounds = rounds;
    B.st->pair_evals = pe;
    B.st->mt = S.mt;
    B.st->nt = S.nt;
  }
}

template <int D, int DP, bool L1>
static int solve_small_t(const SolveBufs& B, const double* a, const double* b, cudaStream_t st) {
  const size_t smem = sizeof(LowdSmem<D, DP, L1>);
  cudaError_t e =
      cudaFuncSetAttribute(k_solve_small<D, DP, L1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return -1;
  k_solve_small<D, DP, L1><<<1, FIN_THREADS, smem, st>>>(B, a, b);
  return 0;
}

int launch_solve_small(const SolveBufs& B, const double* a, const double* b, cudaStream_t st) {
  const bool l1 = B.metric == METRIC_L1;
#define SMALL_CASE(DD, DPP) \
  case DD:                  \
    return l1 ? solve_small_t<DD, DPP, true>(B, a, b, st) : solve_small_t<DD, DPP, false>(B, a, b, st);
  switch (B.d) {
    SMALL_CASE(1, 2) SMALL_CASE(2, 2) SMALL_CASE(3, 4) SMALL_CASE(4, 4)
    SMALL_CASE(5, 8) SMALL_CASE(6, 8) SMALL_CASE(7, 8) SMALL_CASE(8, 8)
    default: return -1;
  }
#undef SMALL_CASE
}

// --------------------------------------------------------------------------
// batched small pairs: one persistent launch, a work queue of pairs, each
// pair solved start to finish by one CTA (Sec. III-D batch processing)
// --------------------------------------------------------------------------

template <int D, int DP, bool L1>
__global__ void __launch_bounds__(FIN_THREADS, 1) k_batched_lowd(BatchArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LowdSmem<D, DP, L1>& L = *reinterpret_cast<LowdSmem<D, DP, L1>*>(smem_raw);
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
    double cost = 0.0;
    long long rounds = 0, pe = 0;
    const bool ok = cta_solve_pair(L.S, L.G, L.G.xs, L.G.ys, A.x + xo * A.d, A.a + xo, m, A.y + yo * A.d, A.b + yo,
                                   n, A.d, A.metric, A.err, cost, rounds, pe, A.protocol, A.seed);
    if (tid == 0) {
      A.costs[pr] = ok ? cost : CUDART_NAN;
      if (A.rounds) A.rounds[pr] = rounds;
      if (A.pair_evals) A.pair_evals[pr] = pe;
    }
    __syncthreads();
  }
}

template <int D, int DP, bool L1>
static int batched_t(const BatchArgs& A, int grid, cudaStream_t st) {
  const size_t smem = sizeof(LowdSmem<D, DP, L1>);
  cudaError_t e =
      cudaFuncSetAttribute(k_batched_lowd<D, DP, L1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return -1;
  k_batched_lowd<D, DP, L1><<<grid, FIN_THREADS, smem, st>>>(A);
  return 0;
}

int launch_batched_lowd(const BatchArgs& A, int grid, cudaStream_t st) {
  const bool l1 = A.metric == METRIC_L1;
#define BAT_CASE(DD, DPP) \
  case DD:                \
    return l1 ? batched_t<DD, DPP, true>(A, grid, st) : batched_t<DD, DPP, false>(A, grid, st);
  switch (A.d) {
    BAT_CASE(1, 2) BAT_CASE(2, 2) BAT_CASE(3, 4) BAT_CASE(4, 4)
    BAT_CASE(5, 8) BAT_CASE(6, 8) BAT_CASE(7, 8) BAT_CASE(8, 8)
    default: return -1;
  }
#undef BAT_CASE
}

}  // namespace nnsemd

// --------------------------------------------------------------------------
// nnsemd_solve_small_noalloc: one small pair solved by the one-CTA solver
// without any memory allocation.
//
// Some callers cannot call cudaMalloc: a plugin that runs inside another
// framework's launch callback, where allocating is not allowed; a process
// whose device memory is already claimed in full by a caching allocator; a
// latency-critical path that cannot afford cudaMalloc's implicit device
// synchronisation.  For them this entry point keeps its few words of scratch
// (error bits and round counters) in a file-scope __device__ array that is
// part of the loaded module, so a call allocates nothing.  Everything else
// lives in the CTA's shared memory, as in the batched kernel above.
//
// Every GPU that loads the library holds this array until the process exits.
// All calls share it and it keeps the last call's contents; the kernel clears
// it itself before use.  Calls that overlap on the GPU (different streams, or
// several host threads) race on it: serialise them.
// --------------------------------------------------------------------------

#include <mutex>

#include "nnsemd.h"

namespace nnsemd {

struct NoAllocScratch {
  unsigned err;          // ErrFlag bits of the last call
  unsigned pad;
  long long rounds;      // rounds of the last call
  long long pair_evals;  // sum of m_t * n_t of the last call
};

constexpr size_t NOALLOC_SCRATCH_BYTES = 256;
static_assert(sizeof(NoAllocScratch) <= NOALLOC_SCRATCH_BYTES, "scratch too small");
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

template <int D, int DP, bool L1>
__global__ void __launch_bounds__(FIN_THREADS, 1)
    k_small_noalloc(const float* x, const double* a, int m, const float* y, const double* b, int n, int d,
                    int metric, double* cost_out, NoAllocScratch* scr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LowdSmem<D, DP, L1>& L = *reinterpret_cast<LowdSmem<D, DP, L1>*>(smem_raw);
  const int tid = threadIdx.x;
  if (tid == 0) {
    scr->err = 0;
    scr->rounds = 0;
    scr->pair_evals = 0;
  }
  __syncthreads();
  double cost = 0.0;
  long long rounds = 0, pe = 0;
  const bool ok = cta_solve_pair(L.S, L.G, L.G.xs, L.G.ys, x, a, m, y, b, n, d, metric, &scr->err, cost, rounds, pe);
  if (tid == 0) {
    *cost_out = ok ? cost : CUDART_NAN;
    scr->rounds = rounds;
    scr->pair_evals = pe;
  }
}

template <int D, int DP, bool L1>
static cudaError_t small_noalloc_t(const float* x, const double* a, int m, const float* y, const double* b, int n,
                                   int metric, double* cost_out, NoAllocScratch* scr, cudaStream_t st) {
  k_small_noalloc<D, DP, L1><<<1, FIN_THREADS, sizeof(LowdSmem<D, DP, L1>), st>>>(x, a, m, y, b, n, D, metric,
                                                                                 cost_out, scr);
  return cudaGetLastError();
}

template <int D, int DP>
static cudaError_t noalloc_allow_smem() {
  cudaError_t e = cudaFuncSetAttribute(k_small_noalloc<D, DP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(LowdSmem<D, DP, false>));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_small_noalloc<D, DP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(LowdSmem<D, DP, true>));
  return e;
}

// One-time set-up per device, with that device current: the device address
// of the scratch array (in host code the array's name is only a stand-in)
// and the shared-memory limit of every instantiation of the kernel.
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[256];

static cudaError_t noalloc_setup(int device, NoAllocScratch** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (device < 0 || device >= 256) return cudaErrorInvalidDevice;
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e == cudaSuccess) e = noalloc_allow_smem<1, 2>();
    if (e == cudaSuccess) e = noalloc_allow_smem<2, 2>();
    if (e == cudaSuccess) e = noalloc_allow_smem<3, 4>();
    if (e == cudaSuccess) e = noalloc_allow_smem<4, 4>();
    if (e == cudaSuccess) e = noalloc_allow_smem<5, 8>();
    if (e == cudaSuccess) e = noalloc_allow_smem<6, 8>();
    if (e == cudaSuccess) e = noalloc_allow_smem<7, 8>();
    if (e == cudaSuccess) e = noalloc_allow_smem<8, 8>();
    if (e != cudaSuccess) return e;
    g_noalloc_addr[device] = p;
  }
  *out = static_cast<NoAllocScratch*>(g_noalloc_addr[device]);
  return cudaSuccess;
}

}  // namespace nnsemd

extern "C" int nnsemd_solve_small_noalloc(const float* x, const double* a, int64_t m, const float* y,
                                          const double* b, int64_t n, int32_t d, int32_t metric, double* cost_out,
                                          void* stream) {
  using namespace nnsemd;
  if (!x || !a || !y || !b || !cost_out) return NNSEMD_ERR_INVALID_ARG;
  if (m < 1 || n < 1 || d < 1 || metric < 0 || metric > 2) return NNSEMD_ERR_INVALID_ARG;
  if (m > NNSEMD_NOALLOC_MAX_POINTS || n > NNSEMD_NOALLOC_MAX_POINTS || d > NNSEMD_NOALLOC_MAX_D)
    return NNSEMD_ERR_UNSUPPORTED;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return NNSEMD_ERR_CUDA;
  NoAllocScratch* scr = nullptr;
  if (noalloc_setup(device, &scr) != cudaSuccess) return NNSEMD_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const bool l1 = metric == METRIC_L1;
  const int mi = (int)m, ni = (int)n;
  cudaError_t e;
#define NOALLOC_CASE(DD, DPP)                                                                              \
  case DD:                                                                                                 \
    e = l1 ? small_noalloc_t<DD, DPP, true>(x, a, mi, y, b, ni, metric, cost_out, scr, st)                 \
           : small_noalloc_t<DD, DPP, false>(x, a, mi, y, b, ni, metric, cost_out, scr, st);               \
    break;
  switch (d) {
    NOALLOC_CASE(1, 2) NOALLOC_CASE(2, 2) NOALLOC_CASE(3, 4) NOALLOC_CASE(4, 4)
    NOALLOC_CASE(5, 8) NOALLOC_CASE(6, 8) NOALLOC_CASE(7, 8) NOALLOC_CASE(8, 8)
    default: return NNSEMD_ERR_UNSUPPORTED;
  }
#undef NOALLOC_CASE
  if (e != cudaSuccess) return NNSEMD_ERR_CUDA;
  NoAllocScratch h{};
  if (cudaMemcpyAsync(&h, scr, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return NNSEMD_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return NNSEMD_ERR_CUDA;
  if (h.err & EF_NONFINITE) return NNSEMD_ERR_NONFINITE;
  if (h.err & (EF_ZERO_MASS | EF_NEGATIVE)) return NNSEMD_ERR_ZERO_MASS;
  if (h.err & EF_ITER) return NNSEMD_ERR_ITER_LIMIT;
  if (h.err) return NNSEMD_ERR_CUDA;
  return NNSEMD_OK;
}
