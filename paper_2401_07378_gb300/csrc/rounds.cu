// Round kernels of a multi-CTA NNS-EMD solve (sm_103a), one per step of
// Alg. 1 (Sec. III-A) after the NNS operation:
//
//   k_group_count / k_group_alloc / k_group_scatter
//       a_i^(t): bucket the active consumers by the supplier they picked,
//       with one 64-bit member key (key32 bits << 32 | consumer position)
//       per consumer, so that sorting a group orders it by distance and
//       then by consumer index (the greedy protocol's order).
//   k_flow (groups of <= 32: one thread or one warp each; longer: one CTA)
//       sort each group (in one thread's registers for groups of at most 8,
//       a warp-register bitonic network up to 32, a CTA network in shared or
//       global memory beyond that), then walk it in FP64 exactly as the
//       algorithm does: f = min(s_i, c_j),
//       s_i -= f, c_j -= f, until s_i is spent; each flow records its
//       original (i, j) and f.
//   k_final_sums
//       after the last round: the cost term f * D_ij (FP64 ground distance)
//       and plan entry of every recorded flow, R and the leftover mass.
//   k_compact_count / k_compact_scatter
//       weights update: stable compaction of both active lists to the points
//       whose residual is still positive, gathering their coordinates into
//       the other half of a double buffer.
//   k_xs_* exact sums (normalisation totals, R, leftover mass).
#include <math_constants.h>

#include "common.cuh"
#include "kernels.h"

namespace nnsemd {

// --------------------------------------------------------------------------
// exact sums
// --------------------------------------------------------------------------

// Up to three exact sums in one launch: job j adds v_j[0..n_j) (n_j from
// n_dev when given) into acc_j.  The jobs' index ranges are concatenated
// and split over the grid; each warp adds into its own shared-memory copy of
// the accumulators (the values of a job often share an exponent, so the
// limbs they touch are the same: 32 lanes contend per copy instead of the
// whole block), and the block adds the per-warp sums into global memory.
struct XsJob {
  const double* v;
  int64_t n;
  const unsigned long long* n_dev;
  unsigned long long* acc;
};
constexpr int XS_THREADS = 256;

__global__ void __launch_bounds__(XS_THREADS) k_xs_accum_multi(XsJob j0, XsJob j1, XsJob j2, int njobs,
                                                               unsigned* err, int check) {
  constexpr int NW = XS_THREADS / 32;
  __shared__ unsigned long long sacc[3][NW][XS_LIMBS];
  for (int i = threadIdx.x; i < 3 * NW * XS_LIMBS; i += blockDim.x) (&sacc[0][0][0])[i] = 0ULL;
  __syncthreads();
  const int64_t n0 = j0.n_dev ? (int64_t)*j0.n_dev : j0.n;
  const int64_t n1 = njobs > 1 ? (j1.n_dev ? (int64_t)*j1.n_dev : j1.n) : 0;
  const int64_t n2 = njobs > 2 ? (j2.n_dev ? (int64_t)*j2.n_dev : j2.n) : 0;
  const int64_t e1 = n0, e2 = n0 + n1, e3 = n0 + n1 + n2;
  const int w = threadIdx.x >> 5;
  // whole warps per step (xs_add_warp): a lane past the end adds nothing
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < e3; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    int j = -1;
    double v = 0.0;
    if (i < e3) {
      j = i < e1 ? 0 : (i < e2 ? 1 : 2);
      v = j == 0 ? j0.v[i] : (j == 1 ? j1.v[i - e1] : j2.v[i - e2]);
      if (check && !isfinite(v)) {
        atomicOr(err, EF_NONFINITE);
        v = 0.0;
      } else if (check && v < 0.0) {
        atomicOr(err, EF_NEGATIVE);
        v = 0.0;
      }
    }
    for (int jj = 0; jj < njobs; ++jj)
      if (__any_sync(0xffffffffu, j == jj)) xs_add_warp(sacc[jj][w], j == jj ? v : 0.0);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < njobs * XS_LIMBS; i += blockDim.x) {
    const int j = i / XS_LIMBS, L = i - j * XS_LIMBS;
    unsigned long long t = 0;
#pragma unroll
    for (int u = 0; u < NW; ++u) t += sacc[j][u][L];
    if (t) atomicAdd((j == 0 ? j0.acc : (j == 1 ? j1.acc : j2.acc)) + L, t);
  }
}

// The end of a solve in one pass: the leftover mass (residuals s[0..m) and
// c[0..n)) into acc_left, and, for every recorded flow k < nnz, its cost
// term f * D_ij (FP64 ground distance from the original coordinates) into
// acc_cost and its plan entry (when a plan is requested).  The flows of all
// rounds are costed here at once, with every lane busy, instead of inside
// the latency-bound flow steps.
struct FinalArgs {
  const double* s;
  int64_t m;
  const double* c;
  int64_t n;
  const int32_t* fl_i;
  const int32_t* fl_j;
  const double* fl_f;
  const unsigned long long* nnz;
  const float* x;
  const float* y;
  int d, metric;
  int32_t* plan_i;  // nullable
  int32_t* plan_j;
  double* plan_f;
  long long plan_cap;
  unsigned long long* acc_left;
  unsigned long long* acc_cost;
  unsigned* err;
};

__global__ void __launch_bounds__(XS_THREADS) k_final_sums(FinalArgs A) {
  constexpr int NW = XS_THREADS / 32;
  __shared__ unsigned long long sacc[2][NW][XS_LIMBS];
  for (int i = threadIdx.x; i < 2 * NW * XS_LIMBS; i += blockDim.x) (&sacc[0][0][0])[i] = 0ULL;
  __syncthreads();
  const int64_t e1 = A.m, e2 = A.m + A.n, e3 = e2 + (int64_t)*A.nnz;
  const int w = threadIdx.x >> 5;
  bool over = false;
  // whole warps per step (xs_add_warp): a lane past the end adds nothing
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < e3; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    double left = 0.0, term = 0.0;
    if (i < e2) {
      left = i < e1 ? A.s[i] : A.c[i - e1];
    } else if (i < e3) {
      const int64_t k = i - e2;
      const int fi = A.fl_i[k], fj = A.fl_j[k];
      const double f = A.fl_f[k];
      term = __dmul_rn(f, cost_dist64(A.x + (size_t)fi * A.d, A.y + (size_t)fj * A.d, A.d, A.metric));
      if (A.plan_i) {
        if (k < A.plan_cap) {
          A.plan_i[k] = fi;
          A.plan_j[k] = fj;
          A.plan_f[k] = f;
        } else {
          over = true;
        }
      }
    }
    if (__any_sync(0xffffffffu, i < e2)) xs_add_warp(sacc[0][w], left);
    if (__any_sync(0xffffffffu, i >= e2 && i < e3)) xs_add_warp(sacc[1][w], term);
  }
  if (over) atomicOr(A.err, EF_CAPACITY);
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * XS_LIMBS; i += blockDim.x) {
    const int j = i / XS_LIMBS, L = i - j * XS_LIMBS;
    unsigned long long t = 0;
#pragma unroll
    for (int u = 0; u < NW; ++u) t += sacc[j][u][L];
    if (t) atomicAdd((j == 0 ? A.acc_left : A.acc_cost) + L, t);
  }
}

// out0 / out1 = the correctly rounded values of acc0 / acc1.
__global__ void k_xs_round2(unsigned long long* acc0, double* out0, unsigned long long* acc1, double* out1) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *out0 = xs_round(acc0);
  if (blockIdx.x == 0 && threadIdx.x == 32 && acc1) *out1 = xs_round(acc1);
}

// Both sides' normalisation in one launch: blocks [0, ga) take (w0, n0, acc0),
// the others (w1, n1, acc1); each block rounds its side's total itself.
__global__ void k_normalise2(const double* __restrict__ w0, int64_t n0, const unsigned long long* __restrict__ acc0,
                             double* total0, double* __restrict__ out0, const double* __restrict__ w1, int64_t n1,
                             const unsigned long long* __restrict__ acc1, double* total1, double* __restrict__ out1,
                             int ga, unsigned* err) {
  __shared__ unsigned long long a[XS_LIMBS];
  __shared__ double total;
  const bool second = (int)blockIdx.x >= ga;
  const unsigned long long* acc = second ? acc1 : acc0;
  const int bid = second ? blockIdx.x - ga : blockIdx.x, nb = second ? gridDim.x - ga : ga;
  for (int i = threadIdx.x; i < XS_LIMBS; i += blockDim.x) a[i] = acc[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    total = xs_round(a);
    if (bid == 0) {
      *(second ? total1 : total0) = total;
      if (!(total > 0.0)) atomicOr(err, EF_ZERO_MASS);
    }
  }
  __syncthreads();
  const double t = total;
  const double* w = second ? w1 : w0;
  double* out = second ? out1 : out0;
  const int64_t n = second ? n1 : n0;
  for (int64_t i = bid * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)nb * blockDim.x) {
    const double wi = w[i];
    out[i] = (t > 0.0 && isfinite(wi) && wi > 0.0) ? __ddiv_rn(wi, t) : 0.0;
  }
}

static int xs_grid(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > num_sms() * 4) g = num_sms() * 4;
  return (int)(g < 1 ? 1 : g);
}

void launch_setup_sums(const SolveBufs& B, const double* a, const double* b, cudaStream_t st) {
  XsJob ja{a, B.m, nullptr, B.xs_acc}, jb{b, B.n, nullptr, B.xs_acc + XS_LIMBS};
  k_xs_accum_multi<<<xs_grid(B.m + B.n), XS_THREADS, 0, st>>>(ja, jb, jb, 2, &B.st->err, 1);
  const int ga = xs_grid(B.m), gb = xs_grid(B.n);
  k_normalise2<<<ga + gb, 256, 0, st>>>(a, B.m, B.xs_acc, &B.st->total_a, B.s, b, B.n, B.xs_acc + XS_LIMBS,
                                        &B.st->total_b, B.c, ga, &B.st->err);
}

// The leftover mass (residuals of both sides), the cost terms and plan
// entries of every recorded flow, and R (their exact sum) in two launches;
// the accumulators were cleared with the others when the solve started.
void launch_leftover(const SolveBufs& B, cudaStream_t st) {
  unsigned long long* acc = B.xs_acc + 3 * XS_LIMBS;
  unsigned long long* cacc = B.xs_acc + 2 * XS_LIMBS;
  FinalArgs F{B.s,    B.m,    B.c,    B.n,      B.fl_i,   B.fl_j,   B.fl_f,        &B.st->nnz, B.x, B.y,
              B.d,    B.metric, B.plan_i, B.plan_j, B.plan_f, (long long)B.plan_cap, acc, cacc, &B.st->err};
  k_final_sums<<<num_sms() * 2, XS_THREADS, 0, st>>>(F);
  k_xs_round2<<<1, 64, 0, st>>>(acc, &B.st->leftover, cacc, &B.st->cost);
}

// --------------------------------------------------------------------------
// compaction (initial packing and the weights update of every round)
// --------------------------------------------------------------------------

constexpr int CP_THREADS = 256;
constexpr int CP_ITEMS = 4;
constexpr int CP_BLOCK = CP_THREADS * CP_ITEMS;

struct CompactSide {
  const float* pts_in;  // input coordinates, in_stride floats per point
  int in_stride;
  const int* idx_in;    // original index of each input point (nullptr: identity)
  const double* resid;  // residual weight by original index
  float* pts_out;       // packed output, DP floats per point
  int* idx_out;
  int count;            // input points
  int* count_out;       // survivors
  int nblocks;
  int check;            // check coordinates for finiteness
  unsigned long long* key_reset;  // nullable: set key_reset[survivor position] = ~0 (next NNS's argmin keys)
};

struct CompactArgs {
  CompactSide side[2];
  int* blockcounts;     // [side0 blocks + side1 blocks]
  unsigned* err;
  volatile int* notify; // nullable: {seq, side0 count, side1 count, error bits} in mapped host memory
  int notify_seq;
  unsigned* ticket;     // zero before the count launch; the last block resets it
};

NNS_DEV int cp_block_side(const CompactArgs& A, int b, int& local) {
  if (b < A.side[0].nblocks) { local = b; return 0; }
  local = b - A.side[0].nblocks;
  return 1;
}

__global__ void __launch_bounds__(CP_THREADS) k_compact_count(CompactArgs A) {
  int lb;
  const int sd = cp_block_side(A, blockIdx.x, lb);
  const CompactSide& S = A.side[sd];
  int c = 0;
  bool bad = false;
  const int base = lb * CP_BLOCK + threadIdx.x * CP_ITEMS;
#pragma unroll
  for (int k = 0; k < CP_ITEMS; ++k) {
    const int pos = base + k;
    if (pos < S.count) {
      const int orig = S.idx_in ? S.idx_in[pos] : pos;
      c += S.resid[orig] > 0.0;
      // with `check`, every point's coordinates are checked here (zero
      // weight or not), so that the early notification carries the error
      if (S.check && S.pts_in)
        for (int e = 0; e < S.in_stride; ++e) bad |= !isfinite(S.pts_in[(size_t)pos * S.in_stride + e]);
    }
  }
  // (thread 0 raises the flag, before its fence and ticket below)
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(A.err, EF_NONFINITE);
  // block reduction
  __shared__ int red[CP_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < CP_THREADS / 32; ++w) t += red[w];
    A.blockcounts[blockIdx.x] = t;
  }
  if (!A.notify) return;
  // The last block to finish adds up both sides' counts and publishes them
  // with the error bits (every block fenced its count before its ticket).
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(A.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x >= 32) return;
  __threadfence();
  const volatile int* bc = A.blockcounts;
  const int nb0 = A.side[0].nblocks, nb = nb0 + A.side[1].nblocks;
  int t0 = 0, t1 = 0;
  for (int b = threadIdx.x; b < nb; b += 32) (b < nb0 ? t0 : t1) += bc[b];
  for (int o = 16; o > 0; o >>= 1) {
    t0 += __shfl_xor_sync(0xffffffffu, t0, o);
    t1 += __shfl_xor_sync(0xffffffffu, t1, o);
  }
  if (threadIdx.x == 0) {
    A.notify[1] = t0;
    A.notify[2] = t1;
    A.notify[3] = (int)*(volatile unsigned*)A.err;
    __threadfence_system();
    A.notify[0] = A.notify_seq;
    *A.ticket = 0u;
  }
}

template <int DP>
__global__ void __launch_bounds__(CP_THREADS) k_compact_scatter(CompactArgs A) {
  int lb;
  const int sd = cp_block_side(A, blockIdx.x, lb);
  const CompactSide& S = A.side[sd];
  const int first = sd == 0 ? 0 : A.side[0].nblocks;
  __shared__ int s_off;
  __shared__ int wsum[CP_THREADS / 32 + 1];
  if (threadIdx.x == 0) {
    int o = 0;
    for (int b = first; b < first + lb; ++b) o += A.blockcounts[b];
    s_off = o;
  }
  // flags of this thread's items
  int flags[CP_ITEMS];
  int origs[CP_ITEMS];
  int mine = 0;
  const int base = lb * CP_BLOCK + threadIdx.x * CP_ITEMS;
#pragma unroll
  for (int k = 0; k < CP_ITEMS; ++k) {
    const int pos = base + k;
    flags[k] = 0;
    origs[k] = 0;
    if (pos < S.count) {
      const int orig = S.idx_in ? S.idx_in[pos] : pos;
      origs[k] = orig;
      flags[k] = S.resid[orig] > 0.0;
    }
    mine += flags[k];
  }
  // block exclusive scan of per-thread counts
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = mine;
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int i = 0; i < CP_THREADS / 32; ++i) {
      int t = wsum[i];
      wsum[i] = run;
      run += t;
    }
    wsum[CP_THREADS / 32] = run;
  }
  __syncthreads();
  int pos_out = s_off + wsum[w] + x - mine;
  bool bad = false;
#pragma unroll
  for (int k = 0; k < CP_ITEMS; ++k) {
    if (!flags[k]) continue;
    const int pos = base + k;
    if (S.key_reset) S.key_reset[pos_out] = ~0ULL;
    if (!S.pts_in) {  // index-only list (d > 8: coordinates stay in place)
      S.idx_out[pos_out++] = origs[k];
      continue;
    }
    float v[DP];
#pragma unroll
    for (int e = 0; e < DP; ++e) {
      float t = e < S.in_stride ? S.pts_in[(size_t)pos * S.in_stride + e] : 0.f;
      if (S.check && !isfinite(t)) bad = true;
      v[e] = t;
    }
    if (DP == 2) {
      reinterpret_cast<float2*>(S.pts_out)[pos_out] = make_float2(v[0], v[1]);
    } else {
#pragma unroll
      for (int e = 0; e < DP; e += 4)
        reinterpret_cast<float4*>(S.pts_out + (size_t)pos_out * DP)[e / 4] = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
    }
    S.idx_out[pos_out] = origs[k];
    ++pos_out;
  }
  if (bad) atomicOr(A.err, EF_NONFINITE);
  // the last block of a side publishes the count and NaN-pads the tail
  if (lb == S.nblocks - 1) {
    const int total = s_off + wsum[CP_THREADS / 32];
    if (threadIdx.x == 0) *S.count_out = total;
    const int padded = S.pts_out ? (int)pad_points(total) : 0;
    for (int p = total + threadIdx.x; p < padded; p += CP_THREADS)
#pragma unroll
      for (int e = 0; e < DP; ++e) S.pts_out[(size_t)p * DP + e] = CUDART_NAN_F;
  }
}

static void compact_launch(CompactArgs& A, int dp, cudaStream_t st) {
  for (int s = 0; s < 2; ++s) A.side[s].nblocks = (A.side[s].count + CP_BLOCK - 1) / CP_BLOCK;
  const int nb = A.side[0].nblocks + A.side[1].nblocks;
  if (nb == 0) return;
  k_compact_count<<<nb, CP_THREADS, 0, st>>>(A);
  if (dp == 2) k_compact_scatter<2><<<nb, CP_THREADS, 0, st>>>(A);
  else if (dp == 4) k_compact_scatter<4><<<nb, CP_THREADS, 0, st>>>(A);
  else k_compact_scatter<8><<<nb, CP_THREADS, 0, st>>>(A);
}

__global__ void k_check_finite(const float* __restrict__ v, int64_t count, unsigned* err) {
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(v[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, EF_NONFINITE);
}

void launch_check_finite(const float* v, int64_t count, unsigned* err, cudaStream_t st) {
  int64_t g = (count + 1023) / 1024;
  if (g > num_sms() * 8) g = num_sms() * 8;
  k_check_finite<<<(int)(g < 1 ? 1 : g), 256, 0, st>>>(v, count, err);
}

int launch_initial_pack(SolveBufs& B, cudaStream_t st) {
  CompactArgs A{};
  const bool packed = B.dp > 0;  // d > 8 keeps index-only active lists
  if (!packed) {
    launch_check_finite(B.x, B.m * B.d, &B.st->err, st);
    launch_check_finite(B.y, B.n * B.d, &B.st->err, st);
  }
  A.side[0] = CompactSide{packed ? B.x : nullptr, B.d, nullptr, B.s, packed ? B.xa[B.cur] : nullptr, B.ia[B.cur],
                          (int)B.m, &B.st->mt, 0, 1};
  A.side[1] = CompactSide{packed ? B.y : nullptr, B.d, nullptr, B.c, packed ? B.ya[B.cur] : nullptr, B.ja[B.cur],
                          (int)B.n, &B.st->nt, 0, 1, B.nnkey};
  A.blockcounts = B.blockcounts;
  A.notify = B.notify;
  A.notify_seq = B.notify_seq;
  A.ticket = &B.st->ticket;
  A.err = &B.st->err;
  compact_launch(A, B.dp, st);
  return 0;
}

// --------------------------------------------------------------------------
// grouping
// --------------------------------------------------------------------------

__global__ void k_group_count(const unsigned long long* __restrict__ nnkey, int nt, int mt, int* __restrict__ cnt,
                              unsigned* err, DevState* st) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q == 0) {  // this round's group lists start empty (read from k_group_alloc on)
    st->nseg = 0;
    st->nbig = 0;
    st->nmed = 0;
    st->seg_cursor = 0;
  }
  if (q >= nt) return;
  const unsigned p = (unsigned)(nnkey[q] & 0xffffffffULL);
  if (p >= (unsigned)mt) { atomicOr(err, EF_INTERNAL); return; }
  atomicAdd(cnt + p, 1);
}

// Groups of at most FLOW_THREAD_MAX consumers are served by one thread each:
// the greedy walk is a chain of dependent FP64 operations, and a lane-level
// chain costs the FP64 pipe one instruction per 32 groups instead of one per
// group.
constexpr int FLOW_THREAD_MAX = 8;

__global__ void k_group_alloc(const int* __restrict__ cnt, int mt, int2* __restrict__ seg, int* __restrict__ seglist,
                              int* __restrict__ biglist, int* __restrict__ medlist, DevState* st) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int L = p < mt ? cnt[p] : 0;
  int x = L;
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  unsigned base = 0;
  if (lane == 31 && x) base = atomicAdd(&st->seg_cursor, (unsigned)x);
  base = __shfl_sync(0xffffffffu, base, 31);
  const unsigned lt = (1u << lane) - 1u;
  const unsigned ne = __ballot_sync(0xffffffffu, L > 0);
  unsigned sb = 0;
  if (lane == 0 && ne) sb = atomicAdd((unsigned*)&st->nseg, (unsigned)__popc(ne));
  sb = __shfl_sync(0xffffffffu, sb, 0);
  const unsigned big = __ballot_sync(0xffffffffu, L > 32);
  unsigned bb = 0;
  if (lane == 0 && big) bb = atomicAdd((unsigned*)&st->nbig, (unsigned)__popc(big));
  bb = __shfl_sync(0xffffffffu, bb, 0);
  const unsigned med = __ballot_sync(0xffffffffu, L > FLOW_THREAD_MAX && L <= 32);
  unsigned mb = 0;
  if (lane == 0 && med) mb = atomicAdd((unsigned*)&st->nmed, (unsigned)__popc(med));
  mb = __shfl_sync(0xffffffffu, mb, 0);
  if (p < mt) {
    seg[p] = make_int2((int)(base + x - L), L);
    if (L > 0) seglist[sb + __popc(ne & lt)] = p;
    if (L > 32) biglist[bb + __popc(big & lt)] = p;
    if (L > FLOW_THREAD_MAX && L <= 32) medlist[mb + __popc(med & lt)] = p;
  }
}

// Member key: the serving order (greedy: the distance key bits; random:
// the round's SplitMix64 key of the consumer) << 32 | consumer position.
__global__ void k_group_scatter(const unsigned long long* __restrict__ nnkey, int nt, int* __restrict__ cnt,
                                const int2* __restrict__ seg, unsigned long long* __restrict__ member,
                                const int* __restrict__ ja, int protocol, unsigned long long seed, long long round) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nt) return;
  const unsigned long long key = nnkey[q];
  const int p = (int)(key & 0xffffffffULL);
  const int slot = seg[p].x + atomicSub(cnt + p, 1) - 1;
  const unsigned long long order =
      protocol == 1 ? ((unsigned long long)rp_key32(seed, round, ja[q]) << 32) : (key & 0xffffffff00000000ULL);
  member[slot] = order | (unsigned)q;
}

// --------------------------------------------------------------------------
// greedy flow
// --------------------------------------------------------------------------

struct FlowArgs {
  const int* ia;   // current active lists
  const int* ja;
  const int2* seg;
  const int* seglist;
  const int* biglist;
  const int* medlist;
  unsigned long long* member;
  double* s;
  double* c;
  // flow record, slot = running flow count (original i, j and f); the cost
  // terms and plan entries of all flows are made in one pass after the
  // last round (k_final_sums)
  int32_t* fl_i;
  int32_t* fl_j;
  double* fl_f;
  DevState* st;
};

// Warp-wide ascending sort of one 64-bit key per lane (bitonic network in
// which every comparator puts the smaller key on the lower lane).
NNS_DEV unsigned long long warp_sort_u64(unsigned long long key) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
    {
      const int partner = lane ^ (k - 1);
      const unsigned long long o = __shfl_sync(0xffffffffu, key, partner);
      key = lane < partner ? (o < key ? o : key) : (o > key ? o : key);
    }
#pragma unroll
    for (int j = k >> 2; j > 0; j >>= 1) {
      const int partner = lane ^ j;
      const unsigned long long o = __shfl_sync(0xffffffffu, key, partner);
      key = lane < partner ? (o < key ? o : key) : (o > key ? o : key);
    }
  }
  return key;
}

// Serve up to 32 sorted members (one per lane, `cnt` valid) from supplier i
// whose residual is `s` (uniform).  Returns how many were served.
NNS_DEV int warp_serve(const FlowArgs& A, int i, double& s, unsigned long long key, int cnt) {
  const int lane = threadIdx.x & 31;
  int j = 0;
  double c = 0.0;
  if (lane < cnt) {
    const int q = (int)(key & 0xffffffffULL);
    j = A.ja[q];
    c = A.c[j];
  }
  double myf = 0.0, mycn = 0.0;
  int served = 0;
  for (int l = 0; l < cnt; ++l) {
    if (!residual_positive(s)) break;
    double cl = __shfl_sync(0xffffffffu, c, l);
    const double f = greedy_step(s, cl);
    if (lane == l) {
      myf = f;
      mycn = cl;
    }
    served = l + 1;
  }
  unsigned long long base = 0;
  if (lane == 0 && served) base = atomicAdd(&A.st->nnz, (unsigned long long)served);
  base = __shfl_sync(0xffffffffu, base, 0);
  if (lane < served) {
    A.c[j] = mycn;
    const unsigned long long slot = base + lane;
    A.fl_i[slot] = i;
    A.fl_j[slot] = j;
    A.fl_f[slot] = myf;
  }
  return served;
}

// One thread: sort the group's keys (distance bits, position) ascending in
// registers, walk them with the supplier's residual, write the flows.
NNS_DEV void thread_serve(const FlowArgs& A, int p, int2 sg, bool active) {
  const int lane = threadIdx.x & 31;
  unsigned long long key[FLOW_THREAD_MAX];
#pragma unroll
  for (int k = 0; k < FLOW_THREAD_MAX; ++k) key[k] = (active && k < sg.y) ? A.member[sg.x + k] : ~0ULL;
  // insertion network over the fixed-size array (padding ~0 stays last)
#pragma unroll
  for (int a = 1; a < FLOW_THREAD_MAX; ++a)
#pragma unroll
    for (int b = a; b > 0; --b) {
      const unsigned long long lo = key[b - 1], hi = key[b];
      key[b - 1] = lo < hi ? lo : hi;
      key[b] = lo < hi ? hi : lo;
    }
  int i = 0;
  double s = 0.0;
  int jv[FLOW_THREAD_MAX];
  double cv[FLOW_THREAD_MAX];
  if (active) {
    i = A.ia[p];
    s = A.s[i];
  }
#pragma unroll
  for (int k = 0; k < FLOW_THREAD_MAX; ++k) {
    jv[k] = 0;
    cv[k] = 0.0;
    if (active && k < sg.y) {
      jv[k] = A.ja[(int)(key[k] & 0xffffffffULL)];
      cv[k] = A.c[jv[k]];
    }
  }
  double fv[FLOW_THREAD_MAX];
  int served = 0;
  bool live = active;
#pragma unroll
  for (int k = 0; k < FLOW_THREAD_MAX; ++k) {
    fv[k] = 0.0;
    if (live && k < sg.y) {
      if (!residual_positive(s)) {
        live = false;
      } else {
        fv[k] = greedy_step(s, cv[k]);
        served = k + 1;
      }
    }
  }
  // plan slots: one atomic per warp
  int incl = served;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  unsigned long long base = 0;
  if (lane == 31 && incl) base = atomicAdd(&A.st->nnz, (unsigned long long)incl);
  base = __shfl_sync(0xffffffffu, base, 31) + (unsigned long long)(incl - served);
  if (!active) return;
#pragma unroll
  for (int k = 0; k < FLOW_THREAD_MAX; ++k) {
    if (k < served) {
      const int j = jv[k];
      A.c[j] = cv[k];
      const unsigned long long slot = base + k;
      A.fl_i[slot] = i;
      A.fl_j[slot] = j;
      A.fl_f[slot] = fv[k];
    }
  }
  A.s[i] = s;
}

// Groups of at most 32 consumers.  Each warp takes 32 groups of the group
// list at a time and serves those of at most FLOW_THREAD_MAX one per lane;
// then the warps serve the groups of 9..32 one per warp.
NNS_DEV void flow_small_blocks(const FlowArgs& A, int bid, int nblocks) {
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int warp = bid * wpb + (threadIdx.x >> 5), nwarps = nblocks * wpb;
  const int nseg = A.st->nseg;
  for (int w0 = warp * 32; w0 < nseg; w0 += nwarps * 32) {
    const int w = w0 + lane;
    int p = -1;
    int2 sg = make_int2(0, 0);
    if (w < nseg) {
      p = A.seglist[w];
      sg = A.seg[p];
    }
    thread_serve(A, p, sg, p >= 0 && sg.y <= FLOW_THREAD_MAX);
  }
  const int nmed = A.st->nmed;
  for (int w = warp; w < nmed; w += nwarps) {
    const int p = A.medlist[w];
    const int2 sg = A.seg[p];
    unsigned long long key = lane < sg.y ? A.member[sg.x + lane] : ~0ULL;
    key = warp_sort_u64(key);
    const int i = A.ia[p];
    double s = A.s[i];
    warp_serve(A, i, s, key, sg.y);
    if (lane == 0) A.s[i] = s;
  }
}

constexpr int BIG_THREADS = 256;
constexpr int BIG_SMEM_KEYS = 4096;

// Ascending bitonic sort of a[0..L) in place (virtual +inf padding up to a
// power of two; every comparator puts the smaller key at the lower index,
// so padding never moves).  All threads of the block call this.
template <typename Ptr>
NNS_DEV void block_sort_u64(Ptr a, int L) {
  int N = 1;
  while (N < L) N <<= 1;
  for (int k = 2; k <= N; k <<= 1) {
    for (int idx = threadIdx.x; idx < N / 2; idx += blockDim.x) {
      const int h = k >> 1;
      const int i = (idx / h) * k + (idx % h);
      const int pr = i ^ (k - 1);
      if (pr < L) {
        const unsigned long long u = a[i], v = a[pr];
        if (v < u) { a[i] = v; a[pr] = u; }
      }
    }
    __syncthreads();
    for (int j = k >> 2; j > 0; j >>= 1) {
      for (int idx = threadIdx.x; idx < N / 2; idx += blockDim.x) {
        const int i = (idx / j) * (2 * j) + (idx % j);
        const int pr = i + j;
        if (pr < L) {
          const unsigned long long u = a[i], v = a[pr];
          if (v < u) { a[i] = v; a[pr] = u; }
        }
      }
      __syncthreads();
    }
  }
}

NNS_DEV void flow_big_blocks(const FlowArgs& A, unsigned long long* keys, int bid, int nblocks) {
  const int nbig = A.st->nbig;
  for (int b = bid; b < nbig; b += nblocks) {
    const int p = A.biglist[b];
    const int2 sg = A.seg[p];
    const int L = sg.y;
    unsigned long long* g = A.member + sg.x;
    const bool in_smem = L <= BIG_SMEM_KEYS;
    if (in_smem) {
      for (int r = threadIdx.x; r < L; r += blockDim.x) keys[r] = g[r];
      __syncthreads();
      block_sort_u64(keys, L);
    } else {
      block_sort_u64(g, L);
    }
    if (threadIdx.x < 32) {
      const int i = A.ia[p];
      double s = A.s[i];
      for (int base = 0; base < L && s > 0.0; base += 32) {
        const int cntc = min(32, L - base);
        const unsigned long long key =
            (int)threadIdx.x < cntc ? (in_smem ? keys[base + threadIdx.x] : g[base + threadIdx.x]) : ~0ULL;
        const int served = warp_serve(A, i, s, key, cntc);
        if (served < cntc) break;
      }
      if (threadIdx.x == 0) A.s[i] = s;
    }
    __syncthreads();
  }
}

// The flow step of a multi-CTA round in one launch: the first `nsmall`
// blocks serve the groups of at most 32 consumers, the others the longer
// groups (one block per group, keys sorted in shared memory).
__global__ void __launch_bounds__(BIG_THREADS) k_flow(FlowArgs A, int nsmall) {
  __shared__ unsigned long long keys[BIG_SMEM_KEYS];
  if ((int)blockIdx.x < nsmall) flow_small_blocks(A, blockIdx.x, nsmall);
  else flow_big_blocks(A, keys, blockIdx.x - nsmall, gridDim.x - nsmall);
}

// --------------------------------------------------------------------------
// one multi-CTA round (the NNS operation is launched by the caller)
// --------------------------------------------------------------------------

int launch_big_round(SolveBufs& B, int mt, int nt, long long round, cudaStream_t st) {
  const int cur = B.cur;
  k_group_count<<<(nt + 255) / 256, 256, 0, st>>>(B.nnkey, nt, mt, B.cnt, &B.st->err, B.st);
  k_group_alloc<<<(mt + 255) / 256, 256, 0, st>>>(B.cnt, mt, B.seg, B.seglist, B.biglist, B.medlist, B.st);
  k_group_scatter<<<(nt + 255) / 256, 256, 0, st>>>(B.nnkey, nt, B.cnt, B.seg, B.member, B.ja[cur], B.protocol,
                                                    B.seed, round);
  FlowArgs F{B.ia[cur], B.ja[cur], B.seg,  B.seglist, B.biglist, B.medlist, B.member,
             B.s,       B.c,       B.fl_i, B.fl_j,    B.fl_f,    B.st};
  // enough warps for every group of 9..32 at once (at most nt / 9 of them);
  // the thread-per-group pass needs nt / 32
  int warps = (nt + 8) / 9;
  int blocks = (warps + 7) / 8;
  const int nsm = num_sms();
  if (blocks > nsm * 16) blocks = nsm * 16;
  k_flow<<<blocks + nsm, BIG_THREADS, 0, st>>>(F, blocks);
  // weights update: compact into the other buffer
  CompactArgs A{};
  const bool packed = B.dp > 0;
  A.side[0] = CompactSide{packed ? B.xa[cur] : nullptr, B.dp, B.ia[cur], B.s, packed ? B.xa[cur ^ 1] : nullptr,
                          B.ia[cur ^ 1], mt, &B.st->mt, 0, 0};
  A.side[1] = CompactSide{packed ? B.ya[cur] : nullptr, B.dp, B.ja[cur], B.c, packed ? B.ya[cur ^ 1] : nullptr,
                          B.ja[cur ^ 1], nt, &B.st->nt, 0, 0, B.nnkey};
  A.blockcounts = B.blockcounts;
  A.err = &B.st->err;
  A.notify = B.notify;
  A.notify_seq = B.notify_seq;
  A.ticket = &B.st->ticket;
  compact_launch(A, B.dp, st);
  return 0;
}

}  // namespace nnsemd
