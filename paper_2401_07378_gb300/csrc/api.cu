// C-ABI entry points of the NNS-EMD library (declared in include/nnsemd.h):
// context and workspace management, argument checks, and the host-side
// orchestration of the rounds of Alg. 1 (Sec. III-A).
//
// A single-pair solve runs
//   setup    exact totals of a and b, normalisation (Sec. II-A), packing of
//            the initial active sets (positive weight);
//   rounds   while both active sets are larger than one CTA can hold: the
//            multi-CTA round (K1 NNS, grouping, greedy flow, compaction);
//   tail     once they fit, every remaining round in one launch: for d <= 8
//            on a thread-block cluster (k_finish_cl, up to 2048 points per
//            side) where the device can co-schedule one, else in one CTA
//            (k_finish, k_finish_hd);
//   final    R and the leftover mass as correctly rounded sums.
// The host reads the two active counts of each multi-CTA round to size the
// next round's grids: the compaction's count kernel writes them into mapped
// host memory as soon as they are known, and the host launches the next
// round while the scatter still runs (no stream synchronisation per round).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "ctx.h"
#include "kernels.h"
#include "nnsemd.h"
#include "proposal.h"

using namespace nnsemd;

namespace {

constexpr int64_t FIN_PAIRS = 1LL << 19;     // d <= 8 tail threshold on m_t * n_t
constexpr int64_t FIN_HD_WORK = 1LL << 23;   // d > 8 tail threshold on m_t * n_t * d
constexpr double KC_BUDGET_BYTES = 8.0e9;    // largest workspace of the batched distance caches
thread_local std::string g_create_err;

int fail(nnsemd_ctx* ctx, int status, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(nnsemd_ctx* ctx, int status, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  else g_create_err = buf;
  return status;
}

}  // namespace

int nnsemd::num_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
  if (dev < 64) {
    const int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int count = 0;
  if (cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || count < 1) {
    cudaGetLastError();
    count = 1;
  }
  if (dev < 64) cache[dev].store(count, std::memory_order_relaxed);
  return count;
}

int nnsemd::ctx_fail(nnsemd_ctx* ctx, int status, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  else g_create_err = buf;
  return status;
}

namespace {

int cuda_fail(nnsemd_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, NNSEMD_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
  } while (0)

// The same inside a solve whose first kernels are already queued: the call
// returns only once its stream has drained (drained() waits for it), so no
// work of the failed call outlives it.
#define CKD(call)                                                      \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) return drained(cuda_fail(ctx, e_, #call));  \
  } while (0)

// Bump allocator over the context workspace (256-byte aligned slices).
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(void* b) : base((char*)b) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

int ensure_ws(nnsemd_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return NNSEMD_OK;
  if (ctx->ws) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  size_t want = bytes + bytes / 8;
  cudaError_t e = cudaMalloc(&ctx->ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->ws = nullptr;
    return fail(ctx, NNSEMD_ERR_OOM, "workspace of %zu bytes: %s", want, cudaGetErrorString(e));
  }
  ctx->ws_bytes = want;
  return NNSEMD_OK;
}

// Lay out the buffers of a single-pair solve; with base == nullptr only the
// size is computed.
size_t layout_solve(void* base, int64_t m, int64_t n, int d, SolveBufs& B, int precision = 0,
                    const nnsemd_proposal* P = nullptr, LearnedBufs* L = nullptr) {
  Carve C(base);
  const int dp = d <= 8 ? padded_dim(d) : 0;
  B.precision = precision;
  if (P && L) {
    const int K = P->cells, h = P->hidden;
    L->P = P;
    L->chunk = 4096;
    L->cell_of_x = C.take<int>(m);
    L->radius = C.take<float>(K);
    L->prop_cells = C.take<int>((size_t)n * PROP_LIST);
    L->bound_cells = C.take<int>((size_t)n * PROP_LIST);
    L->bound_vals = C.take<float>((size_t)n * PROP_LIST);
    L->cell_cnt = C.take<int>(K + 1);
    L->cell_off = C.take<int>(K + 1);
    L->cell_fill = C.take<int>(K);
    L->cell_members = C.take<int>(m);
    L->fallback = C.take<int>(n);
    L->nfallback = C.take<int>(1);
    L->fallback2 = C.take<int>(n);
    L->nfallback2 = C.take<int>(1);
    L->tmp = C.take<float>((size_t)2 * L->chunk * h);
    L->tmp2 = C.take<float>((size_t)L->chunk * K);
    L->tmp3 = C.take<float>((size_t)L->chunk * d);
    L->sel_over = C.take<int>(L->chunk);
    L->nsel_over = C.take<int>(1);
    L->lc_cand = C.take<int>((size_t)n * PROP_TAKE);
    L->lc_slot = C.take<int>((size_t)n * PROP_TAKE);
    L->lc_ncand = C.take<int>(n);
    L->lc_bound = C.take<float>(n);
    L->lc_qcnt = C.take<int>(K);
    L->lc_qoff = C.take<int>(K + 1);
    L->lc_work = C.take<int>(K + 1);
    L->lc_nwork = C.take<int>(2);  // the work items' count, then the counter of the next one
    L->lc_qlist = C.take<int>((size_t)n * PROP_TAKE);
    L->lc_best = C.take<unsigned long long>(n);
    L->w3p = C.take<uint8_t>(linear_tc_supported(h) ? linear_tc_packed_bytes(K, h) : 0);
    L->h2p = C.take<uint8_t>(linear_tc_supported(h) ? linear_tc_packed_bytes(L->chunk, h) : 0);
    const bool tc_all = linear_tc_supported(h) && linear_tc_supported(d);
    L->w1p = C.take<uint8_t>(tc_all ? linear_tc_packed_bytes(h, d) : 0);
    L->w2p = C.take<uint8_t>(tc_all ? linear_tc_packed_bytes(h, h) : 0);
    L->xp1 = C.take<uint8_t>(tc_all ? linear_tc_packed_bytes(L->chunk, d) : 0);
    L->h1p = C.take<uint8_t>(tc_all ? linear_tc_packed_bytes(L->chunk, h) : 0);
    L->assign_chunk = 65536;
    const bool tca = linear_tc_supported(d);
    L->mup = C.take<uint8_t>(tca ? linear_tc_packed_bytes(K, d) : 0);
    L->mu_bias = C.take<float>(tca ? K : 0);
    L->xp = C.take<uint8_t>(tca ? linear_tc_packed_bytes(L->assign_chunk, d) : 0);
    L->apart = C.take<unsigned long long>(tca ? (size_t)L->assign_chunk * ((K + 127) / 128) : 0);
    const bool tcb = cell_bounds_tc_supported(d);
    L->mup3 = C.take<uint8_t>(tcb ? linear_tc_packed_bytes(K, 3 * d) : 0);
    L->mu_sq_lo = C.take<float>(tcb ? K : 0);
    L->mu_nrm_up = C.take<float>(tcb ? K : 0);
    L->yp3 = C.take<uint8_t>(tcb ? linear_tc_packed_bytes(L->chunk, 3 * d) : 0);
    L->y_sq_lo = C.take<float>(tcb ? L->chunk : 0);
    L->y_nrm_up = C.take<float>(tcb ? L->chunk : 0);
  }
  if (precision != NNSEMD_FP32) {
    const size_t kb = tc_kb(d, precision);
    const int64_t bn = tc_bn(kb);
    const int64_t qrows = (n + 127) / 128 * 128, srows = (m + bn - 1) / bn * bn;
    TcBufs& T = B.tc;
    T.A = C.take<uint8_t>(qrows * kb);
    T.B = C.take<uint8_t>(srows * kb);
    T.nrm_x = C.take<float>(srows);
    T.nrm_sx = C.take<float>(srows);
    T.nrm_y = C.take<float>(qrows);
    T.scale_x = C.take<float>(srows);
    T.scale_y = C.take<float>(qrows);
    T.stats = C.take<unsigned>(8);
    T.max_chunks = tc_target_ctas();
    const int64_t cand = (tc_target_ctas() + qrows / 128) * 128 * 16;  // chunks x padded consumers x 16 candidates
    T.cand_v = C.take<float>(cand);
    T.cand_p = C.take<int>(cand);
    T.fallback = C.take<int>(n);
    T.nfallback = C.take<int>(1);
    T.ev0 = T.ev1 = nullptr;
  }
  B.st = C.take<DevState>(1);
  B.xs_acc = C.take<unsigned long long>(4 * XS_LIMBS);
  B.s = C.take<double>(m);
  B.c = C.take<double>(n);
  for (int k = 0; k < 2; ++k) {
    B.xa[k] = C.take<float>(pad_points(m) * dp);
    B.ia[k] = C.take<int>(m);
    B.ya[k] = C.take<float>(pad_points(n) * dp);
    B.ja[k] = C.take<int>(n);
  }
  B.nnkey = C.take<unsigned long long>(n);
  B.cnt = C.take<int>(m);
  B.seg = C.take<int2>(m);
  B.seglist = C.take<int>(m);
  B.biglist = C.take<int>(m);
  B.medlist = C.take<int>(m);
  B.member = C.take<unsigned long long>(n);
  B.fl_i = C.take<int32_t>(m + n);
  B.fl_j = C.take<int32_t>(m + n);
  B.fl_f = C.take<double>(m + n);
  B.blockcounts = C.take<int>((m + n) / 1024 + 8);
  return C.off + 256;
}

int map_err_bits(nnsemd_ctx* ctx, unsigned bits) {
  if (!bits) return NNSEMD_OK;
  if (bits & EF_NONFINITE) return fail(ctx, NNSEMD_ERR_NONFINITE, "a coordinate or weight is not finite");
  if (bits & EF_NEGATIVE) return fail(ctx, NNSEMD_ERR_ZERO_MASS, "a weight is negative");
  if (bits & EF_ZERO_MASS) return fail(ctx, NNSEMD_ERR_ZERO_MASS, "a side's weights sum to zero");
  if (bits & EF_CAPACITY) return fail(ctx, NNSEMD_ERR_CAPACITY, "plan capacity too small");
  if (bits & EF_TIMEOUT) return fail(ctx, NNSEMD_ERR_TIMEOUT, "a bounded device wait gave up");
  if (bits & EF_ITER) return fail(ctx, NNSEMD_ERR_ITER_LIMIT, "round limit m + n exceeded");
  return fail(ctx, NNSEMD_ERR_CUDA, "internal consistency check failed on the device (0x%x)", bits);
}

// Wait (spinning) until the compaction of a round has published its active
// counts under sequence number `seq` (mapped host memory, written by the
// last block of the count kernel).  Fails instead of waiting forever if the
// stream stops or two minutes pass.
int wait_counts(nnsemd_ctx* ctx, cudaStream_t st, int seq, int& mt, int& nt, unsigned& err) {
  volatile int* h = ctx->hmap;
  const auto t0 = std::chrono::steady_clock::now();
  for (unsigned it = 1; h[0] != seq; ++it) {
    if ((it & 4095u) != 0) continue;
    const cudaError_t q = cudaStreamQuery(st);
    if (q != cudaSuccess && q != cudaErrorNotReady)
      return fail(ctx, NNSEMD_ERR_CUDA, "waiting for a round: %s", cudaGetErrorString(q));
    if (q == cudaSuccess && h[0] != seq) return fail(ctx, NNSEMD_ERR_CUDA, "a round's counts were not published");
    if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(120))
      return fail(ctx, NNSEMD_ERR_TIMEOUT, "a round did not finish within two minutes");
  }
  std::atomic_thread_fence(std::memory_order_acquire);
  mt = h[1];
  nt = h[2];
  err = (unsigned)h[3];
  return 0;
}

int check_opts(nnsemd_ctx* ctx, const nnsemd_options* opt, int d, int& metric, int* precision = nullptr) {
  metric = NNSEMD_L2;
  if (precision) *precision = NNSEMD_FP32;
  if (opt) {
    metric = opt->metric;
    if (opt->flags & ~(NNSEMD_FLAG_TIME_KERNELS | NNSEMD_FLAG_AUTOTUNE | NNSEMD_FLAG_GRAPH))
      return fail(ctx, NNSEMD_ERR_INVALID_ARG, "unknown options.flags bits");
    if (opt->precision < NNSEMD_FP32 || opt->precision > NNSEMD_BF16X3)
      return fail(ctx, NNSEMD_ERR_INVALID_ARG, "unknown precision %d", opt->precision);
    if (opt->protocol != NNSEMD_PROTOCOL_GREEDY && opt->protocol != NNSEMD_PROTOCOL_RANDOM)
      return fail(ctx, NNSEMD_ERR_INVALID_ARG, "unknown protocol %d", opt->protocol);
    if (opt->reserved != 0) return fail(ctx, NNSEMD_ERR_INVALID_ARG, "options.reserved must be 0");
    if (opt->rerank_k < 0 || opt->rerank_k > NNSEMD_MAX_RERANK_K)
      return fail(ctx, NNSEMD_ERR_INVALID_ARG, "options.rerank_k = %d: outside 0..%d", opt->rerank_k,
                  NNSEMD_MAX_RERANK_K);
    if (opt->precision != NNSEMD_FP32) {
      if (!precision) return fail(ctx, NNSEMD_ERR_UNSUPPORTED, "reduced precision is served by nnsemd_solve only");
      if (d <= 8) return fail(ctx, NNSEMD_ERR_UNSUPPORTED, "reduced precision serves d > 8 (d = %d)", d);
      if (opt->metric == NNSEMD_L1) return fail(ctx, NNSEMD_ERR_UNSUPPORTED, "the L1 distance has no contraction form");
      if (!tc_supported(d, opt->precision))
        return fail(ctx, NNSEMD_ERR_UNSUPPORTED, "d = %d is too large for precision %d's operand tiles", d,
                    opt->precision);
      *precision = opt->precision;
    }
  }
  if (metric < 0 || metric > 2) return fail(ctx, NNSEMD_ERR_INVALID_ARG, "unknown metric %d", metric);
  if (d < 1) return fail(ctx, NNSEMD_ERR_INVALID_ARG, "d must be >= 1");
  if (d > 65536) return fail(ctx, NNSEMD_ERR_UNSUPPORTED, "d = %d: above 65536", d);
  return NNSEMD_OK;
}

// Packed coordinate width of the d <= 8 path; 0 for d > 8 (index-only lists).
int packed_dim(int d) { return d <= 8 ? padded_dim(d) : 0; }

// The device part of a single-pair solve on buffers that are already laid
// out; writes R to *cost and fills the counters.
int run_solve(nnsemd_ctx* ctx, SolveBufs& B, const double* a, const double* b, double* cost, int64_t* nnz,
              nnsemd_stats* stats, int flags = 0, const LearnedBufs* learned = nullptr) {
  cudaStream_t st = ctx->stream;
  long long L = 0;
  const bool timed = (flags & NNSEMD_FLAG_TIME_KERNELS) != 0;
  if (timed && !ctx->ev[0])
    for (int k = 0; k < 4; ++k) CK(cudaEventCreate(&ctx->ev[k]));
  double nns_ms = 0.0, tail_ms = 0.0;
  long long nns_launches = 0, nns_pairs = 0;
  bool tail_ran = false;
  if (B.dp > 0 && B.m <= FIN_MAX && B.n <= FIN_MAX) {
    // small pair: the whole solve in one launch, one host synchronisation
    CK(cudaMemsetAsync(B.st, 0, sizeof(DevState), st));
    if (timed) CK(cudaEventRecord(ctx->ev[2], st));
    if (launch_solve_small(B, a, b, st)) return fail(ctx, NNSEMD_ERR_CUDA, "small-pair launch");
    if (timed) CK(cudaEventRecord(ctx->ev[3], st));
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ctx->hstate, B.st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int rc0 = map_err_bits(ctx, ctx->hstate->err);
    if (rc0) return rc0;
    *cost = ctx->hstate->cost;
    *nnz = (int64_t)ctx->hstate->nnz;
    ctx->launches += 1;
    if (timed) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]));
      tail_ms = ms;
    }
    if (stats) {
      std::memset(stats, 0, sizeof(*stats));
      stats->rounds = ctx->hstate->rounds;
      stats->pair_evals = ctx->hstate->pair_evals;
      stats->leftover_mass = ctx->hstate->leftover;
      stats->kernel_launches = 1;
      stats->tail_kernel_ms = tail_ms;
    }
    return NNSEMD_OK;
  }
  CK(cudaMemsetAsync(B.st, 0, sizeof(DevState), st));
  CK(cudaMemsetAsync(B.xs_acc, 0, 4 * XS_LIMBS * sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(B.cnt, 0, B.m * sizeof(int), st));
  launch_setup_sums(B, a, b, st);
  B.cur = 0;
  // the initial packing publishes the active counts like every round's
  // compaction (with the weight and coordinate checks' error bits)
  B.notify = ctx->dmap;
  B.notify_seq = ++ctx->notify_seq;
  launch_initial_pack(B, st);
  L += B.dp > 0 ? 4 : 6;  // two sums, count + scatter (d > 8: two finiteness checks too)
  // a failure after this point returns only once the stream has drained:
  // no work of this call outlives it
  auto drained = [&](int status) {
    cudaStreamSynchronize(st);
    return status;
  };
  CKD(cudaGetLastError());
  int mt = 0, nt = 0;
  unsigned err0 = 0;
  int rc = wait_counts(ctx, st, B.notify_seq, mt, nt, err0);
  if (!rc) rc = map_err_bits(ctx, err0);
  if (rc) return drained(rc);
  long long rounds = 0, pair_evals = 0;
  const long long round_limit = B.m + B.n;
  const bool lowd = B.dp > 0;
  // the cluster tail takes over once both active sets fit it
  const int clcap = lowd ? finish_cluster_cap(B.d, B.metric) : 0;
  if (learned) {
    // once per solve: supplier cells and radii, consumer proposals and bounds
    if (learned_prepare(*learned, B.x, B.m, B.y, B.n, B.d, &B.st->err, st))
      return drained(fail(ctx, NNSEMD_ERR_CUDA, "proposal preparation"));
    // per chunk: standardisation, three GEMMs, the centroid bounds and two
    // selections (one-warp + block pass each, or the block pass alone)
    const int sel = learned->P->cells >= 2 * PROP_LIST ? 2 : 1;
    // supplier cells: on the tensor cores two set-up kernels, three per pass,
    // and the radii
    const int64_t passes = (B.m + learned->assign_chunk - 1) / learned->assign_chunk;
    const bool tcb = cell_bounds_tc_supported(B.d);
    const bool tch = linear_tc_supported(learned->P->hidden);
    L += (linear_tc_supported(B.d) ? 3 + 3 * passes : 8) + (tch ? 1 : 0) + (tch && linear_tc_supported(B.d) ? 2 : 0) +
         (tcb ? 2 : 0) + (5 + (tcb ? 2 : 0) + 2 * sel) * ((B.n + learned->chunk - 1) / learned->chunk);
  }
  while (mt > 0 && nt > 0) {
    const bool tail = clcap ? (mt <= clcap && nt <= clcap)
                      : lowd ? (mt <= FIN_MAX && nt <= FIN_MAX && (int64_t)mt * nt <= FIN_PAIRS)
                             : (mt <= FIN_MAX_HD && nt <= FIN_MAX_HD && (int64_t)mt * nt * B.d <= FIN_HD_WORK);
    if (tail) {
      if (timed) CKD(cudaEventRecord(ctx->ev[2], st));
      B.round0 = rounds;
      const int lrc = clcap  ? launch_finish_cluster(B, round_limit - rounds, st)
                      : lowd ? launch_finish(B, round_limit - rounds, st)
                             : launch_finish_hd(B, round_limit - rounds, st);
      if (lrc) return drained(fail(ctx, NNSEMD_ERR_CUDA, "finisher launch"));
      if (timed) CKD(cudaEventRecord(ctx->ev[3], st));
      tail_ran = true;
      L += 1;
      break;
    }
    if (rounds >= round_limit) return drained(fail(ctx, NNSEMD_ERR_ITER_LIMIT, "round limit m + n exceeded"));
    // B.nnkey[0 .. nt) is all ones here: the compaction that produced the
    // active lists reset the key of every surviving consumer
    int nrc;
    if (learned) {
      if (timed) CKD(cudaEventRecord(ctx->ev[0], st));
      nrc = launch_nns_learned(B, *learned, mt, nt, st);
      if (timed) CKD(cudaEventRecord(ctx->ev[1], st));
      L += learned_cell_scan(B.d, B.x, B.y) ? 11 : 6;
    } else if (B.precision != NNSEMD_FP32) {
      // tensor-core candidates + exact re-rank + certificate + FP32 rescan;
      // the timing events bracket the tensor-core kernel alone
      B.tc.ev0 = timed ? ctx->ev[0] : nullptr;
      B.tc.ev1 = timed ? ctx->ev[1] : nullptr;
      nrc = launch_nns_tc(B, B.tc, mt, nt, B.precision, st);
      L += 5;
    } else {
      if (timed) CKD(cudaEventRecord(ctx->ev[0], st));
      nrc = lowd ? launch_nns_lowd(B, mt, nt, st) : launch_nns_f32(B, mt, nt, nullptr, nullptr, st);
      if (timed) CKD(cudaEventRecord(ctx->ev[1], st));
      L += 1;
    }
    if (nrc) return drained(fail(ctx, NNSEMD_ERR_UNSUPPORTED, "NNS launch failed for d=%d (%d)", B.d, nrc));
    // the compaction's count kernel publishes the next active counts as soon
    // as they are known; the host sizes and launches the next round while
    // the scatter still runs
    B.notify = ctx->dmap;
    B.notify_seq = ++ctx->notify_seq;
    launch_big_round(B, mt, nt, rounds, st);
    L += 6;  // group count / alloc / scatter, flow, compaction count / scatter
    CKD(cudaGetLastError());
    B.cur ^= 1;
    rounds += 1;
    pair_evals += (long long)mt * nt;
    nns_launches += 1;
    nns_pairs += (long long)mt * nt;
    unsigned err_bits = 0;
    rc = wait_counts(ctx, st, B.notify_seq, mt, nt, err_bits);
    if (rc) return drained(rc);
    if (timed) {
      float ms = 0.f;
      CKD(cudaEventSynchronize(ctx->ev[1]));
      CKD(cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]));
      nns_ms += ms;
    }
    rc = map_err_bits(ctx, err_bits);
    if (rc) return drained(rc);
  }
  launch_leftover(B, st);
  L += 2;
  CKD(cudaGetLastError());
  CKD(cudaMemcpyAsync(ctx->hstate, B.st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
  CKD(cudaStreamSynchronize(st));
  rc = map_err_bits(ctx, ctx->hstate->err);
  if (rc) return rc;
  *cost = ctx->hstate->cost;
  *nnz = (int64_t)ctx->hstate->nnz;
  ctx->launches += L;
  if (timed && tail_ran) {
    float ms = 0.f;
    CKD(cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]));
    tail_ms = ms;
  }
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->rounds = rounds + ctx->hstate->rounds;
    stats->pair_evals = pair_evals + ctx->hstate->pair_evals;
    stats->leftover_mass = ctx->hstate->leftover;
    stats->kernel_launches = L;
    stats->certified = (int64_t)ctx->hstate->certified;
    stats->fallbacks = (int64_t)ctx->hstate->fallbacks;
    stats->near_ties = (int64_t)ctx->hstate->near_ties;
    stats->widened = (int64_t)ctx->hstate->widened;
    stats->nns_kernel_ms = nns_ms;
    stats->nns_kernel_launches = nns_launches;
    stats->nns_kernel_pairs = nns_pairs;
    stats->tail_kernel_ms = tail_ms;
  }
  return NNSEMD_OK;
}

int check_sizes(nnsemd_ctx* ctx, int64_t m, int64_t n) {
  if (m < 1 || n < 1) return fail(ctx, NNSEMD_ERR_INVALID_ARG, "m and n must be >= 1 (m=%lld n=%lld)",
                                  (long long)m, (long long)n);
  if (m > (1LL << 30) || n > (1LL << 30)) return fail(ctx, NNSEMD_ERR_UNSUPPORTED, "m or n above 2^30");
  return NNSEMD_OK;
}

// A learned proposal replaces the full NNS scan only where its candidate
// search applies: d > 8, L2 or SQL2, the proposal's own d.  With a reduced
// precision the consumers it cannot certify go to the tensor-core scan.
int check_proposal(nnsemd_ctx* ctx, const nnsemd_options* opt, int d, int metric, int precision,
                   const nnsemd_proposal** out) {
  const nnsemd_proposal* P = opt ? static_cast<const nnsemd_proposal*>(opt->proposal) : nullptr;
  *out = P;
  (void)precision;
  if (P && (d <= 8 || metric == NNSEMD_L1 || P->d != d || !P->codebook_ready))
    return fail(ctx, NNSEMD_ERR_UNSUPPORTED,
                "a proposal needs d > 8, metric L2 or SQL2, its own d and a fitted codebook");
  return NNSEMD_OK;
}

}  // namespace

extern "C" {

int nnsemd_create(nnsemd_ctx** out, const nnsemd_config* cfg) {
  if (!out) return fail(nullptr, NNSEMD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  nnsemd_ctx* ctx = new (std::nothrow) nnsemd_ctx();
  if (!ctx) return fail(nullptr, NNSEMD_ERR_OOM, "context allocation");
  ctx->device = cfg ? cfg->device : 0;
  ctx->stream = cfg ? (cudaStream_t)cfg->stream : nullptr;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess) e = cudaMallocHost(&ctx->hstate, sizeof(DevState));
  if (e == cudaSuccess) {
    void* hm = nullptr;
    e = cudaHostAlloc(&hm, 64, cudaHostAllocMapped);
    if (e == cudaSuccess) {
      std::memset(hm, 0, 64);
      ctx->hmap = static_cast<volatile int*>(hm);
      e = cudaHostGetDevicePointer((void**)&ctx->dmap, hm, 0);
    }
  }
  if (e != cudaSuccess) {
    if (ctx->hmap) cudaFreeHost((void*)ctx->hmap);
    if (ctx->hstate) cudaFreeHost(ctx->hstate);
    int rc = fail(nullptr, NNSEMD_ERR_CUDA, "device %d: %s", ctx->device, cudaGetErrorString(e));
    delete ctx;
    return rc;
  }
  if (cfg && cfg->workspace_bytes_hint) {
    int rc = ensure_ws(ctx, cfg->workspace_bytes_hint);
    if (rc) {
      g_create_err = ctx->err;
      cudaFreeHost(ctx->hstate);
      cudaFreeHost((void*)ctx->hmap);
      delete ctx;
      return rc;
    }
  }
  *out = ctx;
  return NNSEMD_OK;
}

int nnsemd_destroy(nnsemd_ctx* ctx) {
  if (!ctx) return NNSEMD_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->hstate) cudaFreeHost(ctx->hstate);
  if (ctx->hmap) cudaFreeHost((void*)ctx->hmap);
  for (cudaEvent_t e : ctx->ev)
    if (e) cudaEventDestroy(e);
  for (auto& g : ctx->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  delete ctx;
  return NNSEMD_OK;
}

int nnsemd_set_stream(nnsemd_ctx* ctx, void* stream) {
  if (!ctx) return NNSEMD_ERR_INVALID_ARG;
  ctx->stream = (cudaStream_t)stream;
  return NNSEMD_OK;
}

int nnsemd_solve(nnsemd_ctx* ctx, const float* x, const double* a, int64_t m, const float* y, const double* b,
                 int64_t n, int32_t d, const nnsemd_options* opt, double* cost_out, nnsemd_plan* plan,
                 nnsemd_stats* stats) {
  if (!ctx) return NNSEMD_ERR_INVALID_ARG;
  ctx->err.clear();
  int metric, precision;
  int rc = check_opts(ctx, opt, d, metric, &precision);
  if (rc) return rc;
  if ((rc = check_sizes(ctx, m, n))) return rc;
  if (!x || !a || !y || !b || !cost_out) return fail(ctx, NNSEMD_ERR_INVALID_ARG, "null pointer argument");
  if (((uintptr_t)x & 3) || ((uintptr_t)y & 3) || ((uintptr_t)a & 7) || ((uintptr_t)b & 7))
    return fail(ctx, NNSEMD_ERR_INVALID_ARG, "misaligned input pointer");
  if (plan && (!plan->i || !plan->j || !plan->f || plan->capacity < 0))
    return fail(ctx, NNSEMD_ERR_INVALID_ARG, "plan arrays");
  const nnsemd_proposal* P = nullptr;
  if ((rc = check_proposal(ctx, opt, d, metric, precision, &P))) return rc;
  CK(cudaSetDevice(ctx->device));
  SolveBufs B{};
  LearnedBufs Lb{};
  size_t bytes = layout_solve(nullptr, m, n, d, B, precision, P, P ? &Lb : nullptr);
  if ((rc = ensure_ws(ctx, bytes))) return rc;
  layout_solve(ctx->ws, m, n, d, B, precision, P, P ? &Lb : nullptr);
  B.x = x;
  B.y = y;
  B.m = m;
  B.n = n;
  B.d = d;
  B.dp = packed_dim(d);
  B.metric = metric;
  B.protocol = opt ? opt->protocol : 0;
  B.seed = opt ? opt->seed : 0;
  B.plan_i = plan ? plan->i : nullptr;
  B.plan_j = plan ? plan->j : nullptr;
  B.plan_f = plan ? plan->f : nullptr;
  B.plan_cap = plan ? plan->capacity : 0;
  B.tc.rerank_k = opt ? opt->rerank_k : 0;
  int64_t nnz = 0;
  rc = run_solve(ctx, B, a, b, cost_out, &nnz, stats, opt ? opt->flags : 0, P ? &Lb : nullptr);
  if (plan) plan->nnz = rc ? 0 : nnz;
  return rc;
}

int nnsemd_solve_host(nnsemd_ctx* ctx, const float* x, const double* a, int64_t m, const float* y,
                      const double* b, int64_t n, int32_t d, const nnsemd_options* opt, double* cost_out,
                      nnsemd_plan* plan, nnsemd_stats* stats) {
  if (!ctx) return NNSEMD_ERR_INVALID_ARG;
  ctx->err.clear();
  int metric, precision;
  int rc = check_opts(ctx, opt, d, metric, &precision);
  if (rc) return rc;
  if ((rc = check_sizes(ctx, m, n))) return rc;
  if (!x || !a || !y || !b || !cost_out) return fail(ctx, NNSEMD_ERR_INVALID_ARG, "null pointer argument");
  if (plan && (!plan->i || !plan->j || !plan->f || plan->capacity < 0))
    return fail(ctx, NNSEMD_ERR_INVALID_ARG, "plan arrays");
  const nnsemd_proposal* P = nullptr;
  if ((rc = check_proposal(ctx, opt, d, metric, precision, &P))) return rc;
  CK(cudaSetDevice(ctx->device));
  // device staging for the inputs and the plan, placed after the solve buffers
  SolveBufs B{};
  LearnedBufs Lb{};
  size_t solve_bytes = layout_solve(nullptr, m, n, d, B, precision, P, P ? &Lb : nullptr);
  const int64_t cap = plan ? std::min<int64_t>(plan->capacity, m + n) : 0;
  auto stage_layout = [&](void* base, float** xd, double** ad, float** yd, double** bd, int32_t** pi, int32_t** pj,
                          double** pf) {
    Carve C(base);
    C.off = solve_bytes;
    *xd = C.take<float>((size_t)m * d);
    *ad = C.take<double>(m);
    *yd = C.take<float>((size_t)n * d);
    *bd = C.take<double>(n);
    *pi = C.take<int32_t>(cap);
    *pj = C.take<int32_t>(cap);
    *pf = C.take<double>(cap);
    return C.off + 256;
  };
  float *xd, *yd;
  double *ad, *bd, *pf;
  int32_t *pi, *pj;
  size_t bytes = stage_layout(nullptr, &xd, &ad, &yd, &bd, &pi, &pj, &pf);
  if ((rc = ensure_ws(ctx, bytes))) return rc;
  layout_solve(ctx->ws, m, n, d, B, precision, P, P ? &Lb : nullptr);
  stage_layout(ctx->ws, &xd, &ad, &yd, &bd, &pi, &pj, &pf);
  cudaStream_t st = ctx->stream;
  CK(cudaMemcpyAsync(xd, x, (size_t)m * d * sizeof(float), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ad, a, (size_t)m * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(yd, y, (size_t)n * d * sizeof(float), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(bd, b, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st));
  B.x = xd;
  B.y = yd;
  B.m = m;
  B.n = n;
  B.d = d;
  B.dp = packed_dim(d);
  B.metric = metric;
  B.protocol = opt ? opt->protocol : 0;
  B.seed = opt ? opt->seed : 0;
  B.plan_i = plan ? pi : nullptr;
  B.plan_j = plan ? pj : nullptr;
  B.plan_f = plan ? pf : nullptr;
  B.plan_cap = cap;
  B.tc.rerank_k = opt ? opt->rerank_k : 0;
  int64_t nnz = 0;
  rc = run_solve(ctx, B, ad, bd, cost_out, &nnz, stats, opt ? opt->flags : 0, P ? &Lb : nullptr);
  if (rc) {
    if (plan) plan->nnz = 0;
    return rc;
  }
  if (plan) {
    if (nnz > plan->capacity) return fail(ctx, NNSEMD_ERR_CAPACITY, "plan capacity too small");
    CK(cudaMemcpyAsync(plan->i, pi, (size_t)nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(plan->j, pj, (size_t)nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(plan->f, pf, (size_t)nnz * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    plan->nnz = nnz;
  }
  return NNSEMD_OK;
}

// The batched solver.  With y_off == nullptr every pair's consumers are the
// same n_shared rows of y_packed / b_packed (one-to-many).
static int solve_batched_impl(nnsemd_ctx* ctx, int32_t num_pairs, const float* x_packed, const double* a_packed,
                              const int64_t* x_off, const float* y_packed, const double* b_packed,
                              const int64_t* y_off, int64_t n_shared, int32_t d, const nnsemd_options* opt,
                              double* costs_out, nnsemd_stats* stats) {
  if (!ctx) return NNSEMD_ERR_INVALID_ARG;
  ctx->err.clear();
  int metric, precision;
  int rc = check_opts(ctx, opt, d, metric, &precision);
  if (rc) return rc;
  const int flags = opt ? opt->flags : 0;
  const bool tc = precision != NNSEMD_FP32;
  if (num_pairs < 0) return fail(ctx, NNSEMD_ERR_INVALID_ARG, "num_pairs < 0");
  if (num_pairs == 0) {
    if (stats) std::memset(stats, 0, sizeof(*stats));
    return NNSEMD_OK;
  }
  if (!x_packed || !a_packed || !x_off || !y_packed || !b_packed || (!y_off && n_shared < 1) || !costs_out)
    return fail(ctx, NNSEMD_ERR_INVALID_ARG, "null pointer argument");
  if (x_off[0] != 0 || (y_off && y_off[0] != 0)) return fail(ctx, NNSEMD_ERR_INVALID_ARG, "offsets must start at 0");
  if (!y_off && n_shared > (1LL << 30)) return fail(ctx, NNSEMD_ERR_UNSUPPORTED, "n above 2^30");
  if (opt && opt->proposal) return fail(ctx, NNSEMD_ERR_UNSUPPORTED, "proposals serve nnsemd_solve only");
  auto y_begin = [&](int p) -> int64_t { return y_off ? y_off[p] : 0; };
  auto y_len = [&](int p) -> int64_t { return y_off ? y_off[p + 1] - y_off[p] : n_shared; };
  std::vector<int> small, large;
  int64_t small_max = 0, small_mn = 0;
  for (int p = 0; p < num_pairs; ++p) {
    const int64_t m = x_off[p + 1] - x_off[p], n = y_len(p);
    if (m < 1 || n < 1) return fail(ctx, NNSEMD_ERR_INVALID_ARG, "pair %d has an empty side", p);
    const int cap = d <= 8 ? FIN_MAX : FIN_MAX_HD;
    const bool fits = m <= cap && n <= cap;
    (fits ? small : large).push_back(p);
    if (fits) {
      small_max = std::max(small_max, std::max(m, n));
      small_mn = std::max(small_mn, m * n);
    }
  }
  // FP32, d > 8: pairs of at most HD_SMALL_CAP points per side go to the
  // 256-thread kernel (several pairs per SM); they come first in the list
  int ntiny = 0;
  if (!tc && d > 8) {
    std::stable_partition(small.begin(), small.end(), [&](int p) {
      return x_off[p + 1] - x_off[p] <= HD_SMALL_CAP && y_len(p) <= HD_SMALL_CAP;
    });
    for (int p : small)
      if (x_off[p + 1] - x_off[p] <= HD_SMALL_CAP && y_len(p) <= HD_SMALL_CAP) ++ntiny;
  }
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const int nsm = num_sms();
  const int grid = (int)std::min<size_t>(small.size(), (size_t)nsm);
  // tensor-core kernel geometry: capacity class, bytes per packed row, tile
  // rows and pipeline stages (autotuned or default)
  const int cap = small_max <= 512 ? 512 : 2048;
  const int kb = tc ? (int)tc_kb(d, precision) : 0;
  int bn = tc ? tc_bn(kb) : 0;
  int nstage = tc ? batched_tc_max_stages(cap, kb, bn, precision) : 0;
  if (tc && !small.empty() && nstage < 1) return fail(ctx, NNSEMD_ERR_UNSUPPORTED, "d = %d too large for the batched tensor-core kernel", d);
  const auto tkey = std::make_tuple(d, precision, cap);
  int kc_use = 1;
  if (tc && ctx->tuned.count(tkey)) std::tie(bn, nstage, kc_use) = ctx->tuned[tkey];
  // the tensor-core kernel's distance cache: every pair's first round fills
  // it and later rounds read it, when all the batch's cache slots fit the
  // budget (else the kernel runs the tensor cores in every round); the
  // autotuner may also turn it off
  long long kc_cap = tc ? (long long)small_mn : 0;
  auto slot_of = [&](long long kc) {
    return std::max(batched_tc_slot_bytes(cap, kb, 64, kc), batched_tc_slot_bytes(cap, kb, 128, kc));
  };
  if (tc && (double)slot_of(kc_cap) * grid > KC_BUDGET_BYTES) kc_cap = 0;
  const size_t slot = tc ? slot_of(kc_cap) : 0;
  // workspace: offsets, pair list, queue/error/counters, per-pair counters,
  // tensor-core scratch slots, then the buffers of the large pairs
  Carve C(nullptr);
  C.take<int64_t>(num_pairs + 1);
  C.take<int64_t>(num_pairs + 1);
  C.take<int>(small.size() + 1);
  C.take<unsigned long long>(6);
  C.take<long long>(num_pairs);
  C.take<long long>(num_pairs);
  C.take<uint8_t>(tc ? slot * grid : 0);
  // flow records of the d > 8 solvers, one slice per CTA (the tensor-core
  // kernel's grid; the 1,024- and the 256-thread FP32 kernels' grids)
  const long long fl_big = tc ? 2LL * cap : 2LL * FIN_MAX_HD, fl_small = 2LL * HD_SMALL_CAP;
  const size_t fl_n = d <= 8 || small.empty() ? 0 : (size_t)(nsm * fl_big + (tc ? 0 : nsm * 4 * fl_small));
  C.take<int32_t>(fl_n);
  C.take<int32_t>(fl_n);
  C.take<double>(fl_n);
  const size_t head = (C.off + 511) & ~(size_t)255;  // keeps the solve buffers 256-byte aligned
  size_t bytes = head;
  int64_t maxm = 0, maxn = 0;
  for (int p : large) {
    maxm = std::max(maxm, x_off[p + 1] - x_off[p]);
    maxn = std::max(maxn, y_len(p));
  }
  SolveBufs B{};
  if (!large.empty()) bytes += layout_solve(nullptr, maxm, maxn, d, B, precision);
  if ((rc = ensure_ws(ctx, bytes))) return rc;
  Carve W(ctx->ws);
  int64_t* xo_d = W.take<int64_t>(num_pairs + 1);
  int64_t* yo_d = W.take<int64_t>(num_pairs + 1);
  int* ids_d = W.take<int>(small.size() + 1);
  // [0]: queue | err << 32, [1] certified, [2] fallbacks, [3] the 256-thread
  // kernel's queue, [4] near-ties
  unsigned long long* ctr_d = W.take<unsigned long long>(6);
  long long* rounds_d = W.take<long long>(num_pairs);
  long long* pe_d = W.take<long long>(num_pairs);
  uint8_t* scratch = W.take<uint8_t>(tc ? slot * grid : 0);
  int32_t* fl_i = W.take<int32_t>(fl_n);
  int32_t* fl_j = W.take<int32_t>(fl_n);
  double* fl_f = W.take<double>(fl_n);
  unsigned* q_d = reinterpret_cast<unsigned*>(ctr_d);
  unsigned* q2_d = reinterpret_cast<unsigned*>(ctr_d + 3);  // queue of the 256-thread kernel
  CK(cudaMemcpyAsync(xo_d, x_off, (num_pairs + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  if (y_off) CK(cudaMemcpyAsync(yo_d, y_off, (num_pairs + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  if (!small.empty())
    CK(cudaMemcpyAsync(ids_d, small.data(), small.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  long long L = 0;
  // the device work of the small pairs: clear the counters, one persistent launch
  auto issue = [&](cudaStream_t s, int nsmall, int g, int tbn, int tns, long long tkc) -> int {
    if (cudaMemsetAsync(ctr_d, 0, 6 * sizeof(unsigned long long), s) != cudaSuccess) return -1;
    if (cudaMemsetAsync(rounds_d, 0, num_pairs * sizeof(long long), s) != cudaSuccess) return -1;
    if (cudaMemsetAsync(pe_d, 0, num_pairs * sizeof(long long), s) != cudaSuccess) return -1;
    BatchArgs A{x_packed, a_packed, xo_d, y_packed, b_packed, yo_d, ids_d, nsmall, d, metric,
                costs_out, rounds_d, pe_d, q_d, q_d + 1, opt ? opt->protocol : 0, opt ? opt->seed : 0ULL,
                y_off ? 0 : (int)n_shared};
    if (fl_n) {
      A.fl_i = fl_i;
      A.fl_j = fl_j;
      A.fl_f = fl_f;
      A.fl_cap = fl_big;
    }
    if (tc)  // (grid <= one CTA per SM)
      return launch_batched_tc(A, precision, cap, kb, tbn, tns, scratch, slot, ctr_d + 1, ctr_d + 2, ctr_d + 4,
                               opt ? opt->rerank_k : 0, tkc, g, s);
    if (d <= 8) return launch_batched_lowd(A, g, s);
    int r = 0;
    const int nbig = nsmall - ntiny;
    if (nbig > 0) {
      BatchArgs Ab = A;
      Ab.pair_ids = ids_d + ntiny;
      Ab.num = nbig;
      r |= launch_batched_hd(Ab, std::min(nbig, nsm), s);
    }
    if (ntiny > 0) {
      BatchArgs At = A;
      At.num = ntiny;
      At.queue = q2_d;
      if (fl_n) {  // the slices after the 1,024-thread kernel's
        At.fl_i = fl_i + nsm * fl_big;
        At.fl_j = fl_j + nsm * fl_big;
        At.fl_f = fl_f + nsm * fl_big;
        At.fl_cap = fl_small;
      }
      r |= launch_batched_hd_small(At, std::min(ntiny, nsm * 4), s);
    }
    return r;
  };
  if (!small.empty() && tc && (flags & NNSEMD_FLAG_AUTOTUNE) && !ctx->tuned.count(tkey)) {
    // time every feasible (tile rows, stages, cache on / off) on a sample of the batch
    const int nsample = (int)std::min<size_t>(small.size(), 2 * (size_t)nsm);
    const int gs = std::min(nsample, nsm);
    if (!ctx->ev[0])
      for (int k = 0; k < 4; ++k) CK(cudaEventCreate(&ctx->ev[k]));
    float best_ms = 1e30f;
    std::tuple<int, int, int> best{bn, nstage, kc_use};
    for (int tkc = kc_cap ? 1 : 0; tkc >= 0; --tkc)
      for (int tbn : {64, 128}) {
        if (tbn == 128 && kb > 384) continue;
        const int maxs = batched_tc_max_stages(cap, kb, tbn, precision);
        for (int tns = 1; tns <= maxs; ++tns) {
          if (issue(st, nsample, gs, tbn, tns, tkc ? kc_cap : 0))
            return fail(ctx, NNSEMD_ERR_CUDA, "autotune launch");
          CK(cudaEventRecord(ctx->ev[0], st));
          if (issue(st, nsample, gs, tbn, tns, tkc ? kc_cap : 0))
            return fail(ctx, NNSEMD_ERR_CUDA, "autotune launch");
          CK(cudaEventRecord(ctx->ev[1], st));
          CK(cudaEventSynchronize(ctx->ev[1]));
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]));
          if (ms < best_ms) {
            best_ms = ms;
            best = {tbn, tns, tkc};
          }
          L += 2;
        }
      }
    ctx->tuned[tkey] = best;
    std::tie(bn, nstage, kc_use) = best;
  }
  if (!kc_use) kc_cap = 0;
  if (!small.empty()) {
    int brc = 0;
    if (flags & NNSEMD_FLAG_GRAPH) {
      const std::vector<uintptr_t> key = {(uintptr_t)x_packed, (uintptr_t)a_packed, (uintptr_t)y_packed,
                                          (uintptr_t)b_packed, (uintptr_t)costs_out, (uintptr_t)ctx->ws,
                                          (uintptr_t)num_pairs, (uintptr_t)small.size(), (uintptr_t)d,
                                          (uintptr_t)metric, (uintptr_t)precision, (uintptr_t)cap, (uintptr_t)bn,
                                          (uintptr_t)nstage, (uintptr_t)ntiny, (uintptr_t)kc_cap,
                                          (uintptr_t)(opt ? opt->protocol : 0), (uintptr_t)(opt ? opt->seed : 0),
                                          (uintptr_t)(opt ? opt->rerank_k : 0),
                                          (uintptr_t)(y_off ? 0 : n_shared)};
      BatchGraph* g = nullptr;
      for (auto& e : ctx->graphs)
        if (e.key == key) g = &e;
      if (!g) {
        if (!ctx->capture_stream) CK(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
        brc = issue(ctx->capture_stream, (int)small.size(), grid, bn, nstage, kc_cap);
        cudaError_t ce = cudaStreamEndCapture(ctx->capture_stream, &graph);
        if (brc || ce != cudaSuccess) {
          if (graph) cudaGraphDestroy(graph);
          return fail(ctx, NNSEMD_ERR_CUDA, "graph capture of the batched launch failed");
        }
        cudaGraphExec_t exec = nullptr;
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaGraphInstantiate");
        ctx->graphs.push_back({key, exec});
        g = &ctx->graphs.back();
      }
      CK(cudaGraphLaunch(g->exec, st));
    } else {
      brc = issue(st, (int)small.size(), grid, bn, nstage, kc_cap);
    }
    if (brc) return fail(ctx, NNSEMD_ERR_CUDA, "batched launch (%d)", brc);
    CK(cudaGetLastError());
    L += 1;
  }
  long long extra_rounds = 0, extra_pe = 0;
  long long extra_cert = 0, extra_fall = 0, extra_near = 0;
  for (int p : large) {
    layout_solve((char*)ctx->ws + head, maxm, maxn, d, B, precision);
    B.x = x_packed + x_off[p] * d;
    B.y = y_packed + y_begin(p) * d;
    B.m = x_off[p + 1] - x_off[p];
    B.n = y_len(p);
    B.d = d;
    B.dp = packed_dim(d);
    B.metric = metric;
    B.protocol = opt ? opt->protocol : 0;
    B.seed = opt ? opt->seed : 0;
    B.tc.rerank_k = opt ? opt->rerank_k : 0;
    double cost = 0;
    int64_t nnz = 0;
    nnsemd_stats s1{};
    rc = run_solve(ctx, B, a_packed + x_off[p], b_packed + y_begin(p), &cost, &nnz, &s1);
    if (rc) return rc;
    CK(cudaMemcpyAsync(costs_out + p, &B.st->cost, sizeof(double), cudaMemcpyDeviceToDevice, st));
    extra_rounds += s1.rounds;
    extra_pe += s1.pair_evals;
    extra_cert += s1.certified;
    extra_fall += s1.fallbacks;
    extra_near += s1.near_ties;
    L += s1.kernel_launches;
  }
  ctx->launches += L;
  if (stats) {
    unsigned long long ctr[6] = {0, 0, 0, 0, 0, 0};
    std::vector<long long> r(num_pairs), pe(num_pairs);
    CK(cudaMemcpyAsync(ctr, ctr_d, sizeof(ctr), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(r.data(), rounds_d, num_pairs * sizeof(long long), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(pe.data(), pe_d, num_pairs * sizeof(long long), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if ((rc = map_err_bits(ctx, (unsigned)(ctr[0] >> 32)))) return rc;
    std::memset(stats, 0, sizeof(*stats));
    for (int p : small) {
      stats->rounds += r[p];
      stats->pair_evals += pe[p];
    }
    stats->rounds += extra_rounds;
    stats->pair_evals += extra_pe;
    stats->certified = (int64_t)ctr[1] + extra_cert;
    stats->fallbacks = (int64_t)ctr[2] + extra_fall;
    stats->near_ties = (int64_t)ctr[4] + extra_near;
    stats->kernel_launches = L;
  }
  return NNSEMD_OK;
}

int nnsemd_solve_batched(nnsemd_ctx* ctx, int32_t num_pairs, const float* x_packed, const double* a_packed,
                         const int64_t* x_off, const float* y_packed, const double* b_packed, const int64_t* y_off,
                         int32_t d, const nnsemd_options* opt, double* costs_out, nnsemd_stats* stats) {
  if (ctx && !y_off) {
    ctx->err.clear();
    return fail(ctx, NNSEMD_ERR_INVALID_ARG, "null pointer argument");
  }
  return solve_batched_impl(ctx, num_pairs, x_packed, a_packed, x_off, y_packed, b_packed, y_off, 0, d, opt,
                            costs_out, stats);
}

int nnsemd_solve_one_to_many(nnsemd_ctx* ctx, int32_t num_pairs, const float* x_packed, const double* a_packed,
                             const int64_t* x_off, const float* y, const double* b, int64_t n, int32_t d,
                             const nnsemd_options* opt, double* costs_out, nnsemd_stats* stats) {
  if (ctx && n < 1) {
    ctx->err.clear();
    return fail(ctx, NNSEMD_ERR_INVALID_ARG, "the shared consumer set is empty (n=%lld)", (long long)n);
  }
  return solve_batched_impl(ctx, num_pairs, x_packed, a_packed, x_off, y, b, nullptr, n, d, opt, costs_out, stats);
}

const char* nnsemd_last_error(const nnsemd_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

const char* nnsemd_status_string(int status) {
  switch (status) {
    case NNSEMD_OK: return "NNSEMD_OK";
    case NNSEMD_ERR_INVALID_ARG: return "NNSEMD_ERR_INVALID_ARG";
    case NNSEMD_ERR_NONFINITE: return "NNSEMD_ERR_NONFINITE";
    case NNSEMD_ERR_ZERO_MASS: return "NNSEMD_ERR_ZERO_MASS";
    case NNSEMD_ERR_CUDA: return "NNSEMD_ERR_CUDA";
    case NNSEMD_ERR_OOM: return "NNSEMD_ERR_OOM";
    case NNSEMD_ERR_TIMEOUT: return "NNSEMD_ERR_TIMEOUT";
    case NNSEMD_ERR_ITER_LIMIT: return "NNSEMD_ERR_ITER_LIMIT";
    case NNSEMD_ERR_UNSUPPORTED: return "NNSEMD_ERR_UNSUPPORTED";
    case NNSEMD_ERR_CAPACITY: return "NNSEMD_ERR_CAPACITY";
    default: return "NNSEMD_ERR_UNKNOWN";
  }
}

int nnsemd_abi_version(void) { return NNSEMD_ABI_VERSION; }

}  // extern "C"
