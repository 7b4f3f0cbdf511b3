// Host-side launchers of the NNS-EMD kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace nnsemd {

// Supplier tile staged in shared memory by K1, and the granularity every
// packed active list is padded to (with NaN coordinates) so that a tile
// never reads past its buffer.
constexpr int K1_TS = 256;
// Streaming multiprocessors of the current device (the device attribute
// cudaDevAttrMultiProcessorCount, looked up once per device); grids are
// sized in multiples of it.
int num_sms();
// K2 grid target (consumer tiles x supplier chunks): four CTAs per SM.
inline int tc_target_ctas() { return 4 * num_sms(); }
constexpr int PAD_POINTS = K1_TS;
// Largest active set the single-CTA solver keeps in shared memory (d <= 8:
// with coordinates; d > 8: per-point state only, coordinates stay in L2).
constexpr int FIN_MAX = 1024;
constexpr int FIN_MAX_HD = 2048;
// Point capacity per side of the cluster tail (d <= 8): its whole state,
// the coordinates at DP floats per point and the key exchange buffers fit
// one CTA's shared memory up to 2048 points for DP <= 4, 1024 for DP = 8.
constexpr int FIN_CL_MAX = 2048;
__host__ __device__ constexpr int fin_cl_cap(int dp) { return dp <= 4 ? FIN_CL_MAX : 1024; }

__host__ __device__ inline int padded_dim(int d) { return d <= 2 ? 2 : (d <= 4 ? 4 : 8); }
__host__ __device__ inline int64_t pad_points(int64_t n) { return (n + PAD_POINTS - 1) / PAD_POINTS * PAD_POINTS; }

// Buffers of the reduced-precision NNS step (tc.cu).
struct TcBufs {
  uint8_t* A;                  // packed consumer tiles
  uint8_t* B;                  // packed supplier tiles
  float* nrm_x;                // per supplier position (padded), +inf on padding
  float* nrm_sx;               // per supplier position: |x| rounded up, 0 on padding
  float* nrm_y;                // per consumer position
  float* scale_x;
  float* scale_y;
  unsigned* stats;             // [8]: supplier max |x|_2, |x|_1, scale; consumer the same at +4
  float* cand_v;               // [chunks][nt_pad][8]
  int* cand_p;
  int* fallback;               // consumer positions to rescan
  int* nfallback;              // device counter (this round)
  int max_chunks;
  int rerank_k;                // candidates per chunk re-ranked in FP32 (1..16; other values: 16)
  cudaEvent_t ev0, ev1;        // optional: recorded around the tensor-core kernel
};

// Buffers of one single-pair solve (device pointers inside the workspace).
struct SolveBufs {
  int precision;   // nnsemd_precision of the NNS step (0 = FP32)
  int protocol;    // nnsemd_protocol (0 greedy, 1 random)
  unsigned long long seed;  // random protocol seed
  long long round0;         // rounds run before the one-CTA tail (random-protocol keys)
  TcBufs tc;       // used when precision != 0
  const float* x;  // original coordinates [m][d]
  const float* y;  // [n][d]
  int64_t m, n;
  int d, dp, metric;
  double* s;       // residual supplier weights [m] (original index)
  double* c;       // residual consumer weights [n]
  float* xa[2];    // packed active supplier coordinates [pad(m)][dp]
  int* ia[2];      // their original indices
  float* ya[2];
  int* ja[2];
  int cur;         // which of the double buffers is current
  unsigned long long* nnkey;  // [n] per active consumer: key32 bits << 32 | supplier position
  int* cnt;        // [m] consumers per supplier position
  int2* seg;       // [m] (offset, length) of each supplier's group
  int* seglist;    // [m] non-empty groups
  int* biglist;    // [m] groups longer than a warp
  int* medlist;    // [m] groups of 9..32 consumers
  unsigned long long* member;  // [n] group members: key32 bits << 32 | consumer position
  int32_t* fl_i;   // [m+n] flow record of the one-CTA rounds (deferred costing)
  int32_t* fl_j;
  double* fl_f;
  int* blockcounts;            // compaction scratch
  unsigned long long* xs_acc;  // 4 exact-sum accumulators of XS_LIMBS limbs
  // Early notification of the active counts (nullable): the compaction's
  // count kernel writes {seq, m_t, n_t, error bits} of the round here (host
  // memory mapped into the device) as soon as the counts are known, before
  // the scatter that moves the points has run.
  volatile int* notify;
  int notify_seq;
  DevState* st;
  // caller's plan arrays (nullable) and capacity
  int32_t* plan_i;
  int32_t* plan_j;
  double* plan_f;
  int64_t plan_cap;
};

// rounds.cu ---------------------------------------------------------------
// After the last round: the cost terms and plan entries of every recorded
// flow, R into st->cost and the leftover mass into st->leftover.
void launch_leftover(const SolveBufs& B, cudaStream_t st);
// Exact totals of a and b and their normalisation into B.s / B.c (two
// launches; B.xs_acc cleared by the caller).
void launch_setup_sums(const SolveBufs& B, const double* a, const double* b, cudaStream_t st);
// Initial packing of both sides: active = positive weight, coordinates checked.
int launch_initial_pack(SolveBufs& B, cudaStream_t st);
// One multi-CTA round on the current active lists (mt, nt known on the host).
int launch_big_round(SolveBufs& B, int mt, int nt, long long round, cudaStream_t st);

// lowd.cu ------------------------------------------------------------------
int launch_nns_lowd(const SolveBufs& B, int mt, int nt, cudaStream_t st);
// Run all remaining rounds of the current active lists in one CTA.
int launch_finish(const SolveBufs& B, int64_t round_limit, cudaStream_t st);
// The same on a thread-block cluster (k_finish_cl), for active sets of at
// most finish_cluster_cap(d) points per side.  finish_cluster_cap returns 0
// when this device cannot co-schedule the cluster (the one-CTA tail serves).
int finish_cluster_cap(int d, int metric);
int launch_finish_cluster(const SolveBufs& B, int64_t round_limit, cudaStream_t st);
// A whole pair with m, n <= FIN_MAX and d <= 8 in one launch (writes st->cost,
// nnz, rounds, pair_evals, leftover and the plan).
int launch_solve_small(const SolveBufs& B, const double* a, const double* b, cudaStream_t st);

// Batched small pairs (all in one persistent launch), low d.
struct BatchArgs {
  const float* x; const double* a; const int64_t* x_off;
  const float* y; const double* b; const int64_t* y_off;
  const int* pair_ids;   // pairs handled by the CTA solver
  int num;               // number of entries in pair_ids
  int d, metric;
  double* costs;         // [P]
  long long* rounds;     // [P] rounds per pair (nullable)
  long long* pair_evals; // [P] (nullable)
  unsigned* queue;       // work-queue counter (device, zeroed)
  unsigned* err;
  int protocol;          // nnsemd_protocol
  unsigned long long seed;
  int n_shared;          // > 0: every pair's consumers are rows 0..n_shared-1 of y (y_off unused)
  // flow records (nullable): CTA b records a pair's flows in entries
  // [b fl_cap, (b + 1) fl_cap) and costs them once after the pair's last
  // round (d > 8 solvers)
  int32_t* fl_i;
  int32_t* fl_j;
  double* fl_f;
  long long fl_cap;
};
int launch_batched_lowd(const BatchArgs& A, int grid, cudaStream_t st);

// highd.cu (d > 8) ---------------------------------------------------------
// FP32 NNS over all active suppliers for the first `ncons` active consumers,
// or, with `cons`, for the consumer positions listed there (count in
// ncons_dev when given, else ncons).  Merges into B.nnkey with atomicMin.
int launch_nns_f32(const SolveBufs& B, int mt, int ncons, const int* cons, const int* ncons_dev, cudaStream_t st);
int launch_finish_hd(const SolveBufs& B, int64_t round_limit, cudaStream_t st);
int launch_batched_hd(const BatchArgs& A, int grid, cudaStream_t st);
// Batched FP32 solver for pairs of at most HD_SMALL_CAP points per side
// (d > 8), HD_SMALL_THREADS threads per pair, several pairs per SM.
constexpr int HD_SMALL_CAP = 512;
constexpr int HD_SMALL_THREADS = 256;
int launch_batched_hd_small(const BatchArgs& A, int grid, cudaStream_t st);
// All d coordinates of both sides finite (else EF_NONFINITE).
void launch_check_finite(const float* v, int64_t count, unsigned* err, cudaStream_t st);

// tc.cu (reduced precision, d > 8, squared-Euclidean order) ----------------
size_t tc_kb(int d, int precision);  // packed bytes per row
int tc_bn(size_t kb);                // supplier rows per tile
bool tc_supported(int d, int precision);  // the operand tiles of K2 fit its shared memory

// A BF16 linear layer on the tensor cores (tc.cu): Z [rows][N] = X W^T + b
// with FP32 accumulation, X [rows][K] and W [N][K] packed by
// pack_rows_bf16 into linear_tc_packed_bytes(rows, K) bytes each; K a
// multiple of 16 up to 256 (linear_tc_supported).  A wait that gives up
// sets EF_TIMEOUT in *err.
bool linear_tc_supported(int K);
size_t linear_tc_packed_bytes(int rows, int K);
int pack_rows_bf16(const float* src, int rows, int K, uint8_t* out, cudaStream_t st);
int linear_tc(const uint8_t* X, int rows, int K, const uint8_t* W, const float* bias, int N, float* Z, unsigned* err,
              cudaStream_t st);
// The same layer with ReLU, written as the next layer's packed X (BF16,
// tiles of 128 rows, padding rows zero; N a multiple of 16).
int linear_tc_pack_relu(const uint8_t* X, int rows, int K, const uint8_t* W, const float* bias, int N, uint8_t* out,
                        unsigned* err, cudaStream_t st);
// The same layer reduced per row: out[row] = the column of the row's largest
// value of X W^T + b (lowest column on ties); part holds rows x
// ceil(N / 128) partial keys.
int linear_tc_argmax(const uint8_t* X, int rows, int K, const uint8_t* W, const float* bias, int N,
                     unsigned long long* part, int* out, unsigned* err, cudaStream_t st);
// Lower bounds of the squared distance from each row y of [rows][d] to any
// point of each cell (centre mu_c, radius r_c): out[row][c] =
// max(0, |y - mu_c| - r_c)^2 with |y - mu_c| bounded from below through a
// BF16X3 contraction and its error bound, rounded toward the bound.  The
// cells are packed once (cell_bounds_tc_cells: packed into
// linear_tc_packed_bytes(cells, 3d) bytes, |mu|^2 down and |mu| up); the
// rows use scratch of linear_tc_packed_bytes(rows, 3d) bytes and 2 x rows
// floats.  d a multiple of 16 with 3d <= 256 (cell_bounds_tc_supported).
bool cell_bounds_tc_supported(int d);
int cell_bounds_tc_cells(const float* mu, int cells, int d, uint8_t* packed, float* sq_lo, float* nrm_up,
                         cudaStream_t st);
int cell_bounds_tc(const float* y, int rows, int d, uint8_t* packed_y, float* y_sq_lo, float* y_nrm_up,
                   const uint8_t* packed_mu, const float* mu_sq_lo, const float* mu_nrm_up, const float* radius,
                   int cells, float* out, unsigned* err, cudaStream_t st);
// NNS of every active consumer: tensor-core candidates, exact FP32 re-rank,
// certificate, FP32 rescan of the rest.  Writes B.nnkey (must be all ones).
int launch_nns_tc(const SolveBufs& B, const TcBufs& T, int mt, int nt, int precision, cudaStream_t st,
                  const int* sel = nullptr, const int* nsel_dev = nullptr);

// batched_tc.cu: batches of pairs with up to `cap` (512 or 2048) points per
// side, reduced-precision NNS inside each pair's CTA.
// kc_cap: entries of each CTA's distance cache (pairs with m * n <= kc_cap
// are answered from it after their first round; 0 turns it off).
size_t batched_tc_slot_bytes(int cap, int kb, int bn, long long kc_cap);
int batched_tc_max_stages(int cap, int kb, int bn, int precision);
// rerank_k: candidates re-ranked per consumer (1..8; other values: 8);
// certified / fallbacks / near_ties: device counters the launch adds to.
int launch_batched_tc(const BatchArgs& base, int precision, int cap, int kb, int bn, int nstage, uint8_t* scratch,
                      size_t slot_bytes, unsigned long long* certified, unsigned long long* fallbacks,
                      unsigned long long* near_ties, int rerank_k, long long kc_cap, int grid, cudaStream_t st);

}  // namespace nnsemd
