/*
 * nnsemd.h -- C ABI of the GB300 (sm_103a) NNS-EMD solver.
 *
 * NNS-EMD approximates the Earth Mover's Distance between two weighted point
 * sets (Sec. II-A, Eq. objective/inflow/outflow): suppliers S (points x_i,
 * weights a_i, i < m) and consumers C (points y_j, weights b_j, j < n).  The
 * solver runs the paper's Algorithm 1 (Sec. III-A, greedy protocol) in
 * rounds until one side has no mass left:
 *   1. every active consumer finds its nearest active supplier (NNS op.);
 *   2. each supplier serves the consumers that picked it in ascending
 *      distance, moving f = min(s_i, c_j) until s_i is spent (greedy
 *      protocol), and the transport cost f * D_ij is accumulated;
 *   3. points whose residual weight is exactly 0 retire (weights update).
 * It returns R = sum f * D_ij and, optionally, the sparse plan F*.
 *
 * Conventions fixed by this library (the paper leaves them open):
 *  - Weights are normalised to unit mass (Sec. II-A) by dividing each by the
 *    correctly rounded sum of its side.  Zero weights are allowed (the point
 *    never takes part); negative or non-finite weights are errors, and so
 *    is a non-finite coordinate of any point, whatever its weight.
 *  - Argmin ties go to the lowest supplier index, greedy-order ties to the
 *    lowest consumer index.
 *  - Metric NNSEMD_L2 (Euclidean, the paper's choice) and NNSEMD_SQL2 order
 *    candidates by the squared distance; NNSEMD_L1 by the L1 sum.  The cost
 *    uses the metric itself (sqrt for L2), evaluated in FP64.
 *  - Decisions (argmin, greedy order) are taken on FP32 distances computed
 *    by direct differences in a fixed order: t_k = x_k - y_k (FP32),
 *    acc = t_0*t_0, acc = fma(t_k, t_k, acc) for k = 1..d-1 (L1: the
 *    running FP32 sum of |t_k|).  Mass bookkeeping is FP64 and sequential
 *    per supplier exactly as in Algorithm 1.  R is the correctly rounded sum
 *    of the per-flow FP64 terms f * D_ij.
 *  - Reduced precision (BF16/FP16/FP8) only proposes candidates; the final
 *    choice is re-ranked in FP32 and certified, so results equal the FP32
 *    path's (uncertified consumers fall back to the FP32 scan).
 *
 * Memory: every array argument is caller-owned.  Pointers are DEVICE
 * pointers unless the name or comment says host.  The context owns only its
 * workspace (grown on demand, freed by nnsemd_destroy).  Coordinates are
 * float32 row-major [points][d] (4-byte aligned); weights are float64
 * (8-byte aligned).
 *
 * Errors: every function returns an nnsemd_status; nothing throws across
 * the ABI.  nnsemd_last_error(ctx) gives a message for the last failure on
 * that context.  A context is not thread-safe: use one per host thread.
 */
#ifndef NNSEMD_H
#define NNSEMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NNSEMD_ABI_VERSION 4

typedef enum {
  NNSEMD_OK = 0,
  NNSEMD_ERR_INVALID_ARG = 1,  /* bad size, pointer, alignment or option */
  NNSEMD_ERR_NONFINITE = 2,    /* a coordinate or weight is NaN or Inf */
  NNSEMD_ERR_ZERO_MASS = 3,    /* a side's weights sum to zero, or a weight is negative */
  NNSEMD_ERR_CUDA = 4,         /* a CUDA runtime call failed */
  NNSEMD_ERR_OOM = 5,          /* the workspace could not be allocated */
  NNSEMD_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up */
  NNSEMD_ERR_ITER_LIMIT = 7,   /* more than m + n rounds (cannot happen unless corrupted) */
  NNSEMD_ERR_UNSUPPORTED = 8,  /* d or a size beyond what the chosen path serves */
  NNSEMD_ERR_CAPACITY = 9      /* the caller's plan arrays are too small */
} nnsemd_status;

typedef enum { NNSEMD_L2 = 0, NNSEMD_SQL2 = 1, NNSEMD_L1 = 2 } nnsemd_metric;

typedef enum {
  NNSEMD_FP32 = 0,  /* direct-difference FP32 distances on CUDA cores (d <= 8) or tiles (d > 8) */
  NNSEMD_BF16 = 1,  /* tcgen05 BF16 contraction proposes candidates, FP32 re-rank decides */
  NNSEMD_FP16 = 2,  /* the same with FP16 operands */
  NNSEMD_FP8 = 3,   /* the same with E4M3 operands and a per-row scale */
  NNSEMD_BF16X3 = 4 /* BF16 split: each coordinate as a high part h = bf16(v) and a low part
                       l = bf16(v - h); one BF16 contraction of length 3d gives
                       <h(x),h(y)> + <l(x),h(y)> + <h(x),l(y)>, within about 3 * 2^-16 |x||y| of
                       <x,y> (a single BF16 copy: about 2^-7 |x||y|), so far more candidates are
                       certified; three times the tensor work; served for d up to 128 */
} nnsemd_precision;

typedef struct nnsemd_ctx nnsemd_ctx;

#define NNSEMD_MAX_RERANK_K 16

typedef struct {
  int32_t device;               /* CUDA device ordinal */
  void *stream;                 /* cudaStream_t the context launches on; NULL = default stream */
  size_t workspace_bytes_hint;  /* preallocate this much workspace (0 = on demand) */
} nnsemd_config;

/* nnsemd_options.flags bits */
#define NNSEMD_FLAG_TIME_KERNELS 1  /* time the NNS and tail kernels with CUDA events (fills the *_ms stats) */
#define NNSEMD_FLAG_AUTOTUNE 2      /* nnsemd_solve_batched: time the candidate tile shapes on a sample of the
                                       batch the first time a (d, precision, size) class is seen; the winner
                                       is kept in the context for later calls */
#define NNSEMD_FLAG_GRAPH 4         /* nnsemd_solve_batched: capture the device work of the call in a CUDA
                                       graph and replay it while the buffers and sizes repeat */

/* How a supplier serves the consumers that picked it (Sec. III-A):
 * GREEDY (the paper's default, Alg. 1) in ascending distance, equal
 * distances by ascending consumer index; RANDOM in a seeded random order:
 * ascending 32-bit key, the upper half of SplitMix64 (Steele, Lea and Flood
 * 2014) output number c + 1 of the generator seeded with options.seed, for
 * the counter c = (round << 32) | consumer index (rounds counted from 0,
 * original consumer indices), equal keys by ascending consumer index. */
typedef enum { NNSEMD_PROTOCOL_GREEDY = 0, NNSEMD_PROTOCOL_RANDOM = 1 } nnsemd_protocol;

typedef struct {
  int32_t metric;               /* nnsemd_metric */
  int32_t precision;            /* nnsemd_precision */
  int32_t rerank_k;             /* reduced precision: approximate candidates per consumer re-ranked with the
                                   exact FP32 key, 0..NNSEMD_MAX_RERANK_K (0 = all the scan keeps: 16 per
                                   supplier chunk in nnsemd_solve, 8 per pair in the batched kernel, which
                                   also caps larger values at 8; with 1..8 the nnsemd_solve scan keeps
                                   8 per chunk, half the list upkeep).  Fewer candidates make the scan
                                   and the re-rank cheaper and the certificate weaker (more FP32
                                   rescans); results never change.  Outside the range: INVALID_ARG. */
  int32_t flags;                /* NNSEMD_FLAG_* bits, 0 for none */
  const void *proposal;         /* learned candidate proposal, NULL = full scan */
  int32_t protocol;             /* nnsemd_protocol (0 = greedy) */
  int32_t reserved;             /* must be 0 */
  uint64_t seed;                /* random protocol: generator seed */
} nnsemd_options;

typedef struct {
  int64_t capacity;             /* in: entries i, j, f can hold; m + n - 1 always suffices */
  int64_t nnz;                  /* out: entries written (order unspecified, (i, j) unique) */
  int32_t *i;                   /* supplier index of each flow */
  int32_t *j;                   /* consumer index of each flow */
  double *f;                    /* flow amount (normalised mass) */
} nnsemd_plan;

typedef struct {
  int64_t rounds;               /* NNS rounds run (Alg. 1 iterations); batched: summed over pairs */
  int64_t pair_evals;           /* sum over rounds of m_t * n_t (the paper's NNS work, Thm. 3) */
  double leftover_mass;         /* residual mass left on both sides (rounding only) */
  int64_t certified;            /* reduced precision: consumer searches settled by the re-rank */
  int64_t fallbacks;            /* reduced precision: consumer searches redone by the FP32 scan */
  int64_t kernel_launches;      /* CUDA kernels this call launched */
  double nns_kernel_ms;         /* NNSEMD_FLAG_TIME_KERNELS: summed duration of the multi-CTA NNS launches */
  int64_t nns_kernel_launches;  /* number of those launches */
  int64_t nns_kernel_pairs;     /* sum of m_t * n_t they evaluated */
  double tail_kernel_ms;        /* NNSEMD_FLAG_TIME_KERNELS: duration of the one-CTA tail kernel */
  int64_t near_ties;            /* reduced precision: consumer searches whose exact FP32 re-rank picked
                                   another supplier than the one the operand-precision distances ranked
                                   first (ties at that precision).  0 on the FP32 paths: their decisions
                                   are the FP32 decisions themselves (the FP32 / FP64 near-ties of the
                                   method are the oracle's to count). */
  int64_t widened;              /* learned proposal: consumer searches certified by the second tier (the
                                   cells of the bound list beyond the proposed candidates, in bound order);
                                   included in `certified`.  certified - widened is what the proposal's
                                   own candidates certified. */
} nnsemd_stats;

/* Create a context bound to cfg->device and cfg->stream.  *out receives the
 * handle (NULL on failure).  cfg may be NULL (device 0, default stream). */
int nnsemd_create(nnsemd_ctx **out, const nnsemd_config *cfg);

/* Free the context and its workspace.  Waits for its stream.  NULL is a no-op. */
int nnsemd_destroy(nnsemd_ctx *ctx);

/* Re-bind the context to another stream of the same device. */
int nnsemd_set_stream(nnsemd_ctx *ctx, void *stream);

/* Solve one pair (Alg. 1, Sec. III-A).
 *   x [m][d], a [m]: suppliers S (device); y [n][d], b [n]: consumers C (device).
 *   1 <= d; d <= 8 runs on CUDA cores, larger d on the tiled / tensor-core path.
 *   cost_out: HOST pointer receiving R; the call returns when R is known.
 *   plan (nullable): device arrays i/j/f of plan->capacity entries; plan->nnz set.
 *   stats (nullable, host): filled on return.
 * Errors: INVALID_ARG (sizes, null or misaligned pointers, bad options),
 * NONFINITE, ZERO_MASS, CAPACITY, UNSUPPORTED, CUDA, OOM, TIMEOUT. */
int nnsemd_solve(nnsemd_ctx *ctx,
                 const float *x, const double *a, int64_t m,
                 const float *y, const double *b, int64_t n,
                 int32_t d, const nnsemd_options *opt,
                 double *cost_out, nnsemd_plan *plan, nnsemd_stats *stats);

/* The same solve from HOST buffers: x, a, y, b and the plan arrays are host
 * memory (pinned memory gives the fastest copies).  The inputs are copied to
 * the context's device workspace, solved, and the plan copied back. */
int nnsemd_solve_host(nnsemd_ctx *ctx,
                      const float *x, const double *a, int64_t m,
                      const float *y, const double *b, int64_t n,
                      int32_t d, const nnsemd_options *opt,
                      double *cost_out, nnsemd_plan *plan, nnsemd_stats *stats);

/* Solve P independent pairs packed back to back (Sec. III-D, batch
 * processing).  Pair p's suppliers are rows x_off[p] .. x_off[p+1]-1 of
 * x_packed / a_packed, its consumers rows y_off[p] .. y_off[p+1]-1 of
 * y_packed / b_packed.  x_off and y_off are HOST arrays of P+1 entries
 * starting at 0; every pair needs >= 1 point on each side.  costs_out is a
 * DEVICE array of P doubles.  The call is asynchronous on the context's
 * stream unless stats is non-NULL (then it waits to fill stats). */
int nnsemd_solve_batched(nnsemd_ctx *ctx, int32_t num_pairs,
                         const float *x_packed, const double *a_packed, const int64_t *x_off,
                         const float *y_packed, const double *b_packed, const int64_t *y_off,
                         int32_t d, const nnsemd_options *opt,
                         double *costs_out, nnsemd_stats *stats);

/* ---- one histogram against many -----------------------------------------
 * The EMD-kNN primitive of the paper's classification and retrieval
 * experiments (Sec. IV-B, IV-C): one query histogram compared with every
 * histogram of a collection.  Pair p has suppliers x_packed rows
 * x_off[p] .. x_off[p+1]-1 (weights a_packed, device) and, as consumers, the
 * same n points y / b (device) for every p, which are stored once.  Offsets
 * are HOST arrays of P+1 entries starting at 0; costs_out is a DEVICE array
 * of P doubles.  Everything else (options, statistics, errors, the
 * asynchrony) is as for nnsemd_solve_batched, whose results it equals. */
int nnsemd_solve_one_to_many(nnsemd_ctx *ctx, int32_t num_pairs,
                             const float *x_packed, const double *a_packed, const int64_t *x_off,
                             const float *y, const double *b, int64_t n,
                             int32_t d, const nnsemd_options *opt,
                             double *costs_out, nnsemd_stats *stats);

/* ---- colour transfer (the application of Sec. IV-D) ---------------------
 * The pipeline: quantise both images' colours with nnsemd_kmeans, solve the
 * NNS-EMD between the palettes (reference palette = suppliers with the
 * cluster sizes as weights, source palette = consumers) with a plan, map
 * every source palette colour to the barycentre of the reference colours it
 * receives (nnsemd_barycentric), and recolour the source pixels
 * (nnsemd_recolour).  All pointers are device pointers; every step is
 * deterministic (exact sums), and the calls return when the work is done.
 * Coordinates must be finite and >= 0 (NONFINITE otherwise). */

/* k-means of pts [N][d] into k clusters: initial centroids are the points
 * at indices floor((2c+1) N / 2k); each of `iters` steps assigns every point
 * to its nearest centroid (the NNS operation's FP32 squared-distance key,
 * lowest index on ties) and sets each centroid coordinate to
 * float(correctly rounded sum of its points' coordinates / count) (a
 * centroid without points keeps its value); then a final assignment.
 * Outputs: centroids_out [k][d] float, labels_out [N] int32 (the final
 * assignment), counts_out [k] int64 (points per label).  Errors:
 * INVALID_ARG (k > N, sizes), NONFINITE, OOM, CUDA. */
int nnsemd_kmeans(nnsemd_ctx *ctx, const float *pts, int64_t N, int32_t d, int32_t k, int32_t iters,
                  float *centroids_out, int32_t *labels_out, int64_t *counts_out);

/* Barycentric map of a plan (device arrays plan->i / j / f, plan->nnz
 * entries, i into x [m][d], j into y [n][d]): y_out[j] = float(S_j / W_j),
 * S_j the correctly rounded sum over the flows into j of f * x_i (FP64
 * products), W_j the correctly rounded sum of their f; consumers without a
 * flow keep y[j].  Errors: INVALID_ARG, NONFINITE, OOM, CUDA. */
int nnsemd_barycentric(nnsemd_ctx *ctx, const nnsemd_plan *plan, const float *x, int64_t m, const float *y,
                       int64_t n, int32_t d, float *y_out);

/* out [N][d] = palette[labels[p]] ([k][d]).  Errors: INVALID_ARG (a label
 * outside [0, k)), CUDA. */
int nnsemd_recolour(nnsemd_ctx *ctx, const int32_t *labels, int64_t N, const float *palette, int32_t k,
                    int32_t d, float *out);

/* ---- the NNS operation alone --------------------------------------------
 * Round one of Alg. 1 (Sec. III-A, NNS step): for every consumer j, the
 * nearest supplier nn_out[j] (device int32 [n]), ties to the lowest index,
 * decided on the FP32 key of this header's conventions.  x [m][d], y [n][d]
 * device.  Used to build the training traces of the learned proposal. */
int nnsemd_nearest(nnsemd_ctx *ctx, const float *x, int64_t m, const float *y, int64_t n,
                   int32_t d, int32_t metric, int32_t *nn_out);

/* ---- learned candidate proposal ------------------------------------------
 * Not in the paper.  A fixed codebook of `cells` centroids (k-means) and an
 * MLP d -> hidden -> hidden -> cells (ReLU) that scores the cells most likely
 * to hold a consumer's nearest supplier.  Passed as nnsemd_options.proposal
 * to nnsemd_solve or nnsemd_solve_host (d > 8, metric L2 or SQL2), it
 * replaces the full NNS scan of every round by an exact FP32 scan of the
 * suppliers in each consumer's first 32 proposed non-empty cells, certified
 * by a triangle-inequality bound on every other non-empty cell; consumers
 * that cannot be certified are scanned in full: in FP32 (precision FP32) or
 * by the reduced-precision tensor-core scan with its own certificate and
 * FP32 rescan (precision BF16 / FP16 / FP8).  Results equal the FP32 path's;
 * stats.certified counts the searches settled by a certificate (proposal or
 * tensor-core), stats.fallbacks those rescanned in FP32.  Training runs on the GPU (Adam over
 * minibatches of the softmax cross-entropy, the label being the cell of the
 * consumer's nearest supplier).  All pointers are device pointers unless
 * stated.  Errors: INVALID_ARG, OOM, CUDA. */
typedef struct nnsemd_proposal nnsemd_proposal;

/* New proposal with seeded He-uniform weights (64 <= cells <= 8192). */
int nnsemd_proposal_create(nnsemd_ctx *ctx, int32_t d, int32_t cells, int32_t hidden, uint64_t seed,
                           nnsemd_proposal **out);
int nnsemd_proposal_destroy(nnsemd_proposal *p);
/* k-means (seeded picks, `iters` Lloyd steps) of pts [N][d] into the
 * codebook; also sets the network's input standardisation from pts. */
int nnsemd_proposal_fit(nnsemd_ctx *ctx, nnsemd_proposal *p, const float *pts, int64_t N, int32_t iters,
                        uint64_t seed);
/* Train on N consumer points y [N][d] whose nearest suppliers are x_nn
 * [N][d]; `epochs` passes of shuffled minibatches of `batch`, Adam with
 * learning rate lr.  *loss_out (host, nullable): mean loss of the last epoch. */
int nnsemd_proposal_train(nnsemd_ctx *ctx, nnsemd_proposal *p, const float *y, const float *x_nn, int64_t N,
                          int32_t epochs, int32_t batch, float lr, uint64_t seed, double *loss_out);
/* Mean softmax cross-entropy of N samples (y [N][d], labels [N] cell ids)
 * into *loss_out (host) and its gradient with respect to every parameter
 * into grad_out (device float [nparams], the layout of nnsemd_proposal_params). */
int nnsemd_proposal_loss_grad(nnsemd_ctx *ctx, const nnsemd_proposal *p, const float *y, const int32_t *labels,
                              int64_t N, double *loss_out, float *grad_out);
/* Shape of a proposal (host outputs, each nullable). */
int nnsemd_proposal_info(const nnsemd_proposal *p, int32_t *d, int32_t *cells, int32_t *hidden, int64_t *nparams);
/* Copy the parameters to (set = 0) or from (set = 1) the HOST buffer, laid
 * out as W1 [hidden][d], b1 [hidden], W2 [hidden][hidden], b2 [hidden],
 * W3 [cells][hidden], b3 [cells]. */
int nnsemd_proposal_params(nnsemd_ctx *ctx, nnsemd_proposal *p, float *host, int32_t set);
/* Checkpoint: a flat binary file (header, centroids, standardisation,
 * parameters). */
int nnsemd_proposal_save(nnsemd_ctx *ctx, const nnsemd_proposal *p, const char *path);
int nnsemd_proposal_load(nnsemd_ctx *ctx, const char *path, nnsemd_proposal **out);

/* Solve one small pair without allocating any memory.  The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc (a plugin
 * running inside another framework's launch callback, a process whose device
 * memory a caching allocator has already claimed, a latency-critical path
 * that cannot take cudaMalloc's implicit synchronisation).
 *   x [m][d], a [m], y [n][d], b [n]: device inputs as for nnsemd_solve;
 *   1 <= m, n <= NNSEMD_NOALLOC_MAX_POINTS, 1 <= d <= NNSEMD_NOALLOC_MAX_D,
 *   larger sizes return NNSEMD_ERR_UNSUPPORTED;
 *   metric: an nnsemd_metric;  cost_out: DEVICE pointer to one double (R);
 *   stream: cudaStream_t to launch on (NULL = default); the call copies an
 *   error word back and waits for the stream before it returns.
 * No context is needed.  Scratch (a few error and counter words) lives in a
 * 256-byte __device__ array of the library, held by every GPU that loads it
 * until the process exits; the kernel clears it at the start of each call.
 * The first call on a device does a one-time set-up with that device current:
 * it looks up the array's device address (cudaGetSymbolAddress) and sets the
 * kernel's shared-memory limit.  All calls share the array, so calls that
 * overlap on the GPU race: serialise them.  R equals nnsemd_solve's. */
#define NNSEMD_NOALLOC_MAX_POINTS 1024
#define NNSEMD_NOALLOC_MAX_D 8
int nnsemd_solve_small_noalloc(const float *x, const double *a, int64_t m,
                               const float *y, const double *b, int64_t n,
                               int32_t d, int32_t metric, double *cost_out, void *stream);

/* Message for the last failure on ctx (never NULL; "" after success).  The
 * string stays valid until the next call on ctx.  ctx may be NULL for
 * failures of nnsemd_create. */
const char *nnsemd_last_error(const nnsemd_ctx *ctx);

/* Static name of a status code. */
const char *nnsemd_status_string(int status);

/* NNSEMD_ABI_VERSION of the loaded library. */
int nnsemd_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NNSEMD_H */
