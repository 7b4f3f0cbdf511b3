// The learned candidate proposal (device side).  Not in the paper: the NNS
// operation of Alg. 1 (Sec. III-A) scans every active supplier; here a small
// network proposes a few cells of a fixed codebook that probably hold a
// consumer's nearest supplier, the suppliers of those cells are ranked with
// the exact FP32 key, and a cell lower bound certifies the choice (or the
// full scan runs).  Certified choices equal the full scan's.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

struct nnsemd_proposal {
  int d = 0;          // point dimension
  int cells = 0;      // codebook size (MLP outputs)
  int hidden = 0;     // MLP width
  float* centroids = nullptr;  // [cells][d]
  float* in_mean = nullptr;    // [d] input standardisation
  float* in_scale = nullptr;   // [d]
  // parameters, one buffer: W1 [hidden][d], b1 [hidden], W2 [hidden][hidden],
  // b2 [hidden], W3 [cells][hidden], b3 [cells]
  float* params = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  long long nparams = 0;
  long long adam_step = 0;
  bool codebook_ready = false;
  int device = 0;
  long long off_W1() const { return 0; }
  long long off_b1() const { return (long long)hidden * d; }
  long long off_W2() const { return off_b1() + hidden; }
  long long off_b2() const { return off_W2() + (long long)hidden * hidden; }
  long long off_W3() const { return off_b2() + hidden; }
  long long off_b3() const { return off_W3() + (long long)cells * hidden; }
};

namespace nnsemd {

constexpr int PROP_LIST = 64;  // cells kept per consumer (by score and by bound)
constexpr int PROP_TAKE = 32;  // non-empty proposed cells scanned per round
constexpr int PROP_MAX_CELLS = 8192;  // per-row selection keeps every cell's key in shared memory

// Per-solve buffers of the learned NNS step.
struct LearnedBufs {
  const nnsemd_proposal* P;
  int* cell_of_x;       // [m] cell of each supplier (original index)
  float* radius;        // [cells] max |x - mu_c| over the instance's suppliers (rounded up)
  int* prop_cells;      // [n][PROP_LIST] proposed cells of each consumer (original index), best first
  int* bound_cells;     // [n][PROP_LIST] cells by increasing lower bound
  float* bound_vals;    // [n][PROP_LIST] their lower bounds of the squared distance
  int* cell_cnt;        // [cells + 1] active suppliers per cell (this round)
  int* cell_off;        // [cells + 1]
  int* cell_fill;       // [cells]
  int* cell_members;    // [m] active supplier positions grouped by cell
  int* fallback;        // [n]
  int* nfallback;
  int* fallback2;       // [n] the consumers the second tier of the cell scan leaves
  int* nfallback2;
  // scratch for the per-solve passes
  float* tmp;           // [chunk][max(cells, hidden)] and friends
  float* tmp2;
  float* tmp3;
  int* sel_over;        // [chunk] rows the one-warp selection hands to the block selection
  int* nsel_over;
  // the cell-by-cell scan (learned.cu)
  int* lc_cand;         // [n][PROP_TAKE]
  int* lc_slot;         // [n][PROP_TAKE]
  int* lc_ncand;        // [n]
  float* lc_bound;      // [n]
  int* lc_qcnt;         // [cells]
  int* lc_qoff;         // [cells + 1]
  int* lc_work;         // [cells + 1]
  int* lc_nwork;         // [2]: work items, next work item
  int* lc_qlist;        // [n * PROP_TAKE]
  unsigned long long* lc_best;  // [n]
  uint8_t* w3p;         // the scoring layer's weights packed for linear_tc
  uint8_t* h2p;         // [chunk] hidden rows packed for linear_tc
  uint8_t* w1p;         // the two narrow layers' weights packed for linear_tc
  uint8_t* w2p;
  uint8_t* xp1;         // [chunk] standardised inputs packed
  uint8_t* h1p;         // [chunk] first hidden layer packed
  // the supplier-to-cell assignment on the tensor cores
  int assign_chunk;     // suppliers per pass
  uint8_t* mup;         // centroids packed for linear_tc
  float* mu_bias;       // [cells] -|mu_c|^2 / 2
  uint8_t* xp;          // [assign_chunk] supplier rows packed
  unsigned long long* apart;  // [assign_chunk][cells / 128] partial row maxima
  // the cell bounds on the tensor cores
  uint8_t* mup3;        // centroids packed as BF16X3 splits
  float* mu_sq_lo;      // [cells]
  float* mu_nrm_up;     // [cells]
  uint8_t* yp3;         // [chunk] consumer rows packed as BF16X3 splits
  float* y_sq_lo;       // [chunk]
  float* y_nrm_up;      // [chunk]
  int chunk;            // consumers per pass
};

// Per-solve preparation: supplier cells and radii, consumer proposals and
// cell bounds (x, y original coordinates, d; m suppliers, n consumers).
int learned_prepare(const LearnedBufs& L, const float* x, int64_t m, const float* y, int64_t n, int d, unsigned* err,
                    cudaStream_t st);
// One round: CSR of active suppliers by cell, candidate scan + certificate,
// FP32 rescan of the rest.  Writes B.nnkey (all ones on entry).
int launch_nns_learned(const SolveBufs& B, const LearnedBufs& L, int mt, int nt, cudaStream_t st);
// Whether a round takes the cell-by-cell scan (d of 32, 64 or 128, 16-byte
// aligned coordinates; else one warp per consumer): 10 launches per round
// before any fallback, against 5.
bool learned_cell_scan(int d, const float* x, const float* y);

// Training / inference building blocks (learned.cu).
int mlp_forward(const nnsemd_proposal* P, const float* X, int rows, float* H1, float* H2, float* Z, cudaStream_t st);
// loss (host) and gradient of the mean softmax cross-entropy over `rows`
// samples with integer labels; grad has nparams entries (device).
int mlp_loss_grad(const nnsemd_proposal* P, const float* X, const int* labels, int rows, float* H1, float* H2,
                  float* Z, float* dbuf1, float* dbuf2, float* grad, double* loss_dev, cudaStream_t st);
void adam_update(nnsemd_proposal* P, const float* grad, float lr, cudaStream_t st);
// k-means (Lloyd) of pts [N][d] into P->cells centroids (seeded initial picks).
int kmeans_fit(nnsemd_proposal* P, const float* pts, int64_t N, int iters, uint64_t seed, int* assign_buf,
               float* sums, int* counts, cudaStream_t st);
// cell of each point (nearest centroid, FP32 direct differences)
int assign_cells(const nnsemd_proposal* P, const float* pts, int64_t N, int* out, cudaStream_t st);
// nearest supplier of every consumer (round one of Alg. 1), positions into x
int nearest_all(const float* x, int64_t m, const float* y, int64_t n, int d, int metric, int* iota_m,
                unsigned long long* keys, int* out, cudaStream_t st);

}  // namespace nnsemd
