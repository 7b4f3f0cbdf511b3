// The learned candidate proposal (not in the paper; see proposal.h).
//
// Training and inference of the proposal network run in the kernels below:
// a tiled FP32 GEMM with fused bias / ReLU / ReLU-mask epilogues for the
// forward and backward passes of a 3-layer MLP, a row-wise softmax
// cross-entropy, column sums for the bias gradients and an Adam step.  The
// codebook is fitted by Lloyd's k-means (assignment = a nearest-centroid
// search with the same tiled FP32 distance routine as the NNS operation).
//
// Per solve the network's scores give each consumer its 64 best cells, and a
// pass over the centroids gives it the 64 cells with the smallest lower
// bound max(0, |y - mu_c| - r_c)^2 on the squared distance to any supplier
// of the cell (r_c = the largest |x - mu_c| over the instance's suppliers in
// c; the triangle inequality makes it a bound).  Per round every active
// consumer scans, with the exact FP32 key, the active suppliers of its first
// 32 proposed cells that still hold any; the best key is certified when it
// is strictly below the bound of every other cell that still holds an active
// supplier (scaled by the key's own rounding bound), so no supplier outside
// the candidates can win or tie.  Uncertified consumers are scanned in full.
#include <math_constants.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "cta.cuh"
#include "kernels.h"
#include "proposal.h"

namespace nnsemd {

// --------------------------------------------------------------------------
// tiled FP32 GEMM: C[M][N] = sum_k A(m,k) B(k,n), with
//   A(m,k) = TA ? A[k*lda + m] : A[m*lda + k]
//   B(k,n) = TB ? B[n*ldb + k] : B[k*ldb + n]
// and an epilogue: none, +bias[n], relu(+bias[n]), or * (mask[m][n] > 0).
// --------------------------------------------------------------------------

enum Epi : int { EPI_NONE = 0, EPI_BIAS = 1, EPI_BIAS_RELU = 2, EPI_MASK = 3 };

constexpr int GM = 64, GN = 64, GK = 16, GT = 256;

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(GT) k_gemm(const float* __restrict__ A, int lda, const float* __restrict__ B,
                                             int ldb, float* __restrict__ C, int ldc, int M, int N, int K,
                                             const float* __restrict__ aux) {
  __shared__ float As[GK][GM + 4];
  __shared__ float Bs[GK][GN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * GM, n0 = blockIdx.x * GN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += GK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int idx = tid + i * GT;
      int mm, kk;
      if (TA) { kk = idx / GM; mm = idx % GM; } else { mm = idx / GK; kk = idx % GK; }
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < K) ? (TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k]) : 0.f;
      int nn, kb;
      if (TB) { nn = idx / GK; kb = idx % GK; } else { kb = idx / GN; nn = idx % GN; }
      const int n = n0 + nn, k2 = k0 + kb;
      Bs[kb][nn] = (n < N && k2 < K) ? (TB ? B[(size_t)n * ldb + k2] : B[(size_t)k2 * ldb + n]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      float v = acc[i][j];
      if (EPI == EPI_BIAS) v += aux[n];
      if (EPI == EPI_BIAS_RELU) v = fmaxf(v + aux[n], 0.f);
      if (EPI == EPI_MASK) v = aux[(size_t)m * ldc + n] > 0.f ? v : 0.f;
      C[(size_t)m * ldc + n] = v;
    }
  }
}

template <bool TA, bool TB, int EPI>
static void gemm(const float* A, int lda, const float* B, int ldb, float* C, int ldc, int M, int N, int K,
                 const float* aux, cudaStream_t st) {
  dim3 grid((N + GN - 1) / GN, (M + GM - 1) / GM);
  k_gemm<TA, TB, EPI><<<grid, GT, 0, st>>>(A, lda, B, ldb, C, ldc, M, N, K, aux);
}

// standardise rows: out = (x - mean) * scale
__global__ void k_standardise(const float* __restrict__ x, int rows, int d, const float* __restrict__ mean,
                              const float* __restrict__ scale, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)rows * d;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(i % d);
    out[i] = (x[i] - mean[k]) * scale[k];
  }
}

int mlp_forward(const nnsemd_proposal* P, const float* Xs, int rows, float* H1, float* H2, float* Z, cudaStream_t st) {
  const float* p = P->params;
  const int d = P->d, h = P->hidden, c = P->cells;
  gemm<false, true, EPI_BIAS_RELU>(Xs, d, p + P->off_W1(), d, H1, h, rows, h, d, p + P->off_b1(), st);
  gemm<false, true, EPI_BIAS_RELU>(H1, h, p + P->off_W2(), h, H2, h, rows, h, h, p + P->off_b2(), st);
  gemm<false, true, EPI_BIAS>(H2, h, p + P->off_W3(), h, Z, c, rows, c, h, p + P->off_b3(), st);
  return 0;
}

// Softmax cross-entropy per row; dZ = (softmax - onehot) / rows; the mean
// loss is added to *loss.
__global__ void k_softmax_xent(const float* __restrict__ Z, const int* __restrict__ labels, int rows, int cols,
                               float* __restrict__ dZ, double* loss) {
  __shared__ float red[32];
  const int r = blockIdx.x;
  const float* z = Z + (size_t)r * cols;
  float mx = -CUDART_INF_F;
  for (int c = threadIdx.x; c < cols; c += blockDim.x) mx = fmaxf(mx, z[c]);
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
  __syncthreads();
  float s = 0.f;
  for (int c = threadIdx.x; c < cols; c += blockDim.x) s += expf(z[c] - mx);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  float sum = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
  const int lab = labels[r];
  const float zl = z[lab];  // read before dZ (which may alias Z) is written
  __syncthreads();
  const float inv = 1.f / (float)rows;
  for (int c = threadIdx.x; c < cols; c += blockDim.x)
    dZ[(size_t)r * cols + c] = (expf(z[c] - mx) / sum - (c == lab ? 1.f : 0.f)) * inv;
  if (threadIdx.x == 0) atomicAdd(loss, ((double)logf(sum) + mx - zl) / rows);
}

// out[c] = sum over rows of M[row][c]
__global__ void k_colsum(const float* __restrict__ M, int rows, int cols, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += M[(size_t)r * cols + c];
  out[c] = s;
}

int mlp_loss_grad(const nnsemd_proposal* P, const float* Xs, const int* labels, int rows, float* H1, float* H2,
                  float* Z, float* dbuf1, float* dbuf2, float* grad, double* loss_dev, cudaStream_t st) {
  const float* p = P->params;
  const int d = P->d, h = P->hidden, c = P->cells;
  mlp_forward(P, Xs, rows, H1, H2, Z, st);
  // dZ in place of Z
  k_softmax_xent<<<rows, 256, 0, st>>>(Z, labels, rows, c, Z, loss_dev);
  float* g = grad;
  // layer 3: dW3 = dZ^T H2, db3 = colsum dZ, dH2 = (dZ W3) masked by H2
  gemm<true, false, EPI_NONE>(Z, c, H2, h, g + P->off_W3(), h, c, h, rows, nullptr, st);
  k_colsum<<<(c + 255) / 256, 256, 0, st>>>(Z, rows, c, g + P->off_b3());
  gemm<false, false, EPI_MASK>(Z, c, p + P->off_W3(), h, dbuf2, h, rows, h, c, H2, st);
  // layer 2
  gemm<true, false, EPI_NONE>(dbuf2, h, H1, h, g + P->off_W2(), h, h, h, rows, nullptr, st);
  k_colsum<<<(h + 255) / 256, 256, 0, st>>>(dbuf2, rows, h, g + P->off_b2());
  gemm<false, false, EPI_MASK>(dbuf2, h, p + P->off_W2(), h, dbuf1, h, rows, h, h, H1, st);
  // layer 1
  gemm<true, false, EPI_NONE>(dbuf1, h, Xs, d, g + P->off_W1(), d, h, d, rows, nullptr, st);
  k_colsum<<<(h + 255) / 256, 256, 0, st>>>(dbuf1, rows, h, g + P->off_b1());
  return 0;
}

__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, long long n, float lr, float b1, float b2, float c1, float c2,
                       float eps) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

void adam_update(nnsemd_proposal* P, const float* grad, float lr, cudaStream_t st) {
  P->adam_step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)P->adam_step), c2 = 1.f - powf(b2, (float)P->adam_step);
  k_adam<<<num_sms() * 8, 256, 0, st>>>(P->params, P->adam_m, P->adam_v, grad, P->nparams, lr, b1, b2, c1, c2, 1e-8f);
}

// --------------------------------------------------------------------------
// nearest neighbour over a whole set (k-means assignment, round one of
// Alg. 1 for training traces)
// --------------------------------------------------------------------------

template <bool L1>
__global__ void __launch_bounds__(TG_THREADS)
    k_nearest(const float* __restrict__ x, const int* __restrict__ iota, int m, int chunk,
              const float* __restrict__ y, int n, int d, unsigned long long* __restrict__ keys) {
  __shared__ TileSmem T;
  const int c0 = blockIdx.x * TG_M;
  const int p0 = blockIdx.y * chunk;
  const int p1 = min(p0 + chunk, m);
  if (c0 >= n || p0 >= p1) return;
  unsigned long long out[4];
  group_nns_tile<L1>(x, iota, p0, p1, y, iota, nullptr, c0, min(TG_M, n - c0), d, T, threadIdx.x, 0, out);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  if (tx == 0)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int q = c0 + ty * 4 + i;
      if (q < n) atomicMin(keys + q, out[i]);
    }
}

__global__ void k_iota(int* v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (int)i;
}

__global__ void k_keys_to_index(const unsigned long long* keys, int64_t n, int* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int)(keys[i] & 0xffffffffULL);
}

// `iota_m` must hold 0..max(m, n)-1.
int nearest_all(const float* x, int64_t m, const float* y, int64_t n, int d, int metric, int* iota_m,
                unsigned long long* keys, int* out, cudaStream_t st) {
  if (cudaMemsetAsync(keys, 0xff, n * sizeof(unsigned long long), st) != cudaSuccess) return -1;
  const int gx = (int)((n + TG_M - 1) / TG_M);
  int gy = (num_sms() * 6 + gx - 1) / gx;
  const int tiles = (int)((m + TG_N - 1) / TG_N);
  if (gy > tiles) gy = tiles;
  const int chunk = ((tiles + gy - 1) / gy) * TG_N;
  gy = (int)((m + chunk - 1) / chunk);
  dim3 grid(gx, gy);
  if (metric == METRIC_L1) k_nearest<true><<<grid, TG_THREADS, 0, st>>>(x, iota_m, (int)m, chunk, y, (int)n, d, keys);
  else k_nearest<false><<<grid, TG_THREADS, 0, st>>>(x, iota_m, (int)m, chunk, y, (int)n, d, keys);
  k_keys_to_index<<<std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, num_sms() * 8)), 256, 0, st>>>(keys, n, out);
  return 0;
}

// --------------------------------------------------------------------------
// k-means
// --------------------------------------------------------------------------

__global__ void k_km_accum(const float* __restrict__ pts, int64_t N, int d, const int* __restrict__ assign,
                           float* __restrict__ sums, int* __restrict__ counts) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N * d; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / d;
    const int k = (int)(i % d);
    const int c = assign[p];
    atomicAdd(sums + (size_t)c * d + k, pts[i]);
    if (k == 0) atomicAdd(counts + c, 1);
  }
}

__global__ void k_km_divide(float* __restrict__ cent, const float* __restrict__ sums, const int* __restrict__ counts,
                            int cells, int d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cells * d; i += gridDim.x * blockDim.x) {
    const int c = i / d;
    if (counts[c] > 0) cent[i] = sums[i] / (float)counts[c];
  }
}

__global__ void k_gather_rows(const float* __restrict__ src, const int* __restrict__ rows, int count, int d,
                              float* __restrict__ dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count * d; i += gridDim.x * blockDim.x)
    dst[i] = src[(size_t)rows[i / d] * d + (i % d)];
}

int assign_cells(const nnsemd_proposal* P, const float* pts, int64_t N, int* out, cudaStream_t st);

// iota / key scratch for the nearest-centroid search live at the end of the
// k-means scratch: assign_buf holds N ints, then N 64-bit keys follow the
// sums array (sized by the caller: cells*d floats + cells ints + N keys).
static int* g_dummy = nullptr;

int kmeans_fit(nnsemd_proposal* P, const float* pts, int64_t N, int iters, uint64_t seed, int* assign_buf,
               float* sums, int* counts, cudaStream_t st) {
  const int K = P->cells, d = P->d;
  if (N < K) return -1;
  // seeded distinct initial picks (partial Fisher-Yates on the host)
  std::vector<int> idx(N);
  for (int64_t i = 0; i < N; ++i) idx[i] = (int)i;
  uint64_t s = seed * 0x9E3779B97F4A7C15ULL + 1;
  for (int i = 0; i < K; ++i) {
    s ^= s >> 12; s ^= s << 25; s ^= s >> 27;
    const uint64_t r = (s * 0x2545F4914F6CDD1DULL) % (uint64_t)(N - i);
    std::swap(idx[i], idx[i + r]);
  }
  int* dpick = assign_buf;  // temporarily holds the K picks
  if (cudaMemcpyAsync(dpick, idx.data(), K * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess) return -1;
  k_gather_rows<<<(K * d + 255) / 256, 256, 0, st>>>(pts, dpick, K, d, P->centroids);
  if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
  for (int it = 0; it < iters; ++it) {
    if (assign_cells(P, pts, N, assign_buf, st)) return -1;
    cudaMemsetAsync(sums, 0, (size_t)K * d * sizeof(float), st);
    cudaMemsetAsync(counts, 0, (size_t)K * sizeof(int), st);
    k_km_accum<<<num_sms() * 8, 256, 0, st>>>(pts, N, d, assign_buf, sums, counts);
    k_km_divide<<<(K * d + 255) / 256, 256, 0, st>>>(P->centroids, sums, counts, K, d);
  }
  (void)g_dummy;
  return 0;
}

// The nearest centroid of every point.  Uses its own temporary buffers.
int assign_cells(const nnsemd_proposal* P, const float* pts, int64_t N, int* out, cudaStream_t st) {
  const int64_t big = std::max<int64_t>(N, P->cells);
  int* iota = nullptr;
  unsigned long long* keys = nullptr;
  if (cudaMallocAsync(&iota, big * sizeof(int), st) != cudaSuccess) return -1;
  if (cudaMallocAsync(&keys, N * sizeof(unsigned long long), st) != cudaSuccess) return -1;
  k_iota<<<num_sms() * 4, 256, 0, st>>>(iota, big);
  const int rc = nearest_all(P->centroids, P->cells, pts, N, P->d, METRIC_SQL2, iota, keys, out, st);
  cudaFreeAsync(iota, st);
  cudaFreeAsync(keys, st);
  return rc;
}

// --------------------------------------------------------------------------
// per-row top-K selection (K = PROP_LIST) by radix select on order-preserving
// 32-bit keys; output in descending key order, ties by ascending column
// --------------------------------------------------------------------------

NNS_DEV unsigned ordered_bits(float v) {
  const unsigned u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// LARGEST: keep the K largest values; otherwise the K smallest.  One block
// per row: a radix select over all of the row's keys.  With row_list /
// n_rows it serves the rows row_list[0 .. *n_rows) (blocks past the count
// leave at once): the rows the one-warp selection below hands over.
template <bool LARGEST>
__global__ void __launch_bounds__(256) k_select_rows(const float* __restrict__ V, int rows, int cols, int* __restrict__ out_idx,
                                                     float* __restrict__ out_val, int out_stride,
                                                     const int* __restrict__ row_list, const int* __restrict__ n_rows) {
  extern __shared__ unsigned sk[];  // cols keys
  __shared__ unsigned hist[256];
  __shared__ unsigned s_prefix, s_mask, s_need;
  __shared__ int s_cnt;
  __shared__ unsigned sel_key[PROP_LIST];
  __shared__ int sel_idx[PROP_LIST];
  if (row_list && (int)blockIdx.x >= *n_rows) return;
  const int r = row_list ? row_list[blockIdx.x] : blockIdx.x;
  const int tid = threadIdx.x;
  for (int c = tid; c < cols; c += blockDim.x) {
    const unsigned o = ordered_bits(V[(size_t)r * cols + c]);
    sk[c] = LARGEST ? o : ~o;
  }
  if (tid == 0) {
    s_prefix = 0u;
    s_mask = 0u;
    s_need = PROP_LIST;
    s_cnt = 0;
  }
  __syncthreads();
  // find the K-th largest key, 8 bits at a time from the top
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int i = tid; i < 256; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    const unsigned pre = s_prefix, msk = s_mask;
    for (int c = tid; c < cols; c += blockDim.x) {
      const unsigned k = sk[c];
      if ((k & msk) == pre) atomicAdd(&hist[(k >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    if (tid == 0) {
      unsigned need = s_need, acc = 0u;
      int dig = 255;
      for (; dig > 0; --dig) {
        if (acc + hist[dig] >= need) break;
        acc += hist[dig];
      }
      s_need = need - acc;
      s_prefix = pre | ((unsigned)dig << shift);
      s_mask = msk | (0xffu << shift);
    }
    __syncthreads();
  }
  const unsigned kth = s_prefix;  // the K-th largest key (exact)
  const unsigned need_eq = s_need;  // how many keys equal to kth to take (lowest columns first)
  // gather: keys > kth, then the first need_eq keys == kth in column order
  for (int c = tid; c < cols; c += blockDim.x) {
    if (sk[c] > kth) {
      const int slot = atomicAdd(&s_cnt, 1);
      sel_key[slot] = sk[c];
      sel_idx[slot] = c;
    }
  }
  __syncthreads();
  if (tid == 0) {
    unsigned taken = 0u;
    for (int c = 0; c < cols && taken < need_eq; ++c)
      if (sk[c] == kth) {
        sel_key[s_cnt] = kth;
        sel_idx[s_cnt] = c;
        ++s_cnt;
        ++taken;
      }
  }
  __syncthreads();
  // rank sort of the K selected (descending key, ascending column)
  if (tid < PROP_LIST) {
    const unsigned k = sel_key[tid];
    const int c = sel_idx[tid];
    int rank = 0;
    for (int u = 0; u < PROP_LIST; ++u) {
      const unsigned ku = sel_key[u];
      rank += (ku > k) || (ku == k && sel_idx[u] < c);
    }
    out_idx[(size_t)r * out_stride + rank] = c;
    if (out_val) out_val[(size_t)r * out_stride + rank] = V[(size_t)r * cols + c];
  }
}

constexpr int SEL_WARPS = 8;   // rows per block of the one-warp selection
constexpr int SEL_CAP = 256;   // candidates a warp keeps in shared memory

// The same selection (the PROP_LIST largest keys, lowest column first among
// equal keys, written in that order), one warp per row, with no atomics:
//  1. the row's columns fall into 64 groups (lane x half of the row); the
//     two largest keys of every group form a set S, and T is the 64th
//     largest key of S, so at least 64 keys of the row are >= T;
//  2. the keys > T are gathered; with fewer than 64 of
//     them, the first keys == T in column order complete the 64 (exactly
//     the selection's tie rule), else the 64 are among the gathered ones;
//  3. each gathered key's rank by (key descending, column ascending) places
//     the 64 first.
// A row with more than SEL_CAP keys > T is left to k_select_rows through
// over_rows / n_over.  Needs cols >= 2 * PROP_LIST.
template <bool LARGEST>
__global__ void __launch_bounds__(32 * SEL_WARPS, 4) k_select_rows_warp(const float* __restrict__ V, int rows, int cols,
                                                                   int* __restrict__ out_idx, float* __restrict__ out_val,
                                                                   int out_stride, int* __restrict__ over_rows,
                                                                   int* __restrict__ n_over) {
  __shared__ unsigned s_key[SEL_WARPS][4 * 32];
  __shared__ unsigned c_key[SEL_WARPS][SEL_CAP];
  __shared__ int c_col[SEL_WARPS][SEL_CAP];
  __shared__ int s_cnt[SEL_WARPS];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * SEL_WARPS + w;
  if (r >= rows) return;
  const float* row = V + (size_t)r * cols;
  auto key = [&](int c) -> unsigned {
    const unsigned o = ordered_bits(row[c]);
    return LARGEST ? o : ~o;
  };
  // 1. the two largest keys of each group (lane, half); every group holds
  // at least two columns (cols >= 128), so all 128 entries are real keys
  // (starting both at 0, the smallest key, gives the two largest of any
  // group of two or more keys).  Rows whose columns split into whole
  // 16-byte vectors per lane and half are read 16 bytes at a time (the
  // group of a lane is then its vectors in that half).
  const int half = cols / 2;
  const bool vec = (cols & 255) == 0 && (reinterpret_cast<uintptr_t>(row) & 15) == 0;
  auto top2 = [](unsigned k, unsigned& a1, unsigned& a2) {
    if (k > a1) {
      a2 = a1;
      a1 = k;
    } else if (k > a2) {
      a2 = k;
    }
  };
  for (int h = 0; h < 2; ++h) {
    unsigned a1 = 0u, a2 = 0u;
    if (vec) {
      const float4* r4 = reinterpret_cast<const float4*>(row);
      for (int f = h * (half / 4) + lane; f < (h + 1) * (half / 4); f += 32) {
        const float4 v = r4[f];
        const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const unsigned o = ordered_bits(e[u]);
          top2(LARGEST ? o : ~o, a1, a2);
        }
      }
    } else {
      for (int c = h * half + lane; c < (h ? cols : half); c += 32) top2(key(c), a1, a2);
    }
    s_key[w][h * 64 + lane] = a1;
    s_key[w][h * 64 + 32 + lane] = a2;
  }
  __syncwarp();
  // T: the largest key of S with at least 64 keys of S at or above it,
  // bit by bit from the top (the count of keys >= t only falls as t grows,
  // so the largest t that keeps it at 64 is the 64th largest key of S)
  const unsigned s0 = s_key[w][lane], s1 = s_key[w][32 + lane], s2 = s_key[w][64 + lane], s3 = s_key[w][96 + lane];
  unsigned T = 0u;
  for (int bit = 31; bit >= 0; --bit) {
    const unsigned t = T | (1u << bit);
    const unsigned ge = (s0 >= t) + (s1 >= t) + (s2 >= t) + (s3 >= t);
    if (__reduce_add_sync(0xffffffffu, ge) >= PROP_LIST) T = t;
  }
  // 2. keys > T (ranked in step 3, so their order here does not matter)
  int n = 0;
  if (vec) {
    // four consecutive columns per lane; the keys above T go to the list in
    // any order (step 3 ranks them by key and column), each lane taking
    // its places from a shared counter
    if (lane == 0) s_cnt[w] = 0;
    __syncwarp();
    const float4* r4 = reinterpret_cast<const float4*>(row);
    for (int f = lane; f < cols / 4; f += 32) {
      const float4 v = r4[f];
      const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const unsigned o = ordered_bits(e[u]);
        const unsigned k = LARGEST ? o : ~o;
        if (k > T) {
          const int pos = atomicAdd(&s_cnt[w], 1);
          if (pos < SEL_CAP) {
            c_key[w][pos] = k;
            c_col[w][pos] = 4 * f + u;
          }
        }
      }
    }
    __syncwarp();
    n = s_cnt[w];
  } else {
    for (int base = 0; base < cols; base += 32) {
      const int c = base + lane;
      const unsigned k = c < cols ? key(c) : 0u;
      const bool p = c < cols && k > T;
      const unsigned bal = __ballot_sync(0xffffffffu, p);
      const int pos = n + __popc(bal & ((1u << lane) - 1u));
      if (p && pos < SEL_CAP) {
        c_key[w][pos] = k;
        c_col[w][pos] = c;
      }
      n += __popc(bal);
    }
  }
  if (n > SEL_CAP) {
    if (lane == 0) over_rows[atomicAdd(n_over, 1)] = r;
    return;
  }
  // ... completed by the first keys == T when fewer than 64 exceed it
  for (int base = 0; base < cols && n < PROP_LIST; base += 32) {
    const int c = base + lane;
    const bool p = c < cols && key(c) == T;
    const unsigned bal = __ballot_sync(0xffffffffu, p);
    const int pos = n + __popc(bal & ((1u << lane) - 1u));
    if (p && pos < PROP_LIST) {
      c_key[w][pos] = T;
      c_col[w][pos] = c;
    }
    n = min(PROP_LIST, n + __popc(bal));
  }
  __syncwarp();
  // 3. ranks; the first PROP_LIST are written
  for (int i = lane; i < n; i += 32) {
    const unsigned ki = c_key[w][i];
    const int ci = c_col[w][i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const unsigned kj = c_key[w][j];
      rank += (kj > ki) || (kj == ki && c_col[w][j] < ci);
    }
    if (rank < PROP_LIST) {
      out_idx[(size_t)r * out_stride + rank] = ci;
      if (out_val) out_val[(size_t)r * out_stride + rank] = row[ci];
    }
  }
}

// --------------------------------------------------------------------------
// per-solve preparation
// --------------------------------------------------------------------------

// radius[c] = max over the points assigned to c of |p - mu_c|, rounded up
__global__ void k_cell_radius(const float* __restrict__ pts, int64_t N, int d, const int* __restrict__ cell,
                              const float* __restrict__ mu, unsigned* __restrict__ radius_bits) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    const int c = cell[p];
    const float k2 = key32<METRIC_SQL2>(pts + (size_t)p * d, mu + (size_t)c * d, d);
    const float r = sqrtf(k2) * (1.f + 1e-4f) + 1e-30f;
    atomicMax(radius_bits + c, __float_as_uint(r));
  }
}

// bias[c] = -|mu_c|^2 / 2 (FP32), the offset of the supplier-to-cell scores
__global__ void k_half_sq_norms(const float* __restrict__ mu, int cells, int d, float* __restrict__ bias) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cells) return;
  float s = 0.f;
  for (int k = 0; k < d; ++k) s = fmaf(mu[(size_t)c * d + k], mu[(size_t)c * d + k], s);
  bias[c] = -0.5f * s;
}

// Lower bounds of the squared distance from each row of Y [rows][d] to any
// supplier of each cell, out[rows][cells]: max(0, |y - mu_c| - r_c)^2.
// |y - mu_c|^2 is computed in FP32 (direct differences, fma in ascending k,
// 4 x 4 per thread); the computed D satisfies D <= |y - mu|^2 (1 + gamma_{d+1})
// (each difference adds a relative error of at most u = 2^-24 before it is
// squared, the d-term sum at most gamma_{d-1}), so |y - mu| >=
// sqrt(D (1 - gamma_{d+2})); every later step rounds down (r_c is rounded up
// when it is formed), so the result is at most the bound it stands for.
__global__ void __launch_bounds__(256) k_centroid_lb(const float* __restrict__ Y, int rows, const float* __restrict__ MU,
                                                     int cells, int d, const unsigned* __restrict__ radius_bits,
                                                     float* __restrict__ out) {
  __shared__ float Ys[TG_K][TG_PAD];
  __shared__ float Ms[TG_K][TG_PAD];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
  const int lr = tid & 63, lk = (tid >> 6) * 8;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < d; k0 += TG_K) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = k0 + lk + e;
      Ys[lk + e][lr] = (r0 + lr < rows && k < d) ? Y[(size_t)(r0 + lr) * d + k] : 0.f;
      Ms[lk + e][lr] = (c0 + lr < cells && k < d) ? MU[(size_t)(c0 + lr) * d + k] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < TG_K; ++k) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float t = __fsub_rn(Ms[k][tx * 4 + j], Ys[k][ty * 4 + i]);
          acc[i][j] = __fmaf_rn(t, t, acc[i][j]);
        }
    }
    __syncthreads();
  }
  const double ud = (d + 2) * 0x1p-24;
  const float shrink = __double2float_rd(1.0 - ud / (1.0 - ud));  // 1 - gamma_{d+2}, rounded down
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = c0 + tx * 4 + j;
    if (c >= cells) continue;
    const float rc = __uint_as_float(radius_bits[c]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + ty * 4 + i;
      if (r >= rows) continue;
      const float gap = __fsub_rd(__fsqrt_rd(__fmul_rd(acc[i][j], shrink)), rc);
      out[(size_t)r * cells + c] = gap > 0.f ? __fmul_rd(gap, gap) : 0.f;
    }
  }
}

// The PROP_LIST best of every row of V [rows][cols]: one warp per row
// (k_select_rows_warp), the rows it hands over by the block selection.
template <bool LARGEST>
static void select_rows(const float* V, int rows, int cols, int* out_idx, float* out_val, const LearnedBufs& L,
                        cudaStream_t st) {
  if (cols >= 2 * PROP_LIST) {
    cudaMemsetAsync(L.nsel_over, 0, sizeof(int), st);
    k_select_rows_warp<LARGEST><<<(rows + SEL_WARPS - 1) / SEL_WARPS, 32 * SEL_WARPS, 0, st>>>(
        V, rows, cols, out_idx, out_val, PROP_LIST, L.sel_over, L.nsel_over);
    k_select_rows<LARGEST><<<rows, 256, cols * sizeof(unsigned), st>>>(V, rows, cols, out_idx, out_val, PROP_LIST,
                                                                       L.sel_over, L.nsel_over);
  } else {
    k_select_rows<LARGEST><<<rows, 256, cols * sizeof(unsigned), st>>>(V, rows, cols, out_idx, out_val, PROP_LIST,
                                                                       nullptr, nullptr);
  }
}

int learned_prepare(const LearnedBufs& L, const float* x, int64_t m, const float* y, int64_t n, int d, unsigned* err,
                    cudaStream_t st) {
  const nnsemd_proposal* P = L.P;
  const int K = P->cells, h = P->hidden;
  // the scoring layer (hidden -> cells, the widest) runs on the tensor
  // cores in BF16 where its width allows: its scores only rank the cells a
  // consumer scans, every choice is still certified with exact keys
  const bool tc3 = linear_tc_supported(h);
  if (tc3 && pack_rows_bf16(P->params + P->off_W3(), K, h, L.w3p, st)) return -1;
  // with d on the tensor cores too, all three layers run there, each
  // writing the next one's packed BF16 input (ReLU applied)
  const bool tc_all = tc3 && linear_tc_supported(d);
  if (tc_all && (pack_rows_bf16(P->params + P->off_W1(), h, d, L.w1p, st) ||
                 pack_rows_bf16(P->params + P->off_W2(), h, h, L.w2p, st)))
    return -1;
  // the cell of each supplier: any assignment keeps the bounds sound (the
  // radii below are taken over the cells as assigned), so on the tensor
  // cores in BF16 where d allows: the largest <x, mu_c> - |mu_c|^2 / 2
  if (linear_tc_supported(d)) {
    k_half_sq_norms<<<(K + 255) / 256, 256, 0, st>>>(P->centroids, K, d, L.mu_bias);
    if (pack_rows_bf16(P->centroids, K, d, L.mup, st)) return -1;
    for (int64_t r0 = 0; r0 < m; r0 += L.assign_chunk) {
      const int rows = (int)std::min<int64_t>(L.assign_chunk, m - r0);
      if (pack_rows_bf16(x + (size_t)r0 * d, rows, d, L.xp, st) ||
          linear_tc_argmax(L.xp, rows, d, L.mup, L.mu_bias, K, L.apart, L.cell_of_x + r0, err, st))
        return -1;
    }
  } else if (assign_cells(P, x, m, L.cell_of_x, st)) {
    return -1;
  }
  cudaMemsetAsync(L.radius, 0, K * sizeof(float), st);
  k_cell_radius<<<num_sms() * 4, 256, 0, st>>>(x, m, d, L.cell_of_x, P->centroids, reinterpret_cast<unsigned*>(L.radius));
  // the cell bounds on the tensor cores (a BF16X3 contraction with its error
  // bound) where d allows, else by FP32 direct differences
  const bool tcb = cell_bounds_tc_supported(d);
  if (tcb && cell_bounds_tc_cells(P->centroids, K, d, L.mup3, L.mu_sq_lo, L.mu_nrm_up, st)) return -1;
  for (int64_t r0 = 0; r0 < n; r0 += L.chunk) {
    const int rows = (int)std::min<int64_t>(L.chunk, n - r0);
    const float* yc = y + (size_t)r0 * d;
    // proposals: the network's best cells
    float* Xs = L.tmp3;              // rows x d (standardised input)
    float* H1 = L.tmp;               // rows x h
    float* H2 = L.tmp + (size_t)L.chunk * h;
    float* Z = L.tmp2;               // rows x K
    k_standardise<<<num_sms() * 4, 256, 0, st>>>(yc, rows, d, P->in_mean, P->in_scale, Xs);
    if (tc_all) {
      const float* p = P->params;
      if (pack_rows_bf16(Xs, rows, d, L.xp1, st) ||
          linear_tc_pack_relu(L.xp1, rows, d, L.w1p, p + P->off_b1(), h, L.h1p, err, st) ||
          linear_tc_pack_relu(L.h1p, rows, h, L.w2p, p + P->off_b2(), h, L.h2p, err, st) ||
          linear_tc(L.h2p, rows, h, L.w3p, p + P->off_b3(), K, Z, err, st))
        return -1;
    } else if (tc3) {
      const float* p = P->params;
      gemm<false, true, EPI_BIAS_RELU>(Xs, d, p + P->off_W1(), d, H1, h, rows, h, d, p + P->off_b1(), st);
      gemm<false, true, EPI_BIAS_RELU>(H1, h, p + P->off_W2(), h, H2, h, rows, h, h, p + P->off_b2(), st);
      if (pack_rows_bf16(H2, rows, h, L.h2p, st) || linear_tc(L.h2p, rows, h, L.w3p, p + P->off_b3(), K, Z, err, st))
        return -1;
    } else {
      mlp_forward(P, Xs, rows, H1, H2, Z, st);
    }
    select_rows<true>(Z, rows, K, L.prop_cells + r0 * PROP_LIST, nullptr, L, st);
    // bounds: the cells with the smallest lower bound
    if (tcb) {
      if (cell_bounds_tc(yc, rows, d, L.yp3, L.y_sq_lo, L.y_nrm_up, L.mup3, L.mu_sq_lo, L.mu_nrm_up, L.radius, K, Z,
                         err, st))
        return -1;
    } else {
      dim3 g2((K + 63) / 64, (rows + 63) / 64);
      k_centroid_lb<<<g2, 256, 0, st>>>(yc, rows, P->centroids, K, d, reinterpret_cast<const unsigned*>(L.radius), Z);
    }
    select_rows<false>(Z, rows, K, L.bound_cells + r0 * PROP_LIST, L.bound_vals + r0 * PROP_LIST, L, st);
  }
  (void)h;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// --------------------------------------------------------------------------
// per round
// --------------------------------------------------------------------------

__global__ void k_cell_count(const int* __restrict__ ia, int mt, const int* __restrict__ cell_of_x,
                             int* __restrict__ cnt) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < mt) atomicAdd(cnt + cell_of_x[ia[p]], 1);
}

// exclusive scan of cnt[0..K) into off (single block), off[K] = total
__global__ void k_cell_scan(const int* __restrict__ cnt, int K, int* __restrict__ off, int* __restrict__ fill) {
  __shared__ int wt[33];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < K; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = i < K ? cnt[i] : 0;
    int tot;
    const int ex = block_scan_excl(v, wt, tot);
    if (i < K) {
      off[i] = carry + ex;
      fill[i] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) off[K] = carry;
}

__global__ void k_cell_scatter(const int* __restrict__ ia, int mt, const int* __restrict__ cell_of_x,
                               const int* __restrict__ off, int* __restrict__ fill, int* __restrict__ members) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= mt) return;
  const int c = cell_of_x[ia[p]];
  members[off[c] + atomicAdd(fill + c, 1)] = p;
}

struct LearnedArgs {
  const float* x;
  const float* y;
  const int* ia;
  const int* ja;
  int d, nt;
  const int* prop_cells;
  const int* bound_cells;
  const float* bound_vals;
  const int* cell_off;   // [K+1]
  const int* members;
  unsigned long long* nnkey;
  int* fallback;
  int* nfallback;
  unsigned long long* ncert;
  unsigned long long* nfall;
};

constexpr int LN_YMAX = 256;  // consumer rows up to this d are staged in shared memory

// One warp per active consumer.  When d % 4 == 0, d <= LN_YMAX and the
// coordinates are 16-byte aligned, the consumer's row is staged in shared
// memory (every lane reads it: broadcast) and the supplier rows are read
// 16 bytes at a time; the key is the same FP32 chain either way.
__global__ void __launch_bounds__(256) k_learned_nns(LearnedArgs A) {
  __shared__ int cand[8][PROP_TAKE];
  __shared__ __align__(16) float ysm[8][LN_YMAX];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int q = blockIdx.x * 8 + wib;
  if (q >= A.nt) return;
  const int j = A.ja[q];
  const float* yrow = A.y + (size_t)j * A.d;
  const bool vec = (A.d & 3) == 0 && A.d <= LN_YMAX && (reinterpret_cast<uintptr_t>(A.x) & 15) == 0;
  if (vec)
    for (int k = lane; k < A.d; k += 32) ysm[wib][k] = yrow[k];
  // the first PROP_TAKE proposed cells that still hold active suppliers
  const int* pl = A.prop_cells + (size_t)j * PROP_LIST;
  int ncand = 0;
  for (int base = 0; base < PROP_LIST && ncand < PROP_TAKE; base += 32) {
    const int c = pl[base + lane];
    const bool ne = A.cell_off[c + 1] > A.cell_off[c];
    const unsigned bal = __ballot_sync(0xffffffffu, ne);
    const int pos = ncand + __popc(bal & ((1u << lane) - 1u));
    if (ne && pos < PROP_TAKE) cand[wib][pos] = c;
    ncand = min(PROP_TAKE, ncand + __popc(bal));
  }
  __syncwarp();
  // exact FP32 key over the candidates' suppliers
  unsigned long long best = ~0ULL;
  for (int k = 0; k < ncand; ++k) {
    const int c = cand[wib][k];
    const int b = A.cell_off[c], e = A.cell_off[c + 1];
    for (int u = b + lane; u < e; u += 32) {
      const int p = A.members[u];
      const float* xr = A.x + (size_t)A.ia[p] * A.d;
      const float key = vec ? key32_sql2_v4(xr, ysm[wib], A.d) : key32<METRIC_SQL2>(xr, yrow, A.d);
      const unsigned long long kk = pack_key(key, (unsigned)p);
      best = kk < best ? kk : best;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
    best = ob < best ? ob : best;
  }
  // smallest bound of a non-candidate cell that still holds active suppliers
  const int* bl = A.bound_cells + (size_t)j * PROP_LIST;
  const float* bv = A.bound_vals + (size_t)j * PROP_LIST;
  float bound = bv[PROP_LIST - 1];  // every cell outside the list is at least this far
  for (int base = 0; base < PROP_LIST; base += 32) {
    const int c = bl[base + lane];
    bool ok = A.cell_off[c + 1] > A.cell_off[c];
    for (int k = 0; k < ncand && ok; ++k) ok = cand[wib][k] != c;
    const float v = ok ? bv[base + lane] : CUDART_INF_F;
    float mn = v;
    for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    bound = fminf(bound, mn);
  }
  if (lane != 0) return;
  const double gam = A.d * 0x1p-24 / (1.0 - A.d * 0x1p-24);
  const bool certified =
      best != ~0ULL && (double)__uint_as_float((unsigned)(best >> 32)) < (double)bound * (1.0 - gam) * (1.0 - 0x1p-30);
  if (certified) {
    A.nnkey[q] = best;
    atomicAdd(A.ncert, 1ULL);
  } else {
    A.fallback[atomicAdd(A.nfallback, 1)] = q;
    if (A.nfall) atomicAdd(A.nfall, 1ULL);
  }
}

// --------------------------------------------------------------------------
// The same step, cell by cell (d of 32, 64 or 128, 16-byte aligned rows): the
// candidate cells and the bound of every consumer first (k_learned_plan), the
// consumers grouped by candidate cell (k_lc_offsets, k_lc_group), then one
// CTA per (cell, up to LC_THREADS of its consumers) stages the cell's active
// suppliers in shared memory once for all of them (k_lc_keys), and the
// certificate last (k_learned_cert).  Candidates, keys, bound and
// certificate are those of k_learned_nns, so the results are the same.
// --------------------------------------------------------------------------

constexpr int LC_THREADS = 128;  // consumers of one cell per work item (one per thread)
constexpr int LC_TILE = 64;      // suppliers staged at a time

struct LcArgs {
  const float* x;
  const float* y;
  const int* ia;
  const int* ja;
  int d, nt, cells;
  const int* prop_cells;
  const int* bound_cells;
  const float* bound_vals;
  const int* cell_off;     // [K+1] active suppliers by cell
  const int* members;
  int* cand;               // [nt][PROP_TAKE] candidate cells of each consumer
  int* slot;               // [nt][PROP_TAKE] the consumer's place in each candidate cell's list
  int* ncand;              // [nt]
  float* bound;            // [nt] smallest bound of a non-candidate cell holding active suppliers
  int* qcnt;               // [K] consumers per cell
  int* qoff;               // [K+1]
  int* work_off;           // [K+1] work items (chunks of LC_THREADS consumers) before each cell
  int* nwork;
  int* work_next;          // the next work item to take (zero at launch)
  int* qlist;              // consumers grouped by cell
  unsigned long long* best;  // [nt] smallest packed key over the candidates (all ones on entry)
  unsigned long long* nnkey;
  int* fallback;
  int* nfallback;
  unsigned long long* ncert;
  unsigned long long* nfall;
  unsigned long long* nwiden;  // certified by the second tier
};

// One warp per active consumer: the first PROP_TAKE proposed cells that
// still hold active suppliers, their places in the cells' lists, and the
// bound of the other cells (as k_learned_nns takes them).
__global__ void __launch_bounds__(256) k_learned_plan(LcArgs A) {
  __shared__ int cand[8][PROP_TAKE];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int q = blockIdx.x * 8 + wib;
  if (q >= A.nt) return;
  const int j = A.ja[q];
  const int* pl = A.prop_cells + (size_t)j * PROP_LIST;
  int ncand = 0;
  for (int base = 0; base < PROP_LIST && ncand < PROP_TAKE; base += 32) {
    const int c = pl[base + lane];
    const bool ne = A.cell_off[c + 1] > A.cell_off[c];
    const unsigned bal = __ballot_sync(0xffffffffu, ne);
    const int pos = ncand + __popc(bal & ((1u << lane) - 1u));
    if (ne && pos < PROP_TAKE) {
      cand[wib][pos] = c;
      A.cand[(size_t)q * PROP_TAKE + pos] = c;
      A.slot[(size_t)q * PROP_TAKE + pos] = atomicAdd(A.qcnt + c, 1);
    }
    ncand = min(PROP_TAKE, ncand + __popc(bal));
  }
  __syncwarp();
  const int* bl = A.bound_cells + (size_t)j * PROP_LIST;
  const float* bv = A.bound_vals + (size_t)j * PROP_LIST;
  float bound = bv[PROP_LIST - 1];
  for (int base = 0; base < PROP_LIST; base += 32) {
    const int c = bl[base + lane];
    bool ok = A.cell_off[c + 1] > A.cell_off[c];
    for (int k = 0; k < ncand && ok; ++k) ok = cand[wib][k] != c;
    const float v = ok ? bv[base + lane] : CUDART_INF_F;
    float mn = v;
    for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    bound = fminf(bound, mn);
  }
  if (lane == 0) {
    A.ncand[q] = ncand;
    A.bound[q] = bound;
  }
}

// Single block: qoff = exclusive scan of qcnt, work_off = exclusive scan of
// the work items per cell (ceil(qcnt / LC_THREADS)), *nwork = their total.
__global__ void k_lc_offsets(LcArgs A) {
  __shared__ int wt[33];
  __shared__ int carry_q, carry_w;
  if (threadIdx.x == 0) carry_q = carry_w = 0;
  __syncthreads();
  for (int base = 0; base < A.cells; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = i < A.cells ? A.qcnt[i] : 0;
    const int wv = (v + LC_THREADS - 1) / LC_THREADS;
    int tot, wtot;
    const int ex = block_scan_excl(v, wt, tot);
    __syncthreads();
    const int wex = block_scan_excl(wv, wt, wtot);
    if (i < A.cells) {
      A.qoff[i] = carry_q + ex;
      A.work_off[i] = carry_w + wex;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry_q += tot;
      carry_w += wtot;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    A.qoff[A.cells] = carry_q;
    A.work_off[A.cells] = carry_w;
    *A.nwork = carry_w;
  }
}

// One thread per (consumer, candidate): the consumer into its cell's list.
__global__ void k_lc_group(LcArgs A) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)A.nt * PROP_TAKE) return;
  const int q = (int)(i / PROP_TAKE), k = (int)(i % PROP_TAKE);
  if (k >= A.ncand[q]) return;
  const int c = A.cand[i];
  A.qlist[A.qoff[c] + A.slot[i]] = q;
}

// The cell scan.  CTAs take work items from a counter; a work item is up to
// LC_THREADS consumers of one cell, one per thread, each with its row in
// registers; the cell's active suppliers pass through shared memory
// LC_TILE rows at a time and every thread runs the key32<SQL2> chain of
// four suppliers at once against its row.
template <int D>
__global__ void __launch_bounds__(LC_THREADS) k_lc_keys(LcArgs A) {
  __shared__ __align__(16) float xs[LC_TILE][D];
  __shared__ int ps[LC_TILE];
  __shared__ int s_wi;
  const int tid = threadIdx.x;
  const int nw = *A.nwork;
  for (;;) {
    __syncthreads();  // the previous item's reads of s_wi and of the tiles are done
    if (tid == 0) s_wi = atomicAdd(A.work_next, 1);
    __syncthreads();
    const int wi = s_wi;
    if (wi >= nw) break;
    // the cell of this work item: the last c with work_off[c] <= wi
    int lo = 0, hi = A.cells;  // work_off[lo] <= wi < work_off[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (A.work_off[mid] <= wi) lo = mid; else hi = mid;
    }
    const int c = lo;
    const int qi = (wi - A.work_off[c]) * LC_THREADS + tid;
    const bool has = qi < A.qoff[c + 1] - A.qoff[c];
    const int q = has ? A.qlist[A.qoff[c] + qi] : 0;
    float yr[D];
    if (has) {
      const float4* y4 = reinterpret_cast<const float4*>(A.y + (size_t)A.ja[q] * D);
#pragma unroll
      for (int k = 0; k < D / 4; ++k) {
        const float4 v = y4[k];
        yr[4 * k] = v.x;
        yr[4 * k + 1] = v.y;
        yr[4 * k + 2] = v.z;
        yr[4 * k + 3] = v.w;
      }
    }
    unsigned long long best = ~0ULL;
    const int s0 = A.cell_off[c], ns = A.cell_off[c + 1] - s0;
    for (int t0 = 0; t0 < ns; t0 += LC_TILE) {
      const int tn = min(LC_TILE, ns - t0);
      __syncthreads();
      for (int i = tid; i < tn * (D / 4); i += LC_THREADS) {
        const int r = i / (D / 4), k4 = i % (D / 4);
        const int p = A.members[s0 + t0 + r];
        reinterpret_cast<float4*>(xs[r])[k4] = reinterpret_cast<const float4*>(A.x + (size_t)A.ia[p] * D)[k4];
        if (k4 == 0) ps[r] = p;
      }
      __syncthreads();
      if (has) {
        for (int r = 0; r < tn; r += 4) {
          const float4* row[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) row[u] = reinterpret_cast<const float4*>(xs[min(r + u, tn - 1)]);
          float acc[4];
#pragma unroll
          for (int k4 = 0; k4 < D / 4; ++k4) {
            const unsigned long long y01 = f2_pack(yr[4 * k4], yr[4 * k4 + 1]);
            const unsigned long long y23 = f2_pack(yr[4 * k4 + 2], yr[4 * k4 + 3]);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              // the differences two coordinates per packed FP32x2 step (each
              // lane rounds as the scalar form), the squares in order
              const float4 xv = row[u][k4];
              const unsigned long long t01 = f2_sub(f2_pack(xv.x, xv.y), y01);
              const unsigned long long t23 = f2_sub(f2_pack(xv.z, xv.w), y23);
              const float t[4] = {f2_lo(t01), f2_hi(t01), f2_lo(t23), f2_hi(t23)};
#pragma unroll
              for (int e = 0; e < 4; ++e)
                acc[u] = (k4 == 0 && e == 0) ? __fmul_rn(t[e], t[e]) : __fmaf_rn(t[e], t[e], acc[u]);
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (r + u < tn) {
              const unsigned long long kk = pack_key(acc[u], (unsigned)ps[r + u]);
              best = kk < best ? kk : best;
            }
        }
      }
    }
    if (has) atomicMin(A.best + q, best);
  }
}

// As many CTAs of the cell scan as the GPU holds at once (they take work
// items from a counter until none is left).
template <int D>
static int lc_grid() {
  static const int per_sm = [] {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_lc_keys<D>, LC_THREADS, 0) != cudaSuccess || b < 1) b = 1;
    return b;
  }();
  return per_sm * num_sms();
}

// One thread per active consumer: the certificate of k_learned_nns.
__global__ void k_learned_cert(LcArgs A) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= A.nt) return;
  const unsigned long long best = A.best[q];
  const double gam = A.d * 0x1p-24 / (1.0 - A.d * 0x1p-24);
  const bool certified = best != ~0ULL && (double)__uint_as_float((unsigned)(best >> 32)) <
                                              (double)A.bound[q] * (1.0 - gam) * (1.0 - 0x1p-30);
  if (certified) {
    A.nnkey[q] = best;
    atomicAdd(A.ncert, 1ULL);
  } else {
    A.fallback[atomicAdd(A.nfallback, 1)] = q;
    if (A.nfall) atomicAdd(A.nfall, 1ULL);
  }
}

// One warp per consumer the cell scan left uncertified (list[0 .. count)):
// the cells of its bound list (smallest bound first) that still hold active
// suppliers and were not among its candidates are scanned one after another
// with the same FP32 key, until the best key is strictly below the bound of
// the next such cell (every cell not scanned then lies at or above that
// bound, the ones outside the list at or above its last), or the list runs
// out and the last bound decides.  The rest go to out_list for the full
// scan.  The key, the packed minimum and the margin are those of
// k_learned_cert, so a certified choice is the full scan's.
__global__ void __launch_bounds__(256) k_learned_widen(LcArgs A, const int* __restrict__ list, int count,
                                                       int* __restrict__ out_list, int* __restrict__ out_count) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int idx = blockIdx.x * 8 + wib;
  if (idx >= count) return;
  const int q = list[idx];
  const int j = A.ja[q];
  const float* yrow = A.y + (size_t)j * A.d;
  const int nc = A.ncand[q];
  static_assert(PROP_TAKE <= 32, "one candidate per lane");
  const int mycand = lane < nc ? A.cand[(size_t)q * PROP_TAKE + lane] : -1;
  const int* bl = A.bound_cells + (size_t)j * PROP_LIST;
  const float* bv = A.bound_vals + (size_t)j * PROP_LIST;
  const double gam = A.d * 0x1p-24 / (1.0 - A.d * 0x1p-24);
  auto below = [&](unsigned long long key, float bound) {
    return key != ~0ULL && (double)__uint_as_float((unsigned)(key >> 32)) < (double)bound * (1.0 - gam) * (1.0 - 0x1p-30);
  };
  unsigned long long best = A.best[q];
  bool done = false;
  for (int t = 0; t < PROP_LIST && !done; ++t) {
    const int c = bl[t];
    const int b = A.cell_off[c], e = A.cell_off[c + 1];
    if (e == b || __any_sync(0xffffffffu, mycand == c)) continue;  // empty, or scanned already
    if (below(best, bv[t])) {
      done = true;
      break;
    }
    for (int u = b + lane; u < e; u += 32) {
      const int p = A.members[u];
      const unsigned long long kk = pack_key(key32_sql2_v4(A.x + (size_t)A.ia[p] * A.d, yrow, A.d), (unsigned)p);
      best = kk < best ? kk : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
      best = ob < best ? ob : best;
    }
  }
  if (!done) done = below(best, bv[PROP_LIST - 1]);
  if (lane != 0) return;
  if (done) {
    A.nnkey[q] = best;
    atomicAdd(A.ncert, 1ULL);
    atomicAdd(A.nwiden, 1ULL);
  } else {
    out_list[atomicAdd(out_count, 1)] = q;
    if (A.nfall) atomicAdd(A.nfall, 1ULL);
  }
}

// Consumers left after the second tier at or below which the full scan
// runs in FP32 rather than on the tensor cores.
constexpr int LC_TC_MIN = 256;

__global__ void k_add_count(unsigned long long* ctr, unsigned long long v) { *ctr += v; }

bool learned_cell_scan(int d, const float* x, const float* y) {
  return (d == 32 || d == 64 || d == 128) && ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15) == 0;
}

// The consumers the proposal cannot certify are scanned in full: in FP32,
// or with a reduced-precision solve precision by the tensor-core scan (its
// own certificate and FP32 rescan), restricted to them.
int launch_nns_learned(const SolveBufs& B, const LearnedBufs& L, int mt, int nt, cudaStream_t st) {
  const int K = L.P->cells;
  const int* ia = B.ia[B.cur];
  cudaMemsetAsync(L.cell_cnt, 0, (K + 1) * sizeof(int), st);
  k_cell_count<<<(mt + 255) / 256, 256, 0, st>>>(ia, mt, L.cell_of_x, L.cell_cnt);
  k_cell_scan<<<1, 1024, 0, st>>>(L.cell_cnt, K, L.cell_off, L.cell_fill);
  k_cell_scatter<<<(mt + 255) / 256, 256, 0, st>>>(ia, mt, L.cell_of_x, L.cell_off, L.cell_fill, L.cell_members);
  cudaMemsetAsync(L.nfallback, 0, sizeof(int), st);
  unsigned long long* nfall = B.precision == 0 ? &B.st->fallbacks : nullptr;
  if (learned_cell_scan(B.d, B.x, B.y)) {
    LcArgs C{B.x,        B.y,          ia,          B.ja[B.cur], B.d,       nt,        K,
             L.prop_cells, L.bound_cells, L.bound_vals, L.cell_off, L.cell_members, L.lc_cand, L.lc_slot,
             L.lc_ncand,   L.lc_bound,   L.lc_qcnt,   L.lc_qoff,  L.lc_work,  L.lc_nwork, L.lc_nwork + 1,
             L.lc_qlist,   L.lc_best,    B.nnkey,     L.fallback, L.nfallback, &B.st->certified, nfall,
             &B.st->widened};
    cudaMemsetAsync(L.lc_qcnt, 0, K * sizeof(int), st);
    cudaMemsetAsync(L.lc_nwork + 1, 0, sizeof(int), st);
    cudaMemsetAsync(L.lc_best, 0xff, (size_t)nt * sizeof(unsigned long long), st);
    k_learned_plan<<<(nt + 7) / 8, 256, 0, st>>>(C);
    k_lc_offsets<<<1, 1024, 0, st>>>(C);
    k_lc_group<<<(int)(((int64_t)nt * PROP_TAKE + 255) / 256), 256, 0, st>>>(C);
    if (B.d == 32) k_lc_keys<32><<<lc_grid<32>(), LC_THREADS, 0, st>>>(C);
    else if (B.d == 64) k_lc_keys<64><<<lc_grid<64>(), LC_THREADS, 0, st>>>(C);
    else k_lc_keys<128><<<lc_grid<128>(), LC_THREADS, 0, st>>>(C);
    LcArgs Cc = C;
    Cc.nfall = nullptr;  // the consumers it leaves are counted after the second tier
    k_learned_cert<<<(nt + 255) / 256, 256, 0, st>>>(Cc);
    // the second tier: more cells, in bound order, for the consumers left
    int nf = 0;
    if (cudaMemcpyAsync(&nf, L.nfallback, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return -1;
    cudaMemsetAsync(L.nfallback2, 0, sizeof(int), st);
    if (nf > 0) k_learned_widen<<<(nf + 7) / 8, 256, 0, st>>>(C, L.fallback, nf, L.fallback2, L.nfallback2);
    if (B.precision == 0) {  // FP32
      launch_nns_f32(B, mt, nt, L.fallback2, L.nfallback2, st);
    } else {
      int nf2 = 0;
      if (nf > 0 && (cudaMemcpyAsync(&nf2, L.nfallback2, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                     cudaStreamSynchronize(st) != cudaSuccess))
        return -1;
      if (nf2 > LC_TC_MIN) {
        if (launch_nns_tc(B, B.tc, mt, nf2, B.precision, st, L.fallback2, nullptr)) return -1;
      } else if (nf2 > 0) {
        // a few consumers: the FP32 scan costs less than packing every
        // active supplier for the tensor cores (counted as fallbacks)
        k_add_count<<<1, 1, 0, st>>>(&B.st->fallbacks, (unsigned long long)nf2);
        launch_nns_f32(B, mt, nt, L.fallback2, L.nfallback2, st);
      }
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
  } else {
    LearnedArgs A{B.x,          B.y,          ia,          B.ja[B.cur], B.d,       nt,
                  L.prop_cells, L.bound_cells, L.bound_vals, L.cell_off, L.cell_members, B.nnkey,
                  L.fallback,   L.nfallback,   &B.st->certified, nfall};
    k_learned_nns<<<(nt + 7) / 8, 256, 0, st>>>(A);
  }
  if (B.precision == 0) {  // FP32
    launch_nns_f32(B, mt, nt, L.fallback, L.nfallback, st);
  } else {
    int nfall = 0;
    if (cudaMemcpyAsync(&nfall, L.nfallback, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return -1;
    if (nfall > 0 && launch_nns_tc(B, B.tc, mt, nfall, B.precision, st, L.fallback, nullptr)) return -1;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace nnsemd
