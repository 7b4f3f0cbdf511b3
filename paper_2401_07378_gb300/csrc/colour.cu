// The colour-transfer application of NNS-EMD (Sec. IV-D): k-means colour
// quantisation, the barycentric map of a transport plan and the recolouring
// of an image, as C-ABI entry points (declared in nnsemd.h).
//
// Every step is deterministic, so the result does not depend on the order
// in which threads run:
//   k-means   assignment: the nearest centroid by the FP32 squared-distance
//             key of the NNS operation, lowest index on ties (nearest_all);
//             update: each coordinate's sum over a cluster in an exact
//             integer accumulator, centroid = float(correctly rounded sum /
//             count); initial centroids: the points at floor((2c+1) N / 2k);
//   map       y'_j = float(S_j / W_j) with S_j = exact sum of f * x_i over the
//             flows into consumer j (FP64 products) and W_j = exact sum of f;
//   recolour  out[p] = palette[label[p]].
// Coordinates must be finite and non-negative (colours); weights of flows
// are non-negative by construction.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "kernels.h"
#include "nnsemd.h"
#include "proposal.h"

using namespace nnsemd;

namespace {

#define CCK(call)                                                                                          \
  do {                                                                                                     \
    cudaError_t e_ = (call);                                                                               \
    if (e_ != cudaSuccess) return ctx_fail(ctx, NNSEMD_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

struct Scratch {
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  T* get(size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
};

__global__ void k_check_colours(const float* __restrict__ v, int64_t count, unsigned* err) {
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    bad |= !(isfinite(v[i]) && v[i] >= 0.f);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, EF_NONFINITE);
}

__global__ void k_init_centroids(const float* __restrict__ pts, int64_t N, int k, int d, float* __restrict__ cent) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k * d; i += gridDim.x * blockDim.x) {
    const int c = i / d, t = i % d;
    const int64_t p = ((2 * (int64_t)c + 1) * N) / (2 * (int64_t)k);
    cent[i] = pts[p * d + t];
  }
}

__global__ void k_km_exact_accum(const float* __restrict__ pts, int64_t N, int d, const int* __restrict__ lab,
                                 unsigned long long* __restrict__ acc, unsigned long long* __restrict__ count) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    const int c = lab[p];
    for (int t = 0; t < d; ++t) xs_add(acc + ((size_t)c * d + t) * XS_LIMBS, (double)pts[p * d + t]);
    atomicAdd(count + c, 1ULL);
  }
}

__global__ void k_km_exact_finish(unsigned long long* __restrict__ acc, const unsigned long long* __restrict__ count,
                                  int k, int d, float* __restrict__ cent) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k * d; i += gridDim.x * blockDim.x) {
    const unsigned long long n = count[i / d];
    if (n) cent[i] = __double2float_rn(__ddiv_rn(xs_round(acc + (size_t)i * XS_LIMBS), (double)n));
  }
}

__global__ void k_count(const int* __restrict__ lab, int64_t N, long long* __restrict__ counts) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(reinterpret_cast<unsigned long long*>(counts + lab[p]), 1ULL);
}

__global__ void k_bary_accum(const int32_t* __restrict__ pi, const int32_t* __restrict__ pj,
                             const double* __restrict__ pf, int64_t nnz, const float* __restrict__ x, int d,
                             unsigned long long* __restrict__ acc) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = pi[e], j = pj[e];
    const double f = pf[e];
    unsigned long long* a = acc + (size_t)j * (d + 1) * XS_LIMBS;
    for (int t = 0; t < d; ++t) xs_add(a + (size_t)t * XS_LIMBS, __dmul_rn(f, (double)x[(size_t)i * d + t]));
    xs_add(a + (size_t)d * XS_LIMBS, f);
  }
}

__global__ void k_bary_finish(unsigned long long* __restrict__ acc, const float* __restrict__ y, int64_t n, int d,
                              float* __restrict__ out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long* a = acc + (size_t)j * (d + 1) * XS_LIMBS;
    const double w = xs_round(a + (size_t)d * XS_LIMBS);
    for (int t = 0; t < d; ++t)
      out[j * d + t] = w > 0.0 ? __double2float_rn(__ddiv_rn(xs_round(a + (size_t)t * XS_LIMBS), w)) : y[j * d + t];
  }
}

__global__ void k_recolour(const int* __restrict__ lab, int64_t N, const float* __restrict__ palette, int k, int d,
                           float* __restrict__ out, unsigned* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N * d; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = lab[i / d];
    if (c < 0 || c >= k) {
      atomicOr(err, EF_INTERNAL);
      continue;
    }
    out[i] = palette[(size_t)c * d + (i % d)];
  }
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, num_sms() * 8)); }

int read_err(nnsemd_ctx* ctx, unsigned* err_d, cudaStream_t st) {
  unsigned h = 0;
  CCK(cudaMemcpyAsync(&h, err_d, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  CCK(cudaStreamSynchronize(st));
  if (h & EF_NONFINITE) return ctx_fail(ctx, NNSEMD_ERR_NONFINITE, "a coordinate is negative or not finite");
  if (h) return ctx_fail(ctx, NNSEMD_ERR_INVALID_ARG, "a label is out of range");
  return NNSEMD_OK;
}

}  // namespace

extern "C" {

int nnsemd_kmeans(nnsemd_ctx* ctx, const float* pts, int64_t N, int32_t d, int32_t k, int32_t iters,
                  float* centroids_out, int32_t* labels_out, int64_t* counts_out) {
  if (!ctx) return NNSEMD_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!pts || !centroids_out || !labels_out || !counts_out || N < 1 || d < 1 || k < 1 || k > N || iters < 0 ||
      N > (1LL << 30) || k > (1 << 20))
    return ctx_fail(ctx, NNSEMD_ERR_INVALID_ARG, "kmeans arguments");
  CCK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  Scratch S;
  unsigned* err = S.get<unsigned>(1);
  int* iota = S.get<int>(std::max<int64_t>(N, k));
  unsigned long long* keys = S.get<unsigned long long>(N);
  unsigned long long* acc = S.get<unsigned long long>((size_t)k * d * XS_LIMBS);
  unsigned long long* cnt = S.get<unsigned long long>(k);
  if (!err || !iota || !keys || !acc || !cnt) return ctx_fail(ctx, NNSEMD_ERR_OOM, "kmeans scratch");
  CCK(cudaMemsetAsync(err, 0, sizeof(unsigned), st));
  k_check_colours<<<grid_for(N * d), 256, 0, st>>>(pts, N * d, err);
  if (int rc = read_err(ctx, err, st)) return rc;
  {
    std::vector<int> h(std::max<int64_t>(N, k));
    for (size_t i = 0; i < h.size(); ++i) h[i] = (int)i;
    CCK(cudaMemcpyAsync(iota, h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    CCK(cudaStreamSynchronize(st));
  }
  k_init_centroids<<<grid_for((int64_t)k * d), 256, 0, st>>>(pts, N, k, d, centroids_out);
  if (nearest_all(centroids_out, k, pts, N, d, METRIC_SQL2, iota, keys, labels_out, st))
    return ctx_fail(ctx, NNSEMD_ERR_CUDA, "assignment launch");
  for (int it = 0; it < iters; ++it) {
    CCK(cudaMemsetAsync(acc, 0, (size_t)k * d * XS_LIMBS * sizeof(unsigned long long), st));
    CCK(cudaMemsetAsync(cnt, 0, (size_t)k * sizeof(unsigned long long), st));
    k_km_exact_accum<<<grid_for(N), 256, 0, st>>>(pts, N, d, labels_out, acc, cnt);
    k_km_exact_finish<<<grid_for((int64_t)k * d), 256, 0, st>>>(acc, cnt, k, d, centroids_out);
    if (nearest_all(centroids_out, k, pts, N, d, METRIC_SQL2, iota, keys, labels_out, st))
      return ctx_fail(ctx, NNSEMD_ERR_CUDA, "assignment launch");
  }
  CCK(cudaMemsetAsync(counts_out, 0, (size_t)k * sizeof(int64_t), st));
  k_count<<<grid_for(N), 256, 0, st>>>(labels_out, N, reinterpret_cast<long long*>(counts_out));
  CCK(cudaGetLastError());
  CCK(cudaStreamSynchronize(st));
  return NNSEMD_OK;
}

int nnsemd_barycentric(nnsemd_ctx* ctx, const nnsemd_plan* plan, const float* x, int64_t m, const float* y,
                       int64_t n, int32_t d, float* y_out) {
  if (!ctx) return NNSEMD_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!plan || !x || !y || !y_out || m < 1 || n < 1 || d < 1 || plan->nnz < 0 || (plan->nnz && (!plan->i || !plan->j || !plan->f)))
    return ctx_fail(ctx, NNSEMD_ERR_INVALID_ARG, "barycentric arguments");
  CCK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  Scratch S;
  unsigned* err = S.get<unsigned>(1);
  unsigned long long* acc = S.get<unsigned long long>((size_t)n * (d + 1) * XS_LIMBS);
  if (!err || !acc) return ctx_fail(ctx, NNSEMD_ERR_OOM, "barycentric scratch");
  CCK(cudaMemsetAsync(err, 0, sizeof(unsigned), st));
  k_check_colours<<<grid_for(m * d), 256, 0, st>>>(x, m * d, err);
  if (int rc = read_err(ctx, err, st)) return rc;
  CCK(cudaMemsetAsync(acc, 0, (size_t)n * (d + 1) * XS_LIMBS * sizeof(unsigned long long), st));
  if (plan->nnz) k_bary_accum<<<grid_for(plan->nnz), 256, 0, st>>>(plan->i, plan->j, plan->f, plan->nnz, x, d, acc);
  k_bary_finish<<<grid_for(n), 256, 0, st>>>(acc, y, n, d, y_out);
  CCK(cudaGetLastError());
  CCK(cudaStreamSynchronize(st));
  return NNSEMD_OK;
}

int nnsemd_recolour(nnsemd_ctx* ctx, const int32_t* labels, int64_t N, const float* palette, int32_t k, int32_t d,
                    float* out) {
  if (!ctx) return NNSEMD_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!labels || !palette || !out || N < 1 || k < 1 || d < 1) return ctx_fail(ctx, NNSEMD_ERR_INVALID_ARG, "recolour arguments");
  CCK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  Scratch S;
  unsigned* err = S.get<unsigned>(1);
  if (!err) return ctx_fail(ctx, NNSEMD_ERR_OOM, "recolour scratch");
  CCK(cudaMemsetAsync(err, 0, sizeof(unsigned), st));
  k_recolour<<<grid_for(N * d), 256, 0, st>>>(labels, N, palette, k, d, out, err);
  return read_err(ctx, err, st);
}

}  // extern "C"
