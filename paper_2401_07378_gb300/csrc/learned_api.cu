// C-ABI entry points of the learned candidate proposal (not in the paper;
// see proposal.h) and of the stand-alone NNS operation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "ctx.h"
#include "kernels.h"
#include "nnsemd.h"
#include "proposal.h"

using namespace nnsemd;

namespace {

#define PCK(call)                                                                                          \
  do {                                                                                                     \
    cudaError_t e_ = (call);                                                                               \
    if (e_ != cudaSuccess) return ctx_fail(ctx, NNSEMD_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// SplitMix64 (Steele, Lea, Flood 2014) for seeded parameter initialisation.
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

double uniform01(uint64_t& s) { return (double)(splitmix(s) >> 11) * 0x1p-53; }

struct DeviceScratch {
  std::vector<void*> ptrs;
  ~DeviceScratch() {
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

__global__ void k_gather_std(const float* __restrict__ src, const int* __restrict__ rows, int count, int d,
                             const float* __restrict__ mean, const float* __restrict__ scale, float* __restrict__ dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count * d; i += gridDim.x * blockDim.x) {
    const int k = i % d;
    dst[i] = (src[(size_t)rows[i / d] * d + k] - mean[k]) * scale[k];
  }
}

__global__ void k_gather_int(const int* __restrict__ src, const int* __restrict__ rows, int count, int* __restrict__ dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) dst[i] = src[rows[i]];
}

__global__ void k_moments(const float* __restrict__ pts, int64_t N, int d, double* __restrict__ sum,
                          double* __restrict__ sq) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N * d; i += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(i % d);
    const double v = pts[i];
    atomicAdd(sum + k, v);
    atomicAdd(sq + k, v * v);
  }
}

int check_prop(nnsemd_ctx* ctx, const nnsemd_proposal* P) {
  if (!ctx) return NNSEMD_ERR_INVALID_ARG;
  if (!P) return ctx_fail(ctx, NNSEMD_ERR_INVALID_ARG, "proposal is NULL");
  return NNSEMD_OK;
}

constexpr uint32_t kMagic = 0x50534E4EU;  // file tag of a saved proposal

}  // namespace

extern "C" {

int nnsemd_proposal_create(nnsemd_ctx* ctx, int32_t d, int32_t cells, int32_t hidden, uint64_t seed,
                           nnsemd_proposal** out) {
  if (!ctx || !out) return NNSEMD_ERR_INVALID_ARG;
  ctx->err.clear();
  *out = nullptr;
  if (d < 1 || cells < PROP_LIST || cells > PROP_MAX_CELLS || hidden < 1 || hidden > 8192)
    return ctx_fail(ctx, NNSEMD_ERR_INVALID_ARG, "bad proposal shape d=%d cells=%d hidden=%d", d, cells, hidden);
  PCK(cudaSetDevice(ctx->device));
  nnsemd_proposal* P = new nnsemd_proposal();
  P->d = d;
  P->cells = cells;
  P->hidden = hidden;
  P->device = ctx->device;
  P->nparams = P->off_b3() + cells;
  bool ok = cudaMalloc(&P->centroids, (size_t)cells * d * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&P->in_mean, d * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&P->in_scale, d * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&P->params, P->nparams * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&P->adam_m, P->nparams * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&P->adam_v, P->nparams * sizeof(float)) == cudaSuccess;
  if (!ok) {
    nnsemd_proposal_destroy(P);
    return ctx_fail(ctx, NNSEMD_ERR_OOM, "proposal buffers");
  }
  // He-uniform weights (bound sqrt(6 / fan_in)), zero biases, seeded
  std::vector<float> h(P->nparams, 0.f);
  uint64_t s = seed;
  auto fill = [&](long long off, long long count, int fan_in) {
    const double b = std::sqrt(6.0 / fan_in);
    for (long long i = 0; i < count; ++i) h[off + i] = (float)((2.0 * uniform01(s) - 1.0) * b);
  };
  fill(P->off_W1(), (long long)hidden * d, d);
  fill(P->off_W2(), (long long)hidden * hidden, hidden);
  fill(P->off_W3(), (long long)cells * hidden, hidden);
  std::vector<float> zero_d(d, 0.f), one_d(d, 1.f);
  cudaStream_t st = ctx->stream;
  PCK(cudaMemcpyAsync(P->params, h.data(), P->nparams * sizeof(float), cudaMemcpyHostToDevice, st));
  PCK(cudaMemsetAsync(P->adam_m, 0, P->nparams * sizeof(float), st));
  PCK(cudaMemsetAsync(P->adam_v, 0, P->nparams * sizeof(float), st));
  PCK(cudaMemcpyAsync(P->in_mean, zero_d.data(), d * sizeof(float), cudaMemcpyHostToDevice, st));
  PCK(cudaMemcpyAsync(P->in_scale, one_d.data(), d * sizeof(float), cudaMemcpyHostToDevice, st));
  PCK(cudaMemsetAsync(P->centroids, 0, (size_t)cells * d * sizeof(float), st));
  PCK(cudaStreamSynchronize(st));
  *out = P;
  return NNSEMD_OK;
}

int nnsemd_proposal_destroy(nnsemd_proposal* P) {
  if (!P) return NNSEMD_OK;
  cudaSetDevice(P->device);
  cudaFree(P->centroids);
  cudaFree(P->in_mean);
  cudaFree(P->in_scale);
  cudaFree(P->params);
  cudaFree(P->adam_m);
  cudaFree(P->adam_v);
  delete P;
  return NNSEMD_OK;
}

int nnsemd_proposal_fit(nnsemd_ctx* ctx, nnsemd_proposal* P, const float* pts, int64_t N, int32_t iters,
                        uint64_t seed) {
  int rc = check_prop(ctx, P);
  if (rc) return rc;
  ctx->err.clear();
  if (!pts || N < P->cells || iters < 0) return ctx_fail(ctx, NNSEMD_ERR_INVALID_ARG, "fit needs >= cells points");
  PCK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  DeviceScratch S;
  int* assign = S.get<int>(N);
  float* sums = S.get<float>((size_t)P->cells * P->d);
  int* counts = S.get<int>(P->cells);
  double* mom = S.get<double>(2 * P->d);
  if (!assign || !sums || !counts || !mom) return ctx_fail(ctx, NNSEMD_ERR_OOM, "fit scratch");
  if (kmeans_fit(P, pts, N, iters, seed, assign, sums, counts, st))
    return ctx_fail(ctx, NNSEMD_ERR_CUDA, "k-means failed");
  // input standardisation of the network from the same points
  PCK(cudaMemsetAsync(mom, 0, 2 * P->d * sizeof(double), st));
  k_moments<<<num_sms() * 4, 256, 0, st>>>(pts, N, P->d, mom, mom + P->d);
  std::vector<double> hm(2 * P->d);
  PCK(cudaMemcpyAsync(hm.data(), mom, 2 * P->d * sizeof(double), cudaMemcpyDeviceToHost, st));
  PCK(cudaStreamSynchronize(st));
  std::vector<float> mean(P->d), scale(P->d);
  for (int k = 0; k < P->d; ++k) {
    const double mu = hm[k] / N, var = hm[P->d + k] / N - mu * mu;
    mean[k] = (float)mu;
    scale[k] = (float)(1.0 / std::sqrt(std::max(var, 1e-12)));
  }
  PCK(cudaMemcpyAsync(P->in_mean, mean.data(), P->d * sizeof(float), cudaMemcpyHostToDevice, st));
  PCK(cudaMemcpyAsync(P->in_scale, scale.data(), P->d * sizeof(float), cudaMemcpyHostToDevice, st));
  PCK(cudaStreamSynchronize(st));
  P->codebook_ready = true;
  return NNSEMD_OK;
}

int nnsemd_proposal_loss_grad(nnsemd_ctx* ctx, const nnsemd_proposal* P, const float* y, const int32_t* labels,
                              int64_t N, double* loss_out, float* grad_out) {
  int rc = check_prop(ctx, P);
  if (rc) return rc;
  ctx->err.clear();
  if (!y || !labels || !grad_out || N < 1 || N > (1 << 20))
    return ctx_fail(ctx, NNSEMD_ERR_INVALID_ARG, "loss_grad arguments");
  PCK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  DeviceScratch S;
  const int n = (int)N, d = P->d, h = P->hidden, c = P->cells;
  int* rows = S.get<int>(n);
  float* Xs = S.get<float>((size_t)n * d);
  float* H1 = S.get<float>((size_t)n * h);
  float* H2 = S.get<float>((size_t)n * h);
  float* Z = S.get<float>((size_t)n * c);
  float* d1 = S.get<float>((size_t)n * h);
  float* d2 = S.get<float>((size_t)n * h);
  double* loss = S.get<double>(1);
  if (!rows || !Xs || !H1 || !H2 || !Z || !d1 || !d2 || !loss) return ctx_fail(ctx, NNSEMD_ERR_OOM, "loss_grad scratch");
  std::vector<int> iota(n);
  for (int i = 0; i < n; ++i) iota[i] = i;
  PCK(cudaMemcpyAsync(rows, iota.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
  k_gather_std<<<num_sms() * 4, 256, 0, st>>>(y, rows, n, d, P->in_mean, P->in_scale, Xs);
  PCK(cudaMemsetAsync(loss, 0, sizeof(double), st));
  mlp_loss_grad(P, Xs, labels, n, H1, H2, Z, d1, d2, grad_out, loss, st);
  double hl = 0;
  PCK(cudaMemcpyAsync(&hl, loss, sizeof(double), cudaMemcpyDeviceToHost, st));
  PCK(cudaStreamSynchronize(st));
  if (loss_out) *loss_out = hl;
  return NNSEMD_OK;
}

int nnsemd_proposal_train(nnsemd_ctx* ctx, nnsemd_proposal* P, const float* y, const float* x_nn, int64_t N,
                          int32_t epochs, int32_t batch, float lr, uint64_t seed, double* loss_out) {
  int rc = check_prop(ctx, P);
  if (rc) return rc;
  ctx->err.clear();
  if (!P->codebook_ready) return ctx_fail(ctx, NNSEMD_ERR_INVALID_ARG, "fit the codebook first");
  if (!y || !x_nn || N < 1 || epochs < 0 || batch < 1 || batch > 65536 || !(lr > 0.f))
    return ctx_fail(ctx, NNSEMD_ERR_INVALID_ARG, "train arguments");
  PCK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  DeviceScratch S;
  const int d = P->d, h = P->hidden, c = P->cells;
  int* labels = S.get<int>(N);
  int* order = S.get<int>(N);
  int* blab = S.get<int>(batch);
  float* Xs = S.get<float>((size_t)batch * d);
  float* H1 = S.get<float>((size_t)batch * h);
  float* H2 = S.get<float>((size_t)batch * h);
  float* Z = S.get<float>((size_t)batch * c);
  float* d1 = S.get<float>((size_t)batch * h);
  float* d2 = S.get<float>((size_t)batch * h);
  float* grad = S.get<float>(P->nparams);
  double* loss = S.get<double>(1);
  if (!labels || !order || !blab || !Xs || !H1 || !H2 || !Z || !d1 || !d2 || !grad || !loss)
    return ctx_fail(ctx, NNSEMD_ERR_OOM, "train scratch");
  // label: the cell of each consumer's nearest supplier
  if (assign_cells(P, x_nn, N, labels, st)) return ctx_fail(ctx, NNSEMD_ERR_CUDA, "labels");
  std::vector<int> perm(N);
  uint64_t s = seed ^ 0xA5A5A5A5ULL;
  double last = 0.0;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int64_t i = 0; i < N; ++i) perm[i] = (int)i;
    for (int64_t i = N - 1; i > 0; --i) std::swap(perm[i], perm[splitmix(s) % (uint64_t)(i + 1)]);
    PCK(cudaMemcpyAsync(order, perm.data(), N * sizeof(int), cudaMemcpyHostToDevice, st));
    PCK(cudaMemsetAsync(loss, 0, sizeof(double), st));
    int nb = 0;
    for (int64_t b0 = 0; b0 + batch <= N; b0 += batch, ++nb) {
      k_gather_std<<<num_sms() * 4, 256, 0, st>>>(y, order + b0, batch, d, P->in_mean, P->in_scale, Xs);
      k_gather_int<<<(batch + 255) / 256, 256, 0, st>>>(labels, order + b0, batch, blab);
      mlp_loss_grad(P, Xs, blab, batch, H1, H2, Z, d1, d2, grad, loss, st);
      adam_update(P, grad, lr, st);
    }
    double hl = 0;
    PCK(cudaMemcpyAsync(&hl, loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    last = nb ? hl / nb : 0.0;
  }
  PCK(cudaGetLastError());
  if (loss_out) *loss_out = last;
  return NNSEMD_OK;
}

int nnsemd_proposal_info(const nnsemd_proposal* P, int32_t* d, int32_t* cells, int32_t* hidden, int64_t* nparams) {
  if (!P) return NNSEMD_ERR_INVALID_ARG;
  if (d) *d = P->d;
  if (cells) *cells = P->cells;
  if (hidden) *hidden = P->hidden;
  if (nparams) *nparams = P->nparams;
  return NNSEMD_OK;
}

int nnsemd_proposal_params(nnsemd_ctx* ctx, nnsemd_proposal* P, float* host, int32_t set) {
  int rc = check_prop(ctx, P);
  if (rc) return rc;
  if (!host) return ctx_fail(ctx, NNSEMD_ERR_INVALID_ARG, "host buffer is NULL");
  PCK(cudaSetDevice(ctx->device));
  if (set) PCK(cudaMemcpy(P->params, host, P->nparams * sizeof(float), cudaMemcpyHostToDevice));
  else PCK(cudaMemcpy(host, P->params, P->nparams * sizeof(float), cudaMemcpyDeviceToHost));
  return NNSEMD_OK;
}

int nnsemd_proposal_save(nnsemd_ctx* ctx, const nnsemd_proposal* P, const char* path) {
  int rc = check_prop(ctx, P);
  if (rc) return rc;
  if (!path) return ctx_fail(ctx, NNSEMD_ERR_INVALID_ARG, "path is NULL");
  PCK(cudaSetDevice(ctx->device));
  std::vector<float> cent((size_t)P->cells * P->d), mean(P->d), scale(P->d), par(P->nparams);
  PCK(cudaMemcpy(cent.data(), P->centroids, cent.size() * sizeof(float), cudaMemcpyDeviceToHost));
  PCK(cudaMemcpy(mean.data(), P->in_mean, P->d * sizeof(float), cudaMemcpyDeviceToHost));
  PCK(cudaMemcpy(scale.data(), P->in_scale, P->d * sizeof(float), cudaMemcpyDeviceToHost));
  PCK(cudaMemcpy(par.data(), P->params, par.size() * sizeof(float), cudaMemcpyDeviceToHost));
  FILE* f = std::fopen(path, "wb");
  if (!f) return ctx_fail(ctx, NNSEMD_ERR_INVALID_ARG, "cannot open %s", path);
  const uint32_t hdr[6] = {kMagic, 1u, (uint32_t)P->d, (uint32_t)P->cells, (uint32_t)P->hidden,
                           (uint32_t)P->codebook_ready};
  bool ok = std::fwrite(hdr, sizeof(hdr), 1, f) == 1 && std::fwrite(cent.data(), sizeof(float), cent.size(), f) == cent.size() &&
            std::fwrite(mean.data(), sizeof(float), mean.size(), f) == mean.size() &&
            std::fwrite(scale.data(), sizeof(float), scale.size(), f) == scale.size() &&
            std::fwrite(par.data(), sizeof(float), par.size(), f) == par.size();
  ok = (std::fclose(f) == 0) && ok;
  return ok ? NNSEMD_OK : ctx_fail(ctx, NNSEMD_ERR_INVALID_ARG, "write failed: %s", path);
}

int nnsemd_proposal_load(nnsemd_ctx* ctx, const char* path, nnsemd_proposal** out) {
  if (!ctx || !path || !out) return NNSEMD_ERR_INVALID_ARG;
  ctx->err.clear();
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return ctx_fail(ctx, NNSEMD_ERR_INVALID_ARG, "cannot open %s", path);
  uint32_t hdr[6];
  if (std::fread(hdr, sizeof(hdr), 1, f) != 1 || hdr[0] != kMagic || hdr[1] != 1u) {
    std::fclose(f);
    return ctx_fail(ctx, NNSEMD_ERR_INVALID_ARG, "%s is not a saved proposal", path);
  }
  nnsemd_proposal* P = nullptr;
  int rc = nnsemd_proposal_create(ctx, (int)hdr[2], (int)hdr[3], (int)hdr[4], 0, &P);
  if (rc) {
    std::fclose(f);
    return rc;
  }
  std::vector<float> cent((size_t)P->cells * P->d), mean(P->d), scale(P->d), par(P->nparams);
  bool ok = std::fread(cent.data(), sizeof(float), cent.size(), f) == cent.size() &&
            std::fread(mean.data(), sizeof(float), mean.size(), f) == mean.size() &&
            std::fread(scale.data(), sizeof(float), scale.size(), f) == scale.size() &&
            std::fread(par.data(), sizeof(float), par.size(), f) == par.size();
  std::fclose(f);
  if (!ok) {
    nnsemd_proposal_destroy(P);
    return ctx_fail(ctx, NNSEMD_ERR_INVALID_ARG, "%s is truncated", path);
  }
  PCK(cudaMemcpy(P->centroids, cent.data(), cent.size() * sizeof(float), cudaMemcpyHostToDevice));
  PCK(cudaMemcpy(P->in_mean, mean.data(), mean.size() * sizeof(float), cudaMemcpyHostToDevice));
  PCK(cudaMemcpy(P->in_scale, scale.data(), scale.size() * sizeof(float), cudaMemcpyHostToDevice));
  PCK(cudaMemcpy(P->params, par.data(), par.size() * sizeof(float), cudaMemcpyHostToDevice));
  P->codebook_ready = hdr[5] != 0;
  *out = P;
  return NNSEMD_OK;
}

int nnsemd_nearest(nnsemd_ctx* ctx, const float* x, int64_t m, const float* y, int64_t n, int32_t d, int32_t metric,
                   int32_t* nn_out) {
  if (!ctx) return NNSEMD_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!x || !y || !nn_out || m < 1 || n < 1 || d < 1 || m > (1LL << 30) || n > (1LL << 30) || metric < 0 ||
      metric > 2)
    return ctx_fail(ctx, NNSEMD_ERR_INVALID_ARG, "nearest arguments");
  PCK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  DeviceScratch S;
  int* iota = S.get<int>(std::max(m, n));
  unsigned long long* keys = S.get<unsigned long long>(n);
  if (!iota || !keys) return ctx_fail(ctx, NNSEMD_ERR_OOM, "nearest scratch");
  std::vector<int> h(std::max(m, n));
  for (size_t i = 0; i < h.size(); ++i) h[i] = (int)i;
  PCK(cudaMemcpyAsync(iota, h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  if (nearest_all(x, m, y, n, d, metric == NNSEMD_L1 ? METRIC_L1 : METRIC_SQL2, iota, keys, nn_out, st))
    return ctx_fail(ctx, NNSEMD_ERR_CUDA, "nearest launch");
  PCK(cudaStreamSynchronize(st));
  return NNSEMD_OK;
}

}  // extern "C"
