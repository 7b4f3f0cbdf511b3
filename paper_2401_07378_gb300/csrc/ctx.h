// The library context (opaque to callers of include/nnsemd.h) and the error
// helpers shared by the entry-point files.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "nnsemd.h"

// A captured batched launch (NNSEMD_FLAG_GRAPH), valid while every pointer
// and size in the key repeats.
struct BatchGraph {
  std::vector<uintptr_t> key;
  cudaGraphExec_t exec = nullptr;
};

struct nnsemd_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  nnsemd::DevState* hstate = nullptr;  // pinned mirror of the device state
  volatile int* hmap = nullptr;        // mapped pinned words: a round's active counts (host view)
  int* dmap = nullptr;                 // the same words, device view
  int notify_seq = 0;                  // sequence number of the last requested notification
  std::string err;
  long long launches = 0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // kernel timing (NNSEMD_FLAG_TIME_KERNELS)
  // autotuner: (d, precision, cap) -> (bn, stages, distance cache on) of the
  // batched tensor-core kernel
  std::map<std::tuple<int, int, int>, std::tuple<int, int, int>> tuned;
  std::vector<BatchGraph> graphs;
  cudaStream_t capture_stream = nullptr;
};

namespace nnsemd {
// Record a formatted message on ctx (or the thread's create-error slot when
// ctx is null) and return `status`.
int ctx_fail(nnsemd_ctx* ctx, int status, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
}  // namespace nnsemd
