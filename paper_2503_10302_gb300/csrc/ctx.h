// The context object behind pc_ctx* and its device-memory holders.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "internal.h"

namespace pc {

// Owning device buffer (cudaMalloc / cudaFree).
template <typename T>
struct DevBuf {
  T *p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { reset(); }
  void reset() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  int alloc(size_t count) {
    reset();
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      return fail(PC_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    n = count;
    return PC_OK;
  }
  int zero(cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(p, 0, n * sizeof(T), st);
    return e == cudaSuccess ? PC_OK : fail(PC_ECUDA, cudaGetErrorString(e));
  }
};

// Owning pinned host buffer (cudaMallocHost / cudaFreeHost) used to stage
// host->device copies.
template <typename T>
struct PinnedBuf {
  T *p = nullptr;
  size_t n = 0;
  PinnedBuf() = default;
  PinnedBuf(const PinnedBuf &) = delete;
  PinnedBuf &operator=(const PinnedBuf &) = delete;
  ~PinnedBuf() { reset(); }
  void reset() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    n = 0;
  }
  int reserve(size_t count) {
    if (count <= n && p) return PC_OK;
    reset();
    cudaError_t e = cudaMallocHost(&p, (count ? count : 1) * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      return fail(PC_ENOMEM, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
    }
    n = count ? count : 1;
    return PC_OK;
  }
};

struct SqaState {
  bool ready = false;
  Lattice lat{};
  int P = 0, S = 0;
  double T = 0;
  std::vector<uint32_t> table;   // [S][24]
  std::vector<int32_t> jq;       // [S]
  DevBuf<uint16_t> d_jneg;
  int nbonds = 0;
  DevBuf<uint32_t> d_table;
  PinnedBuf<uint8_t> stage;       // pinned staging of jneg + tables
  DevBuf<int32_t> d_E;            // per-call output scratch of pc_sqa_run
  DevBuf<int8_t> d_spins;
  DevBuf<uint32_t> d_state;       // run states between chunks of the persistent schedule
  DevBuf<int> d_sync;             // [R] chunks done, queue counter, error flag
  int *last_err = nullptr;        // error flag of the last persistent anneal
  void release() {
    ready = false;
    d_jneg.reset();
    d_table.reset();
    d_E.reset();
    d_spins.reset();
    d_state.reset();
    d_sync.reset();
    last_err = nullptr;
  }
};

// Bookkeeping of the loaded APT batch; the batch itself (device arrays,
// CUDA graph) lives in apt_api.cpp behind pc_ctx::apt_impl.
struct AptState {
  bool ready = false;
  int n = 0, A = 0;
  int64_t sweeps = 0, swaps = 0;
};

}  // namespace pc

struct pc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint64_t seed = 0;
  int sms = 0;
  int smem_optin = 0;
  pc::SqaState sqa;
  pc::AptState apt;
  void *apt_impl = nullptr;
  void *graph_impl = nullptr;   // APT batch on general graphs (graph_api.cpp)
};

void pc_apt_release_impl(pc_ctx *c);
void pc_graph_release_impl(pc_ctx *c);
