// Shared helpers of the CUDA library: status propagation, device buffers,
// the device error word and small launch utilities.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/geneo.h"

namespace geneo {

// An exception carrying a public status code; caught at the C-ABI boundary.
struct Error : std::runtime_error {
  int status;
  Error(int s, const std::string &m) : std::runtime_error(m), status(s) {}
};

#define GENEO_CUDA(call)                                                                   \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      throw ::geneo::Error(e_ == cudaErrorMemoryAllocation ? GENEO_ERR_OOM : GENEO_ERR_CUDA, \
                           std::string(#call) + ": " + cudaGetErrorString(e_));            \
  } while (0)

#define GENEO_CHECK_LAUNCH() GENEO_CUDA(cudaGetLastError())

// Owning device allocation.
template <class T>
struct DevBuf {
  T *p = nullptr;
  int64_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  DevBuf(DevBuf &&o) noexcept : p(o.p), n(o.n) {
    o.p = nullptr;
    o.n = 0;
  }
  DevBuf &operator=(DevBuf &&o) noexcept {
    if (this != &o) {
      release();
      p = o.p;
      n = o.n;
      o.p = nullptr;
      o.n = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  void alloc(int64_t count) {
    release();
    n = count;
    if (count > 0) GENEO_CUDA(cudaMalloc((void **)&p, sizeof(T) * (size_t)count));
  }
  void zero(cudaStream_t s = 0) {
    if (n) GENEO_CUDA(cudaMemsetAsync(p, 0, sizeof(T) * (size_t)n, s));
  }
  void upload(const std::vector<T> &h, cudaStream_t s = 0) {
    alloc((int64_t)h.size());
    if (n) GENEO_CUDA(cudaMemcpyAsync(p, h.data(), sizeof(T) * (size_t)n, cudaMemcpyHostToDevice, s));
  }
  std::vector<T> download(cudaStream_t s = 0) const {
    std::vector<T> h((size_t)n);
    if (n) {
      GENEO_CUDA(cudaMemcpyAsync(h.data(), p, sizeof(T) * (size_t)n, cudaMemcpyDeviceToHost, s));
      GENEO_CUDA(cudaStreamSynchronize(s));
    }
    return h;
  }
  int64_t bytes() const { return n * (int64_t)sizeof(T); }
};

// Event record that also works while the stream is being captured into a
// CUDA graph (it then becomes an event record node fired at every replay).
inline void record_event(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  GENEO_CUDA(cudaStreamIsCapturing(s, &st));
  if (st == cudaStreamCaptureStatusActive)
    GENEO_CUDA(cudaEventRecordWithFlags(e, s, cudaEventRecordExternal));
  else
    GENEO_CUDA(cudaEventRecord(e, s));
}

inline unsigned grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 0x7fffffff) g = 0x7fffffff;
  return (unsigned)g;
}

// Device-side error word: kernels record the first failure here and the host
// turns it into a status after synchronising.
enum DevErr : int {
  kDevOk = 0,
  kDevNotSPD = 1,   // non-positive pivot
  kDevTimeout = 2,  // a bounded mbarrier wait gave up
};

constexpr int kTile = 64;             // tile edge of the packed symmetric matrices
constexpr int kTileElems = kTile * kTile;
constexpr int kTcMaxBlocks = 16;      // tensor-core local solves: n_i <= 16 * 128

}  // namespace geneo
