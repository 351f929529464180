// Allocation-free SYMV of one tile-packed symmetric matrix.
//
// Some callers cannot allocate device memory at the point where they need a
// dense symmetric apply: code running inside a memory pool or arena that
// forbids new allocations, real-time loops where cudaMalloc / cudaFree would
// synchronise the device or stall, and embedding hosts whose allocator owns
// all device memory.  This entry point serves them: the caller passes the
// matrix, x and y, and the only scratch (the streaming SYMV's row and column
// partial sums plus its error word) lives in a file-scope __device__ array
// of fixed size that every GPU loading the library keeps until exit.
//
// The kernels are a single-matrix variant of the batched streaming SYMV
// (dense.cu): 64x64 tiles streamed into shared memory by cp.async.bulk on
// mbarriers, row partials per tile row, column partials per tile, then a
// deterministic reduction.
#include <mutex>

#include "common.cuh"

namespace geneo {
namespace {

constexpr int kNaMaxDim = 4096;                          // largest dimension accepted
constexpr int kNaMaxNt = kNaMaxDim / kTile;              // 64 tiles per side
constexpr int kNaMaxTiles = kNaMaxNt * (kNaMaxNt + 1) / 2;
constexpr int kNaStages = 4;
// scratch layout (doubles): [0, kNaMaxDim) row partials, then kTile column
// partials per stored tile, then one slot holding the error word
constexpr int64_t kNaColOff = kNaMaxDim;
constexpr int64_t kNaErrOff = kNaColOff + (int64_t)kNaMaxTiles * kTile;
constexpr int64_t kNaScratch = kNaErrOff + 1;
constexpr int kNaDrainLost = 0x7fff;  // error word: a drain wait gave up too

static __device__ __align__(256) double g_noalloc_scratch[kNaScratch];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

__device__ __forceinline__ uint32_t na_smem(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ bool na_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, "
      "0, p;\n}" : "=r"(ok) : "r"(na_smem(bar)), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool na_wait(uint64_t *bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!na_try_wait(bar, parity))
    if (clock64() - t0 > 4000000000LL) return false;
  return true;
}

// strips (tile rows) I = blockIdx.x, blockIdx.x + gridDim.x, ...
__global__ void __launch_bounds__(256, 1)
    k_na_symv(const double *__restrict__ tiles, int nt, int dim, const double *__restrict__ x,
              double *__restrict__ scratch) {
  extern __shared__ __align__(128) unsigned char smraw[];
  double *stage = reinterpret_cast<double *>(smraw);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smraw + (size_t)kNaStages * kTileElems * 8);
  double *red = reinterpret_cast<double *>(bar + kNaStages);
  double *rowpart = scratch, *colpart = scratch + kNaColOff;
  int *err = reinterpret_cast<int *>(scratch + kNaErrOff);
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  if (blockIdx.x >= nt) return;
  if (tid == 0) {
    for (int i = 0; i < kNaStages; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(na_smem(&bar[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  int pI = blockIdx.x, pJ = 0;
  long long issued = 0, consumed = 0;
  auto issue = [&]() {
    if (pI >= nt) return;
    const double *src = tiles + ((int64_t)pI * (pI + 1) / 2 + pJ) * kTileElems;
    const int st = (int)(issued % kNaStages);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(na_smem(&bar[st])),
                 "r"(kTileElems * 8)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(na_smem(stage + (size_t)st * kTileElems)),
        "l"(src), "r"(kTileElems * 8), "r"(na_smem(&bar[st]))
        : "memory");
    ++issued;
    if (++pJ > pI) {
      pJ = 0;
      pI += gridDim.x;
    }
  };
  if (tid == 0)
    for (int q = 0; q < kNaStages; ++q) issue();
  bool failed = false;
  for (int I = blockIdx.x; I < nt && !failed; I += gridDim.x) {
    double xi[8], rp[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int row = I * kTile + w * 8 + r;
      xi[r] = row < dim ? x[row] : 0.0;
      rp[r] = 0.0;
    }
    for (int J = 0; J <= I; ++J) {
      const int st = (int)(consumed % kNaStages);
      const bool ok = na_wait(&bar[st], (uint32_t)((consumed / kNaStages) & 1));
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicCAS(err, 0, kDevTimeout);
        failed = true;
        break;
      }
      const double *t = stage + (size_t)st * kTileElems;
      const int c0 = J * kTile + 2 * l;
      const double xj0 = c0 < dim ? x[c0] : 0.0, xj1 = c0 + 1 < dim ? x[c0 + 1] : 0.0;
      double a0 = 0, a1 = 0;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const double2 v = *reinterpret_cast<const double2 *>(t + (w * 8 + r) * kTile + 2 * l);
        rp[r] = fma(v.x, xj0, fma(v.y, xj1, rp[r]));
        a0 = fma(v.x, xi[r], a0);
        a1 = fma(v.y, xi[r], a1);
      }
      if (J < I) {
        red[w * kTile + 2 * l] = a0;
        red[w * kTile + 2 * l + 1] = a1;
      }
      __syncthreads();
      if (J < I && tid < kTile) {
        double sum = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) sum += red[q * kTile + tid];
        colpart[((int64_t)I * (I + 1) / 2 + J) * kTile + tid] = sum;
      }
      ++consumed;
      if (tid == 0) issue();
    }
    if (failed) break;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      double v = rp[r];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (l == 0) rowpart[I * kTile + w * 8 + r] = v;
    }
  }
  // drain the copies still in flight before the CTA leaves; a drain wait
  // that gives up as well is recorded separately: a copy may then still land
  // in this CTA's shared memory after it exits, so the host reports the
  // context as lost (GENEO_ERR_CUDA) instead of a recoverable timeout
  if (failed && tid == 0)
    while (consumed < issued) {
      if (!na_wait(&bar[consumed % kNaStages], (uint32_t)((consumed / kNaStages) & 1)))
        atomicExch(err, kNaDrainLost);
      ++consumed;
    }
}

// y[I*64 + r] = rowpart + sum_{K > I} colpart(K, I), rows below dim only
__global__ void k_na_reduce(int nt, int dim, const double *__restrict__ scratch,
                            double *__restrict__ y) {
  const int I = blockIdx.x, r = threadIdx.x;
  const int row = I * kTile + r;
  if (row >= dim) return;
  const double *colpart = scratch + kNaColOff;
  double v = scratch[row];
  for (int K = I + 1; K < nt; ++K) v += colpart[((int64_t)K * (K + 1) / 2 + I) * kTile + r];
  y[row] = v;
}

}  // namespace
}  // namespace geneo

extern "C" int geneo_symv_packed_noalloc(const double *tiles, int32_t dim, const double *x,
                                         double *y, void *stream) {
  using namespace geneo;
  if (!tiles || !x || !y) return GENEO_ERR_INVALID_ARG;
  if (dim < 1 || dim > kNaMaxDim) return GENEO_ERR_INVALID_ARG;
  // cp.async.bulk reads the tiles from 16-byte aligned addresses only; x and
  // y are read and written as float64
  if (((uintptr_t)tiles & 15) != 0 || ((uintptr_t)x & 7) != 0 || ((uintptr_t)y & 7) != 0)
    return GENEO_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GENEO_ERR_CUDA;
  const size_t smem = (size_t)kNaStages * kTileElems * 8 + kNaStages * 8 + 8 * kTile * 8;
  {
    // once per device, with that device current: the device address of the
    // static scratch, the SM count and the shared-memory opt-in
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GENEO_ERR_CUDA;
      int sms = 0;
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GENEO_ERR_CUDA;
      if (cudaFuncSetAttribute(k_na_symv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem) != cudaSuccess)
        return GENEO_ERR_CUDA;
      g_sm_count[dev] = sms;
      g_scratch_ptr[dev] = static_cast<double *>(p);
    }
  }
  double *scratch = g_scratch_ptr[dev];
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int nt = (dim + kTile - 1) / kTile;
  // the error word must start at zero; every partial sum read later in the
  // call is written earlier in the same call
  if (cudaMemsetAsync(scratch + kNaErrOff, 0, sizeof(double), s) != cudaSuccess)
    return GENEO_ERR_CUDA;
  const int grid = nt < g_sm_count[dev] ? nt : g_sm_count[dev];
  k_na_symv<<<grid, 256, smem, s>>>(tiles, nt, dim, x, scratch);
  k_na_reduce<<<nt, kTile, 0, s>>>(nt, dim, scratch, y);
  if (cudaGetLastError() != cudaSuccess) return GENEO_ERR_CUDA;
  // the call is synchronous so that a device-side wait that gave up is
  // reported here
  int e = 0;
  if (cudaStreamSynchronize(s) != cudaSuccess) return GENEO_ERR_CUDA;
  if (cudaMemcpy(&e, scratch + kNaErrOff, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return GENEO_ERR_CUDA;
  if (e == kNaDrainLost) return GENEO_ERR_CUDA;
  return e ? GENEO_ERR_TIMEOUT : GENEO_OK;
}
