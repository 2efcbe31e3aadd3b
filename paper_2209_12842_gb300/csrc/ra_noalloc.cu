// Allocation-free softmin-weighted update, for callers that cannot allocate
// device memory (see ra_mppi_softmin_update_noalloc in include/ra_mppi.h).
//
// The same block partials and last-block merge as the handle-based update
// (ra_softmin.cuh): each block takes its own minimum of the costs and
// accumulates e_k = exp(-(S~_k - m_b) / lambda), sum e_k and sum e_k U[k, :]
// in compensated FP32; the last block to arrive rescales the block partials
// to the global minimum and divides, with the normalisation sum in FP64.  The
// only difference is where the per-block partials and the arrival counter
// live: in g_noalloc_scratch below, a file-scope device array that every GPU
// loading this library holds until the process exits, instead of in a
// handle's cudaMalloc'ed workspace.
#include <cmath>
#include <mutex>

#include <cuda_runtime.h>

#include "ra_mppi.h"
#include "ra_softmin.cuh"

namespace {

using ramppi::SoftminShared;

constexpr int kNaMaxBlocks = 64;                      // blocks of the update grid
constexpr int kNaMaxCols = RA_MPPI_NOALLOC_MAX_COLS;  // T * nu
constexpr int kNaStride = 2 + kNaMaxCols;             // (m_b, s_b, y_b[T nu]) per block
constexpr int kNaHeader = 64;                         // floats before the partials
constexpr int kNaFloats = kNaHeader + kNaMaxBlocks * kNaStride;
constexpr int kNaMaxDevices = 64;
static_assert(kNaMaxCols <= ramppi::kSoftminMaxCols, "columns fit the shared block sums");
static_assert(kNaMaxBlocks <= ramppi::kSoftminMaxBlocks, "the merge rescales every block");

// The scratch: word 0 is the arrival counter (must be 0 when a launch
// starts); the partials follow the header, packed with stride 2 + T nu of
// the call.  About 130 KB per device.
static __device__ __align__(256) float g_noalloc_scratch[kNaFloats];

__global__ void __launch_bounds__(ramppi::kSoftminThreads, 2)
softmin_update_noalloc_kernel(const float* __restrict__ S_tilde, const float* __restrict__ U, int K, int TN,
                              float inv_lambda, float* __restrict__ V_out, float* scratch) {
  __shared__ SoftminShared sh;
  unsigned int* arrive = reinterpret_cast<unsigned int*>(scratch);
  float* partials = scratch + kNaHeader;
  const int per = (K + gridDim.x - 1) / gridDim.x;
  const int kb = blockIdx.x * per;
  const int ke = min(K, kb + per);

  float mloc = __int_as_float(0x7F800000);
  for (int k = kb + threadIdx.x; k < ke; k += blockDim.x) {
    const float st = S_tilde[k];
    if (isfinite(st)) mloc = fminf(mloc, st);
  }
  const float mb = ramppi::softmin_block_min(mloc, sh.red);
  ramppi::softmin_block_partials(S_tilde, U, kb, ke, TN, inv_lambda, mb, partials + (size_t)blockIdx.x * (2 + TN),
                                 sh);
  if (!ramppi::softmin_arrive_last(arrive, (int)gridDim.x, sh)) return;
  float m;
  double s_tot;
  ramppi::softmin_merge(partials, (int)gridDim.x, TN, inv_lambda, V_out, &m, &s_tot, sh);
  if (threadIdx.x == 0) *arrive = 0u;
}

// Device address of the scratch array, looked up once per device with that
// device current.  In host code g_noalloc_scratch names a host-side stand-in,
// so its address must come from the runtime, never from &g_noalloc_scratch.
// The cached address belongs to the device's current context: after
// cudaDeviceReset the module loads again and the cache would be stale, so a
// process that resets a device must not call this entry point afterwards.
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kNaMaxDevices] = {};

cudaError_t scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int ra_mppi_softmin_update_noalloc(const float* S_tilde, const float* U, int32_t K, int32_t T,
                                              int32_t nu, float lambda, float* V_out, void* stream) {
  if (S_tilde == nullptr || U == nullptr || V_out == nullptr) return RA_MPPI_EINVAL;
  if (K < 1 || K > (1 << 24) || T < 1 || nu < 1 || (int64_t)T * nu > kNaMaxCols) return RA_MPPI_EINVAL;
  if (!(lambda > 0.0f) || !std::isfinite(lambda)) return RA_MPPI_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the scratch is the current device's: a stream of another device would
  // run the kernel there on a foreign address
  int dev = 0, sdev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RA_MPPI_ECUDA;
  if (cudaStreamGetDevice(s, &sdev) != cudaSuccess) return RA_MPPI_ECUDA;
  if (sdev != dev) return RA_MPPI_EINVAL;
  void* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) return RA_MPPI_ECUDA;
  // the arrival counter must start at zero; clearing it is not an allocation
  e = cudaMemsetAsync(scratch, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return RA_MPPI_ECUDA;
  int blocks = (K + ramppi::kSoftminThreads - 1) / ramppi::kSoftminThreads;
  if (blocks > kNaMaxBlocks) blocks = kNaMaxBlocks;
  softmin_update_noalloc_kernel<<<blocks, ramppi::kSoftminThreads, 0, s>>>(S_tilde, U, K, T * nu, 1.0f / lambda,
                                                                             V_out, static_cast<float*>(scratch));
  return cudaGetLastError() == cudaSuccess ? RA_MPPI_OK : RA_MPPI_ECUDA;
}
