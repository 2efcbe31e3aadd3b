// Allocation-free softmin-weighted update, for callers that cannot allocate
// device memory (see ra_mppi_softmin_update_noalloc in include/ra_mppi.h).
//
// Same arithmetic as the handle-based update kernel: each block takes its own
// minimum of the costs and accumulates e_k = exp(-(S~_k - m_b) / lambda),
// sum e_k and sum e_k U[k, :] in compensated FP32; the last block to arrive
// rescales the block partials to the global minimum and divides, with the
// normalisation sum in FP64.  The only difference is where the per-block
// partials and the arrival counter live: in g_noalloc_scratch below, a
// file-scope device array that every GPU loading this library holds until
// the process exits, instead of in a handle's cudaMalloc'ed workspace.
#include <cmath>
#include <mutex>

#include <cuda_runtime.h>

#include "ra_mppi.h"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaWarps = kNaThreads / 32;
constexpr int kNaMaxBlocks = 64;                      // blocks of the update grid
constexpr int kNaMaxCols = RA_MPPI_NOALLOC_MAX_COLS;  // T * nu
constexpr int kNaStride = 2 + kNaMaxCols;             // (m_b, s_b, y_b[T nu]) per block
constexpr int kNaColChunks = kNaMaxCols / 32;
constexpr int kNaHeader = 64;                         // floats before the partials
constexpr int kNaFloats = kNaHeader + kNaMaxBlocks * kNaStride;
constexpr int kNaMaxDevices = 64;

// The scratch: word 0 is the arrival counter (must be 0 when a launch
// starts); the partials follow the header.  About 130 KB per device.
static __device__ __align__(256) float g_noalloc_scratch[kNaFloats];

__device__ __forceinline__ void na_neumaier(float& sum, float& comp, float v) {
  const float t = sum + v;
  if (fabsf(sum) >= fabsf(v)) comp += (sum - t) + v;
  else comp += (v - t) + sum;
  sum = t;
}

__device__ __forceinline__ float na_block_min(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < kNaWarps ? red[lane] : __int_as_float(0x7F800000);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  v = red[0];
  __syncthreads();
  return v;
}

__device__ __forceinline__ double na_block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < kNaWarps ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  v = red[0];
  __syncthreads();
  return v;
}

__global__ void __launch_bounds__(kNaThreads)
softmin_update_noalloc_kernel(const float* __restrict__ S_tilde, const float* __restrict__ U, int K, int TN,
                              float inv_lambda, float* __restrict__ V_out, float* scratch) {
  __shared__ float red[32];
  __shared__ double redd[32];
  __shared__ float e_s[kNaThreads];
  __shared__ float col_s[kNaWarps * kNaMaxCols];
  __shared__ float scale_s[kNaMaxBlocks];
  __shared__ unsigned int is_last;
  unsigned int* arrive = reinterpret_cast<unsigned int*>(scratch);
  float* partials = scratch + kNaHeader;
  const int per = (K + gridDim.x - 1) / gridDim.x;
  const int kb = blockIdx.x * per;
  const int ke = min(K, kb + per);
  float* part = partials + (size_t)blockIdx.x * kNaStride;

  float mloc = __int_as_float(0x7F800000);
  for (int k = kb + threadIdx.x; k < ke; k += blockDim.x) {
    const float st = S_tilde[k];
    if (isfinite(st)) mloc = fminf(mloc, st);
  }
  const float mb = na_block_min(mloc, red);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nj = (TN + 31) >> 5;
  float s_sum = 0.0f, s_comp = 0.0f;
  float y_sum[kNaColChunks], y_comp[kNaColChunks];
#pragma unroll
  for (int j = 0; j < kNaColChunks; ++j) { y_sum[j] = 0.0f; y_comp[j] = 0.0f; }
  for (int k0 = kb; k0 < ke; k0 += blockDim.x) {
    const int k = k0 + threadIdx.x;
    float e = 0.0f;
    if (k < ke) {
      const float st = S_tilde[k];
      if (isfinite(st) && isfinite(mb)) e = expf((mb - st) * inv_lambda);
    }
    e_s[threadIdx.x] = e;
    na_neumaier(s_sum, s_comp, e);
    __syncthreads();
    const int n = min((int)blockDim.x, ke - k0);
    for (int i0 = warp; i0 < n; i0 += 4 * kNaWarps) {
      float ev[4];
      const float* rows[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * kNaWarps;
        ev[u] = i < n ? e_s[i] : 0.0f;
        rows[u] = U + (size_t)(k0 + (i < n ? i : 0)) * TN;
      }
#pragma unroll
      for (int j = 0; j < kNaColChunks; ++j) {
        const int col = lane + 32 * j;
        if (j < nj && col < TN) {
          float v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u] = ev[u] != 0.0f ? rows[u][col] : 0.0f;
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (ev[u] != 0.0f) na_neumaier(y_sum[j], y_comp[j], ev[u] * v[u]);
        }
      }
    }
    __syncthreads();
  }
  const double sb = na_block_sum((double)s_sum + (double)s_comp, redd);
#pragma unroll
  for (int j = 0; j < kNaColChunks; ++j) {
    const int col = lane + 32 * j;
    if (j < nj && col < TN) col_s[warp * kNaMaxCols + col] = y_sum[j] + y_comp[j];
  }
  __syncthreads();
  for (int col = threadIdx.x; col < TN; col += blockDim.x) {
    float y = 0.0f, yc = 0.0f;
#pragma unroll
    for (int w = 0; w < kNaWarps; ++w) na_neumaier(y, yc, col_s[w * kNaMaxCols + col]);
    part[2 + col] = y + yc;
  }
  if (threadIdx.x == 0) {
    part[0] = mb;
    part[1] = (float)sb;
  }

  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int ticket = atomicAdd(arrive, 1u);
    is_last = (ticket == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();

  const int nb = gridDim.x;
  const volatile float* parts = partials;
  float m = __int_as_float(0x7F800000);
  for (int b = threadIdx.x; b < nb; b += blockDim.x) m = fminf(m, parts[(size_t)b * kNaStride]);
  m = na_block_min(m, red);
  double s_loc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const float mbb = parts[(size_t)b * kNaStride];
    const float sbb = parts[(size_t)b * kNaStride + 1];
    const float sc = (isfinite(mbb) && sbb > 0.0f) ? expf((m - mbb) * inv_lambda) : 0.0f;
    scale_s[b] = sc;
    s_loc += (double)sbb * (double)sc;
  }
  const double s_tot = na_block_sum(s_loc, redd);
  const bool ok = isfinite(m) && s_tot > 0.0 && isfinite(s_tot);
  for (int col = threadIdx.x; col < TN; col += blockDim.x) {
    float y = 0.0f, yc = 0.0f;
    for (int b = 0; b < nb; ++b) {
      const float sc = scale_s[b];
      if (sc != 0.0f) na_neumaier(y, yc, parts[(size_t)b * kNaStride + 2 + col] * sc);
    }
    if (ok) V_out[col] = (float)(((double)y + (double)yc) / s_tot);
  }
  if (threadIdx.x == 0) *arrive = 0u;
}

// Device address of the scratch array, looked up once per device with that
// device current.  In host code g_noalloc_scratch names a host-side stand-in,
// so its address must come from the runtime, never from &g_noalloc_scratch.
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
  void* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) return RA_MPPI_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the arrival counter must start at zero; clearing it is not an allocation
  e = cudaMemsetAsync(scratch, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return RA_MPPI_ECUDA;
  int blocks = (K + kNaThreads - 1) / kNaThreads;
  if (blocks > kNaMaxBlocks) blocks = kNaMaxBlocks;
  softmin_update_noalloc_kernel<<<blocks, kNaThreads, 0, s>>>(S_tilde, U, K, T * nu, 1.0f / lambda, V_out,
                                                               static_cast<float*>(scratch));
  return cudaGetLastError() == cudaSuccess ? RA_MPPI_OK : RA_MPPI_ECUDA;
}
