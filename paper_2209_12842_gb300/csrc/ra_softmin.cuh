// Softmin weights and the weighted update over K samples (Eqs. 4, 5, 17),
// the block-level pieces shared by every kernel that forms V+: the
// handle-based update (ra_update.cu, which first forms S~ from S and CVaR),
// the batched update, and the allocation-free update (ra_noalloc.cu).
//
// Each block owns a contiguous range of samples [kb, ke).  It takes its own
// minimum m_b of the finite S~ and accumulates e_k = exp(-(S~_k - m_b) /
// lambda), s_b = sum e_k and y_b[t, j] = sum e_k U[k, t, j] in FP32 with
// Neumaier compensation (non-finite S~_k gets e_k = 0).  The last block to
// finish (arrival counter, no waiting) merges the partials: with
// m = min_b m_b every partial is rescaled by exp(-(m_b - m) / lambda), so the
// result equals subtracting the global minimum first (Eq. 17); the column
// sums merge in compensated FP32, the normalisation sum over K in FP64, and
// V+ = sum y / sum s (Eq. 4).
#pragma once

#include <cuda_runtime.h>

namespace ramppi {

constexpr int kSoftminThreads = 256;
constexpr int kSoftminWarps = kSoftminThreads / 32;
constexpr int kSoftminMaxCols = 512;       // T nu (RA_MPPI_MAX_T x 2)
constexpr int kSoftminMaxBlocks = 256;     // blocks that one merge can rescale
constexpr int kSoftminColChunks = kSoftminMaxCols / 32;
// Loads in flight before their sums: U rows per warp in the block partials
// (RIF) and partials per column in the merge (MIF).  More in flight shortens
// a single problem's update, a latency-bound launch of a few blocks; the
// batched update, many blocks at once, keeps the smaller counts and the
// registers they need.  The order of every sum is the same for any count.
constexpr int kRowsInFlight = 8, kMergeInFlight = 16;
constexpr int kBatchRowsInFlight = 4, kBatchMergeInFlight = 8;

// Shared memory of one block of a softmin update.
struct SoftminShared {
  float red[32];
  double redd[32];
  float e[kSoftminThreads];
  float col[kSoftminWarps * kSoftminMaxCols];
  float scale[kSoftminMaxBlocks];
  unsigned int is_last;
};

__device__ __forceinline__ void neumaier_add(float& sum, float& comp, float v) {
  const float t = sum + v;
  if (fabsf(sum) >= fabsf(v)) comp += (sum - t) + v;
  else comp += (v - t) + sum;
  sum = t;
}

__device__ __forceinline__ float softmin_block_min(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : __int_as_float(0x7F800000);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  v = red[0];
  __syncthreads();
  return v;
}

__device__ __forceinline__ double softmin_block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  v = red[0];
  __syncthreads();
  return v;
}

// The partials (m_b, s_b, y_b[TN]) of samples [kb, ke) into part[2 + TN],
// given the block minimum mb of their finite S~.  Threads take samples
// k0 + threadIdx.x, k0 = kb, kb + blockDim, ...; warps take rows of each
// chunk of blockDim samples and lanes the columns l, l + 32, ..., RIF
// rows in flight (a warp adds its rows w, w + 8, w + 16, ... in that order
// whatever the number in flight).  Called by all threads of a block of
// kSoftminThreads.
template <int RIF = kRowsInFlight>
__device__ __forceinline__ void softmin_block_partials(const float* __restrict__ S_tilde,
                                                       const float* __restrict__ U, int kb, int ke, int TN,
                                                       float inv_lambda, float mb, float* part,
                                                       SoftminShared& sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nj = (TN + 31) >> 5;
  float s_sum = 0.0f, s_comp = 0.0f;
  float y_sum[kSoftminColChunks], y_comp[kSoftminColChunks];
#pragma unroll
  for (int j = 0; j < kSoftminColChunks; ++j) { y_sum[j] = 0.0f; y_comp[j] = 0.0f; }
  for (int k0 = kb; k0 < ke; k0 += blockDim.x) {
    const int k = k0 + threadIdx.x;
    float e = 0.0f;
    if (k < ke) {
      const float st = S_tilde[k];
      if (isfinite(st) && isfinite(mb)) e = expf((mb - st) * inv_lambda);
    }
    sh.e[threadIdx.x] = e;
    neumaier_add(s_sum, s_comp, e);
    __syncthreads();
    const int n = min((int)blockDim.x, ke - k0);
    for (int i0 = warp; i0 < n; i0 += RIF * kSoftminWarps) {
      float ev[RIF];
      const float* rows[RIF];
#pragma unroll
      for (int u = 0; u < RIF; ++u) {
        const int i = i0 + u * kSoftminWarps;
        ev[u] = i < n ? sh.e[i] : 0.0f;
        rows[u] = U + (size_t)(k0 + (i < n ? i : 0)) * TN;
      }
#pragma unroll
      for (int j = 0; j < kSoftminColChunks; ++j) {
        const int col = lane + 32 * j;
        if (j < nj && col < TN) {
          float v[RIF];
#pragma unroll
          for (int u = 0; u < RIF; ++u) v[u] = ev[u] != 0.0f ? rows[u][col] : 0.0f;
#pragma unroll
          for (int u = 0; u < RIF; ++u)
            if (ev[u] != 0.0f) neumaier_add(y_sum[j], y_comp[j], ev[u] * v[u]);
        }
      }
    }
    __syncthreads();
  }
  // block total of e in FP64 (one value per thread, so the compensation is exact enough)
  const double sb = softmin_block_sum((double)s_sum + (double)s_comp, sh.redd);
  // merge the warps' column sums through shared memory
#pragma unroll
  for (int j = 0; j < kSoftminColChunks; ++j) {
    const int col = lane + 32 * j;
    if (j < nj && col < TN) sh.col[warp * kSoftminMaxCols + col] = y_sum[j] + y_comp[j];
  }
  __syncthreads();
  for (int col = threadIdx.x; col < TN; col += blockDim.x) {
    float y = 0.0f, yc = 0.0f;
#pragma unroll
    for (int w = 0; w < kSoftminWarps; ++w) neumaier_add(y, yc, sh.col[w * kSoftminMaxCols + col]);
    part[2 + col] = y + yc;
  }
  if (threadIdx.x == 0) {
    part[0] = mb;
    part[1] = (float)sb;
  }
}

// Publishes this block's partials and takes a ticket: true in the block that
// arrives last (after every other block's partials are visible), which then
// merges.  No block waits for another.
__device__ __forceinline__ bool softmin_arrive_last(unsigned int* arrive, int nblocks, SoftminShared& sh) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int ticket = atomicAdd(arrive, 1u);
    sh.is_last = (ticket == (unsigned int)nblocks - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!sh.is_last) return false;
  __threadfence();
  return true;
}

// The last block's merge of nb partials (stride 2 + TN floats): rescales each
// to the global minimum m by exp(-(m_b - m) / lambda), sums the columns in
// compensated FP32 and the normaliser in FP64, and writes V+ when some weight
// survived (ok).  Returns ok; *m_out, *s_out receive m and the normaliser.
// The other blocks' partials are read through L2 (ld.global.cg): they were
// stored before those blocks' fence and arrival, and L1 may hold nothing
// newer; unlike volatile loads these can be in flight together.
template <int MIF = kMergeInFlight>
__device__ __forceinline__ bool softmin_merge(const float* parts, int nb, int TN, float inv_lambda,
                                              float* __restrict__ V_out, float* m_out, double* s_out,
                                              SoftminShared& sh) {
  const int stride = 2 + TN;
  float m = __int_as_float(0x7F800000);
  for (int b = threadIdx.x; b < nb; b += blockDim.x) m = fminf(m, __ldcg(parts + (size_t)b * stride));
  m = softmin_block_min(m, sh.red);
  double s_loc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const float mbb = __ldcg(parts + (size_t)b * stride);
    const float sbb = __ldcg(parts + (size_t)b * stride + 1);
    const float sc = (isfinite(mbb) && sbb > 0.0f) ? expf((m - mbb) * inv_lambda) : 0.0f;
    sh.scale[b] = sc;
    s_loc += (double)sbb * (double)sc;
  }
  // the normalisation sum over all K samples, in FP64
  const double s_tot = softmin_block_sum(s_loc, sh.redd);
  const bool ok = isfinite(m) && s_tot > 0.0 && isfinite(s_tot);
  for (int col = threadIdx.x; col < TN; col += blockDim.x) {
    float y = 0.0f, yc = 0.0f;
#pragma unroll MIF
    for (int b = 0; b < nb; ++b) {
      const float sc = sh.scale[b];
      const float v = __ldcg(parts + (size_t)b * stride + 2 + col);
      if (sc != 0.0f) neumaier_add(y, yc, v * sc);
    }
    if (ok) V_out[col] = (float)(((double)y + (double)yc) / s_tot);
  }
  *m_out = m;
  *s_out = s_tot;
  return ok;
}

}  // namespace ramppi
