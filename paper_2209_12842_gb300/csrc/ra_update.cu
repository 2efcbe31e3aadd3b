// Softmin weights and the weighted update of the RA-MPPI controls
// (Eqs. 4, 5, 14-17).
//
// Each block owns a contiguous range of samples.  It forms
// S~_k = S_k + A CVaR_k 1{CVaR_k > C_u}, takes its own minimum m_b, and
// accumulates e_k = exp(-(S~_k - m_b) / lambda), s_b = sum e_k and
// y_b[t, j] = sum e_k U[k, t, j] in FP32 with Neumaier compensation.  The
// last block to finish (arrival counter, no waiting) merges the partials:
// with m = min_b m_b every partial is rescaled by exp(-(m_b - m) / lambda),
// so the result equals subtracting the global minimum first (Eq. 17); the
// column sums merge in compensated FP32, the normalisation sum over K in
// FP64, and V+ = sum y / sum s (Eq. 4).
#include "ra_kernels.h"

namespace ramppi {

namespace {

__device__ __forceinline__ void neumaier_add(float& sum, float& comp, float v) {
  const float t = sum + v;
  if (fabsf(sum) >= fabsf(v)) comp += (sum - t) + v;
  else comp += (v - t) + sum;
  sum = t;
}

__device__ __forceinline__ float block_min(float v, float* red) {
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

__device__ __forceinline__ double block_sum_d(double v, double* red) {
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

__device__ __forceinline__ float s_tilde_of(const DevParams& p, float S, float cv) {
  // violation cost J_C = A CVaR 1{CVaR > C_u} (Eqs. 14, 15)
  return S + ((cv > p.C_u) ? p.A * cv : 0.0f);
}

}  // namespace

// One block of the update of one problem: `block` of `nblocks` blocks that
// share the problem's samples, partials and arrival counter.
__device__ __forceinline__ void update_block(const DevParams& p, const UpdateArgs& a, int K, int TN, int block,
                                             int nblocks) {
  __shared__ float red[32];
  __shared__ double redd[32];
  __shared__ float e_s[kUpdateThreads];
  __shared__ float col_s[(kUpdateThreads / 32) * 2 * RA_MPPI_MAX_T_DEV];
  __shared__ float scale_s[kMaxUpdateBlocks];
  __shared__ unsigned int is_last;
  const int per = (K + nblocks - 1) / nblocks;
  const int kb = block * per;
  const int ke = min(K, kb + per);
  float* part = a.partials + (size_t)block * (2 + TN);

  // block minimum of the finite S~ (non-finite samples get zero weight)
  float mloc = __int_as_float(0x7F800000);
  for (int k = kb + threadIdx.x; k < ke; k += blockDim.x) {
    const float st = s_tilde_of(p, a.S[k], a.cvar[k]);
    a.S_tilde[k] = st;
    if (isfinite(st)) mloc = fminf(mloc, st);
    else atomicOr(&a.st->status, kStatusNonFinite);
  }
  const float mb = block_min(mloc, red);

  // compensated partial sums over this block's samples, 256 at a time.
  // Columns (t, j) of U: warp w takes rows i = w, w + 8, ... of each chunk and
  // lane l the columns l, l + 32, ...; four rows are in flight per iteration.
  constexpr int kWarps = kUpdateThreads / 32;
  constexpr int kColChunks = (2 * RA_MPPI_MAX_T_DEV + 31) / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nj = (TN + 31) >> 5;
  float s_sum = 0.0f, s_comp = 0.0f;
  float y_sum[kColChunks], y_comp[kColChunks];
#pragma unroll
  for (int j = 0; j < kColChunks; ++j) { y_sum[j] = 0.0f; y_comp[j] = 0.0f; }
  for (int k0 = kb; k0 < ke; k0 += blockDim.x) {
    const int k = k0 + threadIdx.x;
    float e = 0.0f;
    if (k < ke) {
      const float st = a.S_tilde[k];
      if (isfinite(st) && isfinite(mb)) e = expf((mb - st) * p.inv_lambda);
    }
    e_s[threadIdx.x] = e;
    neumaier_add(s_sum, s_comp, e);
    __syncthreads();
    const int n = min((int)blockDim.x, ke - k0);
    for (int i0 = warp; i0 < n; i0 += 4 * kWarps) {
      float ev[4];
      const float* rows[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * kWarps;
        ev[u] = i < n ? e_s[i] : 0.0f;
        rows[u] = a.U + (size_t)(k0 + (i < n ? i : 0)) * TN;
      }
#pragma unroll
      for (int j = 0; j < kColChunks; ++j) {
        const int col = lane + 32 * j;
        if (j < nj && col < TN) {
          float v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u] = ev[u] != 0.0f ? rows[u][col] : 0.0f;
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (ev[u] != 0.0f) neumaier_add(y_sum[j], y_comp[j], ev[u] * v[u]);
        }
      }
    }
    __syncthreads();
  }
  // block total of e in FP64 (one value per thread, so the compensation is exact enough)
  const double sb = block_sum_d((double)s_sum + (double)s_comp, redd);
  // merge the 8 warps' column sums through shared memory
#pragma unroll
  for (int j = 0; j < kColChunks; ++j) {
    const int col = lane + 32 * j;
    if (j < nj && col < TN) col_s[warp * 2 * RA_MPPI_MAX_T_DEV + col] = y_sum[j] + y_comp[j];
  }
  __syncthreads();
  for (int col = threadIdx.x; col < TN; col += blockDim.x) {
    float y = 0.0f, yc = 0.0f;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) neumaier_add(y, yc, col_s[w * 2 * RA_MPPI_MAX_T_DEV + col]);
    part[2 + col] = y + yc;
  }
  if (threadIdx.x == 0) {
    part[0] = mb;
    part[1] = (float)sb;
  }

  // last block merges the partials
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int ticket = atomicAdd(&a.st->arrive, 1u);
    is_last = (ticket == (unsigned int)nblocks - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();

  // rescale each block's partials to the global minimum: exp(-(m_b - m) / lambda).
  // The other blocks' partials are read through L2 (ld.global.cg): they were
  // stored before those blocks' fence and arrival, and L1 may hold nothing
  // newer; unlike volatile loads these can be in flight together.
  const int nb = nblocks;
  const int stride = 2 + TN;
  const float* parts = a.partials;
  float m = __int_as_float(0x7F800000);
  for (int b = threadIdx.x; b < nb; b += blockDim.x) m = fminf(m, __ldcg(parts + (size_t)b * stride));
  m = block_min(m, red);
  double s_loc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const float mbb = __ldcg(parts + (size_t)b * stride);
    const float sbb = __ldcg(parts + (size_t)b * stride + 1);
    const float sc = (isfinite(mbb) && sbb > 0.0f) ? expf((m - mbb) * p.inv_lambda) : 0.0f;
    scale_s[b] = sc;
    s_loc += (double)sbb * (double)sc;
  }
  // the normalisation sum over all K samples, in FP64
  const double s_tot = block_sum_d(s_loc, redd);
  const bool ok = isfinite(m) && s_tot > 0.0 && isfinite(s_tot);
  for (int col = threadIdx.x; col < TN; col += blockDim.x) {
    float y = 0.0f, yc = 0.0f;
#pragma unroll 8
    for (int b = 0; b < nb; ++b) {
      const float sc = scale_s[b];
      const float v = __ldcg(parts + (size_t)b * stride + 2 + col);
      if (sc != 0.0f) neumaier_add(y, yc, v * sc);
    }
    if (ok) a.V_out[col] = (float)(((double)y + (double)yc) / s_tot);
  }
  if (threadIdx.x == 0) {
    if (!ok) atomicOr(&a.st->status, kStatusNoWeight);
    a.st->last_min = m;
    a.st->last_sum = s_tot;
    a.st->arrive = 0u;        // ready for the next launch on this stream
    a.st->iteration += 1ull;  // the next update draws fresh noise
  }
}

__global__ void __launch_bounds__(kUpdateThreads) softmin_update_kernel(const DevParams p, const UpdateArgs a) {
  update_block(p, a, p.K, p.T * p.nu, blockIdx.x, gridDim.x);
}

// Updates of B problems in one launch: problem i owns blocks
// [upd_block_base_i, upd_block_base_i + nb_upd_i).
__global__ void __launch_bounds__(kUpdateThreads) batch_update_kernel(const DevParams p, const BatchUpdateArgs b) {
  int lo = 0, hi = b.B;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (b.desc[mid].upd_block_base <= (int)blockIdx.x) lo = mid;
    else hi = mid;
  }
  const InstDesc& d = b.desc[lo];
  UpdateArgs a;
  a.S = b.S + d.k_off;
  a.cvar = b.cvar + d.k_off;
  a.U = b.U + d.U_off;
  a.S_tilde = b.S_tilde + d.k_off;
  a.V_out = b.V_out + d.V_off;
  a.partials = b.partials + d.part_off;
  a.st = b.st + lo;
  update_block(p, a, d.K, d.T * p.nu, (int)blockIdx.x - d.upd_block_base, d.nb_upd);
}

cudaError_t launch_batch_update(const DevParams& p, const BatchUpdateArgs& a, int nblocks, cudaStream_t s) {
  batch_update_kernel<<<nblocks, kUpdateThreads, 0, s>>>(p, a);
  return cudaGetLastError();
}

cudaError_t launch_update(const DevParams& p, const UpdateArgs& a, int nblocks, cudaStream_t s) {
  softmin_update_kernel<<<nblocks, kUpdateThreads, 0, s>>>(p, a);
  return cudaGetLastError();
}

}  // namespace ramppi
