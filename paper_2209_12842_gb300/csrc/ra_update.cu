// Violation cost, softmin weights and the weighted update of the RA-MPPI
// controls (Eqs. 4, 5, 14-17).
//
// Each block owns a contiguous range of samples.  It forms
// S~_k = S_k + A CVaR_k 1{CVaR_k > C_u} and then runs the block partials and
// the last block's merge of ra_softmin.cuh (min-shifted weights, compensated
// FP32 column sums, FP64 normaliser).
#include "ra_kernels.h"
#include "ra_softmin.cuh"

namespace ramppi {

static_assert(kUpdateThreads == kSoftminThreads, "update blocks are softmin blocks");
static_assert(kMaxUpdateBlocks <= kSoftminMaxBlocks, "the merge rescales every update block");
static_assert(2 * RA_MPPI_MAX_T_DEV <= kSoftminMaxCols, "T nu columns fit the block's column sums");

namespace {

__device__ __forceinline__ float s_tilde_of(const DevParams& p, float S, float cv) {
  // violation cost J_C = A CVaR 1{CVaR > C_u} (Eqs. 14, 15)
  return S + ((cv > p.C_u) ? p.A * cv : 0.0f);
}

}  // namespace

// One block of the update of one problem: `block` of `nblocks` blocks that
// share the problem's samples, partials and arrival counter.
// RIF, MIF: loads in flight in the partials and the merge (ra_softmin.cuh).
template <int RIF, int MIF>
__device__ __forceinline__ void update_block(const DevParams& p, const UpdateArgs& a, int K, int TN, int block,
                                             int nblocks) {
  __shared__ SoftminShared sh;
  const int per = (K + nblocks - 1) / nblocks;
  const int kb = block * per;
  const int ke = min(K, kb + per);

  // S~ of this block's samples and their minimum (non-finite samples get
  // zero weight and set the status word)
  float mloc = __int_as_float(0x7F800000);
  for (int k = kb + threadIdx.x; k < ke; k += blockDim.x) {
    const float st = s_tilde_of(p, a.S[k], a.cvar[k]);
    a.S_tilde[k] = st;
    if (isfinite(st)) mloc = fminf(mloc, st);
    else atomicOr(&a.st->status, kStatusNonFinite);
  }
  const float mb = softmin_block_min(mloc, sh.red);
  // each thread reads back only the S~ it wrote above (same sample mapping)
  softmin_block_partials<RIF>(a.S_tilde, a.U, kb, ke, TN, p.inv_lambda, mb, a.partials + (size_t)block * (2 + TN), sh);
  if (!softmin_arrive_last(&a.st->arrive, nblocks, sh)) return;
  float m;
  double s_tot;
  const bool ok = softmin_merge<MIF>(a.partials, nblocks, TN, p.inv_lambda, a.V_out, &m, &s_tot, sh);
  if (threadIdx.x == 0) {
    if (!ok) atomicOr(&a.st->status, kStatusNoWeight);
    a.st->last_min = m;
    a.st->last_sum = s_tot;
    a.st->arrive = 0u;        // ready for the next launch on this stream
    a.st->iteration += 1ull;  // the next update draws fresh noise
  }
}

__global__ void __launch_bounds__(kUpdateThreads, 2) softmin_update_kernel(const DevParams p, const UpdateArgs a) {
  update_block<kRowsInFlight, kMergeInFlight>(p, a, p.K, p.T * p.nu, blockIdx.x, gridDim.x);
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
  update_block<kBatchRowsInFlight, kBatchMergeInFlight>(p, a, d.K, d.T * p.nu, (int)blockIdx.x - d.upd_block_base,
                                                        d.nb_upd);
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
