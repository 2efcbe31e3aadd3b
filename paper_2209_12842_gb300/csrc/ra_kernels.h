// Internal launch interface between the C ABI (ra_api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>

#include "ra_batch.cuh"
#include "ra_device.cuh"
#include "ra_rollout.cuh"

namespace ramppi {

struct UpdateArgs {
  const float* S;       // [K] nominal costs
  const float* cvar;    // [K]
  const float* U;       // [K][T][nu]
  float* S_tilde;       // [K] out (always written)
  float* V_out;         // [T][nu] out
  float* partials;      // [nblocks][2 + T nu]
  DevState* st;
};

// Rollout kernel launch for one model; ilp in {1, 2, 4}; `pairs`: two
// samples per warp (dynamic model, ilp 2, at most 32 rollouts per sample);
// `is`: importance-sampled rollouts (ilp 1 or 2, not with pairs); `win`: the
// obstacle cull's x window (dynamic model, neither pairs nor is; ignored
// otherwise).
template <int MODEL>
cudaError_t launch_rollout(const DevParams& p, const RolloutArgs& a, int warps, int ilp, bool pairs, bool is,
                           bool win, size_t smem, int grid, cudaStream_t s);
// Raise the dynamic shared memory limit of every instance of a model.
template <int MODEL>
cudaError_t prepare_rollout(size_t smem);
// Resident blocks per SM of the instance launch_rollout runs for these
// arguments (ck: the checkpointing instances of differentiable handles).
template <int MODEL>
cudaError_t rollout_occupancy(int warps, int ilp, bool pairs, bool is, bool win, bool ck, size_t smem, int* blocks);

cudaError_t launch_update(const DevParams& p, const UpdateArgs& a, int nblocks, cudaStream_t s);

// Adjoint of the last update (ra_adjoint.cu).
struct BwdArgs {
  const float* x0;      // [nx] state of the differentiated update
  const float* V;       // [T][nu] its mean controls
  const float* U;       // [K][T][nu] its samples
  const float* S;       // [K]
  const float* cvar;    // [K]
  const float* L;       // [K][M] risk costs of the update (then [K][M] importance weights)
  const float* ck_nom;  // [K][nseg + 1][NX] nominal state checkpoints of the update (x_0, x_8, ..., x_T)
  const float* ck_dist; // [K][nseg][NX][M] disturbed state checkpoints of the update
  const float4* obs;
  DevState* st;
  const float* gVp;     // [T][nu]
  const float* gS;      // [K] or nullptr
  float* dk;            // [K] d_k = <gV+, U_k>
  float* wk;            // [K] the softmin weights w^_k
  unsigned int* arrive; // [2] arrival counter of the reduction (the other is spare)
  float* Gnom;          // [K][T][nu]
  float* mask;          // [K][T][nu]
  float* gUd;           // [K][T][nu]
  float* thn;           // [K][4]
  float* thd;           // [K][4]
  double* red_part;     // [nb_red][3 (T nu + 4) + 1] the reduction's slice partials
  float* gV;            // [T][nu] out
  float* gtheta;        // [4] out
  int nb_nom, obs_cap;  // nb_nom: 128-thread blocks at one lane per nominal rollout
};
// (ev_begin / ev_end: optional events recorded around the main kernel)
cudaError_t launch_backward(int model, const DevParams& p, const BwdArgs& a, int nb_dist, size_t smem, int nb_red,
                            cudaStream_t s, cudaEvent_t ev_begin = nullptr, cudaEvent_t ev_end = nullptr);

// Batched path (ra_batch.cuh, ra_batch.cu): persistent rollout kernel of one
// model, its shared-memory limit and occupancy, and the batched update
// (`is`: importance-sampled rollouts).
template <int MODEL>
cudaError_t launch_batch_rollout(const DevParams& p, const BatchArgs& a, int warps, int ilp, bool is, size_t smem,
                                 int grid, cudaStream_t s);
template <int MODEL>
cudaError_t prepare_batch_rollout(size_t smem);
template <int MODEL>
cudaError_t batch_rollout_occupancy(int warps, int ilp, bool is, size_t smem, int* blocks_per_sm);

struct BatchUpdateArgs {
  const InstDesc* desc;
  int B;
  DevState* st;
  const float* S;
  const float* cvar;
  const float* U;
  float* S_tilde;
  float* V_out;
  float* partials;
};
cudaError_t launch_batch_update(const DevParams& p, const BatchUpdateArgs& a, int nblocks, cudaStream_t s);

// Plant step of the receding-horizon loop (ra_plant.cu).
cudaError_t launch_plant(int model, const DevParams& p, const float4* obs, DevState* st, float* x,
                         const float* V_plus, float* V_next, int* collisions, int shift, cudaStream_t s);

constexpr int kUpdateThreads = 256;
// Update blocks of one problem: 64 samples each (fewer than the block's
// threads: a shorter serial part per block, the update spread over more SMs),
// but at most 256 blocks, beyond which the last block's merge of the partials
// costs more than it saves (GB300: 15 us less per update at K = 4096, 60 us
// more at K = 65536 with 1024 blocks).
constexpr int kUpdateSamplesPerBlock = 64;
constexpr int kUpdateBlocksCap = 256;
__host__ __device__ constexpr int update_blocks(long long K) {
  return (int)((K + kUpdateSamplesPerBlock - 1) / kUpdateSamplesPerBlock < kUpdateBlocksCap
                   ? (K + kUpdateSamplesPerBlock - 1) / kUpdateSamplesPerBlock
                   : kUpdateBlocksCap);
}
constexpr int kMaxUpdateBlocks = kUpdateBlocksCap;  // shared-memory bound of the merge

}  // namespace ramppi
