// Internal launch interface between the C ABI (ra_api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>

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

// Rollout kernel launch for one model; ilp in {1, 2, 4}.
template <int MODEL>
cudaError_t launch_rollout(const DevParams& p, const RolloutArgs& a, int warps, int ilp,
                           size_t smem, int grid, cudaStream_t s);
// Raise the dynamic shared memory limit of every instance of a model.
template <int MODEL>
cudaError_t prepare_rollout(size_t smem);

cudaError_t launch_update(const DevParams& p, const UpdateArgs& a, int nblocks, cudaStream_t s);

constexpr int kUpdateThreads = 256;
constexpr int kMaxUpdateBlocks = 1024;

}  // namespace ramppi
