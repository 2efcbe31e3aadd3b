// Simulated plant of the receding-horizon loop (Algorithm 1, outer loop):
// execute the first control of V+ on x~_{n+1} = F(x~_n, v0+) + w_n with the
// plant's own noise stream, count the steps whose new state is inside an
// obstacle and those off the track, and warm-start the next update from V+ (shifted
// left by one step, the last control repeated, when `shift` is set).
#include "ra_kernels.h"

namespace ramppi {

template <int MODEL>
__global__ void plant_step_kernel(const DevParams p, const float4* __restrict__ obs, DevState* st,
                                  float* __restrict__ x, const float* __restrict__ V_plus,
                                  float* __restrict__ V_next, int* __restrict__ collisions, int shift) {
  // one warp: every lane steps the same state (no divergence, no broadcast
  // needed), then the lanes split the obstacle test and the warm-start copy
  using Md = Model<MODEL>;
  const int lane = threadIdx.x;
  // the update that produced V+ has already advanced the counter: the plant
  // step belongs to the iteration before it
  const uint32_t iter = (uint32_t)(st->iteration - 1ull);
  const uint32_t k0 = p.seed_lo, k1 = p.seed_hi ^ iter;
  float s[Md::NX];
#pragma unroll
  for (int i = 0; i < Md::NX; ++i) s[i] = x[i];
  const float u0 = V_plus[0];
  const float u1 = Md::NU > 1 ? V_plus[1] : 0.0f;
  Md::step_exact(p, s, Md::ctl(p, u0, u1));
  add_process_noise<MODEL>(p, k0, k1, 0u, 0xFFFFFFFEu, 0xFFFFFFFFu, p.instance, s);
  if (MODEL != 2 && collisions != nullptr) {
    bool hit = false;
    const int n_obs = st->n_obs;
    for (int i = lane; i < n_obs; i += 32) {
      const float4 o = obs[i];
      const float dx = s[0] - o.x, dy = s[1] - o.y;
      hit |= fmaf(dx, dx, dy * dy) < o.w;
    }
    hit = __any_sync(0xFFFFFFFFu, hit);
    const bool off = fabsf(track_e(p, s[0], s[1])) > p.track_hw;
    if (lane == 0) {
      if (hit) atomicAdd(collisions, 1);      // inside an obstacle
      if (off) atomicAdd(collisions + 1, 1);  // off the track
    }
  }
  __syncwarp();  // every lane has read x before lane 0 overwrites it
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < Md::NX; ++i) x[i] = s[i];
  }
  const int TN = p.T * p.nu;
  for (int c = lane; c < TN; c += 32) {
    const int src = (shift && c + p.nu < TN) ? c + p.nu : c;
    V_next[c] = V_plus[src];
  }
}

cudaError_t launch_plant(int model, const DevParams& p, const float4* obs, DevState* st, float* x,
                         const float* V_plus, float* V_next, int* collisions, int shift, cudaStream_t s) {
  switch (model) {
    case 0: plant_step_kernel<0><<<1, 32, 0, s>>>(p, obs, st, x, V_plus, V_next, collisions, shift); break;
    case 1: plant_step_kernel<1><<<1, 32, 0, s>>>(p, obs, st, x, V_plus, V_next, collisions, shift); break;
    default: plant_step_kernel<2><<<1, 32, 0, s>>>(p, obs, st, x, V_plus, V_next, collisions, shift); break;
  }
  return cudaGetLastError();
}

}  // namespace ramppi
