// Batched RA-MPPI updates: B independent problems with their own K, M, T,
// seed and obstacle field in one persistent launch, replayed from a CUDA
// graph.  The work items are the single-problem kernel's (nominal: 32
// samples, one per lane; disturbed: one sample per warp); warps pull them
// from one atomic queue, nominal items of every problem first, then the
// disturbed items of the problems in decreasing order of per-sample cost, so
// the longest items start first and the tail is short.
#pragma once

#include "ra_rollout.cuh"

namespace ramppi {

// Per-problem descriptor (device array); offsets index the packed buffers.
struct InstDesc {
  int K, M, T, n_warm, j_var;
  float frac_j, tail_denom;
  uint32_t instance, seed_lo, seed_hi;
  int obs_cap;          // obstacle capacity of this problem
  int nb_upd;           // update blocks of this problem
  int upd_block_base;   // first update block of this problem
  int is_m0;            // importance sampling: first proposal rollout,
  float is_b, is_base;  // proposal fraction, -(draws per rollout) ln s
  int pad_;
  long long x0_off, V_off, U_off, k_off, obs_off, part_off;
};

struct BatchArgs {
  const InstDesc* desc;
  DevState* st;             // [B]
  int B;
  const float* x0;          // packed [B][nx]
  const float* V;           // packed [sum T_i][nu]
  const float4* obs;        // packed [sum obs_cap_i]
  float* U;                 // packed [sum K_i T_i][nu]
  float* S;                 // packed [sum K_i]
  float* cvar;              // packed [sum K_i]
  const long long* seg_base;  // [2B + 1]: first item of each segment
  const int* seg_inst;        // [2B]: problem of each segment
  long long n_items;
  unsigned long long* queue;  // work counter, zeroed before each launch
  int obs_cap_max, T_max, M_max;
};

// float4 slots of one warp's shared memory: obstacles, controls, risk costs
// (and importance weights)
__host__ __device__ inline int batch_warp_f4(int obs_cap_max, int T_max, int M_max, bool is = false) {
  return obs_cap_max + T_max + (M_max + 3) / 4 * (is ? 2 : 1);
}

// IS: importance-sampled rollouts (a separate instantiation).  At least 3
// blocks of 256 threads per SM for the dynamic model, as the single-problem
// kernel: 80 registers, 24 resident warps per SM.  The lighter kinematic and
// linear models fit 64 registers (the importance-sampled instances with a few
// bytes of spill), so they take 4 blocks: 32 resident warps per SM.  (The
// kinematic kernel without a bound took 108 registers and 16 warps; config
// 3's round went 20.05 -> 19.29 ms at 80 registers.)
template <int MODEL, int ILP, bool IS = false>
__global__ void __launch_bounds__(256, MODEL == 1 ? 3 : 4) batch_rollout_kernel(const DevParams p, const BatchArgs a) {
  extern __shared__ float4 smem[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float4* base = smem + (size_t)w * batch_warp_f4(a.obs_cap_max, a.T_max, a.M_max, IS);
  float4* obs_s = base;
  float4* ctl = obs_s + a.obs_cap_max;
  float* Ls = reinterpret_cast<float*>(ctl + a.T_max);
  float* Ws = IS ? Ls + (a.M_max + 3) / 4 * 4 : nullptr;
  int cur = -1, n_obs = 0;
  Inst in{};
  const InstDesc* d = nullptr;
  for (;;) {
    unsigned long long item = 0ull;
    if (lane == 0) item = atomicAdd(a.queue, 1ull);
    item = __shfl_sync(0xFFFFFFFFu, item, 0);
    if ((long long)item >= a.n_items) break;
    int lo = 0, hi = 2 * a.B;  // seg_base[2B] == n_items
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (a.seg_base[mid] <= (long long)item) lo = mid;
      else hi = mid;
    }
    const int seg = lo;
    const long long local = (long long)item - a.seg_base[seg];
    const int i = a.seg_inst[seg];
    if (i != cur) {
      d = a.desc + i;
      n_obs = a.st[i].n_obs;
      __syncwarp();
      for (int o = lane; o < n_obs; o += 32) obs_s[o] = a.obs[d->obs_off + o];
      in.K = d->K;
      in.M = d->M;
      in.T = d->T;
      in.n_warm = d->n_warm;
      in.j_var = d->j_var;
      in.frac_j = d->frac_j;
      in.tail_denom = d->tail_denom;
      in.instance = d->instance;
      in.k0 = d->seed_lo;
      in.k1 = d->seed_hi ^ (uint32_t)a.st[i].iteration;
      in.is_m0 = d->is_m0;
      in.is_b = d->is_b;
      in.is_base = d->is_base;
      cur = i;
      __syncwarp();
    }
    if (seg < a.B) {
      const int k = (int)local * 32 + lane;
      if (k < in.K)
        nominal_rollout<MODEL>(p, in, a.x0 + d->x0_off, a.V + d->V_off, a.U + d->U_off, a.S + d->k_off, k, obs_s,
                               n_obs);
    } else {
      // a problem too small for a proposal rollout (floor(f M) = 0) takes
      // the plain path, as a single-problem handle does
      if (IS && in.is_b > 0.0f)
        disturbed_sample<MODEL, ILP, true>(p, in, a.x0 + d->x0_off, a.V + d->V_off, (int)local, lane, ctl, Ls, obs_s,
                                           n_obs, a.cvar + d->k_off, nullptr, &a.st[i].status, Ws);
      else
        disturbed_sample<MODEL, ILP, false>(p, in, a.x0 + d->x0_off, a.V + d->V_off, (int)local, lane, ctl, Ls,
                                            obs_s, n_obs, a.cvar + d->k_off, nullptr, &a.st[i].status);
    }
    __syncwarp();
  }
}

}  // namespace ramppi
