// Fused sample + rollout + cost + CVaR work of the RA-MPPI update
// (Algorithm 1, the parallel loop over samples and its inner parallel loop
// over disturbed rollouts; Eqs. 3, 6, 9-13, 18, 19).
//
// Two kinds of work items:
//   - nominal: one thread per sample k draws its control sequence, writes
//     U^k to HBM and rolls it out on the nominal dynamics with the full
//     running cost q, giving S_k (Eq. 3);
//   - disturbed: G warps per sample k (G = 1 by default); the lanes redraw
//     U^k into shared memory (same counter, same bits), then each lane runs
//     the rollouts m = lane + 32 r of its warp's rows r on
//     x~_{t+1} = F(x~_t, u_t) + w_t, ILP of them interleaved (two by two in
//     paired FP32 instructions for the dynamic model), with states and noise
//     in registers, and stores the M risk costs L_{k,m} (Eq. 9) in shared
//     memory; one warp then forms CVaR_k by a radix select of VaR = L_(j)
//     and warp reductions of the tail.
// The single-problem kernel below puts nominal blocks first and disturbed
// blocks after them in one launch, so the nominal work (1/M of the total)
// overlaps the disturbed work; the batched kernel (ra_batch.cu) pulls the
// same items from a work queue.  S~_k is formed by the update, the first
// point where both S_k and CVaR_k exist.
#pragma once

#include "ra_device.cuh"

namespace ramppi {

// Per-problem quantities the work items need besides the common DevParams.
struct Inst {
  int K, M, T, n_warm, j_var;
  float frac_j, tail_denom;
  uint32_t instance, k0, k1;  // Philox counter word 3 and key
  // importance sampling: first proposal rollout, proposal fraction b and
  // -(draws per rollout) ln s (they depend on M and T)
  int is_m0;
  float is_b, is_base;
};

__device__ __forceinline__ Inst inst_of(const DevParams& p, uint32_t iteration) {
  Inst in;
  in.K = p.K;
  in.M = p.M;
  in.T = p.T;
  in.n_warm = p.n_warm;
  in.j_var = p.j_var;
  in.frac_j = p.frac_j;
  in.tail_denom = p.tail_denom;
  in.instance = p.instance;
  in.k0 = p.seed_lo;
  in.k1 = p.seed_hi ^ iteration;
  in.is_m0 = p.is_m0;
  in.is_b = p.is_b;
  in.is_base = p.is_base;
  return in;
}

struct RolloutArgs {
  const float* x0;
  const float* V;
  const float4* obs;   // (x, y, r, r^2), capacity obs_cap
  DevState* st;
  float* U;            // [K][T][nu]
  float* S;            // [K]
  float* cvar;         // [K]
  float* L;            // [K][M] or nullptr
  // state checkpoints for the adjoint (nullptr unless differentiable):
  // nominal x_t at t = 0, 8, ... and x_T, [K][nseg + 1][NX]; disturbed x_t at
  // t = 0, 8, ..., [K][nseg][NX][M] (nseg = ceil(T / 8))
  float* ck_nom;
  float* ck_dist;
  int nb_nom;          // number of nominal blocks
  int obs_cap;
  int wps;             // warps per sample in the disturbed blocks (divides the block's warps)
  // tail split: disturbed blocks from nb_head on take wps_tail (> wps) warps
  // per sample, so the last partial wave of the grid is made of smaller units
  // (nb_head = INT_MAX: no split)
  int nb_head;
  int wps_tail;
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  return v;
}

// order-preserving map of finite floats to unsigned keys
__device__ __forceinline__ uint32_t fkey(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

constexpr int kCkSeg = 8;  // checkpoint spacing (steps) of the adjoint's state checkpoints

// Nominal rollout of sample k: writes U^k [T][nu] and S_k (and, for the
// adjoint, the checkpoints x_0, x_8, ... and x_T of sample k into ck).
template <int MODEL>
__device__ __forceinline__ void nominal_rollout(const DevParams& p, const Inst& in, const float* __restrict__ x0,
                                                const float* __restrict__ V, float* __restrict__ U,
                                                float* __restrict__ S_out, int k, const float4* obs_s,
                                                int n_obs, float* __restrict__ ck = nullptr) {
  using Md = Model<MODEL>;
  float x[Md::NX];
#pragma unroll
  for (int i = 0; i < Md::NX; ++i) x[i] = x0[i];
  float S = 0.0f;
  const int nseg = (in.T + kCkSeg - 1) / kCkSeg;
  float* ckk = ck != nullptr ? ck + (size_t)k * (nseg + 1) * Md::NX : nullptr;
  for (int t = 0; t < in.T; ++t) {
    if (ckk != nullptr && t % kCkSeg == 0) {
#pragma unroll
      for (int i = 0; i < Md::NX; ++i) ckk[(t / kCkSeg) * Md::NX + i] = x[i];
    }
    const float v0 = V[t * Md::NU];
    const float v1 = Md::NU > 1 ? V[t * Md::NU + 1] : 0.0f;
    const float2 u = control_sample(p, in.k0, in.k1, k, t, v0, v1, in.n_warm, in.instance);
    float* Uk = U + ((size_t)k * in.T + t) * Md::NU;
    Uk[0] = u.x;
    if (Md::NU > 1) Uk[1] = u.y;
    float ctrl = v0 * p.inv_sig2[0] * u.x;
    if (Md::NU > 1) ctrl = fmaf(v1 * p.inv_sig2[1], u.y, ctrl);
    S += state_cost<MODEL>(p, x, 0xFFFFFFFFu, obs_s, n_obs) + p.gamma * ctrl;
    Md::step(p, x, Md::ctl(p, u.x, u.y));
  }
  S += terminal_cost<MODEL>(p, x);
  S_out[k] = S;
  if (ckk != nullptr) {
#pragma unroll
    for (int i = 0; i < Md::NX; ++i) ckk[nseg * Md::NX + i] = x[i];
  }
}

// Number of obstacles (sorted by x, at most 1024) with x < v (or x <= v when
// `le`), by two ballots: 32 evenly spaced samples locate the stretch that
// holds the boundary, then its (at most 32) entries give the exact count.
// Warp-collective; every lane returns the same count.
constexpr int kWindowMin = 64;  // fewer obstacles: two rounds of the box test at most

__device__ __forceinline__ int sorted_count(const float4* __restrict__ obs, int n, int lane, float v, bool le) {
  const int stride = (n + 31) >> 5;
  const int j1 = lane * stride;
  const bool p1 = j1 < n && (le ? obs[j1].x <= v : obs[j1].x < v);
  const int c1 = __popc(__ballot_sync(0xFFFFFFFFu, p1));
  if (c1 == 0) return 0;
  const int start = (c1 - 1) * stride;
  const int j2 = start + lane;
  const bool p2 = lane < stride && j2 < n && (le ? obs[j2].x <= v : obs[j2].x < v);
  return start + __popc(__ballot_sync(0xFFFFFFFFu, p2));
}

// Indicator obstacle count of the ILP states of every lane of the warp
// (called by all 32 lanes together).  The warp first bounds its positions by
// a box and tests 32 obstacles at a time against the box, the lane per
// obstacle; only obstacles whose disc can reach the box (with a relative
// margin far above float32 rounding) get the exact per-state test.  A skipped
// obstacle cannot contain any state, so the counts equal the full loop's.
//
// Obstacles are stored sorted by x.  WIN (the dynamic model's kernels for
// more than kWindowMin obstacles, where it pays; obs[-1].x then holds the
// largest radius): the warp first narrows the candidates to those with x
// within that radius (plus a margin far above the rounding of the bounds) of
// the box, found by two ballots over the sorted x; any other obstacle would
// fail the box test below anyway, so the counts stay exact.
//
// The box: coordinates shifted by kBoxShift are positive for every state
// that can be inside an obstacle (obstacles lie within a few hundred metres
// of the origin), so their bit patterns order like the values and one
// integer warp min/max finds each bound.  The shift rounds by at most half
// an ulp of 1024 (6.2e-5 m), so each bound is widened by kBoxPad.  A state
// far below -1024 m turns a min bound very negative and leaves the max
// bounds to the states that matter; a NaN (positive pattern, larger than any
// finite value) makes its max bound NaN, which the candidate test treats as
// unbounded.
template <int MODEL, int ILP, bool WIN = false>
__device__ __forceinline__ void obstacle_hits_culled(const DevParams& p, float (&x)[ILP][Model<MODEL>::NX],
                                                     float (&hits)[ILP], const float4* __restrict__ obs,
                                                     int n_obs) {
  const int lane = threadIdx.x & 31;
  float xmn = x[0][0], xmx = x[0][0], ymn = x[0][1], ymx = x[0][1];
#pragma unroll
  for (int i = 1; i < ILP; ++i) {
    xmn = fminf(xmn, x[i][0]);
    xmx = fmaxf(xmx, x[i][0]);
    ymn = fminf(ymn, x[i][1]);
    ymx = fmaxf(ymx, x[i][1]);
  }
  constexpr float kBoxShift = 1024.0f, kBoxPad = 1.25e-4f;
  const auto lo = [](float v) {
    return __int_as_float(__reduce_min_sync(0xFFFFFFFFu, __float_as_int(v + kBoxShift))) - (kBoxShift + kBoxPad);
  };
  const auto hi = [](float v) {
    return __int_as_float(__reduce_max_sync(0xFFFFFFFFu, __float_as_int(v + kBoxShift))) - (kBoxShift - kBoxPad);
  };
  xmn = lo(xmn);
  xmx = hi(xmx);
  ymn = lo(ymn);
  ymx = hi(ymx);
  int o_begin = 0, o_end = n_obs;
  if (WIN && n_obs > kWindowMin) {
    const float rm = fmaf(obs[-1].x, 1.001f, 2e-4f);
    const float wlo = xmn - rm, whi = xmx + rm;
    if (wlo == wlo && whi == whi) {  // a NaN bound keeps every obstacle
      o_begin = sorted_count(obs, n_obs, lane, wlo, false);
      o_end = sorted_count(obs, n_obs, lane, whi, true);
    }
  }
  for (int base = o_begin; base < o_end; base += 32) {
    const int o = base + lane;
    bool cand = false;
    if (o < o_end) {
      const float4 ob = obs[o];
      // distance from the centre to the box; a NaN bound acts as unbounded
      const float dx = fmaxf(fmaxf(xmn - ob.x, ob.x - xmx), 0.0f);
      const float dy = fmaxf(fmaxf(ymn - ob.y, ob.y - ymx), 0.0f);
      cand = fmaf(dx, dx, dy * dy) <= fmaf(ob.w, 1.0001f, 1e-12f);
    }
    unsigned m = __ballot_sync(0xFFFFFFFFu, cand);
    if (p.diag != nullptr && lane == 0 && m != 0u) atomicAdd(p.diag, (unsigned long long)(__popc(m) * ILP));
    while (m != 0u) {
      const int j = __ffs(m) - 1;
      m &= m - 1u;
      const float4 ob = obs[base + j];
#pragma unroll
      for (int i = 0; i < ILP; ++i) {
        const float dx = x[i][0] - ob.x, dy = x[i][1] - ob.y;
        hits[i] += (fmaf(dx, dx, dy * dy) < ob.w) ? 1.0f : 0.0f;
      }
    }
  }
}

// risk cost l of ILP states of every lane (warp-collective for the indicator term)
template <int MODEL, int ILP, bool WIN = false>
__device__ __forceinline__ void risk_cost_ilp(const DevParams& p, float (&x)[ILP][Model<MODEL>::NX],
                                              float (&L)[ILP], const float4* __restrict__ obs,
                                              int n_obs) {
  const unsigned mask = p.risk_mask;
  if (MODEL != 2 && (mask & 4u) && p.obs_mode == 0) {
    float hits[ILP];
#pragma unroll
    for (int i = 0; i < ILP; ++i) hits[i] = 0.0f;
    obstacle_hits_culled<MODEL, ILP, WIN>(p, x, hits, obs, n_obs);
#pragma unroll
    for (int i = 0; i < ILP; ++i) {
      L[i] = fmaf(p.w_obs, hits[i], L[i]);
      if (mask & ~4u) L[i] += state_cost<MODEL>(p, x[i], mask & ~4u, obs, n_obs);
    }
  } else {
#pragma unroll
    for (int i = 0; i < ILP; ++i) L[i] += state_cost<MODEL>(p, x[i], mask, obs, n_obs);
  }
}

// Importance weight of one rollout from its proposal factor f and its draw
// sums: the balance-heuristic weight 1 / ((1 - b) + b q/p) with
// ln q/p = base + cl f A_L + cg f^2 A_G (an overflowing ratio gives 0)
__device__ __forceinline__ float is_weight(const DevParams& p, const Inst& in, float f, float aL, float aG) {
  const float lr = fmaf(p.is_cg * f * f, aG, fmaf(p.is_cl * f, aL, in.is_base));
  return 1.0f / fmaf(in.is_b, expf(lr), 1.0f - in.is_b);
}

// ILP disturbed rollouts of one lane: rollouts lane + 32 (r0 + i rstride),
// i < ILP (rows r0, r0 + rstride, ... of the M rollouts); risk costs to Ls
// (IS: and importance weights to Ws)
// (ck: this sample's checkpoint block [nseg][NX][M] of the adjoint, or nullptr)
template <int MODEL, int ILP, bool IS = false, bool WIN = false, int NT = -1>
__device__ __forceinline__ void rollouts_ilp(const DevParams& p, const Inst& in, const float* x0, int k, int lane,
                                             int r0, int rstride, const float4* ctl, float* Ls,
                                             const float4* obs_s, int n_obs, float* Ws = nullptr,
                                             float* __restrict__ ck = nullptr) {
  using Md = Model<MODEL>;
  float x[ILP][Md::NX];
  float L[ILP];
  uint32_t m[ILP];
  float fis[ILP], aL[ILP], aG[ILP];
#pragma unroll
  for (int i = 0; i < ILP; ++i) {
    m[i] = (uint32_t)(lane + 32 * (r0 + i * rstride));
    L[i] = 0.0f;
    fis[i] = IS && (int)m[i] >= in.is_m0 ? p.is_s : 1.0f;
    aL[i] = aG[i] = 0.0f;
#pragma unroll
    for (int j = 0; j < Md::NX; ++j) x[i][j] = x0[j];
  }
  for (int t = 0; t < in.T; ++t) {
    if (ck != nullptr && t % kCkSeg == 0) {
#pragma unroll
      for (int i = 0; i < ILP; ++i)
        if ((int)m[i] < in.M) {
#pragma unroll
          for (int j = 0; j < Md::NX; ++j) ck[((size_t)(t / kCkSeg) * Md::NX + j) * in.M + m[i]] = x[i][j];
        }
    }
    const float4 c = ctl[t];
    risk_cost_ilp<MODEL, ILP, WIN>(p, x, L, obs_s, n_obs);
    if constexpr (MODEL == 1 && ILP % 2 == 0) {
      // rollouts two by two in paired FP32 instructions (same bits as one by one)
#pragma unroll
      for (int i = 0; i < ILP; i += 2) {
        float2 xx[Md::NX];
#pragma unroll
        for (int j = 0; j < Md::NX; ++j) xx[j] = make_float2(x[i][j], x[i + 1][j]);
        Md::step2(p, xx, c);
#pragma unroll
        for (int j = 0; j < Md::NX; ++j) {
          x[i][j] = xx[j].x;
          x[i + 1][j] = xx[j].y;
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < ILP; ++i) Md::step(p, x[i], c);
    }
#pragma unroll
    for (int i = 0; i < ILP; ++i)
      add_process_noise<MODEL, IS, NT>(p, in.k0, in.k1, (uint32_t)t, m[i], (uint32_t)k, in.instance, x[i], fis[i],
                                       &aL[i], &aG[i]);
  }
#pragma unroll
  for (int i = 0; i < ILP; ++i)
    if ((int)m[i] < in.M) {
      Ls[m[i]] = L[i];
      if constexpr (IS) Ws[m[i]] = is_weight(p, in, fis[i], aL[i], aG[i]);
    }
}

// U^k into shared memory, steps t_first, t_first + t_stride, ... (the nominal
// thread of sample k draws the same bits)
template <int MODEL>
__device__ __forceinline__ void fill_controls(const DevParams& p, const Inst& in, const float* __restrict__ V, int k,
                                              int t_first, int t_stride, float4* ctl) {
  using Md = Model<MODEL>;
  for (int t = t_first; t < in.T; t += t_stride) {
    const float v0 = V[t * Md::NU];
    const float v1 = Md::NU > 1 ? V[t * Md::NU + 1] : 0.0f;
    const float2 u = control_sample(p, in.k0, in.k1, k, t, v0, v1, in.n_warm, in.instance);
    ctl[t] = Md::ctl(p, u.x, u.y);
  }
}

// the rollout rows r_first, r_first + r_stride, ... of sample k (one warp);
// ILP rows interleaved, the rest one at a time
template <int MODEL, int ILP, bool IS = false, bool WIN = false>
__device__ __forceinline__ void run_rollouts(const DevParams& p, const Inst& in, const float* __restrict__ x0g, int k,
                                             int lane, int r_first, int r_stride, const float4* ctl, float* Ls,
                                             const float4* obs_s, int n_obs, float* Ws = nullptr,
                                             float* __restrict__ ck = nullptr) {
  using Md = Model<MODEL>;
  float x0[Md::NX];
#pragma unroll
  for (int i = 0; i < Md::NX; ++i) x0[i] = x0g[i];
  const int R = (in.M + 31) >> 5;
  int r = r_first;
  // the interleaved rows with the noise type fixed at compile time for the
  // mixture (the dynamic workloads) and Gaussian noise
  if (!IS && p.noise_type == 1) {
    for (; r + (ILP - 1) * r_stride < R; r += ILP * r_stride)
      rollouts_ilp<MODEL, ILP, IS, WIN, 1>(p, in, x0, k, lane, r, r_stride, ctl, Ls, obs_s, n_obs, Ws, ck);
  } else if (!IS && p.noise_type == 0) {
    for (; r + (ILP - 1) * r_stride < R; r += ILP * r_stride)
      rollouts_ilp<MODEL, ILP, IS, WIN, 0>(p, in, x0, k, lane, r, r_stride, ctl, Ls, obs_s, n_obs, Ws, ck);
  }
  for (; r + (ILP - 1) * r_stride < R; r += ILP * r_stride)
    rollouts_ilp<MODEL, ILP, IS, WIN>(p, in, x0, k, lane, r, r_stride, ctl, Ls, obs_s, n_obs, Ws, ck);
  if (ILP > 1)
    for (; r < R; r += r_stride)
      rollouts_ilp<MODEL, 1, IS, WIN>(p, in, x0, k, lane, r, r_stride, ctl, Ls, obs_s, n_obs, Ws, ck);
}

// CVaR_k (or the selected risk measure) of the M risk costs in Ls (one warp),
// with RMAX >= ceil(M / 32) rows of costs per lane in registers
template <int RMAX>
__device__ __forceinline__ void risk_from_shared_rows(const DevParams& p, const Inst& in, const float* Ls, int k,
                                                      int lane, float* __restrict__ cvar, float* __restrict__ Lout,
                                                      int* status) {
  // CVaR_k over the M risk costs (Eqs. 10-13, 18, 19)
  uint32_t key[RMAX];
  float val[RMAX];
  bool bad = false;
  float sum = 0.0f;
#pragma unroll
  for (int r = 0; r < RMAX; ++r) {
    const int idx = lane + 32 * r;
    const bool valid = idx < in.M;
    const float v = valid ? Ls[idx] : 0.0f;
    val[r] = v;
    bad |= valid && !isfinite(v);
    sum += v;
    key[r] = valid ? fkey(v) : 0xFFFFFFFFu;
  }
  if (Lout != nullptr) {
    for (int idx = lane; idx < in.M; idx += 32) Lout[(size_t)k * in.M + idx] = Ls[idx];
  }
  if (__any_sync(0xFFFFFFFFu, bad)) {
    if (lane == 0) {
      cvar[k] = __int_as_float(0x7F800000);  // +inf: the sample gets zero weight
      atomicOr(status, kStatusNonFinite);
    }
    __syncwarp();
    return;
  }
  const float mean = warp_sum(sum) / (float)in.M;

  // radix select of the j-th smallest key (VaR = L_(j), Eq. 11)
  uint32_t prefix = 0u;
  int kth = in.j_var - 1;
#pragma unroll 1
  for (int b = 31; b >= 0; --b) {
    const uint32_t hi_mask = (b == 31) ? 0u : (0xFFFFFFFFu << (b + 1));
    int cnt = 0;
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      const uint32_t kk = key[r];
      cnt += ((kk & hi_mask) == prefix && ((kk >> b) & 1u) == 0u && (lane + 32 * r) < in.M) ? 1 : 0;
    }
    cnt = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)cnt);
    if (kth >= cnt) {
      kth -= cnt;
      prefix |= (1u << b);
    }
  }
  const float var = fkey_inv(prefix);

  int c_gt = 0, c_eq = 0;
  float s_gt = 0.0f;
#pragma unroll
  for (int r = 0; r < RMAX; ++r) {
    if (lane + 32 * r < in.M) {
      const float v = val[r];
      if (v > var) { ++c_gt; s_gt += v; }
      else if (v == var) ++c_eq;
    }
  }
  c_gt = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)c_gt);
  c_eq = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)c_eq);
  s_gt = warp_sum(s_gt);
  float cv;
  if (p.cvar_mode == 0) {
    // fractional tail: weight (j - alpha M) on L_(j), 1 on every later order
    // statistic; ties with L_(j) beyond rank j count at full weight
    const float n_eq_tail = (float)(in.M - in.j_var - c_gt);
    cv = (s_gt + (n_eq_tail + in.frac_j) * var) / in.tail_denom;
  } else if (p.cvar_mode == 1) {
    cv = (s_gt + (float)c_eq * var) / (float)(c_gt + c_eq);
  } else if (p.cvar_mode == 2) {
    cv = var;  // VaR_alpha (Eq. 11)
  } else if (p.cvar_mode == 3) {
    // chance measure: fraction of the scaled risk costs above the threshold
    // (B = 1 compares the costs themselves, so no rounding enters the decision)
    int over = 0;
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      const float v = p.B == 1.0f ? val[r] : fmaf(p.B, val[r] - mean, mean);
      if (lane + 32 * r < in.M) over += v > p.risk_param ? 1 : 0;
    }
    cv = (float)__reduce_add_sync(0xFFFFFFFFu, (unsigned)over) / (float)in.M;
  } else if (p.cvar_mode == 4) {
    cv = mean;  // risk-neutral expected risk cost
  } else {
    // mean-variance: mean + kappa B^2 (1/M) sum (L - mean)^2, two-pass variance
    float d2 = 0.0f;
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      const float d = val[r] - mean;
      if (lane + 32 * r < in.M) d2 = fmaf(d, d, d2);
    }
    cv = fmaf(p.risk_param * p.B * p.B, warp_sum(d2) / (float)in.M, mean);
  }
  // sensitivity scaling L_a = B (L - mean) + mean commutes with the tail
  // average and the quantile for B >= 0: rho(L_a) = B rho(L) + (1 - B) mean
  if (p.B != 1.0f && p.cvar_mode <= 2) cv = fmaf(p.B, cv, (1.0f - p.B) * mean);
  if (lane == 0) cvar[k] = cv;
  __syncwarp();
}

// The row count sized to M, so that the 32 select passes loop over the rows
// that hold costs only (rows past M add nothing: the same bits for every
// size class)
__device__ __forceinline__ void risk_from_shared(const DevParams& p, const Inst& in, const float* Ls, int k, int lane,
                                                 float* __restrict__ cvar, float* __restrict__ Lout, int* status) {
  constexpr int RMAX = (RA_MPPI_MAX_M_DEV + 31) / 32;
  if (in.M <= 32) risk_from_shared_rows<1>(p, in, Ls, k, lane, cvar, Lout, status);
  else if (in.M <= 64) risk_from_shared_rows<2>(p, in, Ls, k, lane, cvar, Lout, status);
  else if (in.M <= 128) risk_from_shared_rows<4>(p, in, Ls, k, lane, cvar, Lout, status);
  else if (in.M <= 256) risk_from_shared_rows<8>(p, in, Ls, k, lane, cvar, Lout, status);
  else risk_from_shared_rows<RMAX>(p, in, Ls, k, lane, cvar, Lout, status);
}

// VaR of the weighted empirical distribution of M costs held by one warp
// (key, wt: rows lane + 32 r): the smallest cost whose strictly larger weight
// is at most tau.  A radix select on the order-preserving keys that sums
// weights instead of counting: bit by bit from the top, keep the upper half
// while the weight above it plus its own exceeds tau.  The weight sums
// round: should a near-tie have left the search below every cost of the
// bucket it skipped, the smallest cost at or above the key found is taken
// (in exact arithmetic, the key itself).
template <int RMAX>
__device__ __forceinline__ float weighted_var(const uint32_t* key, const float* wt, int M, int lane, float tau) {
  uint32_t prefix = 0u;
  float above = 0.0f;
#pragma unroll 1
  for (int b = 31; b >= 0; --b) {
    const uint32_t hi_mask = (b == 31) ? 0u : (0xFFFFFFFFu << (b + 1));
    float s1 = 0.0f;
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      const uint32_t kk = key[r];
      if ((kk & hi_mask) == prefix && ((kk >> b) & 1u) != 0u && (lane + 32 * r) < M) s1 += wt[r];
    }
    s1 = warp_sum(s1);
    if (above + s1 > tau) prefix |= (1u << b);
    else above += s1;
  }
  uint32_t kmin = 0xFFFFFFFFu;
#pragma unroll
  for (int r = 0; r < RMAX; ++r)
    if (lane + 32 * r < M && key[r] >= prefix) kmin = min(kmin, key[r]);
  kmin = __reduce_min_sync(0xFFFFFFFFu, kmin);
  return fkey_inv(kmin != 0xFFFFFFFFu ? kmin : prefix);
}

// The risk measure of the weighted empirical distribution of the M risk
// costs in Ls with the importance weights in Ws (one warp).  With
// W = sum w and tau = (1 - alpha) W: VaR from weighted_var, RU CVaR =
// VaR + sum w (L - VaR)+ / tau, TCE the weighted mean of the costs >= VaR, the chance measure the
// weight fraction above the threshold, the mean and mean-variance the
// weighted moments.  Fixed summation order: the bits do not depend on the
// launch shape.
template <int RMAX>
__device__ __forceinline__ void risk_from_shared_w_rows(const DevParams& p, const Inst& in, const float* Ls,
                                                        const float* Ws, int k, int lane, float* __restrict__ cvar,
                                                        float* __restrict__ Lout, int* status) {
  uint32_t key[RMAX];
  float val[RMAX], wt[RMAX];
  bool bad = false;
  float sw = 0.0f, swl = 0.0f;
#pragma unroll
  for (int r = 0; r < RMAX; ++r) {
    const int idx = lane + 32 * r;
    const bool valid = idx < in.M;
    const float v = valid ? Ls[idx] : 0.0f;
    const float w = valid ? Ws[idx] : 0.0f;
    val[r] = v;
    wt[r] = w;
    bad |= valid && !isfinite(v);
    sw += w;
    swl = fmaf(w, v, swl);
    key[r] = valid ? fkey(v) : 0xFFFFFFFFu;
  }
  if (Lout != nullptr) {
    // kept costs, then the weights after all K x M costs
    float* Wout = Lout + (size_t)in.K * in.M;
    for (int idx = lane; idx < in.M; idx += 32) {
      Lout[(size_t)k * in.M + idx] = Ls[idx];
      Wout[(size_t)k * in.M + idx] = Ws[idx];
    }
  }
  if (__any_sync(0xFFFFFFFFu, bad)) {
    if (lane == 0) {
      cvar[k] = __int_as_float(0x7F800000);
      atomicOr(status, kStatusNonFinite);
    }
    __syncwarp();
    return;
  }
  const float W = warp_sum(sw);
  const float mean = warp_sum(swl) / W;
  const float tau = p.one_m_alpha * W;
  const float var = weighted_var<RMAX>(key, wt, in.M, lane, tau);
  float w_gt = 0.0f, w_eq = 0.0f, tail = 0.0f, wl_ge = 0.0f;
#pragma unroll
  for (int r = 0; r < RMAX; ++r) {
    if (lane + 32 * r < in.M) {
      const float v = val[r], w = wt[r];
      if (v > var) {
        w_gt += w;
        tail = fmaf(w, v - var, tail);
        wl_ge = fmaf(w, v, wl_ge);
      } else if (v == var) {
        w_eq += w;
        wl_ge = fmaf(w, v, wl_ge);
      }
    }
  }
  float cv;
  if (p.cvar_mode == 0) {
    cv = var + warp_sum(tail) / tau;
  } else if (p.cvar_mode == 1) {
    cv = warp_sum(wl_ge) / (warp_sum(w_gt) + warp_sum(w_eq));
  } else if (p.cvar_mode == 2) {
    cv = var;
  } else if (p.cvar_mode == 3) {
    float over = 0.0f;
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      const float v = p.B == 1.0f ? val[r] : fmaf(p.B, val[r] - mean, mean);
      if (lane + 32 * r < in.M && v > p.risk_param) over += wt[r];
    }
    cv = warp_sum(over) / W;
  } else if (p.cvar_mode == 4) {
    cv = mean;
  } else {
    float d2 = 0.0f;
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      const float d = val[r] - mean;
      if (lane + 32 * r < in.M) d2 = fmaf(wt[r] * d, d, d2);
    }
    cv = fmaf(p.risk_param * p.B * p.B, warp_sum(d2) / W, mean);
  }
  if (p.B != 1.0f && p.cvar_mode <= 2) cv = fmaf(p.B, cv, (1.0f - p.B) * mean);
  if (lane == 0) cvar[k] = cv;
  __syncwarp();
}

__device__ __forceinline__ void risk_from_shared_w(const DevParams& p, const Inst& in, const float* Ls,
                                                   const float* Ws, int k, int lane, float* __restrict__ cvar,
                                                   float* __restrict__ Lout, int* status) {
  constexpr int RMAX = (RA_MPPI_MAX_M_DEV + 31) / 32;
  if (in.M <= 64) risk_from_shared_w_rows<2>(p, in, Ls, Ws, k, lane, cvar, Lout, status);
  else if (in.M <= 256) risk_from_shared_w_rows<8>(p, in, Ls, Ws, k, lane, cvar, Lout, status);
  else risk_from_shared_w_rows<RMAX>(p, in, Ls, Ws, k, lane, cvar, Lout, status);
}

// One warp: the M disturbed rollouts of sample k and CVaR_k (written to cvar[k]).
// ctl [T] and Ls [M] are this warp's shared-memory scratch.
template <int MODEL, int ILP, bool IS = false, bool WIN = false>
__device__ __forceinline__ void disturbed_sample(const DevParams& p, const Inst& in, const float* __restrict__ x0g,
                                                 const float* __restrict__ V, int k, int lane, float4* ctl, float* Ls,
                                                 const float4* obs_s, int n_obs, float* __restrict__ cvar,
                                                 float* __restrict__ Lout, int* status, float* Ws = nullptr,
                                                 float* __restrict__ ck = nullptr) {
  fill_controls<MODEL>(p, in, V, k, lane, 32, ctl);
  __syncwarp();
  // disturbed rollouts and their risk costs (Eq. 9)
  run_rollouts<MODEL, ILP, IS, WIN>(p, in, x0g, k, lane, 0, 1, ctl, Ls, obs_s, n_obs, Ws, ck);
  __syncwarp();
  if constexpr (IS) risk_from_shared_w(p, in, Ls, Ws, k, lane, cvar, Lout, status);
  else risk_from_shared(p, in, Ls, k, lane, cvar, Lout, status);
}

// One warp, two samples ka, kb of at most 32 rollouts each (the dynamic
// model, interleave 2): lane l steps rollout l of ka and rollout l of kb as
// one pair in paired FP32 instructions, each under its own sample's controls
// (the same bits as one sample per warp).  kb may be past the last sample;
// then its results are not stored.
template <int MODEL>
__device__ __forceinline__ void disturbed_sample_pair(const DevParams& p, const Inst& in, const float* __restrict__ x0g,
                                                      const float* __restrict__ V, int ka, int kb, int lane,
                                                      float4* ctl_a, float4* ctl_b, float* Ls_a, float* Ls_b,
                                                      const float4* obs_s, int n_obs, float* __restrict__ cvar,
                                                      float* __restrict__ Lout, int* status,
                                                      float* __restrict__ ck_a = nullptr,
                                                      float* __restrict__ ck_b = nullptr) {
  using Md = Model<MODEL>;
  fill_controls<MODEL>(p, in, V, ka, lane, 32, ctl_a);
  fill_controls<MODEL>(p, in, V, kb, lane, 32, ctl_b);
  __syncwarp();
  float x[2][Md::NX];
  float L[2] = {0.0f, 0.0f};
#pragma unroll
  for (int j = 0; j < Md::NX; ++j) x[0][j] = x[1][j] = x0g[j];
  const uint32_t m = (uint32_t)lane;
  for (int t = 0; t < in.T; ++t) {
    if (ck_a != nullptr && t % kCkSeg == 0 && (int)m < in.M) {
#pragma unroll
      for (int j = 0; j < Md::NX; ++j) {
        ck_a[((size_t)(t / kCkSeg) * Md::NX + j) * in.M + m] = x[0][j];
        if (kb < in.K) ck_b[((size_t)(t / kCkSeg) * Md::NX + j) * in.M + m] = x[1][j];
      }
    }
    risk_cost_ilp<MODEL, 2>(p, x, L, obs_s, n_obs);
    float2 xx[Md::NX];
#pragma unroll
    for (int j = 0; j < Md::NX; ++j) xx[j] = make_float2(x[0][j], x[1][j]);
    Md::step2x(p, xx, ctl_a[t], ctl_b[t]);
#pragma unroll
    for (int j = 0; j < Md::NX; ++j) {
      x[0][j] = xx[j].x;
      x[1][j] = xx[j].y;
    }
    add_process_noise<MODEL>(p, in.k0, in.k1, (uint32_t)t, m, (uint32_t)ka, in.instance, x[0]);
    add_process_noise<MODEL>(p, in.k0, in.k1, (uint32_t)t, m, (uint32_t)kb, in.instance, x[1]);
  }
  if ((int)m < in.M) {
    Ls_a[m] = L[0];
    Ls_b[m] = L[1];
  }
  __syncwarp();
  risk_from_shared(p, in, Ls_a, ka, lane, cvar, Lout, status);
  if (kb < in.K) risk_from_shared(p, in, Ls_b, kb, lane, cvar, Lout, status);
}

// PAIRS: the instantiation that takes two samples per warp (dynamic model,
// interleave 2, one row per sample); a separate kernel so that its code does
// not raise the register count of the others
// IS: importance-sampled rollouts with weights in shared memory after the
// costs (a separate instantiation; never with PAIRS)
// WIN: the obstacle cull's x window (dynamic model, more than kWindowMin
// obstacles; a separate instantiation so the others keep their code)
// CK: store the state checkpoints the adjoint reads (differentiable handles;
// a separate instantiation, so the others compile without the stores)
// (at least 3 blocks of 256 threads per SM: 80 registers, 24 resident warps
// per SM; without the bound the register count of some instances drifts
// between 64 and 128 with each code change, and the measured kernels are
// fastest at 80.  The two-samples-per-warp instance fits 64 registers
// without spilling, so it takes 4 blocks: 32 resident warps per SM, config
// 5 at M = 32 4.07 -> 3.97 ms; the others spill at 64 and slow down.)
template <int MODEL, int ILP, bool PAIRS = false, bool IS = false, bool WIN = false, bool CK = false>
__global__ void __launch_bounds__(256, PAIRS ? 4 : 3) rollout_cvar_kernel(const DevParams p, const RolloutArgs a) {
  extern __shared__ float4 smem[];
  // WIN: smem[0].x holds the largest obstacle radius and the obstacles start
  // at smem[1]; otherwise at smem[0].  The samples' controls, costs (and
  // weights) follow the obstacles.
  float4* obs_s = smem + (WIN ? 1 : 0);
  float4* const scratch = obs_s + a.obs_cap;
  const int n_obs = a.st->n_obs;
  const Inst in = inst_of(p, (uint32_t)a.st->iteration);
  for (int i = threadIdx.x; i < n_obs; i += blockDim.x) obs_s[i] = a.obs[i];
  __syncthreads();
  if (WIN && n_obs > kWindowMin) {  // only the windowed cull reads it
    if (threadIdx.x < 32) {
      float r = 0.0f;
      for (int i = threadIdx.x; i < n_obs; i += 32) r = fmaxf(r, obs_s[i].z);
      r = warp_max(r);
      if (threadIdx.x == 0) smem[0] = make_float4(r, 0.0f, 0.0f, 0.0f);
    }
    __syncthreads();
  }

  if ((int)blockIdx.x < a.nb_nom) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < in.K) nominal_rollout<MODEL>(p, in, a.x0, a.V, a.U, a.S, k, obs_s, n_obs, CK ? a.ck_nom : nullptr);
    return;
  }
  // disturbed blocks: G = a.wps warps per sample, warps / G samples per block;
  // the blocks of the tail split (from a.nb_head on) take a.wps_tail warps
  // per sample.  (The hardware hands out blocks as SM slots free up; a
  // persistent grid taking samples from a counter was slower: its per-unit
  // barriers cost more.)  The shared-memory slots keep the head's layout.
  const int warps = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int db = (int)blockIdx.x - a.nb_nom;
  const bool tail = db >= a.nb_head;
  const int spb_h = warps / a.wps;
  const int G = tail ? a.wps_tail : a.wps, spb = warps / G, gi = w / G, g = w - gi * G;
  const int k = tail ? a.nb_head * spb_h + (db - a.nb_head) * spb + gi : db * spb_h + gi;
  float4* ctl = scratch + gi * in.T;
  float* Ls = reinterpret_cast<float*>(scratch + spb_h * in.T) + gi * in.M;
  float* Ws = IS ? Ls + spb_h * in.M : nullptr;
  // this sample's block of disturbed checkpoints (adjoint only)
  const size_t ck_per_sample = (size_t)((in.T + kCkSeg - 1) / kCkSeg) * Model<MODEL>::NX * in.M;
  if constexpr (PAIRS) {
    // two samples per warp: slots 2w and 2w + 1 of the block's controls and costs
    const int ka = ((int)blockIdx.x - a.nb_nom) * 2 * warps + 2 * w, kb = ka + 1;
    if (ka >= in.K) return;
    float4* ctl_a = scratch + (2 * w) * in.T;
    float* Ls_a = reinterpret_cast<float*>(scratch + 2 * warps * in.T) + (2 * w) * in.M;
    float* ck_a = CK ? a.ck_dist + (size_t)ka * ck_per_sample : nullptr;
    disturbed_sample_pair<MODEL>(p, in, a.x0, a.V, ka, kb, lane, ctl_a, ctl_a + in.T, Ls_a, Ls_a + in.M, obs_s,
                                 n_obs, a.cvar, a.L, &a.st->status, ck_a, ck_a != nullptr ? ck_a + ck_per_sample : nullptr);
    return;
  } else {
  if (G == 1) {
    if (k >= in.K) return;
    disturbed_sample<MODEL, ILP, IS, WIN>(p, in, a.x0, a.V, k, lane, ctl, Ls, obs_s, n_obs, a.cvar, a.L,
                                     &a.st->status, Ws, CK ? a.ck_dist + (size_t)k * ck_per_sample : nullptr);
    return;
  }
  // a sample's rollout rows split over its G warps; every warp of the block
  // reaches both barriers
  const bool valid = k < in.K;
  if (valid) fill_controls<MODEL>(p, in, a.V, k, g * 32 + lane, 32 * G, ctl);
  __syncthreads();
  if (valid)
    run_rollouts<MODEL, ILP, IS, WIN>(p, in, a.x0, k, lane, g, G, ctl, Ls, obs_s, n_obs, Ws,
                                      CK ? a.ck_dist + (size_t)k * ck_per_sample : nullptr);
  __syncthreads();
  if (valid && g == 0) {
    if constexpr (IS) risk_from_shared_w(p, in, Ls, Ws, k, lane, a.cvar, a.L, &a.st->status);
    else risk_from_shared(p, in, Ls, k, lane, a.cvar, a.L, &a.st->status);
  }
  }
}

}  // namespace ramppi
