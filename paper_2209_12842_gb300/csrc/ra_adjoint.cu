// Adjoint of one RA-MPPI update: the vector-Jacobian product of
// (V+, S~) = update(V, theta) w.r.t. the mean controls V and the cost weights
// theta = (w_dev, w_speed, gamma, w_obs), for fixed noise.
//
// With cotangents gV+ [T][nu] and gS~ [K] the derivative of each forward
// step, in reverse:
//   Eqs. 4, 17:  dV+/dU_k = w^_k I,  dV+/dS~_k = -(w^_k / lambda)(U_k - V+), so
//                S~-bar_k = gS~_k - (w^_k / lambda)(d_k - c),
//                d_k = <gV+, U_k>, c = sum_k w^_k d_k = <gV+, V+>
//   Eqs. 14-16:  S-bar_k = S~-bar_k, CVaR-bar_k = S~-bar_k A 1{CVaR_k > C_u}
//   Eqs. 10-13, 18, 19: CVaR is piecewise linear in the risk costs; its
//                weights are 1/((1-alpha)M) above VaR, the remaining weight
//                shared by the costs equal to VaR, 0 below; the scaling gives
//                B w + (1 - B)/M
//   Eqs. 3, 9:   reverse sweeps through each rollout, the states recomputed
//                from the checkpoints (every 8 steps) that the
//                differentiable forward stored:
//                u-bar_t = (dF/du)' lam_{t+1}, lam_t = c dq/dx + (dF/dx)' lam_{t+1}
//   Alg. 1:      U = clip(V + eps) passes u-bar to V inside the box for the
//                samples drawn around V; the control cost gamma v' S^-1 u
//                depends on V directly as well.
// Every reverse sweep is linear in its sample's cotangent S~-bar_k, so the
// sweeps run at a unit cotangent and the reduction scales them:
//   gU_k = mask_k w^_k gV+ + S~-bar_k (G_nom,k + mask_k G_dist,k)
// with G the unit-cotangent sweeps.  Two launches: main (nominal blocks +
// one warp per sample for the disturbed rollouts, which also form d_k and
// w^_k) and reduce (the sums over samples, with S~-bar_k = a_k + b_k c split as
// a_k = gS~_k - w^_k d_k / lambda, b_k = w^_k / lambda, so that c is only
// needed in the final merge).
// All three models are differentiated (the dynamic one through its Heun
// sub-steps); the indicator obstacle term has zero derivative almost
// everywhere.
#include "ra_kernels.h"

namespace ramppi {

namespace {

constexpr int kSeg = kCkSeg;  // checkpoint spacing (steps), as the forward stores them
constexpr int kGusSlotCols = 128;  // T nu up to which each slot keeps its own row of control cotangents

__device__ __forceinline__ float sgnf(float v) { return v > 0.0f ? 1.0f : (v < 0.0f ? -1.0f : 0.0f); }

// e(x) and its gradient w.r.t. (px, py)
__device__ __forceinline__ float track_e_grad(const DevParams& p, float px, float py, float* de) {
  const float half = 0.5f * p.track_S;
  const float ax = fabsf(px);
  if (ax <= half) {
    de[0] = 0.0f;
    de[1] = py < 0.0f ? -1.0f : 1.0f;
    return fabsf(py) - p.track_R;
  }
  const float dx = ax - half;
  const float r2 = fmaf(dx, dx, py * py);
  const float ir = r2 > 0.0f ? rsqrtf(r2) : 0.0f;  // hardware 1/rho: a gradient needs no more
  de[0] = sgnf(px) * dx * ir;
  de[1] = py * ir;
  return r2 * ir - p.track_R;
}

// gradient of the arc length s(x) w.r.t. (px, py)
__device__ __forceinline__ void track_s_grad(const DevParams& p, float px, float py, float* ds) {
  const float half = 0.5f * p.track_S;
  if (fabsf(px) <= half) {
    ds[0] = py < 0.0f ? 1.0f : -1.0f;
    ds[1] = 0.0f;
    return;
  }
  const float dx = px > half ? px - half : px + half;
  const float r2 = fmaf(dx, dx, py * py);
  const float ir2 = r2 > 0.0f ? __fdividef(p.track_R, r2) : 0.0f;
  ds[0] = -py * ir2;
  ds[1] = dx * ir2;
}

// The obstacle term at x over the obstacles first, first + stride, ...:
// sums of its values (softplus or indicator, before 1/kappa) and of the
// slopes d/dx, d/dy (before w_obs).
// softplus(z) = max(z, 0) + log(1 + e) and sigmoid(z) = 1 / (1 + e) or
// e / (1 + e), both from e = exp(-|z|); no direction at the centre.  The
// obstacles are independent: unrolled, a lone thread overlaps them.
// Hardware exponential, logarithm and reciprocal: a gradient needs no more
// (the log of 1 + e is off by at most about 1e-7 absolute)
__device__ __forceinline__ void obstacle_grad_part(const DevParams& p, const float* x, const float4* __restrict__ obs,
                                                   int n_obs, int first, int stride, float& val, float& g0,
                                                   float& g1) {
  if (p.obs_mode == 0) {
    for (int i = first; i < n_obs; i += stride) {  // indicator: a value, no gradient
      const float4 o = obs[i];
      const float dx = x[0] - o.x, dy = x[1] - o.y;
      val += fmaf(dx, dx, dy * dy) < o.w ? 1.0f : 0.0f;
    }
    return;
  }
#pragma unroll 4
  for (int i = first; i < n_obs; i += stride) {
    const float4 o = obs[i];
    const float dx = x[0] - o.x, dy = x[1] - o.y;
    const float d2 = fmaf(dx, dx, dy * dy);
    const float rd = d2 > 0.0f ? rsqrtf(d2) : 0.0f;
    const float z = p.kappa * (o.z - d2 * rd);
    const float e = __expf(-fabsf(z));
    val += fmaxf(z, 0.0f) + __logf(1.0f + e);
    const float r = __frcp_rn(1.0f + e);
    const float kk = (z > 0.0f ? r : e * r) * rd;
    g0 = fmaf(-kk, dx, g0);
    g1 = fmaf(-kk, dy, g1);
  }
}

// c * d(cost terms in mask)/dx added to g; c * d(cost)/d(w_dev, w_speed, -, w_obs) added to gth
template <int MODEL>
__device__ __forceinline__ void cost_grad(const DevParams& p, const float* x, unsigned mask, float c,
                                          const float4* __restrict__ obs, int n_obs, float* g, float* gth) {
  if (MODEL == 2) {
    if (mask & 16u) g[0] = fmaf(c, p.c_lin, g[0]);
    return;
  }
  if (mask & 9u) {
    float de[2];
    const float e = track_e_grad(p, x[0], x[1], de);
    if (mask & 1u) {
      const float k = c * p.w_dev * 2.0f * e;
      g[0] = fmaf(k, de[0], g[0]);
      g[1] = fmaf(k, de[1], g[1]);
      gth[0] = fmaf(c, e * e, gth[0]);
    }
    if ((mask & 8u) && p.w_bdry != 0.0f) {  // (the boundary weight is not among theta)
      const float d = p.track_hw - fabsf(e);
      const float db = __fdividef(-100.0f / kPi, fmaf(1e4f * d, d, 1.0f));
      const float k = c * p.w_bdry * db * (-sgnf(e));
      g[0] = fmaf(k, de[0], g[0]);
      g[1] = fmaf(k, de[1], g[1]);
    }
  }
  if (mask & 2u) {
    const float dv = x[3] - p.v_target;
    g[3] = fmaf(c * p.w_speed * 2.0f, dv, g[3]);
    gth[1] = fmaf(c, dv * dv, gth[1]);
  }
  if (mask & 4u) {
    float val = 0.0f, g0 = 0.0f, g1 = 0.0f;
    obstacle_grad_part(p, x, obs, n_obs, 0, 1, val, g0, g1);
    if (p.obs_mode != 0) val *= p.inv_kappa;
    g[0] = fmaf(c * p.w_obs, g0, g[0]);
    g[1] = fmaf(c * p.w_obs, g1, g[1]);
    gth[3] = fmaf(c, val, gth[3]);
  }
  if (mask & 16u) g[0] = fmaf(c, p.c_lin, g[0]);
}

// Transposed Jacobians of the dynamic model's derivative f(x, u) at x
// applied to fb: xb += (df/dx)' fb, gu += (df/du)' fb with u = (steer, accel).
// The same formulas as the forward: slip angles atan(y / max(vx, floor)),
// lateral accelerations k sin(C atan(B alpha)) (k = D Fz / m), yaw arms
// l m / Iz; the derivative values use the library arctangent and the
// hardware sine, cosine and quotients (errors of a few 1e-7, far inside the
// adjoint's tolerance).
__device__ __forceinline__ void dyn_deriv_vjp(const DevParams& p, const float* x, const float4 c, const float* fb,
                                              float* xb, float* gu) {
  const float lf = p.mp[2], lr = p.mp[3], Bt = p.mp[4], C = p.mp[5], vfloor = p.mp[7];
  const float sq2 = p.pacejka_c15 ? 1.41421356237f : 1.0f;  // undo the fold of the closed form
  const float kf = p.acc_f * sq2, kr = p.acc_r * sq2;
  const float psi = x[2], vx = x[3], vy = x[4], r = x[5];
  const float sd = c.z, cd = c.w;
  const float vxs = fmaxf(vx, vfloor);
  const float yf = fmaf(lf, r, vy), yr = fmaf(-lr, r, vy);
  const float ivx = __fdividef(1.0f, vxs);
  const float tf = atanf(yf * ivx), tr = atanf(yr * ivx);
  const float zf = fmaf(-Bt, tf, c.x), zr = -Bt * tr;
  const float qf = C * atanf(zf), qr = C * atanf(zr);
  // (hardware sine, cosine and quotients: a gradient needs no more)
  const float ayf = kf * __sinf(qf), ayr = kr * __sinf(qr);
  const float dsf = __fdividef(C * __cosf(qf), fmaf(zf, zf, 1.0f)), dsr = __fdividef(C * __cosf(qr), fmaf(zr, zr, 1.0f));
  float sp, cp;
  heading_sincos(psi, &sp, &cp);
  // f0 = vx cos psi - vy sin psi, f1 = vx sin psi + vy cos psi, f2 = r
  xb[2] += fb[0] * (-vx * sp - vy * cp) + fb[1] * (vx * cp - vy * sp);
  xb[3] += fb[0] * cp + fb[1] * sp - fb[4] * r;
  xb[4] += -fb[0] * sp + fb[1] * cp + fb[3] * r;
  xb[5] += fb[2] + fb[3] * vy - fb[4] * vx;
  // f3 = a - ayf sin d + r vy, f4 = ayf cos d + ayr - r vx, f5 = yaw_f ayf cos d - yaw_r ayr
  gu[1] += fb[3];
  const float ayfb = -fb[3] * sd + fb[4] * cd + fb[5] * p.yaw_f * cd;
  const float ayrb = fb[4] - fb[5] * p.yaw_r;
  gu[0] += -fb[3] * ayf * cd - fb[4] * ayf * sd - fb[5] * p.yaw_f * ayf * sd;
  // z_f = B (steer - atan_f), z_r = -B atan_r
  const float zfb = ayfb * kf * dsf, zrb = ayrb * kr * dsr;
  gu[0] += Bt * zfb;
  const float tfb = -Bt * zfb, trb = -Bt * zrb;
  const float nf = fmaf(vxs, vxs, yf * yf), nr = fmaf(vxs, vxs, yr * yr);
  const float inf_ = __fdividef(1.0f, nf), inr = __fdividef(1.0f, nr);
  const float yfb = tfb * vxs * inf_, yrb = trb * vxs * inr;
  const float vxsb = -tfb * yf * inf_ - trb * yr * inr;
  xb[4] += yfb + yrb;
  xb[5] += lf * yfb - lr * yrb;
  if (vx > vfloor) xb[3] += vxsb;
}

// (dG/ds)' lam and (dG/du)' lam of one integration sub-step G at state s
template <int MODEL>
__device__ __forceinline__ void substep_vjp(const DevParams& p, const float* s, const float4 c, float* lam,
                                            float* gu) {
  if (MODEL == 0) {
    float sp, cp;
    heading_sincos(s[2], &sp, &cp);
    const float h = p.h, v = s[3], L = p.mp[0];
    const float tl = c.z * L;                 // tan(steer)
    const float sec2_over_L = __fdividef(fmaf(tl, tl, 1.0f), L);
    const float l0 = lam[0], l1 = lam[1], l2 = lam[2], l3 = lam[3];
    lam[2] = l2 + h * v * (cp * l1 - sp * l0);
    lam[3] = l3 + h * (cp * l0 + sp * l1 + c.z * l2);
    gu[0] = fmaf(l2 * h * v, sec2_over_L, gu[0]);
    gu[1] = fmaf(l3, h, gu[1]);
  } else if (MODEL == 1) {
    // Heun: x1 = s + h f(s), G = s + h/2 (f(s) + f(x1)); x1 recomputed as the forward does
    float k1[6], x1[6];
    Model<1>::deriv<float>(p, s, c, k1);
#pragma unroll
    for (int i = 0; i < 6; ++i) x1[i] = __fmaf_rn(p.h, k1[i], s[i]);
    float fb[6], x1b[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < 6; ++i) fb[i] = 0.5f * p.h * lam[i];
    dyn_deriv_vjp(p, x1, c, fb, x1b, gu);  // through f(x1)
    float fa[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      fa[i] = fmaf(p.h, x1b[i], fb[i]);  // f(s) enters G with h/2 and x1 with h
      lam[i] += x1b[i];
    }
    dyn_deriv_vjp(p, s, c, fa, lam, gu);  // through f(s)
  } else {
    gu[0] = fmaf(lam[0], p.h, gu[0]);
  }
}

// reverse through one control step from x_t (sub-steps recomputed)
template <int MODEL>
__device__ __forceinline__ void step_vjp(const DevParams& p, const float* xt, const float4 c, float* lam,
                                         float* gu) {
  using Md = Model<MODEL>;
  if (p.substeps == 1) {
    substep_vjp<MODEL>(p, xt, c, lam, gu);
    return;
  }
  for (int i = p.substeps - 1; i >= 0; --i) {
    float s[Md::NX];
#pragma unroll
    for (int a = 0; a < Md::NX; ++a) s[a] = xt[a];
    for (int j = 0; j < i; ++j) Md::substep(p, s, c);
    substep_vjp<MODEL>(p, s, c, lam, gu);
  }
}

__device__ __forceinline__ float s_tilde_of(const DevParams& p, float S, float cv) {
  return S + ((cv > p.C_u) ? p.A * cv : 0.0f);
}

}  // namespace

// w^_k = exp(-(S~_k - min S~) / lambda) / sum, from the shift and sum the
// update kept (0 for a non-finite S~_k)
__device__ __forceinline__ float weight_of(const DevParams& p, const BwdArgs& a, int k) {
  const float m = a.st->last_min;
  const double s_tot = a.st->last_sum;
  const float st = s_tilde_of(p, a.S[k], a.cvar[k]);
  return (isfinite(st) && s_tot > 0.0) ? (float)((double)expf((m - st) * p.inv_lambda) / s_tot) : 0.0f;
}

// d_k = <gV+, U_k> and w^_k of sample k into a.dk, a.wk (one warp; the
// lanes read U_k's row together and sum it in a fixed shuffle tree)
__device__ __forceinline__ void softmin_terms(const DevParams& p, const BwdArgs& a, int k, int TN, int lane) {
  const float* Uk = a.U + (size_t)k * TN;
  float d = 0.0f;
  for (int c = lane; c < TN; c += 32) d = fmaf(a.gVp[c], Uk[c], d);
  d = warp_sum(d);
  if (lane == 0) {
    a.dk[k] = d;
    a.wk[k] = weight_of(p, a, k);
  }
}

// lanes per nominal rollout in the adjoint: they carry the same state and
// cotangent and split the obstacles of the cost gradient (with one lane per
// rollout, K = 1024 samples leave 32 warps, each on a long serial chain).
// The dynamic model keeps one lane: its Heun sub-steps, repeated on every
// lane of a group, cost more than the split saves
constexpr int kNomLanes = 4;
template <int MODEL>
constexpr int nom_lanes() { return MODEL == 1 ? 1 : kNomLanes; }

// Per warp, the steps of the segments being reversed: 32 lanes x 8 steps x
// (2 NX + 2 NU) floats, whatever the lanes per rollout (32 / lpr rollouts of
// lpr segments each).  Per step: the state x_t, the control u_t and mean
// control v_t (nominal chains), and the cost gradient g_t.
template <int MODEL>
constexpr int step_floats() { return 2 * Model<MODEL>::NX + 2 * Model<MODEL>::NU; }
template <int MODEL>
constexpr int xbuf_floats() { return 32 * kSeg * step_floats<MODEL>(); }

// The cost gradients of steps [tb0, tb1) held in buf (stride step_floats):
// c d(cost terms in mask)/dx at x_t into the step's g_t, the theta partials
// into gth.  They do not depend on the adjoint state, so the L lanes of a
// group split the steps (lane sub takes t = tb0 + sub, tb0 + sub + L, ...)
// and the serial reverse sweep only adds them.
template <int MODEL>
__device__ __forceinline__ void step_cost_grads(const DevParams& p, float* buf, int tb0, int tb1, int sub, int L,
                                                unsigned mask, float c, const float4* __restrict__ obs, int n_obs,
                                                float* gth) {
  constexpr int NX = Model<MODEL>::NX, SW = step_floats<MODEL>(), GO = NX + 2 * Model<MODEL>::NU;
  for (int t = tb0 + sub; t < tb1; t += L) {
    float* st = buf + (t - tb0) * SW;
    float x[NX], g[NX];
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      x[i] = st[i];
      g[i] = 0.0f;
    }
    cost_grad<MODEL>(p, x, mask, c, obs, n_obs, g, gth);
#pragma unroll
    for (int i = 0; i < NX; ++i) st[GO + i] = g[i];
  }
}

// nominal sample k, reversed by nom_lanes lanes (sub = 0 .. nom_lanes - 1;
// all 32 lanes of the warp take part, a lane past K on a copy of sample
// K - 1 that writes nothing), at a unit cotangent of S~_k: cotangents of U_k
// from the nominal cost and the control cost, and the clip mask; theta
// partials of S_k.  The states
// come from the forward's checkpoints: the lanes of a group replay up to
// nom_lanes segments at once (lane sub the segment slo + sub) into the warp's
// state buffer xbuf, then reverse them step by step.  The clip of
// U = clip(V + eps) passes the cotangent iff V + eps lies strictly inside the
// box, which is the case iff U does, so the mask is read off U.
template <int MODEL>
__device__ void bwd_nominal(const DevParams& p, const Inst& in, const BwdArgs& a, int k, int sub, bool writes,
                            const float4* obs_s, int n_obs, float* xbuf) {
  using Md = Model<MODEL>;
  constexpr int NX = Md::NX, NU = Md::NU, NL = nom_lanes<MODEL>();
  const int T = in.T, TN = T * NU;
  const int nseg = (T + kSeg - 1) / kSeg;
  constexpr int SW = step_floats<MODEL>(), GO = NX + 2 * NU;  // per step: x_t, u_t, v_t, g_t
  float* gbuf = xbuf + ((threadIdx.x & 31) / NL) * (NL * kSeg * SW);
  const float sbar = 1.0f;  // unit cotangent: the reduction scales by S~-bar_k
  const float* Uk = a.U + (size_t)k * TN;
  const float* ck = a.ck_nom + (size_t)k * (nseg + 1) * NX;
  const bool warm = k < in.n_warm;
  float lam[NX];
#pragma unroll
  for (int i = 0; i < NX; ++i) lam[i] = 0.0f;
  float gth[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  if (MODEL != 2 && p.c5 != 0.0f) {
    float ds[2];
    track_s_grad(p, ck[nseg * NX], ck[nseg * NX + 1], ds);  // at x_T
    lam[0] = -sbar * p.c5 * ds[0];
    lam[1] = -sbar * p.c5 * ds[1];
  }
  for (int shi = nseg - 1; shi >= 0; shi -= NL) {
    const int slo = max(0, shi - NL + 1);
    const int tb0 = slo * kSeg, tb1 = min(T, (shi + 1) * kSeg);
    const int sr = slo + sub;
    if (sr <= shi) {
      const int t0 = sr * kSeg, t1 = min(T, t0 + kSeg);
      float* dst = gbuf + (t0 - tb0) * SW;
      // the segment's controls and mean controls first: independent loads,
      // in flight together, and the reverse reads them from shared memory
      for (int t = t0; t < t1; ++t) {
#pragma unroll
        for (int j = 0; j < NU; ++j) {
          dst[(t - t0) * SW + NX + j] = Uk[t * NU + j];
          dst[(t - t0) * SW + NX + NU + j] = a.V[t * NU + j];
        }
      }
      float x[NX];
#pragma unroll
      for (int i = 0; i < NX; ++i) x[i] = ck[sr * NX + i];
      for (int t = t0; t < t1; ++t) {
#pragma unroll
        for (int i = 0; i < NX; ++i) dst[(t - t0) * SW + i] = x[i];
        if (t + 1 < t1)
          Md::step(p, x, Md::ctl(p, dst[(t - t0) * SW + NX], NU > 1 ? dst[(t - t0) * SW + NX + 1] : 0.0f));
      }
    }
    __syncwarp();
    // the cost gradients of the batch's steps, split over the group's lanes,
    // with the control cost's theta partial gamma v_t' S^-1 u_t
    step_cost_grads<MODEL>(p, gbuf, tb0, tb1, sub, NL, 0xFFFFFFFFu, sbar, obs_s, n_obs, gth);
    for (int t = tb0 + sub; t < tb1; t += NL) {
      const float* st = gbuf + (t - tb0) * SW;
      gth[2] = fmaf(sbar, st[NX + NU] * p.inv_sig2[0] * st[NX] +
                              (NU > 1 ? st[NX + NU + 1] * p.inv_sig2[1] * st[NX + 1] : 0.0f), gth[2]);
    }
    __syncwarp();
    // the serial reverse sweep: lam_t = (dF/dx)' lam_{t+1} + g_t
    for (int t = tb1 - 1; t >= tb0; --t) {
      const float* st = gbuf + (t - tb0) * SW;
      float xs[NX];
#pragma unroll
      for (int i = 0; i < NX; ++i) xs[i] = st[i];
      const float u0 = st[NX], u1 = NU > 1 ? st[NX + 1] : 0.0f;
      float gu[2] = {0.0f, 0.0f};
      step_vjp<MODEL>(p, xs, Md::ctl(p, u0, u1), lam, gu);
#pragma unroll
      for (int i = 0; i < NX; ++i) lam[i] += st[GO + i];
      // the clip of U = clip(V + eps) and the control cost
      const float vv[2] = {st[NX + NU], NU > 1 ? st[NX + NU + 1] : 0.0f}, uu[2] = {u0, u1};
#pragma unroll
      for (int j = 0; j < NU; ++j) {
        const float msk = (warm && uu[j] > p.u_lo[j] && uu[j] < p.u_hi[j]) ? 1.0f : 0.0f;
        const float gc = p.gamma * p.inv_sig2[j];
        const size_t idx = (size_t)k * TN + t * NU + j;
        if (writes && sub == 0) {
          a.mask[idx] = msk;
          a.Gnom[idx] = msk * (gu[j] + sbar * gc * vv[j]) + sbar * gc * uu[j];
        }
      }
    }
    __syncwarp();
  }
  // the theta partials are split over the group's lanes (by step)
#pragma unroll
  for (int o = 1; o < nom_lanes<MODEL>(); o <<= 1) {
#pragma unroll
    for (int i = 0; i < 4; ++i) gth[i] += __shfl_xor_sync(0xFFFFFFFFu, gth[i], o);
  }
  if (writes && sub == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) a.thn[(size_t)k * 4 + i] = gth[i];
  }
}

// process noise of rollout m at step t as the forward added it: scaled by
// the rollout's proposal factor when importance sampling is on
template <int MODEL, bool IS>
__device__ __forceinline__ void replay_noise(const DevParams& p, const Inst& in, int t, int m, int k, float* x) {
  if constexpr (IS) {
    float aL = 0.0f, aG = 0.0f;
    add_process_noise<MODEL, true>(p, in.k0, in.k1, (uint32_t)t, (uint32_t)m, (uint32_t)k, in.instance, x,
                                   m >= in.is_m0 ? p.is_s : 1.0f, &aL, &aG);
  } else {
    add_process_noise<MODEL>(p, in.k0, in.k1, (uint32_t)t, (uint32_t)m, (uint32_t)k, in.instance, x);
  }
}

// The weights of the risk measure in sample k's M scaled risk costs, times
// the CVaR cotangent cvbar (one warp): VaR by a radix select over
// order-preserving keys (ties at VaR share its weight), then each rollout's
// cotangent.  The rollouts with a nonzero cotangent are packed, (index,
// cotangent) into (act[], Ls[]); returns their count.  With importance
// sampling the weights Ws (beside Ls) enter every weight of the measure.
// RMAX >= ceil(M / 32) rows of costs per lane: sized to M, so the 32 select
// passes loop over rows that hold costs only.
template <bool IS, int RMAX>
__device__ __forceinline__ int bwd_tail(const DevParams& p, const Inst& in, int lane, float cvbar, float* Ls,
                                        const float* Ws, int* act) {
  const int M = in.M;
  const int R = (M + 31) >> 5;
  uint32_t key[RMAX];
  float val[RMAX];
  float sum = 0.0f;
#pragma unroll
  for (int r = 0; r < RMAX; ++r) {
    const int idx = lane + 32 * r;
    const bool valid = idx < M;
    val[r] = valid ? Ls[idx] : 0.0f;
    sum += val[r];
    key[r] = valid ? fkey(val[r]) : 0xFFFFFFFFu;
  }
  uint32_t prefix = 0u;
  int kth = in.j_var - 1;
#pragma unroll 1
  for (int b = 31; b >= 0; --b) {
    const uint32_t hi_mask = (b == 31) ? 0u : (0xFFFFFFFFu << (b + 1));
    int cnt = 0;
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      const uint32_t kk = key[r];
      cnt += ((kk & hi_mask) == prefix && ((kk >> b) & 1u) == 0u && (lane + 32 * r) < M) ? 1 : 0;
    }
    cnt = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)cnt);
    if (kth >= cnt) {
      kth -= cnt;
      prefix |= (1u << b);
    }
  }
  const float var = fkey_inv(prefix);
  int c_gt = 0, c_eq = 0;
#pragma unroll
  for (int r = 0; r < RMAX; ++r) {
    if (lane + 32 * r < M) {
      if (val[r] > var) ++c_gt;
      else if (val[r] == var) ++c_eq;
    }
  }
  c_gt = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)c_gt);
  c_eq = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)c_eq);
  // weights of the risk measure in each scaled cost: above VaR, equal to VaR
  float w_gt, w_eq, w_all = 0.0f;
  if (p.cvar_mode == 0) {
    w_gt = 1.0f / in.tail_denom;
    w_eq = ((float)(M - in.j_var - c_gt) + in.frac_j) / in.tail_denom / (float)c_eq;
  } else if (p.cvar_mode == 1) {
    w_gt = w_eq = 1.0f / (float)(c_gt + c_eq);
  } else if (p.cvar_mode == 2) {
    w_gt = 0.0f;
    w_eq = 1.0f / (float)c_eq;
  } else {
    w_gt = w_eq = 0.0f;  // chance: piecewise constant; mean: uniform weights below
    if (p.cvar_mode >= 4) w_all = 1.0f / (float)M;
  }
  // mean-variance: d rho / d L_a,n = (1 + 2 kappa (L_a,n - mean)) / M with
  // L_a,n - mean = B (L_n - mean)
  float mean = warp_sum(sum) / (float)M;
  float w_dev = p.cvar_mode == 5 ? 2.0f * p.risk_param * p.B / (float)M : 0.0f;
  float base = p.cvar_mode == 3 ? 0.0f : (1.0f - p.B) / (float)M;
  float wts[IS ? RMAX : 1];
  float vw = var;
  if constexpr (IS) {
    // the weighted empirical distribution: every count becomes a weight sum
    // (W in place of M, (1 - alpha) W in place of (1 - alpha) M), and each
    // rollout's weight multiplies its share
    float sw = 0.0f, swl = 0.0f;
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      const bool valid = lane + 32 * r < M;
      wts[r] = valid ? Ws[lane + 32 * r] : 0.0f;
      sw += wts[r];
      swl = fmaf(wts[r], val[r], swl);
    }
    const float W = warp_sum(sw);
    mean = warp_sum(swl) / W;
    const float tau = p.one_m_alpha * W;
    vw = weighted_var<RMAX>(key, wts, M, lane, tau);
    float wgt = 0.0f, weq = 0.0f;
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      if (lane + 32 * r < M) {
        if (val[r] > vw) wgt += wts[r];
        else if (val[r] == vw) weq += wts[r];
      }
    }
    wgt = warp_sum(wgt);
    weq = warp_sum(weq);
    w_all = 0.0f;
    if (p.cvar_mode == 0) {
      w_gt = 1.0f / tau;
      w_eq = (1.0f - wgt / tau) / weq;
    } else if (p.cvar_mode == 1) {
      w_gt = w_eq = 1.0f / (wgt + weq);
    } else if (p.cvar_mode == 2) {
      w_gt = 0.0f;
      w_eq = 1.0f / weq;
    } else {
      w_gt = w_eq = 0.0f;
      if (p.cvar_mode >= 4) w_all = 1.0f / W;
    }
    w_dev = p.cvar_mode == 5 ? 2.0f * p.risk_param * p.B / W : 0.0f;
    base = p.cvar_mode == 3 ? 0.0f : (1.0f - p.B) / W;
  }
  // pack the rollouts with a nonzero cotangent (the costs are in registers
  // now, so Ls can take the cotangents).  A CVaR tail holds about
  // (1 - alpha) M of them, so the reverse sweeps take ceil(n / 32) rows
  // instead of all ceil(M / 32).
  int n_act = 0;
#pragma unroll
  for (int r = 0; r < RMAX; ++r) {
    if (r >= R) break;
    const int m = lane + 32 * r;
    const float Lm = val[r];
    const float wt = m < M ? (Lm > vw ? w_gt : (Lm == vw ? w_eq : 0.0f)) + fmaf(w_dev, Lm - mean, w_all) : 0.0f;
    float lb = m < M ? cvbar * fmaf(p.B, wt, base) : 0.0f;
    if constexpr (IS) lb *= wts[r];
    const unsigned nz = __ballot_sync(0xFFFFFFFFu, lb != 0.0f);
    if (lb != 0.0f) {
      const int pos = n_act + __popc(nz & ((1u << lane) - 1u));
      act[pos] = m;
      Ls[pos] = lb;
    }
    n_act += __popc(nz);
  }
  __syncwarp();
  return n_act;
}

// disturbed rollouts of sample k (one warp), at a unit cotangent of S~_k:
// cotangents of U_k through the CVaR term; theta partials of the risk costs.  With importance sampling the
// importance weights Ws (beside Ls) enter every weight of the risk measure
// (a separate instantiation, so the plain adjoint keeps its registers).
template <int MODEL, bool IS>
__device__ void bwd_disturbed(const DevParams& p, const Inst& in, const BwdArgs& a, int k, int lane, float4* ctl,
                              float* Ls, float* Ws, int* act, float* gus, float* xbuf, const float4* obs_s,
                              int n_obs) {
  using Md = Model<MODEL>;
  constexpr int NX = Md::NX, NU = Md::NU;
  const int T = in.T, TN = T * NU, M = in.M;
  const float cv = a.cvar[k];
  const float cvbar = (cv > p.C_u && isfinite(cv)) ? p.A : 0.0f;  // at a unit cotangent of S~_k
  if (cvbar == 0.0f) {
    for (int c = lane; c < TN; c += 32) a.gUd[(size_t)k * TN + c] = 0.0f;
    if (lane < 4) a.thd[(size_t)k * 4 + lane] = 0.0f;
    softmin_terms(p, a, k, TN, lane);
    return;
  }
  const float* Uk = a.U + (size_t)k * TN;
  for (int t = lane; t < T; t += 32) {
    ctl[t] = Md::ctl(p, Uk[t * NU], NU > 1 ? Uk[t * NU + 1] : 0.0f);
  }
  for (int c = lane; c < (TN <= kGusSlotCols ? 32 * TN : TN); c += 32) gus[c] = 0.0f;
  // the risk costs (and importance weights) the update kept
  for (int m = lane; m < M; m += 32) {
    Ls[m] = a.L[(size_t)k * M + m];
    if constexpr (IS) Ws[m] = a.L[(size_t)in.K * M + (size_t)k * M + m];
  }
  __syncwarp();
  int n_act;
  if (M <= 32) n_act = bwd_tail<IS, 1>(p, in, lane, cvbar, Ls, Ws, act);
  else if (M <= 64) n_act = bwd_tail<IS, 2>(p, in, lane, cvbar, Ls, Ws, act);
  else if (M <= 128) n_act = bwd_tail<IS, 4>(p, in, lane, cvbar, Ls, Ws, act);
  else if (M <= 256) n_act = bwd_tail<IS, 8>(p, in, lane, cvbar, Ls, Ws, act);
  else n_act = bwd_tail<IS, (RA_MPPI_MAX_M_DEV + 31) / 32>(p, in, lane, cvbar, Ls, Ws, act);
  // reverse sweep of every rollout with a nonzero weight.  A short list (a
  // CVaR tail) would leave lanes idle, so each rollout gets lpr lanes that
  // replay up to lpr of its segments at once from the forward's checkpoints
  // and split the steps' cost gradients (32 / lpr rollouts per pass)
  const int lpr = MODEL == 1 ? 1 : (n_act <= 8 ? 4 : (n_act <= 16 ? 2 : 1));  // as nom_lanes
  const int slots = 32 / lpr, slot = lane / lpr, sub = lane % lpr;
  const int nseg = (T + kSeg - 1) / kSeg;
  const float* ckk = a.ck_dist + (size_t)k * nseg * NX * M;
  constexpr int SW = step_floats<MODEL>(), GO = NX + 2 * NU;  // per step: x_t, (unused u, v), g_t
  float* gbuf = xbuf + slot * (lpr * kSeg * SW);
  // the control cotangents: with room for a row per slot (32 T nu floats,
  // T nu <= kGusSlotCols), each group's first lane adds into its own row and
  // the rows are summed once at the end in a fixed order; otherwise a warp
  // sum per step
  const bool slot_rows = TN <= kGusSlotCols;
  float gth[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int c0 = 0; c0 < n_act; c0 += slots) {
    const bool has = c0 + slot < n_act;
    const int m = has ? act[c0 + slot] : 0;  // an idle group replays rollout 0 with no cotangent
    const float lbar = has ? Ls[c0 + slot] : 0.0f;
    float lam[NX];
#pragma unroll
    for (int i = 0; i < NX; ++i) lam[i] = 0.0f;
    for (int shi = nseg - 1; shi >= 0; shi -= lpr) {
      const int slo = max(0, shi - lpr + 1);
      const int tb0 = slo * kSeg, tb1 = min(T, (shi + 1) * kSeg);
      const int sr = slo + sub;
      if (sr <= shi) {
        float x[NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) x[i] = ckk[((size_t)sr * NX + i) * M + m];
        const int t0 = sr * kSeg, t1 = min(T, t0 + kSeg);
        float* dst = gbuf + (t0 - tb0) * SW;
        for (int t = t0; t < t1; ++t) {
#pragma unroll
          for (int i = 0; i < NX; ++i) dst[(t - t0) * SW + i] = x[i];
          if (t + 1 < t1) {
            Md::step(p, x, ctl[t]);
            replay_noise<MODEL, IS>(p, in, t, m, k, x);
          }
        }
      }
      __syncwarp();
      // the risk-cost gradients of the batch's steps, split over the group's lanes
      step_cost_grads<MODEL>(p, gbuf, tb0, tb1, sub, lpr, p.risk_mask, lbar, obs_s, n_obs, gth);
      __syncwarp();
      // the serial reverse sweep: lam_t = (dF/dx)' lam_{t+1} + g_t
      for (int t = tb1 - 1; t >= tb0; --t) {
        const float* st = gbuf + (t - tb0) * SW;
        float xs[NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) xs[i] = st[i];
        float gu[2] = {0.0f, 0.0f};
        step_vjp<MODEL>(p, xs, ctl[t], lam, gu);
#pragma unroll
        for (int i = 0; i < NX; ++i) lam[i] += st[GO + i];
        if (slot_rows) {
          if (sub == 0 && has) {
#pragma unroll
            for (int j = 0; j < NU; ++j) gus[slot * TN + t * NU + j] += gu[j];
          }
        } else {
#pragma unroll
          for (int j = 0; j < NU; ++j) {
            const float s = warp_sum(sub == 0 ? gu[j] : 0.0f);  // one copy per rollout
            if (lane == 0) gus[t * NU + j] += s;
          }
        }
      }
      __syncwarp();
    }
  }
  __syncwarp();
  for (int c = lane; c < TN; c += 32) {
    float v = gus[c];
    if (slot_rows)
      for (int r = 1; r < slots; ++r) v += gus[r * TN + c];
    a.gUd[(size_t)k * TN + c] = v;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float s = warp_sum(gth[i]);
    if (lane == 0) a.thd[(size_t)k * 4 + i] = s;
  }
  softmin_terms(p, a, k, TN, lane);
}

template <int MODEL, bool IS>
__global__ void __launch_bounds__(128) bwd_main_kernel(const DevParams p, const BwdArgs a) {
  extern __shared__ float4 smem[];
  // the obstacles, the warps' state buffers, then the disturbed warps' scratch
  float4* obs_s = smem;
  const int warps = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* xbuf = reinterpret_cast<float*>(obs_s + a.obs_cap) + w * xbuf_floats<MODEL>();
  float4* const scratch = reinterpret_cast<float4*>(reinterpret_cast<float*>(obs_s + a.obs_cap) +
                                                    warps * xbuf_floats<MODEL>());
  const int n_obs = a.st->n_obs;
  // the differentiated update already advanced the counter
  const Inst in = inst_of(p, (uint32_t)(a.st->iteration - 1ull));
  for (int i = threadIdx.x; i < n_obs; i += blockDim.x) obs_s[i] = a.obs[i];
  __syncthreads();

  if ((int)blockIdx.x < a.nb_nom) {
    // nom_lanes lanes per nominal rollout; every lane of a warp with a sample
    // in range takes part in the group shuffles
    constexpr int NL = nom_lanes<MODEL>();
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = gt / NL, sub = gt % NL;
    const int k_warp0 = (gt & ~31) / NL;
    if (k_warp0 < in.K) bwd_nominal<MODEL>(p, in, a, min(k, in.K - 1), sub, k < in.K, obs_s, n_obs, xbuf);
    return;
  }
  const int k = ((int)blockIdx.x - a.nb_nom) * warps + w;
  if (k >= in.K) return;
  float4* ctl = scratch + w * in.T;
  // per warp: risk costs [M], importance weights [M] (when on), packed
  // rollout indices [M], U cotangents [T nu] (a row per slot, [32][T nu],
  // when T nu <= kGusSlotCols)
  const int wcap = IS ? in.M : 0;
  const int TNw = in.T * p.nu;
  const int gcap = TNw <= kGusSlotCols ? 32 * TNw : TNw;
  float* Ls = reinterpret_cast<float*>(scratch + warps * in.T) + w * (2 * in.M + wcap + gcap);
  float* Ws = Ls + in.M;
  int* act = reinterpret_cast<int*>(Ws + wcap);
  float* gus = reinterpret_cast<float*>(act + in.M);
  bwd_disturbed<MODEL, IS>(p, in, a, k, lane, ctl, Ls, Ws, act, gus, xbuf, obs_s, n_obs);
}

// gV and gtheta: sums over the K samples of
//   v_k = mask_k w^_k gV+ + S~-bar_k B_k,  B_k = G_nom,k + mask_k G_dist,k
// (U columns; the theta columns have B_k = the unit theta partials and no
// softmin part).  With S~-bar_k = a_k + b_k c (a_k = gS~_k - w^_k d_k /
// lambda, b_k = w^_k / lambda, c = sum_k w^_k d_k) every column is
// gV+ sum_k mask_k w^_k + sum_k a_k B_k + c sum_k b_k B_k, so one pass over
// the samples forms the three sums and c, and the last block combines them.
// A block takes a slice of the samples in chunks of 32 (d_k and w^_k come
// from the main kernel): the column sums with kRedRows row lanes per
// column, in FP64; the last block to arrive merges the slices.  The order
// depends on K and the grid only.
constexpr int kRedCols = 64, kRedRows = 4;  // 256 threads
constexpr int kRedChunk = 32;
constexpr int kRedColIters = (2 * RA_MPPI_MAX_T_DEV + 4 + kRedCols - 1) / kRedCols;
__global__ void __launch_bounds__(kRedCols * kRedRows) bwd_reduce_kernel(const DevParams p, const BwdArgs a) {
  __shared__ double acc[3][kRedRows][kRedCols];
  __shared__ float ch_w[kRedChunk];
  __shared__ double ch_a[kRedChunk], ch_b[kRedChunk], ch_wd[kRedChunk];
  __shared__ unsigned int is_last;
  const int TN = p.T * p.nu, NC = TN + 4, stride = 3 * NC + 1;
  const int per = (p.K + gridDim.x - 1) / gridDim.x;
  const int kb = blockIdx.x * per, ke = min(p.K, kb + per);
  const int cl = threadIdx.x % kRedCols, rl = threadIdx.x / kRedCols;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double inv_lam = (double)p.inv_lambda;
  double R[kRedColIters], P[kRedColIters], Q[kRedColIters];
#pragma unroll
  for (int j = 0; j < kRedColIters; ++j) R[j] = P[j] = Q[j] = 0.0;
  double wd = 0.0;  // thread 0: the slice's sum of w^_k d_k
  for (int k0 = kb; k0 < ke; k0 += kRedChunk) {
    const int n = min(kRedChunk, ke - k0);
    // the chunk's a_k, b_k from d_k and w^_k (formed by the main kernel)
    if (threadIdx.x < n) {
      const int k = k0 + threadIdx.x;
      const float wk = a.wk[k], d = a.dk[k];
      const double gs = a.gS != nullptr ? (double)a.gS[k] : 0.0;
      ch_w[threadIdx.x] = wk;
      ch_a[threadIdx.x] = gs - (double)wk * (double)d * inv_lam;
      ch_b[threadIdx.x] = (double)wk * inv_lam;
      ch_wd[threadIdx.x] = (double)wk * (double)d;
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int i = 0; i < n; ++i) wd += ch_wd[i];
#pragma unroll
    for (int j = 0; j < kRedColIters; ++j) {
      const int c = j * kRedCols + cl;
      if (c < NC) {
        // (unrolled: the loads of several samples are in flight together)
#pragma unroll 8
        for (int i = rl; i < n; i += kRedRows) {
          const int k = k0 + i;
          float B;
          if (c < TN) {
            const size_t idx = (size_t)k * TN + c;
            const float msk = a.mask[idx];
            B = a.Gnom[idx] + msk * a.gUd[idx];
            R[j] += (double)(msk * ch_w[i]);
          } else {
            B = a.thn[(size_t)k * 4 + (c - TN)] + a.thd[(size_t)k * 4 + (c - TN)];
          }
          P[j] = fma(ch_a[i], (double)B, P[j]);
          Q[j] = fma(ch_b[i], (double)B, Q[j]);
        }
      }
    }
    __syncthreads();
  }
  // the slice's partials: (R, P, Q) per column, then sum w^_k d_k
  double* part = a.red_part + (size_t)blockIdx.x * stride;
#pragma unroll
  for (int j = 0; j < kRedColIters; ++j) {
    if (j * kRedCols >= NC) break;  // uniform across the block
    const int c = j * kRedCols + cl;
    acc[0][rl][cl] = R[j];
    acc[1][rl][cl] = P[j];
    acc[2][rl][cl] = Q[j];
    __syncthreads();
    if (rl < 3 && c < NC)
      part[rl * NC + c] = ((acc[rl][0][cl] + acc[rl][1][cl]) + acc[rl][2][cl]) + acc[rl][3][cl];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[3 * NC] = wd;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(&a.arrive[1], 1u) == gridDim.x - 1 ? 1u : 0u;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  const int nb = (int)gridDim.x;
  __shared__ double c_all;
  if (warp == 0) {
    // c = sum_k w^_k d_k: the slices' sums, lanes strided over the blocks
    // (their loads in flight together), then a fixed shuffle tree
    double c = 0.0;
    for (int b = lane; b < nb; b += 32) c += __ldcg(&a.red_part[(size_t)b * stride + 3 * NC]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if (lane == 0) c_all = c;
  }
  __syncthreads();
  const double c = c_all;
  for (int c0 = 0; c0 < NC; c0 += kRedCols) {
    const int col = c0 + cl;
    double r = 0.0, pp = 0.0, q = 0.0;
    if (col < NC) {
#pragma unroll 4
      for (int b = rl; b < nb; b += kRedRows) {
        const double* pb = a.red_part + (size_t)b * stride;
        r += __ldcg(pb + col);
        pp += __ldcg(pb + NC + col);
        q += __ldcg(pb + 2 * NC + col);
      }
    }
    acc[0][rl][cl] = r;
    acc[1][rl][cl] = pp;
    acc[2][rl][cl] = q;
    __syncthreads();
    if (rl == 0 && col < NC) {
      const double R4 = ((acc[0][0][cl] + acc[0][1][cl]) + acc[0][2][cl]) + acc[0][3][cl];
      const double P4 = ((acc[1][0][cl] + acc[1][1][cl]) + acc[1][2][cl]) + acc[1][3][cl];
      const double Q4 = ((acc[2][0][cl] + acc[2][1][cl]) + acc[2][2][cl]) + acc[2][3][cl];
      const double t = (col < TN ? R4 * (double)a.gVp[col] : 0.0) + P4 + c * Q4;
      if (col < TN) a.gV[col] = (float)t;
      else a.gtheta[col - TN] = (float)t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) a.arrive[1] = 0u;
}

template <int MODEL>
cudaError_t launch_bwd_main(const DevParams& p, const BwdArgs& a, bool is, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e;
  if (is) {
    e = cudaFuncSetAttribute(bwd_main_kernel<MODEL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) bwd_main_kernel<MODEL, true><<<grid, 128, smem, s>>>(p, a);
  } else {
    e = cudaFuncSetAttribute(bwd_main_kernel<MODEL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) bwd_main_kernel<MODEL, false><<<grid, 128, smem, s>>>(p, a);
  }
  return e;
}

cudaError_t launch_backward(int model, const DevParams& p, const BwdArgs& a, int nb_dist, size_t smem, int nb_red,
                            cudaStream_t s, cudaEvent_t ev_begin, cudaEvent_t ev_end) {
  cudaError_t e = cudaSuccess;
  // a.nb_nom counts blocks at one lane per nominal rollout
  BwdArgs b = a;
  if (model == 0) b.nb_nom = a.nb_nom * nom_lanes<0>();
  else if (model == 1) b.nb_nom = a.nb_nom * nom_lanes<1>();
  else b.nb_nom = a.nb_nom * nom_lanes<2>();
  const int grid = b.nb_nom + nb_dist;
  const bool is = p.is_b > 0.0f;
  if (ev_begin != nullptr) {
    e = cudaEventRecord(ev_begin, s);
    if (e != cudaSuccess) return e;
  }
  if (model == 0) e = launch_bwd_main<0>(p, b, is, grid, smem, s);
  else if (model == 1) e = launch_bwd_main<1>(p, b, is, grid, smem, s);
  else e = launch_bwd_main<2>(p, b, is, grid, smem, s);
  if (e != cudaSuccess) return e;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ev_end != nullptr) {
    e = cudaEventRecord(ev_end, s);
    if (e != cudaSuccess) return e;
  }
  bwd_reduce_kernel<<<nb_red, 256, 0, s>>>(p, a);
  return cudaGetLastError();
}

}  // namespace ramppi
