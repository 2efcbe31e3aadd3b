// Device math of the RA-MPPI update: counter-based noise, vehicle models,
// track geometry and running costs.  Everything here runs in registers; the
// kernels in ra_rollout.cuh compose it.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ramppi {

constexpr float kPi = 3.14159265358979323846f;
#define RA_MPPI_MAX_M_DEV 512
#define RA_MPPI_MAX_T_DEV 256

// Constants of one problem, precomputed on the host (ra_api.cu) and passed to
// the kernels by value.
struct DevParams {
  int K, M, T, nu, substeps;
  int noise_type, obs_mode, cvar_mode;
  unsigned risk_mask;
  int n_warm;         // samples k < n_warm are drawn around V (Alg. 1)
  int j_var;          // ceil(alpha M): rank (1-based) of VaR = L_(j) (Eq. 11)
  float frac_j;       // j - alpha M: weight of L_(j) in the fractional tail
  float tail_denom;   // (1 - alpha) M
  float h;            // integration step dt / substeps
  float mp[8];        // model parameters (see ra_mppi.h)
  int pacejka_c15;    // Pacejka shape factor C is exactly 3/2 (closed form below)
  float acc_f, acc_r;  // D Fz / m per axle (times 1/sqrt(2) when pacejka_c15)
  float yaw_f, yaw_r;  // l_f m / Iz, l_r m / Iz
  float nyaw_acc_r;    // -yaw_r acc_r: rear shape to yaw acceleration
  float sigma_u[2], inv_sig2[2], u_lo[2], u_hi[2];
  float w_scale[4];
  uint32_t mix_thresh;    // floor(mix_p 2^32): Gaussian branch iff selector word < it
  float mix_inv_thresh;   // 1 / floor(mix_p 2^32) (0 when the threshold is 0)
  float mix_gauss[4];     // mix_scale * w_scale[s]: std of the Gaussian branch
  float w_dev, w_speed, v_target, gamma, w_obs, w_bdry, c4, c5, c_lin, kappa, inv_kappa;
  float track_S, track_R, track_hw;
  float inv_lambda, A, B, C_u;
  float risk_param;  // threshold of the chance measure; variance weight of mean-variance
  float one_m_alpha;  // 1 - alpha
  // importance-sampled rollouts (see add_process_noise): rollouts m >= is_m0
  // draw their noise at is_s times its size; a rollout's log density ratio
  // is is_base + is_cl f A_L + is_cg f^2 A_G (f its factor, A_L the sum of
  // the unit Laplace magnitudes, A_G of the squared unit normals it drew)
  int is_m0;
  float is_s, is_b;         // proposal scale s, proposal fraction b = (M - is_m0) / M
  float is_base;            // -(draws per rollout) ln s
  float is_cl, is_cg;       // 1 - 1/s, (1 - 1/s^2) / 2
  uint32_t seed_lo, seed_hi, instance;
  unsigned long long* diag;  // optional count of obstacle candidates tested (diagnostics)
};

// Mutable per-handle state in device memory, read at kernel start so that a
// replayed launch sees the current update counter and obstacle count.
struct DevState {
  unsigned long long iteration;
  int status;        // bit 0: non-finite cost, bit 1: all weights vanished
  int n_obs;
  unsigned int arrive;  // last-block-done counter of the update kernel
  float last_min;       // min S~ of the last update (softmin shift)
  double last_sum;      // sum_k exp(-(S~_k - min) / lambda) of the last update
};

enum : int { kStatusNonFinite = 1, kStatusNoWeight = 2 };

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// 4x32 S-box, multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key bumps
// 0x9E3779B9 / 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // one 32 x 32 -> 64 bit product per multiplier (both halves at once)
    const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53u;
    const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57u;
    const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// uniform (x + 1/2) 2^-32 in (0, 1): exact for x < 2^24, otherwise rounded once
__device__ __forceinline__ float u01(uint32_t x) {
  return __fmaf_rn(__uint2float_rn(x), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
}

// Box-Muller pair from two words: sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).
// ln u1 is taken from the word itself: for u1 >= 1/2 as log1p(-(1 - u1)),
// where 1 - u1 = (~a + 1/2) 2^-32 = u01(~a) keeps its full precision (the
// float32 u1 itself would be rounded to a multiple of 2^-24 next to 1, and
// the square root would amplify that near rad = 0).
__device__ __forceinline__ float2 box_muller(uint32_t a, uint32_t b) {
  const float lu = (a >> 31) != 0u ? log1pf(-u01(~a)) : logf(u01(a));
  const float rad = sqrtf(-2.0f * lu);
  float s, c;
  sincospif(2.0f * u01(b), &s, &c);
  return make_float2(__fmul_rn(rad, c), __fmul_rn(rad, s));
}

// ln v of a uniform v in (0, 1] given with w = 1 - v (both exact to one
// rounding): the hardware logarithm, whose absolute error is about 2^-21,
// except next to v = 1 (w < 2^-10), where that error would be large against
// ln v itself and the series log1p(-w) = -w (1 + w/2 + w^2/3 + ...) to the
// cubic term is exact to the float32 rounding (the next term is below
// w^4/4 < 2^-40).  Both are formed and one is selected, so a warp never
// diverges on it.
__device__ __forceinline__ float log_unit(float v, float w) {
  const float series = -w * __fmaf_rn(w, __fmaf_rn(w, 0.333333343f, 0.5f), 1.0f);
  const float hw = __logf(v);
  return w < 9.765625e-4f ? series : hw;
}

// The same pair for process noise, where an absolute error of a few 1e-7 in
// the unit normal is far below the disturbance scale: the angle 2 pi u2 - pi
// lies in (-pi, pi], where the hardware sine and cosine are accurate to about
// 2^-21 absolute, and cos(2 pi u2) = -cos(2 pi u2 - pi) (likewise sin).  The
// radius takes ln u1 from log_unit with 1 - u1 = (~a + 1/2) 2^-32 from the
// word (so its error is not amplified by the square root next to u1 = 1) and
// the square root as x rsqrt(x).
__device__ __forceinline__ float2 box_muller_process(uint32_t a, uint32_t b) {
  const float e = -2.0f * log_unit(u01(a), u01(~a));
  const float rad = e > 0.0f ? e * rsqrtf(e) : 0.0f;
  float s, c;
  __sincosf(fmaf(2.0f * kPi, u01(b), -kPi), &s, &c);
  return make_float2(-rad * c, -rad * s);
}

// Heavy-tailed slot value from a selector word and a value word.  The value
// word gives the tail mass v = 2 min(a, 1 - a) of the uniform
// a = (word + 1/2) 2^-32, computed from the integer so no precision is lost
// near a = 1 (and 1 - v = (r' + 1/2) 2^-31 with r' the 31 low bits of ~r, for
// log_unit), and the sign of a - 1/2.  With the selector at or above
// floor(p 2^32): Laplace(0, b) by its inverse CDF, -b ln v.  Below it:
// N(0, g^2) by Box-Muller from v and the selector itself, which is uniform
// on [0, floor(p 2^32)) given the branch, as the angle
// u2 = (sel + 1/2) / floor(p 2^32).  Both branches share ln v and neither
// diverges within a warp.
__device__ __forceinline__ float mix_value(uint32_t sel, uint32_t word, float b, float g,
                                           uint32_t thresh, float inv_thresh) {
  const bool hi = (word >> 31) != 0u;
  const uint32_t r = hi ? ~word : word;
  const float v = __fmaf_rn(__uint2float_rn(r), 4.656612873077393e-10f, 2.3283064365386963e-10f);
  const float w = __fmaf_rn(__uint2float_rn(~r & 0x7FFFFFFFu), 4.656612873077393e-10f, 2.3283064365386963e-10f);
  const float lv = log_unit(v, w);
  const float e = -2.0f * lv;
  const float rad = e > 0.0f ? e * rsqrtf(e) : 0.0f;
  const float u2 = (__uint2float_rn(sel) + 0.5f) * inv_thresh;
  const float gauss = -g * rad * __cosf(fmaf(2.0f * kPi, u2, -kPi));
  const float mag = sel < thresh ? gauss : -b * lv;
  return hi ? mag : -mag;
}

// mix_value with the unit-scale draw reported for the importance weights:
// adds |u| of a Laplace draw (-ln v) to *aL, or u^2 of a Gaussian one to
// *aG (u the value over its branch's scale).  The returned value has the bits
// of mix_value.
__device__ __forceinline__ float mix_value_is(uint32_t sel, uint32_t word, float b, float g,
                                              uint32_t thresh, float inv_thresh, float* aL, float* aG) {
  const bool hi = (word >> 31) != 0u;
  const uint32_t r = hi ? ~word : word;
  const float v = __fmaf_rn(__uint2float_rn(r), 4.656612873077393e-10f, 2.3283064365386963e-10f);
  const float w = __fmaf_rn(__uint2float_rn(~r & 0x7FFFFFFFu), 4.656612873077393e-10f, 2.3283064365386963e-10f);
  const float lv = log_unit(v, w);
  const float e = -2.0f * lv;
  const float rad = e > 0.0f ? e * rsqrtf(e) : 0.0f;
  const float u2 = (__uint2float_rn(sel) + 0.5f) * inv_thresh;
  const float c = __cosf(fmaf(2.0f * kPi, u2, -kPi));
  const float gauss = -g * rad * c;
  const bool is_gauss = sel < thresh;
  const float zc = rad * c;
  if (is_gauss) *aG = fmaf(zc, zc, *aG);
  else *aL -= lv;
  const float mag = is_gauss ? gauss : -b * lv;
  return hi ? mag : -mag;
}

// sin and cos of a heading angle: reduce to [-pi, pi] with a two-constant
// split of 2 pi (Cody-Waite), then the hardware approximations, whose absolute
// error is about 2^-21 on that interval.
__device__ __forceinline__ void heading_sincos(float a, float* s, float* c) {
  const float n = rintf(__fmul_rn(a, 0.15915494309189535f));  // a / (2 pi)
  float r = __fmaf_rn(n, -6.28318548202514648f, a);            // 2 pi rounded to float
  r = __fmaf_rn(n, 1.7484556e-7f, r);                           // 2 pi - float(2 pi)
  __sincosf(r, s, c);
}

// ---------------------------------------------------------------- lanes x 2
// The dynamic model is written once for T = float (one rollout) and
// T = float2 (two rollouts of a lane side by side).  Every arithmetic step is
// one IEEE operation with round-to-nearest: __fmaf_rn / __fmul_rn /
// __fadd_rn for float, and the sm_100+ paired instructions __ffma2_rn /
// __fmul2_rn / __fadd2_rn for float2, which round each half exactly like
// the scalar ones.  So a pair gives the bits of two scalar evaluations, and
// a launch that interleaves rollouts two by two matches one that does not,
// while issuing one instruction for two FP32 operations.  One rule keeps
// this true: no product is ever added to something as a separate step.  The
// compiler may fuse a paired multiply and a paired add into one FMA (the
// scalar _rn forms are never fused), so every product-plus-term is written as
// an explicit vfma.
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float vneg(float a) { return -a; }
// the hardware reciprocal square root as one PTX instruction, so that no
// compiler rewrite of an expression around it (s * rsqrt(s) as a square
// root, say) can make the scalar and the paired paths differ
__device__ __forceinline__ float rsqrt_hw(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
template <class T> __device__ __forceinline__ T bc(float c);
template <> __device__ __forceinline__ float bc<float>(float c) { return c; }
template <> __device__ __forceinline__ float2 bc<float2>(float c) { return make_float2(c, c); }
// per-rollout application of a scalar function
template <class F> __device__ __forceinline__ float vmap(float a, F f) { return f(a); }
template <class F> __device__ __forceinline__ float2 vmap(float2 a, F f) { return make_float2(f(a.x), f(a.y)); }
__device__ __forceinline__ float vmaxabs(float a) { return fabsf(a); }
__device__ __forceinline__ float vmaxabs(float2 a) { return fmaxf(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ void vsincos(float a, float* s, float* c) { heading_sincos(a, s, c); }
// heading_sincos of two angles, the reduction in paired instructions
__device__ __forceinline__ void vsincos(float2 a, float2* s, float2* c) {
  const float2 y = vmul(a, bc<float2>(0.15915494309189535f));
  const float2 n = make_float2(rintf(y.x), rintf(y.y));
  float2 r = vfma(n, bc<float2>(-6.28318548202514648f), a);
  r = vfma(n, bc<float2>(1.7484556e-7f), r);
  __sincosf(r.x, &s->x, &c->x);
  __sincosf(r.y, &s->y, &c->y);
}

// The heading reduced to [-pi, pi] by the same two-constant split (once per
// control step of the dynamic model, so that its sub-steps can take the
// hardware sine and cosine directly: their argument is scaled by 1/(2 pi) in
// float32, and a heading within a few tenths of a radian of [-pi, pi] keeps
// the absolute error near 2^-21).  A heading already in [-pi, pi] is
// returned unchanged (n = 0).
__device__ __forceinline__ float vwrap(float a) {
  const float n = rintf(__fmul_rn(a, 0.15915494309189535f));
  return __fmaf_rn(n, 1.7484556e-7f, __fmaf_rn(n, -6.28318548202514648f, a));
}
__device__ __forceinline__ float2 vwrap(float2 a) {
  const float2 y = vmul(a, bc<float2>(0.15915494309189535f));
  const float2 n = make_float2(rintf(y.x), rintf(y.y));
  return vfma(n, bc<float2>(1.7484556e-7f), vfma(n, bc<float2>(-6.28318548202514648f), a));
}
// sin and cos of a heading near [-pi, pi] (see vwrap)
__device__ __forceinline__ void vsincos_near(float a, float* s, float* c) { __sincosf(a, s, c); }
__device__ __forceinline__ void vsincos_near(float2 a, float2* s, float2* c) {
  __sincosf(a.x, &s->x, &c->x);
  __sincosf(a.y, &s->y, &c->y);
}

// The per-step control quantities of the dynamic model in the lane type T:
// B steer, accel, and the front axle's -acc_f sin steer and acc_f cos steer
// (its lateral acceleration per unit tyre shape along the body x and y
// axes).  For T = float2 they are either the same for both halves (two
// rollouts of one sample) or the two samples' own (one rollout each of two
// samples).
template <class T>
struct CtlT {
  T bd, a, kns, kc;
};
__device__ __forceinline__ CtlT<float> ctl_of(const DevParams& p, const float4 c, float) {
  return {c.x, c.y, __fmul_rn(-p.acc_f, c.z), __fmul_rn(p.acc_f, c.w)};
}
__device__ __forceinline__ CtlT<float2> ctl_of(const DevParams& p, const float4 c, float2) {
  const CtlT<float> q = ctl_of(p, c, 0.0f);
  return {bc<float2>(q.bd), bc<float2>(q.a), bc<float2>(q.kns), bc<float2>(q.kc)};
}
__device__ __forceinline__ CtlT<float2> ctl_pair(const DevParams& p, const float4 ca, const float4 cb) {
  const CtlT<float> a = ctl_of(p, ca, 0.0f), b = ctl_of(p, cb, 0.0f);
  return {make_float2(a.bd, b.bd), make_float2(a.a, b.a), make_float2(a.kns, b.kns), make_float2(a.kc, b.kc)};
}

// arctangent for the slip angles: z P(z^2) on [0, 1] with P of degree 7 in
// z^2 (coefficients fitted here by iterated weighted least squares on
// Chebyshev nodes for the relative error; max 2.5e-7 in float32), reflected
// as pi/2 - atan(1/|z|) above 1, odd in z.  atan_coef(i) multiplies z^(2i).
__device__ __forceinline__ constexpr float atan_coef(int i) {
  return i == 0 ? 9.999998808e-01f
       : i == 1 ? -3.333199322e-01f
       : i == 2 ? 1.996973604e-01f
       : i == 3 ? -1.401953697e-01f
       : i == 4 ? 9.914427996e-02f
       : i == 5 ? -5.948816240e-02f
       : i == 6 ? 2.425358072e-02f
                : -4.693589173e-03f;
}
// P(s) by Horner (the coefficients as immediates)
template <class T>
__device__ __forceinline__ T atan_q(T s) {
  T q = bc<T>(atan_coef(7));
#pragma unroll
  for (int i = 6; i >= 0; --i) q = vfma(q, s, bc<T>(atan_coef(i)));
  return q;
}
__device__ __forceinline__ float atan_poly(float z) {
  const float a = fabsf(z);
  const bool big = a > 1.0f;
  const float t = big ? __fdividef(1.0f, a) : a;
  float r = vmul(t, atan_q<float>(vmul(t, t)));
  r = big ? __fadd_rn(1.57079632679489662f, -r) : r;
  return copysignf(r, z);
}

// Two arctangents at once (of T, so up to four rollouts' worth).  When no
// active lane has an argument above 1 in magnitude (the common case), the
// warp skips the reflection; z P(z^2) with the odd z equals
// copysign(|z| P(z^2), z) bit for bit (P > 0), so both paths give the same
// bits and the result does not depend on which lanes share a warp.  (A
// shorter polynomial on |z| <= 1/2 was a few per cent faster at small slip
// angles and slower under large disturbances, where few warps stay below
// 1/2.)
template <class T>
__device__ __forceinline__ void atan_pair(T za, T zb, T* ta, T* tb) {
  if (__all_sync(__activemask(), fmaxf(vmaxabs(za), vmaxabs(zb)) <= 1.0f)) {
    *ta = vmul(za, atan_q<T>(vmul(za, za)));
    *tb = vmul(zb, atan_q<T>(vmul(zb, zb)));
  } else {
    *ta = vmap(za, atan_poly);
    *tb = vmap(zb, atan_poly);
  }
}
// Both axles' Pacejka arguments from the slip ratios yf, yr:
// zf = B steer - B atan(yf), zr = -B atan(yr).  (Folding -B into the
// polynomial's coefficients saves two operations but takes them from the
// parameter bank instead of immediates; on GB300 that was slower.)
template <class T>
__device__ __forceinline__ void pacejka_args(const DevParams& p, T yf, T yr, T bd, T* zf, T* zr) {
  T tf, tr;
  atan_pair<T>(yf, yr, &tf, &tr);
  const float Bt = p.mp[4];
  *zf = vfma(bc<T>(-Bt), tf, bd);
  *zr = vmul(bc<T>(-Bt), tr);
}

// ---------------------------------------------------------------- models
// Per-step control quantities shared by all rollouts of a sample:
//   KIN  (steer, accel, tan(steer) / wheelbase, 0)
//   DYN  (steer, accel, sin(steer), cos(steer))
//   LIN  (u, 0, 0, 0)
template <int MODEL>
struct Model;

template <>
struct Model<0> {  // kinematic bicycle, explicit Euler
  static constexpr int NX = 4, NU = 2, NS = 4;
  __device__ static __forceinline__ int slot_dim(int s) { return s; }
  __device__ static __forceinline__ float4 ctl(const DevParams& p, float u0, float u1) {
    return make_float4(u0, u1, tanf(u0) / p.mp[0], 0.0f);
  }
  // one Euler sub-step of size h
  __device__ static __forceinline__ void substep(const DevParams& p, float* x, const float4 c) {
    float sp, cp;
    heading_sincos(x[2], &sp, &cp);
    const float hv = p.h * x[3];
    x[0] = fmaf(hv, cp, x[0]);
    x[1] = fmaf(hv, sp, x[1]);
    x[2] = fmaf(hv, c.z, x[2]);
    x[3] = fmaf(p.h, c.y, x[3]);
  }
  __device__ static __forceinline__ void step(const DevParams& p, float* x, const float4 c) {
    for (int s = 0; s < p.substeps; ++s) substep(p, x, c);
  }
  // the plant's step (the same: every sub-step reduces the heading itself)
  __device__ static __forceinline__ void step_exact(const DevParams& p, float* x, const float4 c) { step(p, x, c); }
  __device__ static __forceinline__ float speed(const float* x) { return x[3]; }
};

template <>
struct Model<1> {  // dynamic single-track with Pacejka lateral tyre forces, Heun
  static constexpr int NX = 6, NU = 2, NS = 3;
  __device__ static __forceinline__ int slot_dim(int s) { return 3 + s; }
  // per-step control quantities: (B steer, accel, sin steer, cos steer)
  __device__ static __forceinline__ float4 ctl(const DevParams& p, float u0, float u1) {
    float s, c;
    sincosf(u0, &s, &c);
    return make_float4(p.mp[4] * u0, u1, s, c);
  }
  // tyre shape sin(C atan z) of one axle; its lateral acceleration is
  // acc_{f,r} times it.  C15: 1 for C = 3/2, 0 for any other C, -1 to read
  // it off the parameters (the step below decides once per control step, so
  // the derivatives carry no branch on it).  For C = 3/2 the shape has the
  // closed form z (q + 2) / (q sqrt(2 q (q + 1))), q = sqrt(1 + z^2)
  // (half-angle identities with cos(atan z) = 1/q; no cancellation near 0).
  // With s = 1 + z^2, 2 q (q + 1) = 2 (s + q) and (q + 2) / q = 1 + 2/q, so
  // it is z (1 + 2u) rsqrt(s + q) / sqrt(2) with u = rsqrt(s) = 1/q; this
  // returns it without the 1/sqrt(2), which the host folds into acc_{f,r}.
  template <class T, int C15 = -1>
  __device__ static __forceinline__ T pacejka(const DevParams& p, T z) {
    if (C15 == 1 || (C15 < 0 && p.pacejka_c15)) {
      const T s = vfma(z, z, bc<T>(1.0f));
      const T u = vmap(s, rsqrt_hw);              // 1 / q, and q = s u
      const T w = vmap(vfma(s, u, s), rsqrt_hw);  // rsqrt(s + q)
      return vmul(vmul(z, vfma(u, bc<T>(2.0f), bc<T>(1.0f))), w);
    }
    const float C = p.mp[5];
    return vmap(z, [C](float v) { return sinf(C * atanf(v)); });
  }
  // f(x, u).  EXACT: the heading's sine and cosine after the full reduction
  // (the plant, whose heading is never wrapped); otherwise the heading lies
  // near [-pi, pi] (step_t wraps it once per control step).
  template <class T, int C15 = -1, bool EXACT = false>
  __device__ static __forceinline__ void deriv(const DevParams& p, const T* x, const CtlT<T>& c, T* f) {
    const float lf = p.mp[2], lr = p.mp[3], vfloor = p.mp[7];
    const T vx = x[3], vy = x[4], r = x[5];
    // slip angles; the floored vx is positive, so atan2(y, vx) = atan(y / vx).
    // Pacejka arguments B alpha_f = B (steer - atan_f), B alpha_r = -B atan_r
    const T inv_vx = vmap(vx, [vfloor](float v) { return __fdividef(1.0f, fmaxf(v, vfloor)); });
    T zf, zr;
    pacejka_args<T>(p, vmul(vfma(bc<T>(lf), r, vy), inv_vx), vmul(vfma(bc<T>(-lr), r, vy), inv_vx), c.bd, &zf, &zr);
    const T sh_f = pacejka<T, C15>(p, zf), sh_r = pacejka<T, C15>(p, zr);
    T sp, cp;
    if (EXACT) vsincos(x[2], &sp, &cp);
    else vsincos_near(x[2], &sp, &cp);
    // (negated factors make the products exact negations: a (-b) = -(a b))
    f[0] = vfma(vx, cp, vmul(vneg(vy), sp));
    f[1] = vfma(vx, sp, vmul(vy, cp));
    f[2] = r;
    const T g = vmul(sh_f, c.kc);  // front force along the body y axis, per unit mass
    f[3] = vfma(sh_f, c.kns, vfma(r, vy, c.a));
    f[4] = vfma(r, vneg(vx), vfma(bc<T>(p.acc_r), sh_r, g));
    f[5] = vfma(bc<T>(p.yaw_f), g, vmul(bc<T>(p.nyaw_acc_r), sh_r));
  }
  // one Heun sub-step of size h: x + h/2 k1 + h/2 k2 with k1 = f(x) and
  // k2 = f(x + h k1), accumulated as (x + h/2 k1) + h/2 k2, so that x and k1
  // are dead while k2 is formed (fewer live registers than x + h/2 (k1 + k2))
  template <class T, int C15 = -1, bool EXACT = false>
  __device__ static __forceinline__ void substep_t(const DevParams& p, T* x, const CtlT<T>& c) {
    T k[6], xp[6];
    deriv<T, C15, EXACT>(p, x, c, k);
    const float hh = 0.5f * p.h;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      xp[i] = vfma(bc<T>(p.h), k[i], x[i]);
      x[i] = vfma(bc<T>(hh), k[i], x[i]);
    }
    deriv<T, C15, EXACT>(p, xp, c, k);
#pragma unroll
    for (int i = 0; i < 6; ++i) x[i] = vfma(bc<T>(hh), k[i], x[i]);
  }
  // one control step: the heading wrapped to [-pi, pi] (the state's other
  // components and every cost are unaffected), then the sub-steps
  template <class T, bool EXACT = false>
  __device__ static __forceinline__ void step_t(const DevParams& p, T* x, const CtlT<T>& c) {
    if (!EXACT) x[2] = vwrap(x[2]);
    if (p.pacejka_c15) {
      for (int s = 0; s < p.substeps; ++s) substep_t<T, 1, EXACT>(p, x, c);
    } else {
      for (int s = 0; s < p.substeps; ++s) substep_t<T, 0, EXACT>(p, x, c);
    }
  }
  // the derivative with one sample's control quantities (heading near [-pi, pi])
  template <class T>
  __device__ static __forceinline__ void deriv(const DevParams& p, const T* x, const float4 c, T* f) {
    deriv<T>(p, x, ctl_of(p, c, T{}), f);
  }
  // one sub-step from a state whose heading is near [-pi, pi]
  __device__ static __forceinline__ void substep(const DevParams& p, float* x, const float4 c) {
    substep_t<float>(p, x, ctl_of(p, c, 0.0f));
  }
  __device__ static __forceinline__ void step(const DevParams& p, float* x, const float4 c) {
    step_t<float>(p, x, ctl_of(p, c, 0.0f));
  }
  // the plant's step: the heading is kept as it is (no wrap) and reduced
  // exactly inside every derivative
  __device__ static __forceinline__ void step_exact(const DevParams& p, float* x, const float4 c) {
    step_t<float, true>(p, x, ctl_of(p, c, 0.0f));
  }
  // two rollouts at once: x[i] = (state i of rollout a, state i of rollout b)
  __device__ static __forceinline__ void step2(const DevParams& p, float2* x, const float4 c) {
    step_t<float2>(p, x, ctl_of(p, c, float2{}));
  }
  // one rollout each of two samples: x[i] = (state i under ca, state i under cb)
  __device__ static __forceinline__ void step2x(const DevParams& p, float2* x, const float4 ca, const float4 cb) {
    step_t<float2>(p, x, ctl_pair(p, ca, cb));
  }
  __device__ static __forceinline__ float speed(const float* x) { return x[3]; }
};

template <>
struct Model<2> {  // linear test system x+ = x + h u
  static constexpr int NX = 1, NU = 1, NS = 1;
  __device__ static __forceinline__ int slot_dim(int s) { return s; }
  __device__ static __forceinline__ float4 ctl(const DevParams&, float u0, float) {
    return make_float4(u0, 0.f, 0.f, 0.f);
  }
  __device__ static __forceinline__ void substep(const DevParams& p, float* x, const float4 c) {
    x[0] = fmaf(p.h, c.x, x[0]);
  }
  __device__ static __forceinline__ void step(const DevParams& p, float* x, const float4 c) {
    for (int s = 0; s < p.substeps; ++s) substep(p, x, c);
  }
  // the plant's step (the same: every sub-step reduces the heading itself)
  __device__ static __forceinline__ void step_exact(const DevParams& p, float* x, const float4 c) { step(p, x, c); }
  __device__ static __forceinline__ float speed(const float*) { return 0.f; }
};

// ---------------------------------------------------------------- noise
// Process noise of rollout m of sample k at step t, added to the state
// (NT: the noise type fixed at compile time, -1 to read it off p):
// counter (t | draw << 16, m, k, instance).  IS: every value is multiplied by
// f (the rollout's proposal factor, 1 or s; f = 1 keeps the bits) and the
// unit-scale draws are summed into *aL (Laplace magnitudes) and *aG (squared
// normals) for the importance weight (Gaussian and mixture noise only).
template <int MODEL, bool IS = false, int NT = -1>
__device__ __forceinline__ void add_process_noise(const DevParams& p, uint32_t k0, uint32_t k1,
                                                  uint32_t t, uint32_t m, uint32_t k, uint32_t instance,
                                                  float* x, float f = 1.0f, float* aL = nullptr,
                                                  float* aG = nullptr) {
  using Md = Model<MODEL>;
  if constexpr (IS) {
    if (p.noise_type == 0) {
      const uint4 w = philox4x32_10(make_uint4(t, m, k, instance), k0, k1);
      const float2 z01 = box_muller_process(w.x, w.y);
      const float2 z23 = Md::NS > 2 ? box_muller_process(w.z, w.w) : make_float2(0.0f, 0.0f);
      const float z[4] = {z01.x, z01.y, z23.x, z23.y};
#pragma unroll
      for (int s = 0; s < Md::NS; ++s) {
        x[Md::slot_dim(s)] = fmaf(p.w_scale[s] * f, z[s], x[Md::slot_dim(s)]);
        if (p.w_scale[s] != 0.0f) *aG = fmaf(z[s], z[s], *aG);
      }
    } else {
      const uint4 sel = philox4x32_10(make_uint4(t, m, k, instance), k0, k1);
      const uint4 val = philox4x32_10(make_uint4(t | (1u << 16), m, k, instance), k0, k1);
      const uint32_t sw[4] = {sel.x, sel.y, sel.z, sel.w};
      const uint32_t vw[4] = {val.x, val.y, val.z, val.w};
#pragma unroll
      for (int s = 0; s < Md::NS; ++s) {
        if (p.w_scale[s] != 0.0f)
          x[Md::slot_dim(s)] += f * mix_value_is(sw[s], vw[s], p.w_scale[s], p.mix_gauss[s], p.mix_thresh,
                                                 p.mix_inv_thresh, aL, aG);
      }
    }
    return;
  }
  const int nt = NT >= 0 ? NT : p.noise_type;
  if (nt == 0) {
    const uint4 w = philox4x32_10(make_uint4(t, m, k, instance), k0, k1);
    const float2 z01 = box_muller_process(w.x, w.y);
    x[Md::slot_dim(0)] = fmaf(p.w_scale[0], z01.x, x[Md::slot_dim(0)]);
    if (Md::NS > 1) {
      x[Md::slot_dim(1)] = fmaf(p.w_scale[1], z01.y, x[Md::slot_dim(1)]);
      const float2 z23 = box_muller_process(w.z, w.w);
      x[Md::slot_dim(2)] = fmaf(p.w_scale[2], z23.x, x[Md::slot_dim(2)]);
      if (Md::NS > 3) x[Md::slot_dim(3)] = fmaf(p.w_scale[3], z23.y, x[Md::slot_dim(3)]);
    }
  } else if (nt == 1) {
    const uint4 sel = philox4x32_10(make_uint4(t, m, k, instance), k0, k1);
    const uint4 val = philox4x32_10(make_uint4(t | (1u << 16), m, k, instance), k0, k1);
    const uint32_t sw[4] = {sel.x, sel.y, sel.z, sel.w};
    const uint32_t vw[4] = {val.x, val.y, val.z, val.w};
#pragma unroll
    for (int s = 0; s < Md::NS; ++s) {
      if (p.w_scale[s] != 0.0f)
        x[Md::slot_dim(s)] += mix_value(sw[s], vw[s], p.w_scale[s], p.mix_gauss[s], p.mix_thresh, p.mix_inv_thresh);
    }
  } else if (nt == 2) {
    // uniform on [-a_s, a_s]: (2u - 1) a_s
    const uint4 w = philox4x32_10(make_uint4(t, m, k, instance), k0, k1);
    const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int s = 0; s < Md::NS; ++s)
      x[Md::slot_dim(s)] += fmaf(2.0f * u01(ww[s]), p.w_scale[s], -p.w_scale[s]);
  } else {
    // impulse: with probability p a jump of per-slot size a_s along a
    // direction uniform on the unit sphere of the active slots
    const uint4 a = philox4x32_10(make_uint4(t, m, k, instance), k0, k1);
    if (a.x < p.mix_thresh) {
      const uint4 b = philox4x32_10(make_uint4(t | (1u << 16), m, k, instance), k0, k1);
      const float2 z01 = box_muller_process(a.y, a.z);
      const float2 z23 = box_muller_process(a.w, b.x);
      const float z[4] = {z01.x, z01.y, z23.x, z23.y};
      float n2 = 0.0f;
#pragma unroll
      for (int s = 0; s < Md::NS; ++s)
        if (p.w_scale[s] != 0.0f) n2 = fmaf(z[s], z[s], n2);
      const float inv = n2 > 0.0f ? rsqrtf(n2) : 0.0f;
#pragma unroll
      for (int s = 0; s < Md::NS; ++s)
        if (p.w_scale[s] != 0.0f) x[Md::slot_dim(s)] = fmaf(p.w_scale[s] * z[s], inv, x[Md::slot_dim(s)]);
    }
  }
}

// Control sample U^k_t = clip(base + sigma eps): counter (t, 0xFFFFFFFF, k, instance).
// Rounding is pinned (explicit _rn intrinsics) so every thread that draws the
// same (k, t) gets the same bits.
__device__ __forceinline__ float2 control_sample(const DevParams& p, uint32_t k0, uint32_t k1, int k,
                                                 int t, float v0, float v1, int n_warm, uint32_t instance) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)t, 0xFFFFFFFFu, (uint32_t)k, instance), k0, k1);
  const float2 z = box_muller(w.x, w.y);
  const bool warm = k < n_warm;
  const float b0 = warm ? v0 : 0.0f, b1 = warm ? v1 : 0.0f;
  float u0 = __fmaf_rn(p.sigma_u[0], z.x, b0);
  float u1 = __fmaf_rn(p.sigma_u[1], z.y, b1);
  u0 = fminf(fmaxf(u0, p.u_lo[0]), p.u_hi[0]);
  u1 = fminf(fmaxf(u1, p.u_lo[1]), p.u_hi[1]);
  return make_float2(u0, u1);
}

// ---------------------------------------------------------------- costs
// Stadium track: lateral deviation e (outward +), CCW arc length s from
// (0, -R), distance to the nearest boundary d = hw - |e|.
__device__ __forceinline__ float track_e(const DevParams& p, float px, float py) {
  const float half = 0.5f * p.track_S;
  const float ax = fabsf(px);
  if (ax <= half) return fabsf(py) - p.track_R;
  const float dx = ax - half;
  return sqrtf(fmaf(dx, dx, py * py)) - p.track_R;
}

__device__ __forceinline__ float track_s(const DevParams& p, float px, float py) {
  const float S = p.track_S, R = p.track_R, half = 0.5f * S;
  const float total = 2.0f * S + 2.0f * kPi * R;
  if (fabsf(px) <= half) {
    if (py < 0.0f) return px >= 0.0f ? px : total + px;
    return half + kPi * R + (half - px);
  }
  if (px > half) return half + R * (atan2f(py, px - half) + 0.5f * kPi);
  const float th = atan2f(py, px + half);
  const float phi = th > 0.0f ? th - 0.5f * kPi : th + 1.5f * kPi;
  return half + kPi * R + S + R * phi;
}

// softplus(z) = log(1 + exp(z)) = max(z, 0) + log(1 + e), e = exp(-|z|) in
// (0, 1], from the hardware exponential (relative error about 2^-22) and,
// for e >= 2^-6, the hardware logarithm of 1 + e (absolute error about 1e-7
// against a value above 0.0155).  Below 2^-6, where that error would be large
// against log(1 + e) itself, the series e (1 - e/2 + e^2/3 - e^3/4 + e^4/5),
// whose first omitted term is below 2^-32 e.  Both are formed and one is
// selected, so a warp never diverges on it.
__device__ __forceinline__ float softplus_fast(float z) {
  const float e = __expf(-fabsf(z));
  const float ser = e * fmaf(e, fmaf(e, fmaf(e, fmaf(e, 0.2f, -0.25f), 0.333333343f), -0.5f), 1.0f);
  const float hw = __logf(1.0f + e);
  return fmaxf(z, 0.0f) + (e < 0.015625f ? ser : hw);
}

// obstacle term: obstacles are (x, y, r, r^2)
__device__ __forceinline__ float obstacle_term(const DevParams& p, float px, float py,
                                               const float4* __restrict__ obs, int n_obs) {
  float acc = 0.0f;
  if (p.obs_mode == 0) {
    for (int i = 0; i < n_obs; ++i) {
      const float4 o = obs[i];
      const float dx = px - o.x, dy = py - o.y;
      acc += (fmaf(dx, dx, dy * dy) < o.w) ? 1.0f : 0.0f;
    }
  } else {
    for (int i = 0; i < n_obs; ++i) {
      const float4 o = obs[i];
      const float dx = px - o.x, dy = py - o.y;
      const float d2 = fmaf(dx, dx, dy * dy);
      const float d = d2 > 0.0f ? d2 * rsqrtf(d2) : 0.0f;
      acc += softplus_fast(p.kappa * (o.z - d));
    }
    acc *= p.inv_kappa;
  }
  return acc;
}

// running cost of the terms in `mask` (Eq. 20 family; Eqs. 21, 22)
template <int MODEL>
__device__ __forceinline__ float state_cost(const DevParams& p, const float* x, unsigned mask,
                                            const float4* __restrict__ obs, int n_obs) {
  float c = 0.0f;
  if (MODEL == 2) {
    if (mask & 16u) c = p.c_lin * x[0];
    return c;
  }
  if (mask & 9u) {  // deviation or boundary needs e(x)
    const float e = track_e(p, x[0], x[1]);
    if (mask & 1u) c = fmaf(p.w_dev, e * e, c);
    if ((mask & 8u) && p.w_bdry != 0.0f) {
      const float d = p.track_hw - fabsf(e);
      const float b = atanf(-100.0f * d) * (1.0f / kPi) + 0.5f;
      c = fmaf(p.w_bdry, fmaxf(b, 0.0f), c);
    }
  }
  if (mask & 2u) {
    const float dv = Model<MODEL>::speed(x) - p.v_target;
    c = fmaf(p.w_speed, dv * dv, c);
  }
  if (mask & 4u) c = fmaf(p.w_obs, obstacle_term(p, x[0], x[1], obs, n_obs), c);
  if (mask & 16u) c = fmaf(p.c_lin, x[0], c);
  return c;
}

// terminal cost phi(x) = c4 - c5 s(x) (Eq. 23)
template <int MODEL>
__device__ __forceinline__ float terminal_cost(const DevParams& p, const float* x) {
  if (MODEL == 2) return 0.0f;
  if (p.c5 == 0.0f) return p.c4;
  return p.c4 - p.c5 * track_s(p, x[0], x[1]);
}

}  // namespace ramppi
