/*
 * ra_mppi.h — C ABI of the GB300 (sm_103a) Risk-Aware MPPI update library.
 *
 * One call of ra_mppi_step performs one control update of RA-MPPI
 * (Yin, Zhang, Tsiotras, "Risk-Aware Model Predictive Path Integral Control
 * Using Conditional Value-at-Risk", arXiv 2209.12842), i.e. one pass of the
 * body of Algorithm 1 minus the state estimate and the actuation:
 *
 *   1. sample K control sequences U^k = clip(V + eps^k), eps ~ N(0, Sigma);
 *      the last eta fraction of samples use U^k = clip(eps^k)   (Alg. 1)
 *   2. roll each out on the nominal dynamics x_{t+1} = F(x_t, u_t) (Eq. 1)
 *      and charge S_k = phi(x_T) + sum_t q(x_t) + gamma v_t' Sigma^-1 u_t
 *                                                                 (Eq. 3)
 *   3. roll out M disturbed trajectories x~_{t+1} = F(x~_t, u_t) + w_t per
 *      sample (Eqs. 6, 7) with risk costs L = sum_t l(x~_t)        (Eq. 9)
 *   4. CVaR_alpha of the M risk costs, after the sensitivity scaling
 *      L_a = B (L - mean) + mean                       (Eqs. 10-13, 18, 19)
 *   5. S~_k = S_k + A CVaR_k 1{CVaR_k > C_u}                 (Eqs. 14-16)
 *   6. w_k = exp(-(S~_k - min S~) / lambda),
 *      V+ = sum_k w_k U^k / sum_k w_k                      (Eqs. 4, 5, 17)
 *
 * Letters: K control samples (the paper's M), M disturbed rollouts per
 * sample (the paper's N), T horizon steps (the paper's K).
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status (ra_mppi_status); the library
 *     never aborts the process.  Invalid arguments return RA_MPPI_EINVAL
 *     before any work is enqueued.
 *   - Arrays are float32, contiguous, row-major.  "device" pointers must be
 *     CUDA device (or managed) memory on the handle's device; "host"
 *     pointers are ordinary host memory (pinned memory gives faster copies).
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy
 *     default stream.  Device-pointer entry points only enqueue work: no
 *     allocation, no synchronisation.  Results are valid once the stream
 *     has reached the call.
 *   - A handle owns its workspace (allocated at create, freed at destroy)
 *     and is not thread-safe; distinct handles are independent.
 *   - The random numbers come from Philox4x32-10 (Salmon et al., SC'11)
 *     keyed by (seed, update iteration) and counted by (t, rollout m,
 *     sample k, instance); the iteration counter lives in the handle and
 *     advances by one per update, so a handle reproduces its sequence
 *     exactly after ra_mppi_set_state.
 */
#ifndef RA_MPPI_H
#define RA_MPPI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RA_MPPI_OK = 0,
  RA_MPPI_EINVAL = -1,       /* invalid argument or size                    */
  RA_MPPI_ENOMEM = -2,       /* device or host allocation failed            */
  RA_MPPI_ECUDA = -3,        /* a CUDA runtime call or launch failed        */
  RA_MPPI_ETIMEOUT = -4,     /* reserved: no kernel of this library waits on
                                another block, so no call returns it         */
  RA_MPPI_ENONFINITE = -5,   /* a cost was NaN/inf or all weights vanished  */
  RA_MPPI_EUNSUPPORTED = -6  /* valid request the library does not support  */
} ra_mppi_status;

/* Dynamics F (Eq. 1).  The paper does not give its vehicle model; these are
 * the three models of this library (state / control layout):
 *   KIN_BICYCLE      x = (px, py, psi, v),           u = (steer, accel),
 *                    explicit Euler; model_params[0] = wheelbase
 *   DYN_SINGLE_TRACK x = (px, py, psi, vx, vy, r),   u = (steer, accel),
 *                    Heun (RK2); model_params = m, Iz, lf, lr, Pacejka B,
 *                    C, D, vx floor of the slip angles; lateral tyre force
 *                    D Fz sin(C atan(B alpha)) with static axle loads Fz
 *   LINEAR_TEST      x = (x),                         u = (u),
 *                    x+ = x + dt u (closed-form checks)
 * `substeps` integration steps of dt / substeps make one control period. */
enum { RA_MPPI_KIN_BICYCLE = 0, RA_MPPI_DYN_SINGLE_TRACK = 1, RA_MPPI_LINEAR_TEST = 2 };

/* Process noise w_t of the disturbed dynamics (Eq. 6), added to the state
 * after each control period.  Slots: KIN (px, py, psi, v); DYN (vx, vy, r);
 * LINEAR (x).  GAUSS: w_s ~ N(0, w_scale[s]^2).  LAPLACE_MIX: w_s ~
 * Laplace(0, w_scale[s]), replaced with probability mix_p by
 * N(0, (mix_scale w_scale[s])^2).  UNIFORM: w_s ~ U[-w_scale[s], w_scale[s]]
 * (the paper's uniform disturbance, Sec. V-B).  IMPULSE: with probability
 * mix_p a jump of size w_scale[s] per slot along a direction uniform on the
 * unit sphere of the slots with w_scale != 0, else none (the paper's
 * impulse disturbance, Sec. V-B). */
enum { RA_MPPI_NOISE_GAUSS = 0, RA_MPPI_NOISE_LAPLACE_MIX = 1, RA_MPPI_NOISE_UNIFORM = 2, RA_MPPI_NOISE_IMPULSE = 3 };

/* Obstacle term of q and l: the indicator 1{d_i < r_i} of Eq. 22, or a
 * smooth barrier softplus(kappa (r_i - d_i)) / kappa. */
enum { RA_MPPI_OBS_INDICATOR = 0, RA_MPPI_OBS_SOFTPLUS = 1 };

/* Risk measure of the M risk costs (field cvar_mode), after the
 * sensitivity scaling (Eqs. 18, 19):
 *   RU     CVaR as the fractional sorted tail [(j - alpha M) L_(j) +
 *          sum_{i>j} L_(i)] / ((1 - alpha) M), j = ceil(alpha M) (equals the
 *          Rockafellar-Uryasev minimum; continuous in L, tie-insensitive)
 *   TCE    CVaR in the literal Monte-Carlo form of Eqs. 12-13: mean of
 *          {L >= VaR}, VaR = L_(j) (Eq. 11)
 *   VAR    VaR_alpha = L_(j) itself (Eq. 11)
 *   CHANCE fraction of the M costs above risk_param (a chance constraint
 *          in place of CVaR; the paper names chance constraints as a
 *          replacement for its Monte-Carlo risk block, Secs. I and III-A)
 *   MEAN   the mean risk cost (risk neutral)
 *   MEANVAR mean-variance: mean + risk_param * (1/M) sum (L_a - mean)^2 of
 *          the scaled costs L_a, risk_param >= 0 (the paper's risk block
 *          admits other metrics, Secs. I and III-A; this classical one is
 *          not among those it names) */
enum { RA_MPPI_CVAR_RU = 0, RA_MPPI_CVAR_TCE = 1, RA_MPPI_RISK_VAR = 2, RA_MPPI_RISK_CHANCE = 3,
       RA_MPPI_RISK_MEAN = 4, RA_MPPI_RISK_MEANVAR = 5 };

/* Bits of risk_mask: the running-cost terms that form the risk cost l
 * (Eq. 9).  The paper's experiments use l = q (all terms). */
enum {
  RA_MPPI_TERM_DEV = 1,   /* w_dev e(x)^2, lateral deviation from the centreline */
  RA_MPPI_TERM_SPEED = 2, /* w_speed (v - v_target)^2 (v = speed, or vx)         */
  RA_MPPI_TERM_OBS = 4,   /* w_obs sum_i obstacle term (Eq. 22)                   */
  RA_MPPI_TERM_BDRY = 8,  /* w_bdry max{0, atan(-100 d(x))/pi + 1/2} (Eq. 21)     */
  RA_MPPI_TERM_LIN = 16   /* c_lin x[0] (linear test cost)                        */
};

/* flags */
enum {
  RA_MPPI_KEEP_RISK_COSTS = 1, /* keep the K x M risk costs L for inspection              */
  RA_MPPI_DIFFERENTIABLE = 2   /* keep what ra_mppi_backward needs (x0, V and the risk costs of each update) */
};

#define RA_MPPI_MAX_M 512
#define RA_MPPI_MAX_T 256
#define RA_MPPI_MAX_OBSTACLES 1024
/* Every obstacle disc must lie in the square |x|, |y| <= RA_MPPI_OBSTACLE_EXTENT
 * metres (|centre| + r within it).  The kernels' obstacle cull is exact under
 * this bound (float32 rounding of shifted coordinates stays below its pad). */
#define RA_MPPI_OBSTACLE_EXTENT 500.0f

/* Problem definition (the quantities of Sec. II-V).  All reals float32. */
typedef struct ra_mppi_problem {
  int32_t model;      /* RA_MPPI_KIN_BICYCLE, ...                            */
  int32_t K;          /* control samples, 1 .. 2^24                          */
  int32_t M;          /* disturbed rollouts per sample, 1 .. RA_MPPI_MAX_M   */
  int32_t T;          /* horizon steps, 1 .. RA_MPPI_MAX_T                   */
  int32_t substeps;   /* integration steps per control period, >= 1          */
  int32_t noise_type; /* RA_MPPI_NOISE_*                                     */
  int32_t obs_mode;   /* RA_MPPI_OBS_*                                       */
  int32_t cvar_mode;  /* RA_MPPI_CVAR_*                                      */
  uint32_t risk_mask; /* RA_MPPI_TERM_* bits forming l                       */
  int32_t flags;      /* RA_MPPI_KEEP_RISK_COSTS                             */
  float dt;           /* control period (s)                                  */
  float model_params[8];
  float sigma_u[2];   /* Sigma = diag(sigma_u^2); sigma 0 = no noise, no cost */
  float u_lo[2], u_hi[2]; /* control box; samples are clipped after noise   */
  float w_scale[4];   /* process-noise scale per slot                        */
  float mix_p, mix_scale;
  float w_dev, w_speed, v_target, gamma, w_obs, w_bdry, c4, c5, c_lin;
  float kappa;        /* softplus barrier sharpness                          */
  float track_straight, track_radius, track_half_width; /* stadium track    */
  float lambda;       /* softmin temperature, > 0 (Eq. 5)                    */
  float alpha;        /* CVaR level in (0, 1) (Eq. 8b)                        */
  float A;            /* CVaR cost gain (Eq. 14)                              */
  float B;            /* risk sensitivity scale, >= 0 (Eq. 18)                */
  float C_u;          /* CVaR bound (Eq. 15)                                  */
  float eta;          /* zero-mean sample fraction in [0, 1) (Alg. 1)         */
  float risk_param;   /* threshold of RISK_CHANCE; variance weight (>= 0) of RISK_MEANVAR */
  int32_t max_obstacles; /* capacity of the obstacle list, 0 .. RA_MPPI_MAX_OBSTACLES */
  uint32_t instance_id;  /* fourth Philox counter word                        */
  uint64_t seed;         /* Philox key                                        */
  /* Importance-sampled rollouts (the paper names importance sampling for
   * alpha near 1 but leaves it out, Sec. III-A).  The last
   * M_s = floor(is_frac M) rollouts of every sample draw each process-noise
   * value at is_scale times its size; with b = M_s / M, rollout m gets the
   * deterministic-mixture weight w_m = 1 / ((1 - b) + b q(W_m)/p(W_m)) of
   * its noise path W_m (p the nominal density, q(w) = p(w/s)/s per value;
   * for the mixture noise the density given the branch drawn), and every
   * risk measure becomes that of the weighted empirical distribution of the
   * M risk costs (VaR: the smallest cost whose strictly larger weight is at
   * most (1 - alpha) sum w; RU CVaR: VaR + sum w (L - VaR)+ / ((1 - alpha)
   * sum w); the others the weighted tail mean, fraction or moments).
   * Off when is_frac = 0 or is_scale = 1 (or M_s = 0).  is_scale in
   * [1, 16], is_frac in [0, 1); Gaussian and mixture noise only.  The
   * batched path applies it per problem (M_s from each problem's M);
   * ra_mppi_backward differentiates the weighted measure (the weights depend
   * on the noise only). */
  float is_scale;
  float is_frac;
} ra_mppi_problem;

typedef struct ra_mppi ra_mppi_t;

/* Size of ra_mppi_problem as compiled into the library (binding check). */
int32_t ra_mppi_problem_size(void);

/* Validate *p (the problem of Secs. II-III: dynamics, costs, Sigma, lambda,
 * alpha, K, M, T) and allocate a handle with all its workspace on CUDA
 * device `device` (-1: the current device).  Every later call on the handle
 * runs on that device, whatever device is current when it is made (the
 * caller's current device is restored on return).  Returns EINVAL for
 * out-of-range sizes or parameters (lambda <= 0, alpha outside (0, 1),
 * B < 0, eta outside [0, 1), M > RA_MPPI_MAX_M, no such device, ...),
 * ENOMEM if allocation fails, ECUDA if the device cannot be used.  *out is
 * set only on success. */
int ra_mppi_create(const ra_mppi_problem* p, int32_t device, ra_mppi_t** out);

/* Release a handle and its workspace.  NULL is allowed. */
void ra_mppi_destroy(ra_mppi_t* h);

/* Set the obstacle circles used by q and l (Eq. 22): xyr[n_obs][3] =
 * (centre x, centre y, radius), host or device pointer.  Synchronous: the
 * copy has completed when the call returns.  EINVAL if n_obs >
 * max_obstacles, a radius is negative, a centre is not finite, or a disc
 * leaves the square of side 2 RA_MPPI_OBSTACLE_EXTENT around the origin.
 * The library keeps them sorted by x (the obstacle cull narrows to an x
 * window); the costs do not depend on the order, except for the rounding of
 * the softplus barrier's sum. */
int ra_mppi_set_obstacles(ra_mppi_t* h, const float* xyr, int32_t n_obs, void* stream);

/* One RA-MPPI update on device buffers (steps 1-6 above).
 *   x0      [nx]      device, current state x(0)
 *   V_in    [T][nu]   device, mean control sequence V
 *   V_out   [T][nu]   device, receives V+ (may alias V_in)
 *   S_tilde [K]       device, optional (NULL): receives S~_k
 *   cvar    [K]       device, optional (NULL): receives CVaR_k
 * Enqueues two kernels on `stream`; advances the iteration counter. */
int ra_mppi_step(ra_mppi_t* h, const float* x0, const float* V_in, float* V_out, float* S_tilde,
                 float* cvar, void* stream);

/* The same update on HOST buffers: copies x0 and V_in to the device, runs
 * ra_mppi_step, copies V+ (and S_tilde if non-NULL) back and waits for
 * `stream`.  This is the end-to-end call of a controller loop (the paper
 * keeps everything but the state and the command on the GPU, Sec. V-C). */
int ra_mppi_step_host(ra_mppi_t* h, const float* x0_host, const float* V_in_host, float* V_out_host,
                      float* S_tilde_host, void* stream);

/* One pass of Algorithm 1's receding-horizon loop on a simulated plant:
 * the state estimate is the plant state x, one update (ra_mppi_step) gives
 * V+, the first control v0+ is executed on the plant
 * x <- F(x, v0+) + w (Eqs. 1, 6; the plant's noise has its own Philox
 * stream, counter (draw << 16, 0xFFFFFFFE, 0xFFFFFFFF, instance) at the
 * update's iteration), and V is warm-started from V+ ("V = V+", Alg. 1),
 * shifted left by one step with the last control repeated when shift != 0.
 *   x          [nx]     device, in: plant state; out: next plant state
 *   V          [T][nu]  device, in: mean controls; out: next warm start
 *   S_tilde    [K]      device or NULL: receives the update's S~_k
 *   collisions [2]      device int32 or NULL: [0] incremented when the new
 *                       plant state lies inside an obstacle (Eq. 22 with
 *                       d < r), [1] when it is off the track (|e| > half width)
 * Enqueued on `stream` (three kernels), no synchronisation. */
int ra_mppi_closed_loop_step(ra_mppi_t* h, float* x, float* V, float* S_tilde, int32_t* collisions,
                             int32_t shift, void* stream);

/* Device views of the last update's workspace, valid until destroy:
 *   U [K][T][nu] sampled (clipped) controls, S [K] nominal costs (Eq. 3),
 *   cvar [K] CVaR values, L [K][M] risk costs (NULL unless the problem had
 *   RA_MPPI_KEEP_RISK_COSTS).  Any output pointer may be NULL. */
int ra_mppi_workspace(ra_mppi_t* h, const float** U, const float** S, const float** cvar,
                      const float** L);

/* Copy the last update's workspace into caller buffers (host or device,
 * any may be NULL): U [K][T][nu], S [K], cvar [K], L [K][M] (EINVAL if L is
 * requested without RA_MPPI_KEEP_RISK_COSTS).  Enqueued on `stream`. */
int ra_mppi_copy_workspace(ra_mppi_t* h, float* U, float* S, float* cvar, float* L, void* stream);

/* Copy the last update's importance weights W [K][M] (the deterministic-
 * mixture weight of every disturbed rollout; see is_scale) into a caller
 * buffer (host or device).  EINVAL unless the problem had
 * RA_MPPI_KEEP_RISK_COSTS and importance sampling on.  Enqueued on `stream`. */
int ra_mppi_copy_weights(ra_mppi_t* h, float* W, void* stream);

/* The handle's resumable state: the update counter that keys the noise
 * (Alg. 1 redraws the samples at every update; the counter makes update n
 * reproducible).  A handle restored with set_state reproduces the updates
 * that followed get_state exactly.  get waits for the device. */
int ra_mppi_get_state(ra_mppi_t* h, uint64_t* iteration);
int ra_mppi_set_state(ra_mppi_t* h, uint64_t iteration);

/* Device status word accumulated since the last call, then cleared: OK,
 * or ENONFINITE when a cost was NaN/inf or every weight vanished.  Waits
 * for the device. */
int ra_mppi_get_status(ra_mppi_t* h);

/* Human-readable reason of the last error on this handle ("" if none). */
const char* ra_mppi_last_error(const ra_mppi_t* h);

/* Launch-shape tuner: times every valid (warps per block in {1..6, 8},
 * interleave in {1, 2, 4}, warps per sample dividing the block) shape that
 * gives each warp at least one full set of interleaved rows (or, dynamic
 * model with M <= 32, interleave 2 and one warp per sample: two samples per
 * warp, stepped as pairs), on the given
 * inputs (x0, V device; `replays` updates each), keeps the fastest and
 * restores the update counter, so later results are unchanged (they never
 * depend on the shape).  Synchronous. */
int ra_mppi_tune(ra_mppi_t* h, const float* x0, const float* V, int32_t replays, float* best_ms);
int ra_mppi_get_launch(ra_mppi_t* h, int32_t* warps_per_block, int32_t* ilp, int32_t* warps_per_sample);

/* Cost weights theta = (w_dev, w_speed, gamma, w_obs) used by the following
 * updates (host-side, no device work).  EINVAL if any is not finite. */
int ra_mppi_set_cost_weights(ra_mppi_t* h, const float* theta);

/* Vector-Jacobian product of the most recent ra_mppi_step of this handle.
 * For the update's fixed noise, (V+, S~) is a function of the mean
 * controls V and of theta; this computes
 *   gV     [T][nu] device = d(<gV_plus, V+> + <gS_tilde, S~>) / dV
 *   gtheta [4]     device = the same derivative w.r.t. theta
 * from gV_plus [T][nu] (device) and gS_tilde [K] (device, or NULL for 0):
 * the derivative of the softmin update (Eqs. 4, 5, 17), of the violation
 * cost (Eqs. 14-16: A where CVaR > C_u, else 0), of the fractional-tail or
 * literal CVaR (Eqs. 10-13: the tail weights, times the importance weights
 * when importance sampling is on; Eqs. 18, 19: the scaling), of
 * the costs and dynamics along every nominal and disturbed rollout (Eqs. 3,
 * 6, 9, 20-23; the risk costs kept by the update, states recomputed from
 * checkpoints every 8 steps), and of the
 * clip U = clip(V + eps) (Alg. 1).  The obstacle indicator (Eq. 22) has
 * zero derivative; use the softplus barrier to differentiate through
 * obstacles.  Needs RA_MPPI_DIFFERENTIABLE; all three models (the dynamic
 * one through its Heun sub-steps).  FP32; the sums over samples accumulate
 * in FP64 (partials over slices of samples stored as FP32) in an order fixed
 * by K, so repeated calls give the same bits; the barrier's slope uses the
 * hardware exponential and logarithm.  Enqueued on `stream`. */
int ra_mppi_backward(ra_mppi_t* h, const float* gV_plus, const float* gS_tilde, float* gV, float* gtheta,
                     void* stream);

/* Kernel launch tuning: disturbed-rollout warps per block (1..8), rollouts
 * each lane interleaves (1, 2 or 4) and warps sharing one sample's M
 * rollouts (1..8, dividing warps_per_block); 0 keeps the current value.
 * Dynamic model, M <= 32, interleave 2 and one warp per sample: each warp
 * takes two samples (the default there).  Results never depend on the shape. */
int ra_mppi_set_launch(ra_mppi_t* h, int32_t warps_per_block, int32_t ilp, int32_t warps_per_sample);

/* Tail split of the rollout launch (on by default; the tuner keeps it only
 * where it is faster): when the grid's last round of disturbed blocks would
 * fill at most half of the GPU's resident-block slots, the samples of that
 * round take twice the warps per sample (half the rows each), so the last
 * round is made of more, shorter blocks.  Results never depend on it. */
int ra_mppi_set_tail_split(ra_mppi_t* h, int32_t enable);
/* The rollout launch ra_mppi_step makes at the current shape: its grid,
 * the first disturbed block of the tail split (-1 without one), the tail's
 * warps per sample and the resident blocks per SM.  Any output may be NULL. */
int ra_mppi_get_launch_plan(ra_mppi_t* h, int32_t* grid, int32_t* nb_head, int32_t* wps_tail, int32_t* blocks_per_sm);

/* Diagnostics: when `candidates` (device uint64) is set, the disturbed
 * rollouts add to it, per step and per row of 32 rollouts, the number of
 * obstacles tested exactly after the warp's bounding-box cull (the work the
 * indicator term actually does; divided by K ceil(M/32) T it is the mean
 * per rollout-step).  NULL turns it off. */
int ra_mppi_set_diagnostics(ra_mppi_t* h, unsigned long long* candidates);

/* Timing hook: when set, ra_mppi_step records the caller's CUDA events
 * (cudaEvent_t passed as void*) immediately before and after the fused
 * rollout kernel on the step's stream, and ra_mppi_backward before and after
 * its main (reverse-sweep) kernel, so the caller can time that kernel alone.
 * NULL, NULL turns the hook off. */
int ra_mppi_set_timing_events(ra_mppi_t* h, void* rollout_begin, void* rollout_end);

/* Pipe-throughput probe for the roofline of the rollout kernel (no
 * counterpart in the paper; a measurement aid).  Runs one probe kernel of
 * `iters` iterations of eight independent chains per thread, on 4 blocks of
 * 256 threads per SM of `device` (-1: current), of one instruction kind:
 *   0 FP32 fused multiply-add     1 paired FP32 multiply-add (2 ops each)
 *   2 rsqrt.approx  3 cos.approx  4 ex2.approx  5 lg2.approx  6 sin.approx
 *                                 (one special-function unit operation each)
 *   7 32-bit integer to float conversion   8 32-bit integer multiply-add
 * and returns its CUDA-event time *ms and the lane-operations it executed
 * (*lane_ops), so that ops / (ms x SM clock x SMs) is the pipe's rate per SM
 * per clock.  Synchronous; allocates a stream and two events. */
int ra_mppi_pipe_probe(int32_t kind, int32_t iters, int32_t device, float* ms, double* lane_ops);

/* ------------------------------------------------------------------ */
/* Batched updates: B independent problems in one persistent launch    */
/* replayed from a CUDA graph.  The paper updates one controller; this  */
/* runs many (different K, M, T, seed and obstacles, common model, cost */
/* and risk parameters) at once, each with exactly the single-problem   */
/* arithmetic.                                                          */
/* ------------------------------------------------------------------ */
typedef struct ra_mppi_instance {
  int32_t K, M, T;          /* sizes of this problem (as in ra_mppi_problem) */
  int32_t max_obstacles;    /* obstacle capacity of this problem            */
  uint64_t seed;            /* Philox key of this problem                   */
  uint32_t instance_id;     /* fourth Philox counter word                   */
  int32_t reserved;
} ra_mppi_instance;

typedef struct ra_mppi_batch ra_mppi_batch_t;

/* Validate every problem (common fields + inst[i]) as ra_mppi_create would,
 * allocate packed buffers on CUDA device `device` (-1: the current device;
 * later calls run there, as for single handles), order the work items
 * (nominal items first, then the disturbed samples of the costliest
 * problems first) and capture the graph (queue reset, persistent rollout
 * kernel, batched update kernel).  Each problem is one RA-MPPI update
 * (Alg. 1); the batch has no counterpart in the paper. */
int ra_mppi_batch_create(const ra_mppi_problem* common, const ra_mppi_instance* inst, int32_t B, int32_t device,
                         ra_mppi_batch_t** out);
void ra_mppi_batch_destroy(ra_mppi_batch_t* b);

/* Offsets of problem i in the packed buffers, offsets[4 i + 0..3] =
 * (x0, V / V_out, per-sample arrays, U), counted in floats except the
 * per-sample offset, counted in samples. */
int ra_mppi_batch_layout(ra_mppi_batch_t* b, int64_t* offsets);

/* Library-owned packed device buffers, stable for the handle's life (the
 * graph reads and writes them): x0 [sum nx], V [sum T_i nu] (input mean
 * controls), V_out [sum T_i nu] (V+), S_tilde [sum K_i]. */
int ra_mppi_batch_buffers(ra_mppi_batch_t* b, float** x0, float** V, float** V_out, float** S_tilde);

/* The batch's packed inputs, owned by the library and stable for the
 * handle's life, so a captured graph and the caller both address them:
 *   x0_packed  receives the device buffer of the states x(0) (Alg. 1's state
 *              estimate) [sum nx], problem i at offsets[4 i + 0];
 *   V_packed   receives the device buffer of the mean controls V [sum T_i nu],
 *              problem i at offsets[4 i + 1] (its V+ is at the same offset
 *              of ra_mppi_batch_buffers' V_out);
 *   offsets    [4 B] int64 or NULL: as ra_mppi_batch_layout.
 * Any output may be NULL. */
int ra_mppi_batch_io(ra_mppi_batch_t* b, float** x0_packed, float** V_packed, int64_t* offsets);

/* Copy packed inputs in (x0 [sum nx], V [sum T_i nu]) and outputs out
 * (V_out [sum T_i nu], S_tilde [sum K_i]) between caller buffers (host or
 * device; NULL skips one) and the library's buffers, on `stream`. */
int ra_mppi_batch_write_inputs(ra_mppi_batch_t* b, const float* x0, const float* V, void* stream);
int ra_mppi_batch_read_outputs(ra_mppi_batch_t* b, float* V_out, float* S_tilde, void* stream);

/* Obstacles of problem i, as ra_mppi_set_obstacles (synchronous). */
int ra_mppi_batch_set_obstacles(ra_mppi_batch_t* b, int32_t i, const float* xyr, int32_t n_obs, void* stream);

/* Timing hook and diagnostics of the batched path, as ra_mppi_set_timing_events
 * and ra_mppi_set_diagnostics: the events are recorded around the persistent
 * rollout kernel by ra_mppi_step_batched_eager (the captured graph holds no
 * events); the counter takes the obstacles tested exactly after the cull, by
 * the eager launches and by the graph captured after the call (the call
 * recaptures it).  NULL turns either off. */
int ra_mppi_batch_set_timing_events(ra_mppi_batch_t* b, void* rollout_begin, void* rollout_end);
int ra_mppi_batch_set_diagnostics(ra_mppi_batch_t* b, unsigned long long* candidates);

/* One update of every problem: replay of the captured graph on `stream`. */
int ra_mppi_step_batched(ra_mppi_batch_t* b, void* stream);
/* The same kernels launched directly (no graph), for comparison. */
int ra_mppi_step_batched_eager(ra_mppi_batch_t* b, void* stream);

/* Packed copies of the last update's U, S and CVaR (any may be NULL). */
int ra_mppi_batch_copy_workspace(ra_mppi_batch_t* b, float* U, float* S, float* cvar, void* stream);

/* Update counter of every problem; status word of all problems (waits). */
int ra_mppi_batch_set_iteration(ra_mppi_batch_t* b, uint64_t iteration);
int ra_mppi_batch_get_status(ra_mppi_batch_t* b);

/* Launch shape of the persistent kernel (warps per block 1..8, rollouts a
 * lane interleaves 1 or 2; the grid fills every SM to its occupancy).  tune
 * times the candidate shapes on the current inputs (`replays` graph replays
 * each), keeps the fastest, recaptures the graph and restores the update
 * counters; results do not depend on the shape. */
int ra_mppi_batch_set_launch(ra_mppi_batch_t* b, int32_t warps_per_block, int32_t ilp);
int ra_mppi_batch_get_launch(ra_mppi_batch_t* b, int32_t* warps_per_block, int32_t* ilp, int32_t* grid);
int ra_mppi_batch_tune(ra_mppi_batch_t* b, int32_t replays, float* best_ms);
const char* ra_mppi_batch_last_error(const ra_mppi_batch_t* b);

/* Allocation-free softmin-weighted update.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * where they run the update, such as a controller on a real-time thread that
 * may not call cudaMalloc/cudaFree (they can block and synchronise the
 * device), or a host program that owns all device memory through its own
 * pool and hands the library only pointers.  It computes step 6 above on
 * caller-supplied inputs:
 *   S_tilde [K]        device, costs S~_k (non-finite entries get weight 0)
 *   U       [K][T][nu] device, sampled controls
 *   V_out   [T][nu]    device, receives V+ = sum_k w_k U^k / sum_k w_k,
 *                      w_k = exp(-(S~_k - min S~) / lambda); left unchanged
 *                      when no S~_k is finite
 * Limits: 1 <= K <= 2^24, 1 <= T nu <= RA_MPPI_NOALLOC_MAX_COLS, lambda > 0
 * and finite; anything else returns RA_MPPI_EINVAL before any work is
 * enqueued.  The call allocates nothing: its per-block partials and arrival
 * counter live in one fixed device array of about 130 KB, which every GPU
 * that loads this library keeps until the process exits; the counter is
 * cleared with cudaMemsetAsync before each launch.  The first call on a
 * device looks up that array's device address with the device current;
 * make this first call before any stream capture.  The address is kept for
 * the life of the device's context: do not call this entry point after
 * cudaDeviceReset in the same process.  `stream` must belong to the current
 * device (EINVAL otherwise).  All calls share the array and it keeps the
 * last call's contents: calls that overlap on the GPU (different streams,
 * or threads without ordering between them) race; calls ordered on one
 * stream do not. */
#define RA_MPPI_NOALLOC_MAX_COLS 512
int ra_mppi_softmin_update_noalloc(const float* S_tilde, const float* U, int32_t K, int32_t T, int32_t nu,
                                   float lambda, float* V_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RA_MPPI_H */
