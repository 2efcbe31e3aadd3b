/*
 * FP64 CPU oracle of one Risk-Aware MPPI (RA-MPPI) control update.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path; it is a plain,
 * slow, obviously-correct restatement of the method for checking it.
 *
 * What it computes (RA-MPPI, Yin, Zhang, Tsiotras; arXiv 2209.12842):
 *   Algorithm 1, one pass of the while-loop body:
 *     - sample K control sequences U^k = V + eps^k (or eps^k for the last
 *       eta fraction), eps ~ N(0, Sigma)                      (Sec. II, Alg. 1)
 *     - roll out each one on the nominal dynamics F (Eq. 1) and form
 *       S_k = phi(x_T) + sum_t q(x_t) + gamma v_t' Sigma^-1 u_t      (Eq. 3)
 *     - roll out M disturbed trajectories per sample on
 *       x~_{t+1} = F(x~_t, u_t) + w_t and form L = sum_t l(x~_t)  (Eqs. 6, 9)
 *     - scale the risk costs L_a = B (L - mean) + mean        (Eqs. 18, 19)
 *     - CVaR_alpha of the M scaled costs                     (Eqs. 10-13)
 *     - S~_k = S_k + A CVaR 1{CVaR > C_u}                    (Eqs. 14-16)
 *   then the softmin-weighted update
 *     w_k = exp(-(S~_k - min S~)/lambda), V+ = sum w U / sum w (Eqs. 4, 5, 17)
 *
 * Letters follow the implementation: K samples (the paper's M), M disturbed
 * rollouts per sample (the paper's N), T horizon steps (the paper's K).
 *
 * Readings of points the paper leaves open (each is listed with its reason
 * in the design notes):
 *   - CVaR estimator: the fractional sorted-tail (Rockafellar-Uryasev) form
 *       CVaR = [(j - alpha M) L_(j) + sum_{i>j} L_(i)] / ((1 - alpha) M),
 *     j = ceil(alpha M), is the default; the literal tail mean over
 *     {L >= VaR} (Eqs. 12, 13) is the alternative mode.  VaR = L_(j) (Eq. 11)
 *   - the mean in Eq. 19 divides by M (the text calls it the mean)
 *   - q and l are charged on x_0 .. x_{T-1}; phi on x_T
 *   - controls are clipped to the box after the noise is added
 *   - the control-cost weight uses 1/sigma^2 and is 0 where sigma = 0
 *   - importance sampling of the process noise (the paper leaves it out,
 *     Sec. III-A, pointing to importance sampling for alpha near 1): the
 *     deterministic-mixture form with a scaled proposal, see orc_is_weights
 *   - the random numbers come from Philox4x32-10 (Salmon, Moraes, Dror,
 *     Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11), keyed by
 *     (seed, iteration) with counter (t | draw << 16, m, k, instance);
 *     m = 0xFFFFFFFF marks control noise, (m, k) = (0xFFFFFFFE, 0xFFFFFFFF)
 *     the simulated plant's noise
 *
 * Parity status: every function below is pinned by the CPU tests against
 * closed forms, invariants, brute force or an independent library routine;
 * none is unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

enum { ORC_KIN = 0, ORC_DYN = 1, ORC_LIN = 2 };
enum { ORC_GAUSS = 0, ORC_LAPLACE_MIX = 1, ORC_UNIFORM = 2, ORC_IMPULSE = 3 };
enum { ORC_OBS_INDICATOR = 0, ORC_OBS_SOFTPLUS = 1 };
enum { ORC_CVAR_RU = 0, ORC_CVAR_TCE = 1, ORC_VAR = 2, ORC_CHANCE = 3, ORC_MEAN = 4, ORC_MEANVAR = 5 };
enum { ORC_R_DEV = 1, ORC_R_SPEED = 2, ORC_R_OBS = 4, ORC_R_BDRY = 8, ORC_R_LIN = 16 };

typedef struct {
  int32_t model, K, M, T, substeps;
  int32_t noise_type, obs_mode, cvar_mode;
  uint32_t risk_mask;
  int32_t n_threads;
  double dt;
  double model_params[8];
  double sigma_u[2], u_lo[2], u_hi[2];
  double w_scale[4];
  double mix_p, mix_scale;
  double w_dev, w_speed, v_target, gamma, w_obs, w_bdry, c4, c5, c_lin;
  double kappa;
  double track_straight, track_radius, track_half_width;
  double lam, alpha, A, B, C_u, eta;
  double band_delta;
  double risk_param;
  uint64_t seed;
  uint64_t iteration;
  uint32_t instance_id;
  uint32_t pad_;
  double is_scale; /* proposal scale s >= 1 of the importance-sampled rollouts */
  double is_frac;  /* fraction of the M rollouts drawn from the proposal, in [0, 1) */
} orc_problem;

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11): 10 rounds of the 4x32 Philox S-box with the   */
/* multipliers 0xD2511F53, 0xCD9E8D57 and the Weyl key increments       */
/* 0x9E3779B9, 0xBB67AE85.                                               */
/* ------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void make_key(const orc_problem* p, uint64_t iteration, uint32_t key[2]) {
  key[0] = (uint32_t)(p->seed & 0xFFFFFFFFu);
  key[1] = (uint32_t)(p->seed >> 32) ^ (uint32_t)(iteration & 0xFFFFFFFFu);
}

/* uniform in (0, 1): (x + 1/2) 2^-32, exact in double */
double orc_uniform(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

/* Box-Muller: two independent standard normals from two words */
void orc_box_muller(uint32_t a, uint32_t b, double out[2]) {
  double u1 = orc_uniform(a), u2 = orc_uniform(b);
  double rad = sqrt(-2.0 * log(u1));
  out[0] = rad * cos(2.0 * ORC_PI * u2);
  out[1] = rad * sin(2.0 * ORC_PI * u2);
}

/* Heavy-tailed slot value (Eq. 6 with the mixture noise of the workload):
 * Laplace(0, b) by its inverse CDF, replaced with probability p by
 * N(0, (mix_scale b)^2).  The value word gives the tail mass
 * v = 2 min(a, 1 - a) of a = (x + 1/2) 2^-32 and the sign of a - 1/2; the
 * Gaussian branch is taken when the selector word is below floor(p 2^32). */
static double mix_value_branch(uint32_t sel, uint32_t word, double b, double p, double mix_scale, int* gauss) {
  uint32_t hi = word >> 31;
  uint32_t r = hi ? ~word : word;                 /* in [0, 2^31) */
  double v = ((double)r + 0.5) * (1.0 / 2147483648.0);
  double sgn = hi ? 1.0 : -1.0;
  double thresh = floor(p * 4294967296.0 > 4294967295.0 ? 4294967295.0 : p * 4294967296.0);
  *gauss = (double)sel < thresh;
  if (*gauss) {
    /* Gaussian branch: Box-Muller with radius from v and angle from the
     * selector, uniform on [0, thresh) given this branch */
    double u2 = ((double)sel + 0.5) / thresh;
    return sgn * (mix_scale * b) * sqrt(-2.0 * log(v)) * cos(2.0 * ORC_PI * u2);
  }
  return sgn * (-b * log(v));
}

double orc_mix_value(uint32_t sel, uint32_t word, double b, double p, double mix_scale) {
  int gauss;
  return mix_value_branch(sel, word, b, p, mix_scale, &gauss);
}

/* log densities of one noise value */
static double log_gauss(double w, double sd) { return -log(sd) - 0.5 * log(2.0 * ORC_PI) - w * w / (2.0 * sd * sd); }
static double log_laplace(double w, double b) { return -log(2.0 * b) - fabs(w) / b; }

static int nx_of(int model) { return model == ORC_KIN ? 4 : model == ORC_DYN ? 6 : 1; }
static int nu_of(int model) { return model == ORC_LIN ? 1 : 2; }
static int nslots_of(int model) { return model == ORC_KIN ? 4 : model == ORC_DYN ? 3 : 1; }
/* which state component noise slot s perturbs */
static int slot_dim(int model, int s) { return model == ORC_DYN ? 3 + s : s; }

/* control noise eps^k_t (Alg. 1: "Sample eps^m"), Sigma = diag(sigma_u^2) */
void orc_control_noise(const orc_problem* p, int32_t k, int32_t t, double eps[2]) {
  uint32_t key[2], ctr[4], w[4];
  make_key(p, p->iteration, key);
  ctr[0] = (uint32_t)t; ctr[1] = 0xFFFFFFFFu; ctr[2] = (uint32_t)k; ctr[3] = p->instance_id;
  orc_philox(ctr, key, w);
  double z[2];
  orc_box_muller(w[0], w[1], z);
  eps[0] = p->sigma_u[0] * z[0];
  eps[1] = p->sigma_u[1] * z[1];
}

/* process noise w_t added to the state (Eq. 6 with F~ = F + w, so Eq. 7 holds) */
static void noise_words(const orc_problem* p, uint64_t iteration, uint32_t c1, uint32_t c2,
                        int32_t t, uint32_t draw, uint32_t w[4]) {
  uint32_t key[2], ctr[4];
  make_key(p, iteration, key);
  ctr[0] = (uint32_t)t | (draw << 16); ctr[1] = c1; ctr[2] = c2; ctr[3] = p->instance_id;
  orc_philox(ctr, key, w);
}

/* the process noise of step t, each value multiplied by g (1, or the
 * proposal scale s for an importance-sampled rollout).  With log_ratio
 * non-NULL (Gaussian and mixture noise only) it adds, for every value w
 * drawn, ln q(w) - ln p(w): p the value's nominal density, q(w) = p(w/s)/s
 * the proposal's (for the mixture, the densities given the branch drawn,
 * whose probabilities the proposal keeps) */
static void process_noise_at(const orc_problem* p, uint64_t iteration, uint32_t c1, uint32_t c2,
                             int32_t t, double g, double* log_ratio, double out[4]) {
  int ns = nslots_of(p->model);
  for (int s = 0; s < 4; ++s) out[s] = 0.0;
  if (p->noise_type == ORC_GAUSS) {
    uint32_t w[4];
    noise_words(p, iteration, c1, c2, t, 0, w);
    double z[4];
    orc_box_muller(w[0], w[1], z);
    orc_box_muller(w[2], w[3], z + 2);
    for (int s = 0; s < ns; ++s) {
      out[s] = g * (p->w_scale[s] * z[s]);
      if (log_ratio && p->w_scale[s] != 0.0)
        *log_ratio += log_gauss(out[s], p->is_scale * p->w_scale[s]) - log_gauss(out[s], p->w_scale[s]);
    }
  } else if (p->noise_type == ORC_LAPLACE_MIX) {
    uint32_t sel[4], val[4];
    noise_words(p, iteration, c1, c2, t, 0, sel);
    noise_words(p, iteration, c1, c2, t, 1, val);
    for (int s = 0; s < ns; ++s) {
      if (p->w_scale[s] == 0.0) {
        out[s] = 0.0;
        continue;
      }
      int gauss;
      out[s] = g * mix_value_branch(sel[s], val[s], p->w_scale[s], p->mix_p, p->mix_scale, &gauss);
      if (log_ratio) {
        if (gauss) {
          const double sd = p->mix_scale * p->w_scale[s];
          *log_ratio += log_gauss(out[s], p->is_scale * sd) - log_gauss(out[s], sd);
        } else {
          *log_ratio += log_laplace(out[s], p->is_scale * p->w_scale[s]) - log_laplace(out[s], p->w_scale[s]);
        }
      }
    }
  } else if (p->noise_type == ORC_UNIFORM) {
    /* w_s ~ U[-a_s, a_s] (the paper's uniform disturbance, Sec. V-B) */
    uint32_t w[4];
    noise_words(p, iteration, c1, c2, t, 0, w);
    for (int s = 0; s < ns; ++s) out[s] = (2.0 * orc_uniform(w[s]) - 1.0) * p->w_scale[s];
  } else {
    /* impulse (Sec. V-B): with probability p a jump of per-slot size a_s
     * along a direction uniform on the unit sphere of the slots with
     * a_s != 0 (a normalised Gaussian vector), otherwise no disturbance */
    uint32_t a[4], b[4];
    noise_words(p, iteration, c1, c2, t, 0, a);
    noise_words(p, iteration, c1, c2, t, 1, b);
    double thr = floor(p->mix_p * 4294967296.0 > 4294967295.0 ? 4294967295.0 : p->mix_p * 4294967296.0);
    if ((double)a[0] < thr) {
      double z[4];
      orc_box_muller(a[1], a[2], z);
      orc_box_muller(a[3], b[0], z + 2);
      double n2 = 0.0;
      for (int s = 0; s < ns; ++s)
        if (p->w_scale[s] != 0.0) n2 += z[s] * z[s];
      double inv = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
      for (int s = 0; s < ns; ++s) out[s] = p->w_scale[s] != 0.0 ? p->w_scale[s] * z[s] * inv : 0.0;
    }
  }
}

void orc_process_noise(const orc_problem* p, int32_t k, int32_t m, int32_t t, double out[4]) {
  process_noise_at(p, p->iteration, (uint32_t)m, (uint32_t)k, t, 1.0, NULL, out);
}

/* ------------------------------------------------------------------ */
/* Importance-sampled rollouts (the paper leaves importance sampling out,  */
/* Sec. III-A, naming it as the remedy when alpha is near 1).  The last    */
/* M_s = floor(is_frac M) rollouts of every sample draw each process-noise */
/* value at is_scale times its nominal size; the others are unchanged.     */
/* With b = M_s / M, rollout m's noise path W_m gets the balance-heuristic */
/* (deterministic-mixture) weight                                          */
/*   w_m = p(W_m) / ((1 - b) p(W_m) + b q(W_m)) = 1 / ((1 - b) + b e^G_m), */
/* G_m = ln q(W_m) - ln p(W_m) summed over the path's values, so that      */
/* sum_m w_m f(W_m) / M is an unbiased estimate of E_p f.  The risk        */
/* measures are then those of the weighted empirical distribution of the   */
/* risk costs.  Off (all weights 1) when M_s = 0 or is_scale = 1.          */
/* ------------------------------------------------------------------ */
static int is_count(const orc_problem* p) {
  if (p->is_scale == 1.0 || p->is_frac <= 0.0) return 0;
  return (int)floor(p->is_frac * (double)p->M);
}

/* proposal factor of rollout m: s for the last M_s rollouts, else 1 */
static double is_factor(const orc_problem* p, int m, int M_s) {
  return m >= p->M - M_s ? p->is_scale : 1.0;
}

static double is_weight(const orc_problem* p, int M_s, double log_ratio) {
  const double b = (double)M_s / (double)p->M;
  return 1.0 / ((1.0 - b) + b * exp(log_ratio));
}

/* the M weights of sample k (noise only: no dynamics); all 1 when off.
 * Returns -6 for noise types without a density ratio (uniform, impulse). */
int32_t orc_is_weights(const orc_problem* p, int32_t k, double* w) {
  const int M_s = is_count(p);
  if (M_s > 0 && p->noise_type != ORC_GAUSS && p->noise_type != ORC_LAPLACE_MIX) return -6;
  for (int m = 0; m < p->M; ++m) {
    if (M_s == 0) {
      w[m] = 1.0;
      continue;
    }
    double G = 0.0, out[4];
    for (int t = 0; t < p->T; ++t)
      process_noise_at(p, p->iteration, (uint32_t)m, (uint32_t)k, t, is_factor(p, m, M_s), &G, out);
    w[m] = is_weight(p, M_s, G);
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Dynamics F (Eq. 1)                                                   */
/* ------------------------------------------------------------------ */
static void dyn_deriv(const double* mp, const double* x, const double* u, double* f) {
  const double m = mp[0], Iz = mp[1], lf = mp[2], lr = mp[3];
  const double Bt = mp[4], Ct = mp[5], Dt = mp[6], vfloor = mp[7];
  const double g = 9.81;
  double psi = x[2], vx = x[3], vy = x[4], r = x[5];
  double delta = u[0], a = u[1];
  double Fzf = m * g * lr / (lf + lr);
  double Fzr = m * g * lf / (lf + lr);
  double vxs = vx > vfloor ? vx : vfloor;
  double alpha_f = delta - atan2(vy + lf * r, vxs);
  double alpha_r = -atan2(vy - lr * r, vxs);
  double Fyf = Dt * Fzf * sin(Ct * atan(Bt * alpha_f));
  double Fyr = Dt * Fzr * sin(Ct * atan(Bt * alpha_r));
  f[0] = vx * cos(psi) - vy * sin(psi);
  f[1] = vx * sin(psi) + vy * cos(psi);
  f[2] = r;
  f[3] = a - Fyf * sin(delta) / m + r * vy;
  f[4] = (Fyf * cos(delta) + Fyr) / m - r * vx;
  f[5] = (lf * Fyf * cos(delta) - lr * Fyr) / Iz;
}

/* one control period of F: `substeps` explicit-Euler (kinematic, linear) or
 * Heun/RK2 (dynamic) steps of dt / substeps */
void orc_dynamics(const orc_problem* p, const double* x, const double* u, double* xn) {
  int nx = nx_of(p->model);
  double s[6];
  for (int i = 0; i < nx; ++i) s[i] = x[i];
  int n = p->substeps > 0 ? p->substeps : 1;
  double h = p->dt / n;
  for (int it = 0; it < n; ++it) {
    if (p->model == ORC_KIN) {
      double L = p->model_params[0];
      double px = s[0], py = s[1], psi = s[2], v = s[3];
      s[0] = px + h * v * cos(psi);
      s[1] = py + h * v * sin(psi);
      s[2] = psi + h * v * tan(u[0]) / L;
      s[3] = v + h * u[1];
    } else if (p->model == ORC_DYN) {
      double k1[6], k2[6], xp[6];
      dyn_deriv(p->model_params, s, u, k1);
      for (int i = 0; i < 6; ++i) xp[i] = s[i] + h * k1[i];
      dyn_deriv(p->model_params, xp, u, k2);
      for (int i = 0; i < 6; ++i) s[i] = s[i] + 0.5 * h * (k1[i] + k2[i]);
    } else {
      s[0] = s[0] + h * u[0];
    }
  }
  for (int i = 0; i < nx; ++i) xn[i] = s[i];
}

/* ------------------------------------------------------------------ */
/* Track geometry (stadium): e lateral deviation (outward +), s arc     */
/* length counter-clockwise from (0, -R), d distance to the boundary.   */
/* ------------------------------------------------------------------ */
void orc_track(const orc_problem* p, double px, double py, double out[3]) {
  double S = p->track_straight, R = p->track_radius, hw = p->track_half_width;
  double half = 0.5 * S;
  double total = 2.0 * S + 2.0 * ORC_PI * R;
  double e, s;
  if (fabs(px) <= half) {
    if (py < 0.0) {
      e = -py - R;
      s = px >= 0.0 ? px : total + px;
    } else {
      e = py - R;
      s = half + ORC_PI * R + (half - px);
    }
  } else if (px > half) {
    double dx = px - half;
    e = sqrt(dx * dx + py * py) - R;
    s = half + R * (atan2(py, dx) + 0.5 * ORC_PI);
  } else {
    double dx = px + half;
    e = sqrt(dx * dx + py * py) - R;
    double th = atan2(py, dx);
    double phi = th > 0.0 ? th - 0.5 * ORC_PI : th + 1.5 * ORC_PI;
    s = half + ORC_PI * R + S + R * phi;
  }
  out[0] = e;
  out[1] = s;
  out[2] = hw - fabs(e);
}

/* ------------------------------------------------------------------ */
/* Running cost q (Eq. 20) and risk cost l (Eq. 9)                     */
/* ------------------------------------------------------------------ */
/* obstacle term: sum_i 1{d_i < r_i + shift} (Eq. 22) or the softplus
 * barrier sum_i softplus(kappa (r_i - d_i)) / kappa */
static double obstacle_term(const orc_problem* p, const double* x, const double* obs, int n_obs,
                            double shift) {
  double acc = 0.0;
  for (int i = 0; i < n_obs; ++i) {
    double dx = x[0] - obs[3 * i + 0], dy = x[1] - obs[3 * i + 1];
    double d = sqrt(dx * dx + dy * dy);
    double r = obs[3 * i + 2];
    if (p->obs_mode == ORC_OBS_INDICATOR) {
      if (d < r + shift) acc += 1.0;
    } else {
      double z = p->kappa * (r - d);
      double sp = z > 0.0 ? z + log1p(exp(-z)) : log1p(exp(z));
      acc += sp / p->kappa;
    }
  }
  return acc;
}

/* cost of state x with the terms in `mask`; `shift` moves the obstacle
 * indicator threshold (0 for the exact cost, -/+ delta for band bounds) */
static double state_cost(const orc_problem* p, const double* x, const double* obs, int n_obs,
                         uint32_t mask, double shift) {
  double c = 0.0;
  if (p->model == ORC_LIN) {
    if (mask & ORC_R_LIN) c += p->c_lin * x[0];
    return c;
  }
  double tr[3];
  orc_track(p, x[0], x[1], tr);
  if (mask & ORC_R_DEV) c += p->w_dev * tr[0] * tr[0];
  if (mask & ORC_R_SPEED) c += p->w_speed * (x[3] - p->v_target) * (x[3] - p->v_target);
  if (mask & ORC_R_OBS) c += p->w_obs * obstacle_term(p, x, obs, n_obs, shift);
  if (mask & ORC_R_BDRY) {
    double b = atan(-100.0 * tr[2]) / ORC_PI + 0.5;
    c += p->w_bdry * (b > 0.0 ? b : 0.0);
  }
  if (mask & ORC_R_LIN) c += p->c_lin * x[0];
  return c;
}

/* terminal cost phi(x) = c4 - c5 s(x) (Eq. 23) */
static double terminal_cost(const orc_problem* p, const double* x) {
  if (p->model == ORC_LIN) return 0.0;
  double tr[3];
  orc_track(p, x[0], x[1], tr);
  return p->c4 - p->c5 * tr[1];
}

/* ------------------------------------------------------------------ */
/* CVaR of a set of M risk costs: Scal, then Max(., 1 - alpha), then     */
/* Average (Alg. 1; Eqs. 10-13, 18, 19)                                  */
/* ------------------------------------------------------------------ */
static int cmp_double(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return (x > y) - (x < y);
}

/* risk measure of M risk costs after the sensitivity scaling (Eqs. 18, 19):
 * RU / TCE the two CVaR forms (Eqs. 10-13), VAR the quantile L_(j)
 * (Eq. 11), CHANCE the fraction of scaled costs above `thr` (a chance
 * constraint in place of CVaR, Sec. III-A), MEAN the risk-neutral mean,
 * MEANVAR the mean plus `thr` times the population variance (a classical
 * mean-variance measure; the risk block admits such metrics, Sec. III-A) */
double orc_risk(const double* L, int32_t M, double alpha, double B, int32_t mode, double thr);

double orc_cvar(const double* L, int32_t M, double alpha, double B, int32_t mode) {
  return orc_risk(L, M, alpha, B, mode, 0.0);
}

double orc_risk(const double* L, int32_t M, double alpha, double B, int32_t mode, double thr) {
  /* a non-finite risk cost (NaN or inf) ranks as the worst outcome: the
   * sample's CVaR is +inf, so it receives zero weight in the update */
  for (int n = 0; n < M; ++n)
    if (!isfinite(L[n])) return INFINITY;
  double* La = (double*)malloc(sizeof(double) * (size_t)M);
  double mean = 0.0;
  for (int n = 0; n < M; ++n) mean += L[n];
  mean /= (double)M;
  for (int n = 0; n < M; ++n) La[n] = B * (L[n] - mean) + mean;
  qsort(La, (size_t)M, sizeof(double), cmp_double);
  double aM = alpha * (double)M; /* exact for float32 alpha and M < 2^29 */
  int j = (int)ceil(aM);
  if (j < 1) j = 1;
  if (j > M) j = M;
  double var = La[j - 1];
  double out;
  if (mode == ORC_VAR) {
    out = var;
  } else if (mode == ORC_CHANCE || mode == ORC_MEAN) {
    double acc = 0.0;
    for (int n = 0; n < M; ++n) {
      double v = (B == 1.0) ? L[n] : B * (L[n] - mean) + mean; /* Eq. 18 with B = 1 is the identity */
      acc += (mode == ORC_CHANCE) ? (v > thr ? 1.0 : 0.0) : v;
    }
    out = acc / (double)M;
  } else if (mode == ORC_MEANVAR) {
    /* mean + kappa * population variance of the scaled costs */
    double m1 = 0.0;
    for (int n = 0; n < M; ++n) m1 += La[n];
    m1 /= (double)M;
    double m2 = 0.0;
    for (int n = 0; n < M; ++n) m2 += (La[n] - m1) * (La[n] - m1);
    out = m1 + thr * (m2 / (double)M);
  } else if (mode == ORC_CVAR_RU) {
    double tail = ((double)j - aM) * var;
    for (int i = j; i < M; ++i) tail += La[i];
    out = tail / ((1.0 - alpha) * (double)M);
  } else {
    double s = 0.0;
    int c = 0;
    for (int n = 0; n < M; ++n)
      if (La[n] >= var) { s += La[n]; ++c; }
    out = s / (double)c;
  }
  free(La);
  return out;
}

/* Risk measure of M risk costs with positive weights w (NULL: all 1), the
 * measure of the weighted empirical distribution sum_m (w_m / W) at L_m,
 * W = sum w.  The costs are scaled first, La = B (L - mean) + mean with the
 * weighted mean (Eqs. 18, 19).  With tau = (1 - alpha) W:
 *   VAR     the smallest La_m whose strictly larger weight W(La > La_m)
 *           is at most tau (with equal weights: L_(ceil(alpha M)))
 *   RU      VaR + sum_m w_m (La_m - VaR)+ / tau, the Rockafellar-Uryasev
 *           objective c + sum w (La - c)+ / tau at its minimiser c = VaR
 *   TCE     the weighted mean of the La_m >= VaR
 *   CHANCE  the weight fraction of La_m above thr; MEAN the weighted mean;
 *   MEANVAR the weighted mean plus thr times the weighted variance.
 * VaR is found by its definition, one weight sum per candidate (O(M^2)). */
double orc_risk_w(const double* L, const double* w, int32_t M, double alpha, double B, int32_t mode, double thr) {
  if (w == NULL) return orc_risk(L, M, alpha, B, mode, thr);
  for (int n = 0; n < M; ++n)
    if (!isfinite(L[n])) return INFINITY;
  double W = 0.0, mean = 0.0;
  for (int n = 0; n < M; ++n) {
    W += w[n];
    mean += w[n] * L[n];
  }
  mean /= W;
  double* La = (double*)malloc(sizeof(double) * (size_t)M);
  for (int n = 0; n < M; ++n) La[n] = B * (L[n] - mean) + mean;
  const double tau = (1.0 - alpha) * W;
  double var = INFINITY;
  for (int c = 0; c < M; ++c) {
    double above = 0.0;
    for (int n = 0; n < M; ++n)
      if (La[n] > La[c]) above += w[n];
    if (above <= tau && La[c] < var) var = La[c];
  }
  double out;
  if (mode == ORC_VAR) {
    out = var;
  } else if (mode == ORC_CVAR_RU) {
    double tail = 0.0;
    for (int n = 0; n < M; ++n)
      if (La[n] > var) tail += w[n] * (La[n] - var);
    out = var + tail / tau;
  } else if (mode == ORC_CVAR_TCE) {
    double s = 0.0, ws = 0.0;
    for (int n = 0; n < M; ++n)
      if (La[n] >= var) { s += w[n] * La[n]; ws += w[n]; }
    out = s / ws;
  } else if (mode == ORC_CHANCE) {
    double over = 0.0;
    for (int n = 0; n < M; ++n) {
      double v = (B == 1.0) ? L[n] : La[n];
      if (v > thr) over += w[n];
    }
    out = over / W;
  } else if (mode == ORC_MEAN) {
    double acc = 0.0;
    for (int n = 0; n < M; ++n) acc += w[n] * La[n];
    out = acc / W;
  } else {
    double m1 = 0.0;
    for (int n = 0; n < M; ++n) m1 += w[n] * La[n];
    m1 /= W;
    double m2 = 0.0;
    for (int n = 0; n < M; ++n) m2 += w[n] * (La[n] - m1) * (La[n] - m1);
    out = m1 + thr * (m2 / W);
  }
  free(La);
  return out;
}

/* ------------------------------------------------------------------ */
/* Per-sample stage (Alg. 1 loop body for sample k)                     */
/* ------------------------------------------------------------------ */
static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

static int n_warm_of(const orc_problem* p) {
  /* Alg. 1: sample k keeps the mean control when k < (1 - eta) K */
  return (int)ceil((1.0 - p->eta) * (double)p->K);
}

/* Outputs for sample index i of the list ks[] (each may be NULL):
 *   U[i][T][nu], S[i], L[i][M], cvar[i], S_tilde[i], and band bounds of S,
 *   CVaR and S~ obtained with the obstacle indicator threshold at r - delta
 *   (lo) and r + delta (hi) along the same trajectories */
int32_t orc_samples(const orc_problem* p, const double* x0, const double* V, const double* obs,
                    int32_t n_obs, const int32_t* ks, int32_t nk, double* U, double* S, double* L,
                    double* cvar, double* S_tilde, double* S_lo, double* S_hi, double* cvar_lo,
                    double* cvar_hi, double* St_lo, double* St_hi) {
  const int nx = nx_of(p->model), nu = nu_of(p->model), T = p->T, M = p->M;
  const int n_warm = n_warm_of(p);
  const int M_s = is_count(p);
  if (M_s > 0 && p->noise_type != ORC_GAUSS && p->noise_type != ORC_LAPLACE_MIX) return -6;
  double inv_sig2[2];
  for (int j = 0; j < 2; ++j) inv_sig2[j] = p->sigma_u[j] > 0.0 ? 1.0 / (p->sigma_u[j] * p->sigma_u[j]) : 0.0;
  int nthreads = p->n_threads > 0 ? p->n_threads : 1;
  (void)nthreads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
  for (int i = 0; i < nk; ++i) {
    const int k = ks[i];
    double* Uk = (double*)malloc(sizeof(double) * (size_t)T * nu);
    double* Lm = (double*)malloc(sizeof(double) * (size_t)M * 3);
    double* Wm = (double*)malloc(sizeof(double) * (size_t)M);
    /* sample the control sequence */
    for (int t = 0; t < T; ++t) {
      double eps[2];
      orc_control_noise(p, k, t, eps);
      for (int j = 0; j < nu; ++j) {
        double mean_part = (k < n_warm) ? V[t * nu + j] : 0.0;
        Uk[t * nu + j] = clampd(mean_part + eps[j], p->u_lo[j], p->u_hi[j]);
      }
    }
    /* nominal rollout and trajectory cost (Eq. 3) */
    double x[6], xn[6];
    for (int a = 0; a < nx; ++a) x[a] = x0[a];
    double Sk = 0.0, Sk_lo = 0.0, Sk_hi = 0.0;
    for (int t = 0; t < T; ++t) {
      double ctrl = 0.0;
      for (int j = 0; j < nu; ++j) ctrl += V[t * nu + j] * inv_sig2[j] * Uk[t * nu + j];
      ctrl *= p->gamma;
      uint32_t all = 0xFFFFFFFFu;
      Sk += state_cost(p, x, obs, n_obs, all, 0.0) + ctrl;
      Sk_lo += state_cost(p, x, obs, n_obs, all, -p->band_delta) + ctrl;
      Sk_hi += state_cost(p, x, obs, n_obs, all, p->band_delta) + ctrl;
      orc_dynamics(p, x, Uk + t * nu, xn);
      for (int a = 0; a < nx; ++a) x[a] = xn[a];
    }
    double phi = terminal_cost(p, x);
    Sk += phi; Sk_lo += phi; Sk_hi += phi;
    /* disturbed rollouts and their risk costs (Eq. 9); importance weights
     * of the rollouts when some draw from the scaled proposal */
    for (int m = 0; m < M; ++m) {
      double xt[6];
      for (int a = 0; a < nx; ++a) xt[a] = x0[a];
      double Lv = 0.0, Llo = 0.0, Lhi = 0.0, G = 0.0;
      for (int t = 0; t < T; ++t) {
        Lv += state_cost(p, xt, obs, n_obs, p->risk_mask, 0.0);
        Llo += state_cost(p, xt, obs, n_obs, p->risk_mask, -p->band_delta);
        Lhi += state_cost(p, xt, obs, n_obs, p->risk_mask, p->band_delta);
        double w[4];
        process_noise_at(p, p->iteration, (uint32_t)m, (uint32_t)k, t, is_factor(p, m, M_s),
                         M_s > 0 ? &G : NULL, w);
        orc_dynamics(p, xt, Uk + t * nu, xn);
        for (int a = 0; a < nx; ++a) xt[a] = xn[a];
        for (int s = 0; s < nslots_of(p->model); ++s) xt[slot_dim(p->model, s)] += w[s];
      }
      Lm[m] = Lv; Lm[M + m] = Llo; Lm[2 * M + m] = Lhi;
      Wm[m] = M_s > 0 ? is_weight(p, M_s, G) : 1.0;
    }
    const double* wts = M_s > 0 ? Wm : NULL;
    double cv = orc_risk_w(Lm, wts, M, p->alpha, p->B, p->cvar_mode, p->risk_param);
    double cv_lo = orc_risk_w(Lm + M, wts, M, p->alpha, p->B, p->cvar_mode, p->risk_param);
    double cv_hi = orc_risk_w(Lm + 2 * M, wts, M, p->alpha, p->B, p->cvar_mode, p->risk_param);
    /* CVaR violation cost and modified trajectory cost (Eqs. 14-16) */
    double st = Sk + ((cv > p->C_u) ? p->A * cv : 0.0);
    if (U) memcpy(U + (size_t)i * T * nu, Uk, sizeof(double) * (size_t)T * nu);
    if (S) S[i] = Sk;
    if (L) memcpy(L + (size_t)i * M, Lm, sizeof(double) * (size_t)M);
    if (cvar) cvar[i] = cv;
    if (S_tilde) S_tilde[i] = st;
    if (S_lo) S_lo[i] = Sk_lo;
    if (S_hi) S_hi[i] = Sk_hi;
    if (St_lo) St_lo[i] = Sk_lo + ((cv_lo > p->C_u) ? p->A * cv_lo : 0.0);
    if (St_hi) St_hi[i] = Sk_hi + ((cv_hi > p->C_u) ? p->A * cv_hi : 0.0);
    if (cvar_lo) cvar_lo[i] = cv_lo;
    if (cvar_hi) cvar_hi[i] = cv_hi;
    free(Uk);
    free(Lm);
    free(Wm);
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Softmin weights and the weighted update (Eqs. 4, 5, 17)              */
/* ------------------------------------------------------------------ */
int32_t orc_update(int32_t K, int32_t T, int32_t nu, double lam, const double* S_tilde, const double* U,
                   double* V_plus, double* weights) {
  double beta = INFINITY;
  for (int k = 0; k < K; ++k)
    if (isfinite(S_tilde[k]) && S_tilde[k] < beta) beta = S_tilde[k];
  if (!isfinite(beta)) return -5;
  double sum = 0.0;
  for (int k = 0; k < K; ++k) {
    double w = isfinite(S_tilde[k]) ? exp(-(S_tilde[k] - beta) / lam) : 0.0;
    if (weights) weights[k] = w;
    sum += w;
  }
  for (int t = 0; t < T; ++t)
    for (int j = 0; j < nu; ++j) {
      double acc = 0.0;
      for (int k = 0; k < K; ++k) {
        double w = isfinite(S_tilde[k]) ? exp(-(S_tilde[k] - beta) / lam) : 0.0;
        acc += w * U[((size_t)k * T + t) * nu + j];
      }
      V_plus[t * nu + j] = acc / sum;
    }
  if (weights)
    for (int k = 0; k < K; ++k) weights[k] /= sum;
  return 0;
}

/* ------------------------------------------------------------------ */
/* Simulated plant for the receding-horizon loop (Alg. 1 outer loop)    */
/* ------------------------------------------------------------------ */
/* x_out = F(x, u) + w with the plant's own noise stream at `iteration`;
 * returns bit 0 when x_out is inside an obstacle, bit 1 when it is off the track */
int32_t orc_plant_step(const orc_problem* p, uint64_t iteration, const double* x, const double* u,
                       const double* obs, int32_t n_obs, double* x_out) {
  int nx = nx_of(p->model);
  double xn[6], w[4];
  orc_dynamics(p, x, u, xn);
  process_noise_at(p, iteration, 0xFFFFFFFEu, 0xFFFFFFFFu, 0, 1.0, NULL, w);
  for (int s = 0; s < nslots_of(p->model); ++s) xn[slot_dim(p->model, s)] += w[s];
  for (int a = 0; a < nx; ++a) x_out[a] = xn[a];
  if (p->model == ORC_LIN) return 0;
  double tr[3];
  orc_track(p, xn[0], xn[1], tr);
  int hit = fabs(tr[0]) > p->track_half_width ? 2 : 0;
  for (int i = 0; i < n_obs; ++i) {
    double dx = xn[0] - obs[3 * i], dy = xn[1] - obs[3 * i + 1];
    if (sqrt(dx * dx + dy * dy) < obs[3 * i + 2]) hit |= 1;
  }
  return hit;
}

/* scalar exports used by the pins */
double orc_state_cost(const orc_problem* p, const double* x, const double* obs, int32_t n_obs, uint32_t mask) {
  return state_cost(p, x, obs, n_obs, mask, 0.0);
}
double orc_terminal_cost(const orc_problem* p, const double* x) { return terminal_cost(p, x); }
int32_t orc_sizeof_problem(void) { return (int32_t)sizeof(orc_problem); }
int32_t orc_n_warm(const orc_problem* p) { return n_warm_of(p); }

/* ------------------------------------------------------------------ */
/* Adjoint (vector-Jacobian product) of one update.                      */
/*                                                                       */
/* For fixed noise, one update maps the mean controls V and the cost      */
/* weights theta = (w_dev, w_speed, gamma, w_obs) to (V+, S~).  Given     */
/* cotangents gV+ [T][nu] and gS~ [K], this returns                      */
/*   gV = d<gV+, V+> / dV + d<gS~, S~> / dV,  gtheta likewise.            */
/* Steps, each the derivative of the corresponding forward step:        */
/*   Eq. 4/17: V+ = sum w U / sum w  =>  dV+/dU_k = w^_k I and            */
/*             dV+/dS~_k = -(w^_k / lambda) (U_k - V+)                    */
/*   Eqs. 14-16: dS~/dS = 1, dS~/dCVaR = A 1{CVaR > C_u}                  */
/*   Eqs. 10-13, 18, 19: CVaR is piecewise linear in L; its weights are   */
/*             1/((1-alpha)M) above VaR, the remaining weight shared      */
/*             equally by the values equal to VaR, 0 below; the scaling   */
/*             adds (1-B)/M to every weight times B                       */
/*   Eqs. 3, 9: reverse sweeps lambda_t = dc/dx_t + (dF/dx)' lambda_{t+1} */
/*             through the stored states, u-bar_t += (dF/du)' lambda_{t+1}*/
/*   Alg. 1:   U = clip(V + eps) passes the cotangent to V inside the box */
/*             for the samples drawn around V; the control cost            */
/*             gamma v' Sigma^-1 u depends on V directly as well.          */
/* The indicator obstacle term has zero derivative almost everywhere.    */
/* The dynamic model's Heun sub-steps are reversed with the analytic     */
/* Jacobian of its derivative (slip angles, Pacejka forces, heading).    */
/* ------------------------------------------------------------------ */

/* gradient of the track deviation e and arc length s w.r.t. (px, py) */
static void track_grad(const orc_problem* p, double px, double py, double de[2], double ds[2]) {
  double half = 0.5 * p->track_straight;
  de[0] = de[1] = ds[0] = ds[1] = 0.0;
  if (fabs(px) <= half) {
    if (py < 0.0) { de[1] = -1.0; ds[0] = 1.0; }
    else { de[1] = 1.0; ds[0] = -1.0; }
  } else {
    double cx = px > half ? half : -half;
    double dx = px - cx, rho = sqrt(dx * dx + py * py);
    if (rho > 0.0) {
      de[0] = dx / rho;
      de[1] = py / rho;
      /* s = const + R atan2(py, dx): ds = R (-py, dx) / rho^2 */
      ds[0] = p->track_radius * (-py) / (rho * rho);
      ds[1] = p->track_radius * dx / (rho * rho);
    }
  }
}

/* gradient w.r.t. the state of the cost terms in mask, scaled by c, added to
 * gx; theta-gradient (dev, speed, -, obs) of the same terms added to gth */
static void state_cost_grad(const orc_problem* p, const double* x, const double* obs, int n_obs,
                            uint32_t mask, double c, double* gx, double* gth) {
  if (p->model == ORC_LIN) {
    if (mask & ORC_R_LIN) gx[0] += c * p->c_lin;
    return;
  }
  double tr[3], de[2], ds[2];
  orc_track(p, x[0], x[1], tr);
  track_grad(p, x[0], x[1], de, ds);
  if (mask & ORC_R_DEV) {
    gx[0] += c * p->w_dev * 2.0 * tr[0] * de[0];
    gx[1] += c * p->w_dev * 2.0 * tr[0] * de[1];
    gth[0] += c * tr[0] * tr[0];
  }
  if (mask & ORC_R_SPEED) {
    gx[3] += c * p->w_speed * 2.0 * (x[3] - p->v_target);
    gth[1] += c * (x[3] - p->v_target) * (x[3] - p->v_target);
  }
  if (mask & ORC_R_OBS) {
    double val = 0.0, g0 = 0.0, g1 = 0.0;
    for (int i = 0; i < n_obs; ++i) {
      double dx = x[0] - obs[3 * i], dy = x[1] - obs[3 * i + 1];
      double d = sqrt(dx * dx + dy * dy), r = obs[3 * i + 2];
      if (p->obs_mode == ORC_OBS_INDICATOR) {
        if (d < r) val += 1.0;
      } else {
        double z = p->kappa * (r - d);
        double sp = z > 0.0 ? z + log1p(exp(-z)) : log1p(exp(z));
        val += sp / p->kappa;
        double sig = 1.0 / (1.0 + exp(-z));
        if (d > 0.0) { g0 += -sig * dx / d; g1 += -sig * dy / d; }
      }
    }
    gx[0] += c * p->w_obs * g0;
    gx[1] += c * p->w_obs * g1;
    gth[3] += c * val;
  }
  if (mask & ORC_R_BDRY) {
    /* b = atan(-100 d)/pi + 1/2 > 0, d = hw - |e| */
    double d = tr[2];
    double db_dd = (-100.0 / ORC_PI) / (1.0 + 1e4 * d * d);
    double sgn = tr[0] > 0.0 ? 1.0 : (tr[0] < 0.0 ? -1.0 : 0.0);
    gx[0] += c * p->w_bdry * db_dd * (-sgn) * de[0];
    gx[1] += c * p->w_bdry * db_dd * (-sgn) * de[1];
  }
  if (mask & ORC_R_LIN) gx[0] += c * p->c_lin;
}

/* transposed Jacobians of the dynamic model's derivative f(x, u) applied to
 * fb: xb += (df/dx)' fb, ub += (df/du)' fb (the same formulas as dyn_deriv) */
static void dyn_deriv_vjp(const double* mp, const double* x, const double* u, const double* fb, double* xb,
                          double* ub) {
  const double m = mp[0], Iz = mp[1], lf = mp[2], lr = mp[3];
  const double Bt = mp[4], Ct = mp[5], Dt = mp[6], vfloor = mp[7];
  const double g = 9.81;
  const double psi = x[2], vx = x[3], vy = x[4], r = x[5];
  const double delta = u[0];
  const double Fzf = m * g * lr / (lf + lr), Fzr = m * g * lf / (lf + lr);
  const double vxs = vx > vfloor ? vx : vfloor;
  const double yf = vy + lf * r, yr = vy - lr * r;
  const double af = delta - atan2(yf, vxs), ar = -atan2(yr, vxs);
  const double Fyf = Dt * Fzf * sin(Ct * atan(Bt * af));
  const double Fyr = Dt * Fzr * sin(Ct * atan(Bt * ar));
  /* dF/dalpha = D Fz cos(C atan(B a)) C B / (1 + (B a)^2) */
  const double dFf = Dt * Fzf * cos(Ct * atan(Bt * af)) * Ct * Bt / (1.0 + Bt * af * Bt * af);
  const double dFr = Dt * Fzr * cos(Ct * atan(Bt * ar)) * Ct * Bt / (1.0 + Bt * ar * Bt * ar);
  const double cp = cos(psi), sp = sin(psi), cd = cos(delta), sd = sin(delta);
  /* f0 = vx cos psi - vy sin psi, f1 = vx sin psi + vy cos psi, f2 = r */
  xb[2] += fb[0] * (-vx * sp - vy * cp) + fb[1] * (vx * cp - vy * sp);
  xb[3] += fb[0] * cp + fb[1] * sp;
  xb[4] += -fb[0] * sp + fb[1] * cp;
  xb[5] += fb[2];
  /* f3 = a - Fyf sin d / m + r vy */
  ub[1] += fb[3];
  xb[5] += fb[3] * vy;
  xb[4] += fb[3] * r;
  /* f4 = (Fyf cos d + Fyr) / m - r vx */
  xb[5] += -fb[4] * vx;
  xb[3] += -fb[4] * r;
  /* forces and steer through f3, f4, f5 = (lf Fyf cos d - lr Fyr) / Iz */
  const double Ffb = -fb[3] * sd / m + fb[4] * cd / m + fb[5] * lf * cd / Iz;
  const double Frb = fb[4] / m - fb[5] * lr / Iz;
  ub[0] += -fb[3] * Fyf * cd / m - fb[4] * Fyf * sd / m - fb[5] * lf * Fyf * sd / Iz;
  const double afb = Ffb * dFf, arb = Frb * dFr;
  ub[0] += afb;
  /* alpha_f = d - atan2(yf, vxs), alpha_r = -atan2(yr, vxs) */
  const double nf = vxs * vxs + yf * yf, nr = vxs * vxs + yr * yr;
  const double yfb = afb * (-vxs / nf), yrb = arb * (-vxs / nr);
  const double vxsb = afb * (yf / nf) + arb * (yr / nr);
  xb[4] += yfb + yrb;
  xb[5] += lf * yfb - lr * yrb;
  if (vx > vfloor) xb[3] += vxsb;
}

/* one integration sub-step G and its transposed Jacobians applied to lam:
 * lam_out = (dG/ds)' lam, gu += (dG/du)' lam */
static void substep_vjp(const orc_problem* p, const double* s, const double* u, const double* lam,
                        double* lam_out, double* gu) {
  double h = p->dt / (p->substeps > 0 ? p->substeps : 1);
  if (p->model == ORC_DYN) {
    /* Heun: x1 = s + h f(s), G = s + h/2 (f(s) + f(x1)) */
    double k1[6], x1[6];
    dyn_deriv(p->model_params, s, u, k1);
    for (int i = 0; i < 6; ++i) x1[i] = s[i] + h * k1[i];
    double fb[6], x1b[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 6; ++i) fb[i] = 0.5 * h * lam[i];
    dyn_deriv_vjp(p->model_params, x1, u, fb, x1b, gu);   /* through f(x1) */
    double fa[6];
    for (int i = 0; i < 6; ++i) fa[i] = 0.5 * h * lam[i] + h * x1b[i];
    for (int i = 0; i < 6; ++i) lam_out[i] = lam[i] + x1b[i];
    dyn_deriv_vjp(p->model_params, s, u, fa, lam_out, gu);  /* through f(s) */
  } else if (p->model == ORC_KIN) {
    double L = p->model_params[0], psi = s[2], v = s[3];
    double cs = cos(psi), sn = sin(psi), tn = tan(u[0]), sec2 = 1.0 / (cos(u[0]) * cos(u[0]));
    lam_out[0] = lam[0];
    lam_out[1] = lam[1];
    lam_out[2] = lam[2] + lam[0] * (-h * v * sn) + lam[1] * (h * v * cs);
    lam_out[3] = lam[3] + lam[0] * (h * cs) + lam[1] * (h * sn) + lam[2] * (h * tn / L);
    gu[0] += lam[2] * h * v * sec2 / L;
    gu[1] += lam[3] * h;
  } else {
    lam_out[0] = lam[0];
    gu[0] += lam[0] * h;
  }
}

static void substep_fwd(const orc_problem* p, const double* s, const double* u, double* out) {
  orc_problem q = *p;
  q.dt = p->dt / (p->substeps > 0 ? p->substeps : 1);
  q.substeps = 1;
  orc_dynamics(&q, s, u, out);
}

/* reverse sweep of one rollout with stored states xs[(T+1)][nx]; cost
 * weight c on the running terms `mask` (and on phi when with_phi);
 * accumulates gU [T][nu] and gth [4] */
static void rollout_vjp(const orc_problem* p, const double* xs, const double* Uk, const double* obs, int n_obs,
                        uint32_t mask, int with_phi, double c, double* gU, double* gth) {
  const int nx = nx_of(p->model), nu = nu_of(p->model), T = p->T;
  const int ns = p->substeps > 0 ? p->substeps : 1;
  double lam[6] = {0, 0, 0, 0, 0, 0};
  if (with_phi && p->model != ORC_LIN && p->c5 != 0.0) {
    double de[2], ds[2];
    const double* xT = xs + (size_t)T * nx;
    track_grad(p, xT[0], xT[1], de, ds);
    lam[0] += c * (-p->c5) * ds[0];
    lam[1] += c * (-p->c5) * ds[1];
  }
  double sub[65][6];
  for (int t = T - 1; t >= 0; --t) {
    const double* xt = xs + (size_t)t * nx;
    const double* ut = Uk + (size_t)t * nu;
    /* through F(x_t, u_t): recompute the sub-step states, reverse them */
    for (int a = 0; a < nx; ++a) sub[0][a] = xt[a];
    for (int i = 0; i < ns; ++i) substep_fwd(p, sub[i], ut, sub[i + 1]);
    for (int i = ns - 1; i >= 0; --i) {
      double lo[6] = {0, 0, 0, 0, 0, 0};
      substep_vjp(p, sub[i], ut, lam, lo, gU + (size_t)t * nu);
      for (int a = 0; a < nx; ++a) lam[a] = lo[a];
    }
    /* running cost at x_t */
    state_cost_grad(p, xt, obs, n_obs, mask, c, lam, gth);
  }
}

int32_t orc_backward(const orc_problem* p, const double* x0, const double* V, const double* obs, int32_t n_obs,
                     const double* gVp, const double* gSt, double* gV, double* gtheta) {
  if (p->substeps > 64) return -1;
  const int M_s = is_count(p);
  if (M_s > 0 && p->noise_type != ORC_GAUSS && p->noise_type != ORC_LAPLACE_MIX) return -6;
  const int K = p->K, M = p->M, T = p->T, nx = nx_of(p->model), nu = nu_of(p->model);
  const int n_warm = n_warm_of(p);
  double inv_sig2[2];
  for (int j = 0; j < 2; ++j) inv_sig2[j] = p->sigma_u[j] > 0.0 ? 1.0 / (p->sigma_u[j] * p->sigma_u[j]) : 0.0;
  double* U = (double*)calloc((size_t)K * T * nu, sizeof(double));
  double* inside = (double*)calloc((size_t)K * T * nu, sizeof(double));
  double* S = (double*)calloc((size_t)K, sizeof(double));
  double* cv = (double*)calloc((size_t)K, sizeof(double));
  double* St = (double*)calloc((size_t)K, sizeof(double));
  double* Xn = (double*)calloc((size_t)K * (T + 1) * nx, sizeof(double));
  double* Xd = (double*)calloc((size_t)K * M * (T + 1) * nx, sizeof(double));
  double* Lm = (double*)calloc((size_t)K * M, sizeof(double));
  double* Wm = (double*)calloc((size_t)K * M, sizeof(double)); /* importance weights (1 when off) */
  /* forward with stored states (same steps as orc_samples) */
  for (int k = 0; k < K; ++k) {
    double* Uk = U + (size_t)k * T * nu;
    for (int t = 0; t < T; ++t) {
      double eps[2];
      orc_control_noise(p, k, t, eps);
      for (int j = 0; j < nu; ++j) {
        double raw = ((k < n_warm) ? V[t * nu + j] : 0.0) + eps[j];
        Uk[t * nu + j] = clampd(raw, p->u_lo[j], p->u_hi[j]);
        inside[(size_t)k * T * nu + t * nu + j] = (k < n_warm && raw > p->u_lo[j] && raw < p->u_hi[j]) ? 1.0 : 0.0;
      }
    }
    double* xs = Xn + (size_t)k * (T + 1) * nx;
    for (int a = 0; a < nx; ++a) xs[a] = x0[a];
    double Sk = 0.0;
    for (int t = 0; t < T; ++t) {
      double ctrl = 0.0;
      for (int j = 0; j < nu; ++j) ctrl += V[t * nu + j] * inv_sig2[j] * Uk[t * nu + j];
      Sk += state_cost(p, xs + (size_t)t * nx, obs, n_obs, 0xFFFFFFFFu, 0.0) + p->gamma * ctrl;
      orc_dynamics(p, xs + (size_t)t * nx, Uk + t * nu, xs + (size_t)(t + 1) * nx);
    }
    Sk += terminal_cost(p, xs + (size_t)T * nx);
    S[k] = Sk;
    for (int m = 0; m < M; ++m) {
      double* xd = Xd + ((size_t)k * M + m) * (T + 1) * nx;
      for (int a = 0; a < nx; ++a) xd[a] = x0[a];
      double Lv = 0.0, G = 0.0;
      for (int t = 0; t < T; ++t) {
        Lv += state_cost(p, xd + (size_t)t * nx, obs, n_obs, p->risk_mask, 0.0);
        double w[4];
        process_noise_at(p, p->iteration, (uint32_t)m, (uint32_t)k, t, is_factor(p, m, M_s), M_s > 0 ? &G : NULL, w);
        orc_dynamics(p, xd + (size_t)t * nx, Uk + t * nu, xd + (size_t)(t + 1) * nx);
        for (int s = 0; s < nslots_of(p->model); ++s) xd[(size_t)(t + 1) * nx + slot_dim(p->model, s)] += w[s];
      }
      Lm[(size_t)k * M + m] = Lv;
      Wm[(size_t)k * M + m] = M_s > 0 ? is_weight(p, M_s, G) : 1.0;
    }
    cv[k] = orc_risk_w(Lm + (size_t)k * M, M_s > 0 ? Wm + (size_t)k * M : NULL, M, p->alpha, p->B, p->cvar_mode,
                       p->risk_param);
    St[k] = S[k] + ((cv[k] > p->C_u) ? p->A * cv[k] : 0.0);
  }
  /* update and its weights */
  double beta = INFINITY;
  for (int k = 0; k < K; ++k) if (isfinite(St[k]) && St[k] < beta) beta = St[k];
  double* wh = (double*)calloc((size_t)K, sizeof(double));
  double* Vp = (double*)calloc((size_t)T * nu, sizeof(double));
  double sum = 0.0;
  for (int k = 0; k < K; ++k) { wh[k] = isfinite(St[k]) ? exp(-(St[k] - beta) / p->lam) : 0.0; sum += wh[k]; }
  for (int k = 0; k < K; ++k) wh[k] /= sum;
  for (int k = 0; k < K; ++k)
    for (int c = 0; c < T * nu; ++c) Vp[c] += wh[k] * U[(size_t)k * T * nu + c];
  for (int c = 0; c < T * nu; ++c) gV[c] = 0.0;
  for (int i = 0; i < 4; ++i) gtheta[i] = 0.0;
  double* gU = (double*)calloc((size_t)T * nu, sizeof(double));
  double* La = (double*)calloc((size_t)M, sizeof(double));
  for (int k = 0; k < K; ++k) {
    const double* Uk = U + (size_t)k * T * nu;
    /* cotangent of S~_k */
    double dot = 0.0;
    for (int c = 0; c < T * nu; ++c) dot += gVp[c] * (Uk[c] - Vp[c]);
    double sbar = (gSt ? gSt[k] : 0.0) - wh[k] / p->lam * dot;
    double cvbar = (cv[k] > p->C_u) ? sbar * p->A : 0.0;
    for (int c = 0; c < T * nu; ++c) gU[c] = wh[k] * gVp[c];
    /* nominal: S_k */
    rollout_vjp(p, Xn + (size_t)k * (T + 1) * nx, Uk, obs, n_obs, 0xFFFFFFFFu, 1, sbar, gU, gtheta);
    for (int t = 0; t < T; ++t) {
      double ctrl = 0.0;
      for (int j = 0; j < nu; ++j) {
        ctrl += V[t * nu + j] * inv_sig2[j] * Uk[t * nu + j];
        gU[t * nu + j] += sbar * p->gamma * inv_sig2[j] * V[t * nu + j];
        gV[t * nu + j] += sbar * p->gamma * inv_sig2[j] * Uk[t * nu + j];
      }
      gtheta[2] += sbar * ctrl;
    }
    /* disturbed: weights of CVaR in each L_{k,m}.  With importance weights
     * w (all 1 when off) every count becomes a weight sum: the measure of
     * the weighted empirical distribution, W = sum w in place of M */
    if (cvbar != 0.0) {
      const double* Lk = Lm + (size_t)k * M;
      const double* wk = Wm + (size_t)k * M;
      double W = 0.0, mean = 0.0;
      for (int m = 0; m < M; ++m) { W += wk[m]; mean += wk[m] * Lk[m]; }
      mean /= W;
      for (int m = 0; m < M; ++m) La[m] = p->B * (Lk[m] - mean) + mean;
      /* VaR: the smallest La_m whose strictly larger weight is at most (1 - alpha) W */
      const double tau = (1.0 - p->alpha) * W;
      double var = INFINITY;
      for (int c = 0; c < M; ++c) {
        double above = 0.0;
        for (int n = 0; n < M; ++n)
          if (La[n] > La[c]) above += wk[n];
        if (above <= tau && La[c] < var) var = La[c];
      }
      double w_gt = 0.0, w_eq = 0.0;
      for (int m = 0; m < M; ++m) { if (La[m] > var) w_gt += wk[m]; else if (La[m] == var) w_eq += wk[m]; }
      for (int m = 0; m < M; ++m) {
        double wa;
        if (p->cvar_mode == ORC_CVAR_RU)
          wa = La[m] > var ? wk[m] / tau : (La[m] == var ? (1.0 - w_gt / tau) * wk[m] / w_eq : 0.0);
        else if (p->cvar_mode == ORC_CVAR_TCE)
          wa = La[m] >= var ? wk[m] / (w_gt + w_eq) : 0.0;
        else if (p->cvar_mode == ORC_VAR)
          wa = La[m] == var ? wk[m] / w_eq : 0.0;
        else if (p->cvar_mode == ORC_MEAN)
          wa = wk[m] / W;
        else if (p->cvar_mode == ORC_MEANVAR)
          wa = wk[m] * (1.0 + 2.0 * p->risk_param * (La[m] - mean)) / W;
        else
          wa = 0.0; /* the chance measure is piecewise constant in L */
        if (p->cvar_mode == ORC_CHANCE) continue;
        double lbar = cvbar * (p->B * wa + (1.0 - p->B) * wk[m] / W);
        if (lbar != 0.0)
          rollout_vjp(p, Xd + ((size_t)k * M + m) * (T + 1) * nx, Uk, obs, n_obs, p->risk_mask, 0, lbar, gU, gtheta);
      }
    }
    /* through U = clip(V + eps) to V */
    for (int c = 0; c < T * nu; ++c) gV[c] += gU[c] * inside[(size_t)k * T * nu + c];
  }
  free(U); free(inside); free(S); free(cv); free(St); free(Xn); free(Xd); free(Lm); free(Wm);
  free(wh); free(Vp); free(gU); free(La);
  return 0;
}

/* set theta = (w_dev, w_speed, gamma, w_obs) on a problem copy */
void orc_set_theta(orc_problem* p, const double* theta) {
  p->w_dev = theta[0];
  p->w_speed = theta[1];
  p->gamma = theta[2];
  p->w_obs = theta[3];
}
