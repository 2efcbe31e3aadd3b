// C ABI of the RA-MPPI update library (declarations and contracts in
// include/ra_mppi.h).  Host side only: validation, workspace, constants and
// kernel launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "ra_host.h"
#include "ra_kernels.h"
#include "ra_mppi.h"

using ramppi::DevParams;
using ramppi::DevState;
using ramppi_api::DeviceScope;

struct ra_mppi {
  ra_mppi_problem prob;
  DevParams dp;
  int device = 0;
  int n_sms = 152;
  int nx = 0, nu = 0;
  int warps = 4, ilp = 1, wps = 1;  // warps per block, rollouts interleaved, warps per sample
  bool tail_split = true;            // the last partial wave in smaller units (see tail_plan)
  int occ_blocks = 0;                // resident rollout blocks per SM at the current shape
  int n_obs_host = 0;                // obstacle count of the last set_obstacles
  int nb_upd = 1;
  int obs_cap = 0;
  size_t smem = 0;
  float* U = nullptr;
  float* S = nullptr;
  float* cvar = nullptr;
  float* S_tilde = nullptr;
  float* partials = nullptr;
  float* L = nullptr;
  float4* obs = nullptr;
  DevState* st = nullptr;
  float* x0_dev = nullptr;  // staging for ra_mppi_step_host
  float* V_dev = nullptr;
  float* V_plus = nullptr;  // V+ of ra_mppi_closed_loop_step before the warm-start shift
  // adjoint (RA_MPPI_DIFFERENTIABLE): inputs of the last update and scratch
  float* keep_x0 = nullptr;
  float* keep_V = nullptr;
  unsigned int* b_arrive = nullptr;
  float* b_dk = nullptr;
  float* b_wk = nullptr;
  float* b_Gnom = nullptr;
  float* b_mask = nullptr;
  float* b_gUd = nullptr;
  float* b_thn = nullptr;
  float* b_thd = nullptr;
  double* b_red = nullptr;
  float* b_ck_nom = nullptr;   // state checkpoints of the last update (every 8 steps)
  float* b_ck_dist = nullptr;
  int nb_red = 0;
  cudaEvent_t ev_begin = nullptr;  // optional timing hook around the rollout kernel
  cudaEvent_t ev_end = nullptr;
  std::string err;
};

namespace {

int fail(ra_mppi* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

int cuda_fail(ra_mppi* h, cudaError_t e, const char* where) {
  return fail(h, RA_MPPI_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Host-side fault injection for tests of the error paths: RAMPPI_FAULT=alloc
// makes create fail as if cudaMalloc had, RAMPPI_FAULT=launch makes step fail
// before enqueueing anything.  Never touches the GPU.
bool fault(const char* what) {
  const char* f = std::getenv("RAMPPI_FAULT");
  return f != nullptr && std::strcmp(f, what) == 0;
}

#define RA_DEVICE_SCOPE(h)                                                   \
  DeviceScope device_scope_((h)->device);                                    \
  if (!device_scope_.ok()) return fail((h), RA_MPPI_ECUDA, "cannot make the handle's device current")

int model_nx(int model) { return model == RA_MPPI_KIN_BICYCLE ? 4 : model == RA_MPPI_DYN_SINGLE_TRACK ? 6 : 1; }
int model_nu(int model) { return model == RA_MPPI_LINEAR_TEST ? 1 : 2; }
int model_slots(int model) { return model == RA_MPPI_KIN_BICYCLE ? 4 : model == RA_MPPI_DYN_SINGLE_TRACK ? 3 : 1; }

bool finite_all(const float* v, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

// returns "" when valid, otherwise the reason
// number of importance-sampled (proposal) rollouts per sample, 0 when off
int is_count(const ra_mppi_problem& p) {
  if (p.is_scale == 1.0f || !(p.is_frac > 0.0f)) return 0;
  return (int)std::floor((double)p.is_frac * (double)p.M);
}

std::string validate(const ra_mppi_problem& p) {
  if (p.model < 0 || p.model > 2) return "model must be 0 (kinematic), 1 (dynamic) or 2 (linear)";
  if (p.K < 1 || p.K > (1 << 24)) return "K must be in [1, 2^24]";
  if (p.M < 1 || p.M > RA_MPPI_MAX_M) return "M must be in [1, 512]";
  if (p.T < 1 || p.T > RA_MPPI_MAX_T) return "T must be in [1, 256]";
  if (p.substeps < 1 || p.substeps > 64) return "substeps must be in [1, 64]";
  if (p.noise_type < RA_MPPI_NOISE_GAUSS || p.noise_type > RA_MPPI_NOISE_IMPULSE) return "unknown noise_type";
  if (p.obs_mode != RA_MPPI_OBS_INDICATOR && p.obs_mode != RA_MPPI_OBS_SOFTPLUS) return "unknown obs_mode";
  if (p.cvar_mode < RA_MPPI_CVAR_RU || p.cvar_mode > RA_MPPI_RISK_MEANVAR) return "unknown risk measure (cvar_mode)";
  if (std::isnan(p.risk_param)) return "risk_param must not be NaN";
  if (p.cvar_mode == RA_MPPI_RISK_MEANVAR && !(p.risk_param >= 0.0f && std::isfinite(p.risk_param)))
    return "the mean-variance weight risk_param must be finite and >= 0";
  if (p.max_obstacles < 0 || p.max_obstacles > RA_MPPI_MAX_OBSTACLES) return "max_obstacles must be in [0, 1024]";
  if (!(p.dt > 0.0f) || !std::isfinite(p.dt)) return "dt must be finite and > 0";
  if (!(p.lambda > 0.0f) || !std::isfinite(p.lambda)) return "lambda must be finite and > 0";
  if (!(p.alpha > 0.0f && p.alpha < 1.0f)) return "alpha must be in (0, 1)";
  if (!(p.B >= 0.0f) || !std::isfinite(p.B)) return "B must be finite and >= 0";
  if (!(p.eta >= 0.0f && p.eta < 1.0f)) return "eta must be in [0, 1)";
  if (!(p.mix_p >= 0.0f && p.mix_p <= 1.0f)) return "mix_p must be in [0, 1]";
  if (!(p.kappa > 0.0f) && p.obs_mode == RA_MPPI_OBS_SOFTPLUS) return "kappa must be > 0";
  for (int j = 0; j < 2; ++j) {
    if (!(p.sigma_u[j] >= 0.0f) || !std::isfinite(p.sigma_u[j])) return "sigma_u must be finite and >= 0";
    if (!(p.u_lo[j] <= p.u_hi[j])) return "u_lo must be <= u_hi";
  }
  for (int s = 0; s < 4; ++s)
    if (!(p.w_scale[s] >= 0.0f) || !std::isfinite(p.w_scale[s])) return "w_scale must be finite and >= 0";
  if (!finite_all(p.model_params, 8)) return "model_params must be finite";
  if (p.model == RA_MPPI_KIN_BICYCLE && !(p.model_params[0] > 0.0f)) return "wheelbase must be > 0";
  if (p.model == RA_MPPI_DYN_SINGLE_TRACK) {
    const float* mp = p.model_params;
    if (!(mp[0] > 0.0f && mp[1] > 0.0f && mp[2] > 0.0f && mp[3] > 0.0f && mp[7] > 0.0f))
      return "dynamic model needs m, Iz, lf, lr and the vx floor > 0";
  }
  const float w[] = {p.w_dev, p.w_speed, p.v_target, p.gamma, p.w_obs, p.w_bdry, p.c4, p.c5, p.c_lin,
                     p.track_straight, p.track_radius, p.track_half_width, p.A, p.C_u, p.mix_scale};
  for (float v : w)
    if (std::isnan(v)) return "cost and track parameters must not be NaN";
  if (!(p.is_scale >= 1.0f && p.is_scale <= 16.0f)) return "is_scale must be in [1, 16]";
  if (!(p.is_frac >= 0.0f && p.is_frac < 1.0f)) return "is_frac must be in [0, 1)";
  if (is_count(p) > 0 && p.noise_type != RA_MPPI_NOISE_GAUSS && p.noise_type != RA_MPPI_NOISE_LAPLACE_MIX)
    return "importance sampling needs Gaussian or mixture process noise";
  return "";
}

DevParams make_params(const ra_mppi_problem& p) {
  DevParams d{};
  d.K = p.K;
  d.M = p.M;
  d.T = p.T;
  d.nu = model_nu(p.model);
  d.substeps = p.substeps;
  d.noise_type = p.noise_type;
  d.obs_mode = p.obs_mode;
  d.cvar_mode = p.cvar_mode;
  d.risk_mask = p.risk_mask;
  // Alg. 1: sample k keeps the mean control when k < (1 - eta) K; the
  // products below are exact in double for float32 inputs
  d.n_warm = (int)std::ceil((1.0 - (double)p.eta) * (double)p.K);
  const double aM = (double)p.alpha * (double)p.M;
  int j = (int)std::ceil(aM);
  j = j < 1 ? 1 : (j > p.M ? p.M : j);
  d.j_var = j;
  d.frac_j = (float)((double)j - aM);
  d.tail_denom = (float)((1.0 - (double)p.alpha) * (double)p.M);
  d.h = p.dt / (float)p.substeps;
  for (int i = 0; i < 8; ++i) d.mp[i] = p.model_params[i];
  if (p.model == RA_MPPI_DYN_SINGLE_TRACK) {
    const double m = p.model_params[0], Iz = p.model_params[1], lf = p.model_params[2], lr = p.model_params[3];
    const double D = p.model_params[6], g = 9.81;
    d.pacejka_c15 = p.model_params[5] == 1.5f ? 1 : 0;
    // lateral accelerations per unit shape, with the 1/sqrt(2) of the C = 3/2
    // closed form folded in; yaw arms l m / Iz
    const double fold = d.pacejka_c15 ? std::sqrt(0.5) : 1.0;
    d.acc_f = (float)(D * g * lr / (lf + lr) * fold);
    d.acc_r = (float)(D * g * lf / (lf + lr) * fold);
    d.yaw_f = (float)(lf * m / Iz);
    d.yaw_r = (float)(lr * m / Iz);
    d.nyaw_acc_r = (float)(-(double)d.yaw_r * (double)d.acc_r);
  }
  for (int j2 = 0; j2 < 2; ++j2) {
    d.sigma_u[j2] = p.sigma_u[j2];
    d.inv_sig2[j2] = p.sigma_u[j2] > 0.0f ? (float)(1.0 / ((double)p.sigma_u[j2] * p.sigma_u[j2])) : 0.0f;
    d.u_lo[j2] = p.u_lo[j2];
    d.u_hi[j2] = p.u_hi[j2];
  }
  const double thr = std::floor(std::fmin((double)p.mix_p * 4294967296.0, 4294967295.0));
  d.mix_thresh = (uint32_t)thr;
  d.mix_inv_thresh = thr > 0.0 ? (float)(1.0 / thr) : 0.0f;
  for (int s = 0; s < 4; ++s) {
    d.w_scale[s] = p.w_scale[s];
    d.mix_gauss[s] = (float)((double)p.mix_scale * (double)p.w_scale[s]);
  }
  d.w_dev = p.w_dev;
  d.w_speed = p.w_speed;
  d.v_target = p.v_target;
  d.gamma = p.gamma;
  d.w_obs = p.w_obs;
  d.w_bdry = p.w_bdry;
  d.c4 = p.c4;
  d.c5 = p.c5;
  d.c_lin = p.c_lin;
  d.kappa = p.kappa;
  d.inv_kappa = p.kappa > 0.0f ? 1.0f / p.kappa : 0.0f;
  d.track_S = p.track_straight;
  d.track_R = p.track_radius;
  d.track_hw = p.track_half_width;
  d.inv_lambda = 1.0f / p.lambda;
  d.A = p.A;
  d.B = p.B;
  d.C_u = p.C_u;
  d.risk_param = p.risk_param;
  d.one_m_alpha = (float)(1.0 - (double)p.alpha);
  {
    // importance sampling: per rollout ln q/p = -(draws) ln s + (1 - 1/s) A_L
    // + (1 - 1/s^2)/2 A_G over its unit-scale Laplace magnitudes A_L and
    // squared normals A_G (q(w) = p(w/s)/s for both densities)
    const int M_s = is_count(p);
    const double s = p.is_scale;
    int slots = 0;
    for (int i = 0; i < model_slots(p.model); ++i) slots += p.w_scale[i] != 0.0f ? 1 : 0;
    d.is_m0 = p.M - M_s;
    d.is_s = p.is_scale;
    d.is_b = (float)((double)M_s / (double)p.M);
    d.is_base = (float)(-(double)p.T * slots * std::log(s));
    d.is_cl = (float)(1.0 - 1.0 / s);
    d.is_cg = (float)(0.5 * (1.0 - 1.0 / (s * s)));
  }
  d.seed_lo = (uint32_t)(p.seed & 0xFFFFFFFFull);
  d.seed_hi = (uint32_t)(p.seed >> 32);
  d.instance = p.instance_id;
  return d;
}

template <typename T>
cudaError_t dalloc(T** ptr, size_t count) {
  if (fault("alloc")) return cudaErrorMemoryAllocation;
  return cudaMalloc(reinterpret_cast<void**>(ptr), sizeof(T) * (count > 0 ? count : 1));
}

void release(ra_mppi* h) {
  cudaFree(h->U);
  cudaFree(h->S);
  cudaFree(h->cvar);
  cudaFree(h->S_tilde);
  cudaFree(h->partials);
  cudaFree(h->L);
  cudaFree(h->obs);
  cudaFree(h->st);
  cudaFree(h->x0_dev);
  cudaFree(h->V_dev);
  cudaFree(h->V_plus);
  cudaFree(h->keep_x0);
  cudaFree(h->keep_V);
  cudaFree(h->b_arrive);
  cudaFree(h->b_dk);
  cudaFree(h->b_wk);
  cudaFree(h->b_Gnom);
  cudaFree(h->b_mask);
  cudaFree(h->b_gUd);
  cudaFree(h->b_thn);
  cudaFree(h->b_thd);
  cudaFree(h->b_red);
  cudaFree(h->b_ck_nom);
  cudaFree(h->b_ck_dist);
}

// The limit is a property of the kernel, shared by every handle: raise it
// to what this handle launches with, never lower it below another handle's.
std::mutex g_smem_mutex;
size_t g_smem_limit[64][3] = {};  // per device, per model

// one row of rollouts per sample and two interleaved, dynamic model: each
// warp takes two samples (one rollout of each per lane, a paired-instruction
// pair; see disturbed_sample_pair)
bool importance(const ra_mppi* h) { return is_count(h->prob) > 0; }

// the obstacle cull's x window: dynamic model with more than 64 obstacles
// (below that the box test takes two rounds at most)
// (differentiable handles run the checkpointing kernel instances, which have
// neither the x window nor sample pairs: those change speed only)
bool differentiable(const ra_mppi* h) { return (h->prob.flags & RA_MPPI_DIFFERENTIABLE) != 0; }

bool windowed(const ra_mppi* h) {
  return h->prob.model == RA_MPPI_DYN_SINGLE_TRACK && h->n_obs_host > 64 && !differentiable(h);
}

bool pairs_samples(const ra_mppi* h) {
  return h->prob.model == RA_MPPI_DYN_SINGLE_TRACK && h->ilp == 2 && h->wps == 1 && h->prob.M <= 32 &&
         !importance(h) && !differentiable(h);
}

// samples per disturbed block
int samples_per_block(const ra_mppi* h) { return (h->warps / h->wps) * (pairs_samples(h) ? 2 : 1); }

size_t rollout_smem(const ra_mppi* h) {
  const size_t spb = (size_t)samples_per_block(h);
  // the largest obstacle radius (read by the windowed cull only), obstacles,
  // then controls, risk costs (and importance weights) per sample
  return (1 + (size_t)h->obs_cap) * sizeof(float4) + spb * h->prob.T * sizeof(float4) +
         spb * h->prob.M * sizeof(float) * (importance(h) ? 2 : 1);
}

cudaError_t occupancy(ra_mppi* h) {
  const int m = h->prob.model;
  const bool ck = differentiable(h);
  int blocks = 0;
  cudaError_t e;
  switch (m) {
    case 0: e = ramppi::rollout_occupancy<0>(h->warps, h->ilp, pairs_samples(h), importance(h), windowed(h), ck, h->smem, &blocks); break;
    case 1: e = ramppi::rollout_occupancy<1>(h->warps, h->ilp, pairs_samples(h), importance(h), windowed(h), ck, h->smem, &blocks); break;
    default: e = ramppi::rollout_occupancy<2>(h->warps, h->ilp, pairs_samples(h), importance(h), windowed(h), ck, h->smem, &blocks); break;
  }
  h->occ_blocks = e == cudaSuccess ? blocks : 0;
  return e;
}

// The tail split of the disturbed blocks.  With Ba blocks of warps / wps
// samples each and S = SMs x resident blocks per SM slots, the grid runs
// floor(Ba / S) full rounds and a last round of Ba mod S blocks; when that
// last round is at most half full, its samples take 2 wps warps each instead
// (half the rows per warp), so the last round is made of twice as many
// shorter blocks and the SMs stay busier to the end.  Needs 2 wps to divide
// the block and leave each warp a row; results do not depend on it.
void tail_plan(const ra_mppi* h, int nb_dist, int* nb_head, int* wps_tail, int* nb_total) {
  *nb_head = 0x7FFFFFFF;
  *wps_tail = h->wps;
  *nb_total = nb_dist;
  const int R = (h->prob.M + 31) / 32, G2 = 2 * h->wps;
  if (!h->tail_split || pairs_samples(h) || h->occ_blocks < 1 || G2 > R || h->warps % G2 != 0) return;
  const long long slots = (long long)h->n_sms * h->occ_blocks;
  const long long rounds = nb_dist / slots, rem = nb_dist - rounds * slots;
  if (rounds < 1 || rem == 0 || 2 * rem > slots) return;
  const int spb_h = h->warps / h->wps, spb_t = h->warps / G2;
  const long long head = rounds * slots, tail_samples = (long long)h->prob.K - head * spb_h;
  if (tail_samples <= 0) return;
  *nb_head = (int)head;
  *wps_tail = G2;
  *nb_total = (int)(head + (tail_samples + spb_t - 1) / spb_t);
}

cudaError_t prepare(ra_mppi* h) {
  h->smem = rollout_smem(h);
  const int m = h->prob.model < 0 || h->prob.model > 2 ? 2 : h->prob.model;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  {
    std::lock_guard<std::mutex> lock(g_smem_mutex);
    if (h->smem > g_smem_limit[dev][m]) {
      cudaError_t e;
      switch (m) {
        case 0: e = ramppi::prepare_rollout<0>(h->smem); break;
        case 1: e = ramppi::prepare_rollout<1>(h->smem); break;
        default: e = ramppi::prepare_rollout<2>(h->smem); break;
      }
      if (e != cudaSuccess) return e;
      g_smem_limit[dev][m] = h->smem;
    }
  }
  return occupancy(h);
}

// largest interleave in {2, 1} that divides the rollouts per lane
int default_ilp(int M, int model) {
  const int R = (M + 31) / 32;
  // measured on GB300: both models are fastest with 2 (the dynamic one steps
  // the pair in paired FP32 instructions); 4 costs registers
  // one row per sample: the dynamic model pairs two samples per warp
  if (model == RA_MPPI_DYN_SINGLE_TRACK && R == 1) return 2;
  const int cap = 2;
  for (int ilp = cap; ilp > 1; ilp >>= 1)
    if (R % ilp == 0) return ilp;
  return 1;
}

}  // namespace

// shared with the batched path (ra_batch.cu)
namespace ramppi_api {
// the disc (x, y, r) lies in |x|, |y| <= RA_MPPI_OBSTACLE_EXTENT
bool obstacle_in_extent(float x, float y, float r) {
  const double e = RA_MPPI_OBSTACLE_EXTENT;
  return std::fabs((double)x) + r <= e && std::fabs((double)y) + r <= e;
}
std::string validate_problem(const ra_mppi_problem& p) { return validate(p); }
DevParams make_params(const ra_mppi_problem& p) { return ::make_params(p); }
}  // namespace ramppi_api

extern "C" {

int32_t ra_mppi_problem_size(void) { return (int32_t)sizeof(ra_mppi_problem); }

int ra_mppi_create(const ra_mppi_problem* p, int32_t device, ra_mppi_t** out) {
  if (p == nullptr || out == nullptr) return RA_MPPI_EINVAL;
  const std::string why = validate(*p);
  if (!why.empty()) {
    std::fprintf(stderr, "ra_mppi_create: %s\n", why.c_str());
    return RA_MPPI_EINVAL;
  }
  if (fault("alloc")) return RA_MPPI_ENOMEM;
  int dev = 0;
  {
    cudaError_t e0 = cudaSuccess;
    if (!ramppi_api::resolve_device(device, &dev, &e0)) {
      if (e0 == cudaSuccess) return RA_MPPI_EINVAL;
      std::fprintf(stderr, "ra_mppi_create: %s\n", cudaGetErrorString(e0));
      return RA_MPPI_ECUDA;
    }
  }
  DeviceScope scope(dev);
  if (!scope.ok()) return RA_MPPI_ECUDA;
  ra_mppi* h = new (std::nothrow) ra_mppi();
  if (h == nullptr) return RA_MPPI_ENOMEM;
  h->device = dev;
  h->prob = *p;
  h->dp = make_params(*p);
  h->nx = model_nx(p->model);
  h->nu = model_nu(p->model);
  h->obs_cap = p->max_obstacles;
  h->ilp = default_ilp(p->M, p->model);
  h->warps = 4;
  // few samples with many rollouts: spread a sample over several warps until
  // the sample warps fill the GPU (24 resident warps per SM at 80 registers,
  // times the device's SM count).  The dynamic model's long rollouts gain from
  // two waves, so the last partial wave is short (config 2, K = 4096,
  // M = 128: 2 warps per sample 0.845 ms, 1 warp 0.893); the cheaper
  // kinematic rollouts from one.
  cudaError_t e = cudaDeviceGetAttribute(&h->n_sms, cudaDevAttrMultiProcessorCount, dev);
  {
    const int R = (p->M + 31) / 32;
    const long long waves = p->model == RA_MPPI_DYN_SINGLE_TRACK ? 2 : 1;
    int g = 1;
    while (g < 4 && (long long)p->K * g < waves * h->n_sms * 24 && R >= 2 * g) g *= 2;
    h->wps = g;
  }
  const size_t K = (size_t)p->K, TN = (size_t)p->T * h->nu;
  h->nb_upd = ramppi::update_blocks((long long)K);
  if (e == cudaSuccess) e = dalloc(&h->U, K * TN);
  if (e == cudaSuccess) e = dalloc(&h->S, K);
  if (e == cudaSuccess) e = dalloc(&h->cvar, K);
  if (e == cudaSuccess) e = dalloc(&h->S_tilde, K);
  if (e == cudaSuccess) e = dalloc(&h->partials, (size_t)h->nb_upd * (2 + TN));
  // kept risk costs [K][M], followed by the importance weights [K][M] when on
  // (also for the adjoint, which reads them instead of recomputing them)
  if (e == cudaSuccess && (p->flags & (RA_MPPI_KEEP_RISK_COSTS | RA_MPPI_DIFFERENTIABLE)))
    e = dalloc(&h->L, K * (size_t)p->M * (is_count(*p) > 0 ? 2 : 1));
  if (e == cudaSuccess) e = dalloc(&h->obs, (size_t)h->obs_cap);
  if (e == cudaSuccess) e = dalloc(&h->st, 1);
  if (e == cudaSuccess) e = dalloc(&h->x0_dev, 8);
  if (e == cudaSuccess) e = dalloc(&h->V_dev, TN);
  if (e == cudaSuccess) e = dalloc(&h->V_plus, TN);
  if (e == cudaSuccess && (p->flags & RA_MPPI_DIFFERENTIABLE)) {
    // the column reduction takes slices of 32 samples, at most 256 slices
    h->nb_red = (int)std::min<size_t>((K + 31) / 32, 256);
    e = dalloc(&h->keep_x0, 8);
    if (e == cudaSuccess) e = dalloc(&h->keep_V, TN);
    if (e == cudaSuccess) e = dalloc(&h->b_arrive, 2);
    if (e == cudaSuccess) e = dalloc(&h->b_dk, K);
    if (e == cudaSuccess) e = dalloc(&h->b_wk, K);
    if (e == cudaSuccess) e = dalloc(&h->b_Gnom, K * TN);
    if (e == cudaSuccess) e = dalloc(&h->b_mask, K * TN);
    if (e == cudaSuccess) e = dalloc(&h->b_gUd, K * TN);
    if (e == cudaSuccess) e = dalloc(&h->b_thn, K * 4);
    if (e == cudaSuccess) e = dalloc(&h->b_thd, K * 4);
    if (e == cudaSuccess) e = dalloc(&h->b_red, (size_t)h->nb_red * (3 * (TN + 4) + 1));
    // the forward's state checkpoints every 8 steps: nominal x_0, x_8, ...
    // and x_T; every disturbed rollout's x_0, x_8, ...
    const size_t nseg = ((size_t)p->T + 7) / 8;
    if (e == cudaSuccess) e = dalloc(&h->b_ck_nom, K * (nseg + 1) * h->nx);
    if (e == cudaSuccess) e = dalloc(&h->b_ck_dist, K * nseg * h->nx * (size_t)p->M);
    if (e == cudaSuccess) e = cudaMemset(h->b_arrive, 0, 2 * sizeof(unsigned int));
  }
  if (e == cudaSuccess) e = cudaMemset(h->st, 0, sizeof(DevState));
  if (e == cudaSuccess) e = cudaMemset(h->U, 0, sizeof(float) * K * TN);
  if (e == cudaSuccess) e = prepare(h);
  if (e != cudaSuccess) {
    const int code = (e == cudaErrorMemoryAllocation) ? RA_MPPI_ENOMEM : RA_MPPI_ECUDA;
    std::fprintf(stderr, "ra_mppi_create: %s\n", cudaGetErrorString(e));
    release(h);
    delete h;
    return code;
  }
  *out = h;
  return RA_MPPI_OK;
}

void ra_mppi_destroy(ra_mppi_t* h) {
  if (h == nullptr) return;
  DeviceScope scope(h->device);
  release(h);
  delete h;
}

int ra_mppi_set_obstacles(ra_mppi_t* h, const float* xyr, int32_t n_obs, void* stream) {
  if (h == nullptr) return RA_MPPI_EINVAL;
  RA_DEVICE_SCOPE(h);
  if (n_obs < 0 || n_obs > h->obs_cap) return fail(h, RA_MPPI_EINVAL, "n_obs exceeds max_obstacles");
  if (n_obs > 0 && xyr == nullptr) return fail(h, RA_MPPI_EINVAL, "xyr is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // packed as (x, y, r, r^2) so the indicator compares squared distances
  float4* host = nullptr;
  if (n_obs > 0) {
    host = static_cast<float4*>(std::malloc(sizeof(float4) * n_obs));
    if (host == nullptr) return fail(h, RA_MPPI_ENOMEM, "host buffer");
    float* tmp = static_cast<float*>(std::malloc(sizeof(float) * 3 * n_obs));
    if (tmp == nullptr) {
      std::free(host);
      return fail(h, RA_MPPI_ENOMEM, "host buffer");
    }
    cudaError_t e = cudaMemcpy(tmp, xyr, sizeof(float) * 3 * n_obs, cudaMemcpyDefault);
    if (e != cudaSuccess) {
      std::free(tmp);
      std::free(host);
      return cuda_fail(h, e, "set_obstacles copy");
    }
    for (int i = 0; i < n_obs; ++i) {
      const float r = tmp[3 * i + 2];
      if (!(r >= 0.0f) || !std::isfinite(tmp[3 * i]) || !std::isfinite(tmp[3 * i + 1])) {
        std::free(tmp);
        std::free(host);
        return fail(h, RA_MPPI_EINVAL, "obstacle radius must be >= 0 and centres finite");
      }
      if (!ramppi_api::obstacle_in_extent(tmp[3 * i], tmp[3 * i + 1], r)) {
        std::free(tmp);
        std::free(host);
        return fail(h, RA_MPPI_EINVAL, "obstacle disc outside |x|, |y| <= RA_MPPI_OBSTACLE_EXTENT");
      }
      host[i] = make_float4(tmp[3 * i], tmp[3 * i + 1], r, r * r);
    }
    std::free(tmp);
    // stored sorted by x: the kernels' obstacle cull narrows to an x window
    std::stable_sort(host, host + n_obs, [](const float4& u, const float4& v) { return u.x < v.x; });
    e = cudaMemcpyAsync(h->obs, host, sizeof(float4) * n_obs, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    std::free(host);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_obstacles upload");
  }
  const cudaError_t e = cudaMemcpyAsync(&h->st->n_obs, &n_obs, sizeof(int32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    const cudaError_t e2 = cudaStreamSynchronize(s);
    if (e2 != cudaSuccess) return cuda_fail(h, e2, "set_obstacles sync");
  } else {
    return cuda_fail(h, e, "set_obstacles count");
  }
  h->n_obs_host = n_obs;
  return RA_MPPI_OK;
}

int ra_mppi_step(ra_mppi_t* h, const float* x0, const float* V_in, float* V_out, float* S_tilde, float* cvar,
                 void* stream) {
  if (h == nullptr) return RA_MPPI_EINVAL;
  RA_DEVICE_SCOPE(h);
  if (x0 == nullptr || V_in == nullptr || V_out == nullptr) return fail(h, RA_MPPI_EINVAL, "x0, V_in and V_out are required");
  if (fault("launch")) return fail(h, RA_MPPI_ECUDA, "injected launch failure");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const ra_mppi_problem& p = h->prob;
  ramppi::RolloutArgs a{};
  a.x0 = x0;
  a.V = V_in;
  a.obs = h->obs;
  a.st = h->st;
  a.U = h->U;
  a.S = h->S;
  a.cvar = h->cvar;
  a.L = h->L;
  a.ck_nom = h->b_ck_nom;
  a.ck_dist = h->b_ck_dist;
  a.nb_nom = (p.K + 32 * h->warps - 1) / (32 * h->warps);
  a.obs_cap = h->obs_cap;
  a.wps = h->wps;
  const int spb = samples_per_block(h);
  int nb_dist = (p.K + spb - 1) / spb;
  tail_plan(h, nb_dist, &a.nb_head, &a.wps_tail, &nb_dist);
  const int grid = a.nb_nom + nb_dist;
  cudaError_t e;
  if (h->keep_x0 != nullptr) {
    e = cudaMemcpyAsync(h->keep_x0, x0, sizeof(float) * h->nx, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->keep_V, V_in, sizeof(float) * (size_t)p.T * h->nu, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "keep inputs");
  }
  if (h->ev_begin != nullptr) {
    e = cudaEventRecord(h->ev_begin, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "timing event");
  }
  switch (p.model) {
    case 0: e = ramppi::launch_rollout<0>(h->dp, a, h->warps, h->ilp, pairs_samples(h), importance(h), windowed(h), h->smem, grid, s); break;
    case 1: e = ramppi::launch_rollout<1>(h->dp, a, h->warps, h->ilp, pairs_samples(h), importance(h), windowed(h), h->smem, grid, s); break;
    default: e = ramppi::launch_rollout<2>(h->dp, a, h->warps, h->ilp, pairs_samples(h), importance(h), windowed(h), h->smem, grid, s); break;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "rollout launch");
  if (h->ev_end != nullptr) {
    e = cudaEventRecord(h->ev_end, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "timing event");
  }
  ramppi::UpdateArgs u{};
  u.S = h->S;
  u.cvar = h->cvar;
  u.U = h->U;
  u.S_tilde = S_tilde != nullptr ? S_tilde : h->S_tilde;
  u.V_out = V_out;
  u.partials = h->partials;
  u.st = h->st;
  e = ramppi::launch_update(h->dp, u, h->nb_upd, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "update launch");
  if (cvar != nullptr) {
    e = cudaMemcpyAsync(cvar, h->cvar, sizeof(float) * p.K, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "cvar copy");
  }
  return RA_MPPI_OK;
}

int ra_mppi_step_host(ra_mppi_t* h, const float* x0_host, const float* V_in_host, float* V_out_host,
                      float* S_tilde_host, void* stream) {
  if (h == nullptr) return RA_MPPI_EINVAL;
  RA_DEVICE_SCOPE(h);
  if (x0_host == nullptr || V_in_host == nullptr || V_out_host == nullptr)
    return fail(h, RA_MPPI_EINVAL, "x0, V_in and V_out are required");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t TN = (size_t)h->prob.T * h->nu;
  cudaError_t e = cudaMemcpyAsync(h->x0_dev, x0_host, sizeof(float) * h->nx, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->V_dev, V_in_host, sizeof(float) * TN, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "step_host upload");
  const int rc = ra_mppi_step(h, h->x0_dev, h->V_dev, h->V_dev, nullptr, nullptr, stream);
  if (rc != RA_MPPI_OK) return rc;
  e = cudaMemcpyAsync(V_out_host, h->V_dev, sizeof(float) * TN, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && S_tilde_host != nullptr)
    e = cudaMemcpyAsync(S_tilde_host, h->S_tilde, sizeof(float) * h->prob.K, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "step_host download");
  return RA_MPPI_OK;
}

int ra_mppi_closed_loop_step(ra_mppi_t* h, float* x, float* V, float* S_tilde, int32_t* collisions,
                             int32_t shift, void* stream) {
  if (h == nullptr) return RA_MPPI_EINVAL;
  RA_DEVICE_SCOPE(h);
  if (x == nullptr || V == nullptr) return fail(h, RA_MPPI_EINVAL, "x and V are required");
  const int rc = ra_mppi_step(h, x, V, h->V_plus, S_tilde, nullptr, stream);
  if (rc != RA_MPPI_OK) return rc;
  const cudaError_t e = ramppi::launch_plant(h->prob.model, h->dp, h->obs, h->st, x, h->V_plus, V, collisions,
                                             shift ? 1 : 0, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(h, e, "plant launch");
  return RA_MPPI_OK;
}

int ra_mppi_workspace(ra_mppi_t* h, const float** U, const float** S, const float** cvar, const float** L) {
  if (h == nullptr) return RA_MPPI_EINVAL;
  if (U) *U = h->U;
  if (S) *S = h->S;
  if (cvar) *cvar = h->cvar;
  if (L) *L = h->L;
  return RA_MPPI_OK;
}

int ra_mppi_copy_workspace(ra_mppi_t* h, float* U, float* S, float* cvar, float* L, void* stream) {
  if (h == nullptr) return RA_MPPI_EINVAL;
  RA_DEVICE_SCOPE(h);
  if (L != nullptr && h->L == nullptr) return fail(h, RA_MPPI_EINVAL, "risk costs were not kept");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t K = (size_t)h->prob.K;
  cudaError_t e = cudaSuccess;
  if (U) e = cudaMemcpyAsync(U, h->U, sizeof(float) * K * h->prob.T * h->nu, cudaMemcpyDefault, s);
  if (e == cudaSuccess && S) e = cudaMemcpyAsync(S, h->S, sizeof(float) * K, cudaMemcpyDefault, s);
  if (e == cudaSuccess && cvar) e = cudaMemcpyAsync(cvar, h->cvar, sizeof(float) * K, cudaMemcpyDefault, s);
  if (e == cudaSuccess && L) e = cudaMemcpyAsync(L, h->L, sizeof(float) * K * h->prob.M, cudaMemcpyDefault, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "copy_workspace");
  return RA_MPPI_OK;
}

int ra_mppi_copy_weights(ra_mppi_t* h, float* W, void* stream) {
  if (h == nullptr || W == nullptr) return RA_MPPI_EINVAL;
  RA_DEVICE_SCOPE(h);
  if (h->L == nullptr || !importance(h))
    return fail(h, RA_MPPI_EINVAL, "weights are kept only with RA_MPPI_KEEP_RISK_COSTS and importance sampling");
  const size_t KM = (size_t)h->prob.K * h->prob.M;
  const cudaError_t e = cudaMemcpyAsync(W, h->L + KM, sizeof(float) * KM, cudaMemcpyDefault,
                                        static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(h, e, "copy_weights");
  return RA_MPPI_OK;
}

int ra_mppi_get_state(ra_mppi_t* h, uint64_t* iteration) {
  if (h == nullptr || iteration == nullptr) return RA_MPPI_EINVAL;
  RA_DEVICE_SCOPE(h);
  unsigned long long it = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&it, &h->st->iteration, sizeof(it), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_state");
  *iteration = it;
  return RA_MPPI_OK;
}

int ra_mppi_set_state(ra_mppi_t* h, uint64_t iteration) {
  if (h == nullptr) return RA_MPPI_EINVAL;
  RA_DEVICE_SCOPE(h);
  const unsigned long long it = iteration;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&h->st->iteration, &it, sizeof(it), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_state");
  return RA_MPPI_OK;
}

int ra_mppi_get_status(ra_mppi_t* h) {
  if (h == nullptr) return RA_MPPI_EINVAL;
  RA_DEVICE_SCOPE(h);
  int status = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&status, &h->st->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(&h->st->status, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(h, e, "get_status");
  return status == 0 ? RA_MPPI_OK : RA_MPPI_ENONFINITE;
}

const char* ra_mppi_last_error(const ra_mppi_t* h) { return h == nullptr ? "null handle" : h->err.c_str(); }

int ra_mppi_set_launch(ra_mppi_t* h, int32_t warps_per_block, int32_t ilp, int32_t warps_per_sample) {
  if (h == nullptr) return RA_MPPI_EINVAL;
  RA_DEVICE_SCOPE(h);
  const int w = warps_per_block == 0 ? h->warps : warps_per_block;
  const int i = ilp == 0 ? h->ilp : ilp;
  const int g = warps_per_sample == 0 ? h->wps : warps_per_sample;
  if (w < 1 || w > 8) return fail(h, RA_MPPI_EINVAL, "warps_per_block must be in [1, 8]");
  if (i != 1 && i != 2 && i != 4) return fail(h, RA_MPPI_EINVAL, "ilp must be 1, 2 or 4");
  if (i == 4 && importance(h)) return fail(h, RA_MPPI_EINVAL, "importance-sampled rollouts interleave 1 or 2");
  if (i == 4 && differentiable(h)) return fail(h, RA_MPPI_EINVAL, "differentiable handles interleave 1 or 2");
  if (g < 1 || g > w || w % g != 0) return fail(h, RA_MPPI_EINVAL, "warps_per_sample must divide warps_per_block");
  const int old_w = h->warps, old_i = h->ilp, old_g = h->wps;
  h->warps = w;
  h->ilp = i;
  h->wps = g;
  const cudaError_t e = prepare(h);
  if (e != cudaSuccess) {
    h->warps = old_w;
    h->ilp = old_i;
    h->wps = old_g;
    prepare(h);
    return cuda_fail(h, e, "set_launch");
  }
  return RA_MPPI_OK;
}


int ra_mppi_get_launch_plan(ra_mppi_t* h, int32_t* grid, int32_t* nb_head, int32_t* wps_tail, int32_t* blocks_per_sm) {
  if (h == nullptr) return RA_MPPI_EINVAL;
  const int nb_nom = (h->prob.K + 32 * h->warps - 1) / (32 * h->warps);
  const int spb = samples_per_block(h);
  int nh = 0, wt = 0, nd = (h->prob.K + spb - 1) / spb;
  tail_plan(h, nd, &nh, &wt, &nd);
  if (grid) *grid = nb_nom + nd;
  if (nb_head) *nb_head = nh == 0x7FFFFFFF ? -1 : nh;
  if (wps_tail) *wps_tail = wt;
  if (blocks_per_sm) *blocks_per_sm = h->occ_blocks;
  return RA_MPPI_OK;
}

int ra_mppi_set_tail_split(ra_mppi_t* h, int32_t enable) {
  if (h == nullptr) return RA_MPPI_EINVAL;
  h->tail_split = enable != 0;
  return RA_MPPI_OK;
}

int ra_mppi_tune(ra_mppi_t* h, const float* x0, const float* V, int32_t replays, float* best_ms) {
  if (h == nullptr || x0 == nullptr || V == nullptr) return RA_MPPI_EINVAL;
  RA_DEVICE_SCOPE(h);
  if (replays < 1) replays = 3;
  unsigned long long saved_it = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&saved_it, &h->st->iteration, sizeof(saved_it), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "tune");
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_fail(h, e, "tune");
  const int R = (h->prob.M + 31) / 32;
  const int old_w = h->warps, old_i = h->ilp, old_g = h->wps;
  h->tail_split = true;
  int bw = old_w, bi = old_i, bg = old_g;
  float best = 1e30f;
  // warps per sample need not be a power of two: M = 300 has 10 rows of 32
  // rollouts, which 5 warps split into one interleaved pair each
  const int warps_c[] = {1, 2, 3, 4, 5, 6, 8};
  const int ilp_c[] = {1, 2, 4};
  const int wps_c[] = {1, 2, 3, 4, 5, 6, 8};
  for (int w : warps_c) {
    for (int il : ilp_c)
    for (int g : wps_c) {
      if (il == 4 && (importance(h) || differentiable(h))) continue;
      // shapes that leave a warp without a full set of interleaved rows add
      // nothing, except one row per sample, which two samples share (dynamic model)
      const bool sample_pairs = h->prob.model == RA_MPPI_DYN_SINGLE_TRACK && R == 1 && il == 2 && g == 1;
      if (g > w || w % g != 0 || (R < g * il && !sample_pairs)) continue;
      h->warps = w;
      h->ilp = il;
      h->wps = g;
      if (prepare(h) != cudaSuccess) continue;
      if (ra_mppi_step(h, x0, V, h->V_plus, nullptr, nullptr, s) != RA_MPPI_OK) continue;
      cudaEventRecord(e0, s);
      for (int r = 0; r < replays; ++r) ra_mppi_step(h, x0, V, h->V_plus, nullptr, nullptr, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) continue;
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= (float)replays;
      if (ms < best) {
        best = ms;
        bw = w;
        bi = il;
        bg = g;
      }
    }
  }
  h->warps = bw;
  h->ilp = bi;
  h->wps = bg;
  e = prepare(h);
  // the tail split at the chosen shape: keep it only if it is faster
  if (e == cudaSuccess) {
    int nh = 0, wt = 0, nt = 0;
    tail_plan(h, (h->prob.K + samples_per_block(h) - 1) / samples_per_block(h), &nh, &wt, &nt);
    if (nh != 0x7FFFFFFF) {
      float t_on = best, t_off = 1e30f;
      h->tail_split = false;
      if (ra_mppi_step(h, x0, V, h->V_plus, nullptr, nullptr, s) == RA_MPPI_OK) {
        cudaEventRecord(e0, s);
        for (int r = 0; r < replays; ++r) ra_mppi_step(h, x0, V, h->V_plus, nullptr, nullptr, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) == cudaSuccess) {
          cudaEventElapsedTime(&t_off, e0, e1);
          t_off /= (float)replays;
        }
      }
      h->tail_split = t_on <= t_off;
      if (!h->tail_split) best = t_off;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (e == cudaSuccess) e = cudaMemcpy(&h->st->iteration, &saved_it, sizeof(saved_it), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(h, e, "tune");
  if (best_ms) *best_ms = best;
  return RA_MPPI_OK;
}

int ra_mppi_get_launch(ra_mppi_t* h, int32_t* warps_per_block, int32_t* ilp, int32_t* warps_per_sample) {
  if (h == nullptr) return RA_MPPI_EINVAL;
  if (warps_per_block) *warps_per_block = h->warps;
  if (ilp) *ilp = h->ilp;
  if (warps_per_sample) *warps_per_sample = h->wps;
  return RA_MPPI_OK;
}

int ra_mppi_set_cost_weights(ra_mppi_t* h, const float* theta) {
  if (h == nullptr || theta == nullptr) return RA_MPPI_EINVAL;
  for (int i = 0; i < 4; ++i)
    if (!std::isfinite(theta[i])) return fail(h, RA_MPPI_EINVAL, "cost weights must be finite");
  h->prob.w_dev = h->dp.w_dev = theta[0];
  h->prob.w_speed = h->dp.w_speed = theta[1];
  h->prob.gamma = h->dp.gamma = theta[2];
  h->prob.w_obs = h->dp.w_obs = theta[3];
  return RA_MPPI_OK;
}

int ra_mppi_backward(ra_mppi_t* h, const float* gV_plus, const float* gS_tilde, float* gV, float* gtheta,
                     void* stream) {
  if (h == nullptr) return RA_MPPI_EINVAL;
  RA_DEVICE_SCOPE(h);
  if (gV_plus == nullptr || gV == nullptr || gtheta == nullptr)
    return fail(h, RA_MPPI_EINVAL, "gV_plus, gV and gtheta are required");
  if (h->keep_x0 == nullptr) return fail(h, RA_MPPI_EINVAL, "the problem was created without RA_MPPI_DIFFERENTIABLE");
  const ra_mppi_problem& p = h->prob;
  ramppi::BwdArgs a{};
  a.x0 = h->keep_x0;
  a.V = h->keep_V;
  a.U = h->U;
  a.S = h->S;
  a.cvar = h->cvar;
  a.L = h->L;
  a.ck_nom = h->b_ck_nom;
  a.ck_dist = h->b_ck_dist;
  a.obs = h->obs;
  a.st = h->st;
  a.gVp = gV_plus;
  a.gS = gS_tilde;
  a.arrive = h->b_arrive;
  a.dk = h->b_dk;
  a.wk = h->b_wk;
  a.Gnom = h->b_Gnom;
  a.mask = h->b_mask;
  a.gUd = h->b_gUd;
  a.thn = h->b_thn;
  a.thd = h->b_thd;
  a.red_part = h->b_red;
  a.gV = gV;
  a.gtheta = gtheta;
  constexpr int kBwdWarps = 4;
  a.nb_nom = (p.K + 32 * kBwdWarps - 1) / (32 * kBwdWarps);
  a.obs_cap = h->obs_cap;
  const int nb_dist = (p.K + kBwdWarps - 1) / kBwdWarps;
  // per warp: the steps of the segments being reversed (32 x 8 steps x
  // (2 nx + 2 nu): state, control, mean control, cost gradient),
  // then controls, risk costs, importance weights (when on), packed rollout
  // indices, U cotangents
  // (the U cotangents: a row per slot, 32 T nu floats, when T nu <= 128)
  const size_t TNb = (size_t)p.T * h->nu, gcap = TNb <= 128 ? 32 * TNb : TNb;
  const size_t smem = (size_t)h->obs_cap * sizeof(float4) + (size_t)kBwdWarps * 32 * 8 * (2 * h->nx + 2 * h->nu) * sizeof(float) +
                      (size_t)kBwdWarps * p.T * sizeof(float4) +
                      (size_t)kBwdWarps * (p.M * (importance(h) ? 3 : 2) + gcap) * sizeof(float);
  const cudaError_t e = ramppi::launch_backward(p.model, h->dp, a, nb_dist, smem, h->nb_red,
                                                static_cast<cudaStream_t>(stream), h->ev_begin, h->ev_end);
  if (e != cudaSuccess) return cuda_fail(h, e, "backward launch");
  return RA_MPPI_OK;
}

int ra_mppi_set_diagnostics(ra_mppi_t* h, unsigned long long* candidates) {
  if (h == nullptr) return RA_MPPI_EINVAL;
  h->dp.diag = candidates;
  return RA_MPPI_OK;
}

int ra_mppi_set_timing_events(ra_mppi_t* h, void* rollout_begin, void* rollout_end) {
  if (h == nullptr) return RA_MPPI_EINVAL;
  if ((rollout_begin == nullptr) != (rollout_end == nullptr))
    return fail(h, RA_MPPI_EINVAL, "set both timing events or neither");
  h->ev_begin = static_cast<cudaEvent_t>(rollout_begin);
  h->ev_end = static_cast<cudaEvent_t>(rollout_end);
  return RA_MPPI_OK;
}

}  // extern "C"
