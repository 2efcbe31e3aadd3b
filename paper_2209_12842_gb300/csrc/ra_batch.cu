// C ABI of the batched path (declarations and contracts in include/ra_mppi.h):
// packed buffers, per-problem descriptors, the ordered work list, the
// captured graph and the launch-shape tuner.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "ra_host.h"
#include "ra_kernels.h"
#include "ra_mppi.h"

using ramppi::BatchArgs;
using ramppi::BatchUpdateArgs;
using ramppi::DevParams;
using ramppi::DevState;
using ramppi::InstDesc;

// defined in ra_api.cu
namespace ramppi_api {
std::string validate_problem(const ra_mppi_problem& p);
DevParams make_params(const ra_mppi_problem& p);
bool obstacle_in_extent(float x, float y, float r);
}  // namespace ramppi_api

struct ra_mppi_batch {
  ra_mppi_problem common;
  DevParams dp;
  int device = 0;
  cudaEvent_t ev_begin = nullptr, ev_end = nullptr;  // optional timing hook (eager launches)
  int B = 0, nx = 0, nu = 0;
  std::vector<InstDesc> desc_h;
  InstDesc* desc = nullptr;
  DevState* st = nullptr;
  float* x0 = nullptr;
  float* V = nullptr;
  float* V_out = nullptr;
  float4* obs = nullptr;
  float* U = nullptr;
  float* S = nullptr;
  float* cvar = nullptr;
  float* S_tilde = nullptr;
  float* partials = nullptr;
  long long* seg_base = nullptr;
  int* seg_inst = nullptr;
  unsigned long long* queue = nullptr;
  long long n_items = 0, n_x0 = 0, n_V = 0, n_U = 0, n_k = 0, n_obs = 0, n_part = 0;
  int obs_cap_max = 0, T_max = 0, M_max = 0, upd_blocks = 0;
  int warps = 4, ilp = 1, blocks_per_sm = 1, n_sms = 1;
  bool is = false;  // importance-sampled rollouts
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::string err;
};

namespace {

int bfail(ra_mppi_batch* b, int code, const std::string& msg) {
  if (b) b->err = msg;
  return code;
}

int bcuda(ra_mppi_batch* b, cudaError_t e, const char* where) {
  return bfail(b, RA_MPPI_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define RA_BATCH_DEVICE_SCOPE(b)                            \
  ramppi_api::DeviceScope device_scope_((b)->device);       \
  if (!device_scope_.ok()) return bfail((b), RA_MPPI_ECUDA, "cannot make the handle's device current")

template <typename T>
cudaError_t balloc(T** p, long long n) {
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)(n > 0 ? n : 1));
}

void release(ra_mppi_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  cudaFree(b->desc);
  cudaFree(b->st);
  cudaFree(b->x0);
  cudaFree(b->V);
  cudaFree(b->V_out);
  cudaFree(b->obs);
  cudaFree(b->U);
  cudaFree(b->S);
  cudaFree(b->cvar);
  cudaFree(b->S_tilde);
  cudaFree(b->partials);
  cudaFree(b->seg_base);
  cudaFree(b->seg_inst);
  cudaFree(b->queue);
}

size_t batch_smem(const ra_mppi_batch* b) {
  return (size_t)b->warps * ramppi::batch_warp_f4(b->obs_cap_max, b->T_max, b->M_max, b->is) * sizeof(float4);
}

// per-kernel dynamic shared-memory limit, shared by all batches: only raised
std::mutex g_bsmem_mutex;
size_t g_bsmem_limit[64][3] = {};  // per device, per model

cudaError_t raise_limit(int model, size_t smem) {
  const int m = model < 0 || model > 2 ? 2 : model;
  std::lock_guard<std::mutex> lock(g_bsmem_mutex);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (smem <= g_bsmem_limit[dev][m]) return cudaSuccess;
  cudaError_t e;
  switch (m) {
    case 0: e = ramppi::prepare_batch_rollout<0>(smem); break;
    case 1: e = ramppi::prepare_batch_rollout<1>(smem); break;
    default: e = ramppi::prepare_batch_rollout<2>(smem); break;
  }
  if (e == cudaSuccess) g_bsmem_limit[dev][m] = smem;
  return e;
}

cudaError_t prepare(ra_mppi_batch* b) {
  const size_t smem = batch_smem(b);
  cudaError_t e = raise_limit(b->common.model, smem);
  if (e != cudaSuccess) return e;
  int bps = 0;
  switch (b->common.model) {
    case 0:
      e = ramppi::batch_rollout_occupancy<0>(b->warps, b->ilp, b->is, smem, &bps);
      break;
    case 1:
      e = ramppi::batch_rollout_occupancy<1>(b->warps, b->ilp, b->is, smem, &bps);
      break;
    default:
      e = ramppi::batch_rollout_occupancy<2>(b->warps, b->ilp, b->is, smem, &bps);
      break;
  }
  if (e != cudaSuccess) return e;
  if (bps < 1) return cudaErrorInvalidConfiguration;
  b->blocks_per_sm = bps;
  return cudaSuccess;
}

BatchArgs rollout_args(const ra_mppi_batch* b) {
  BatchArgs a{};
  a.desc = b->desc;
  a.st = b->st;
  a.B = b->B;
  a.x0 = b->x0;
  a.V = b->V;
  a.obs = b->obs;
  a.U = b->U;
  a.S = b->S;
  a.cvar = b->cvar;
  a.seg_base = b->seg_base;
  a.seg_inst = b->seg_inst;
  a.n_items = b->n_items;
  a.queue = b->queue;
  a.obs_cap_max = b->obs_cap_max;
  a.T_max = b->T_max;
  a.M_max = b->M_max;
  return a;
}

// queue reset, persistent rollout launch and batched update on stream s
// (timed: the timing hook's events around the rollout launch)
cudaError_t enqueue(ra_mppi_batch* b, cudaStream_t s, bool timed = false) {
  cudaError_t e = cudaMemsetAsync(b->queue, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const BatchArgs a = rollout_args(b);
  const size_t smem = batch_smem(b);
  const int grid = b->blocks_per_sm * b->n_sms;
  if (timed && b->ev_begin != nullptr) {
    e = cudaEventRecord(b->ev_begin, s);
    if (e != cudaSuccess) return e;
  }
  switch (b->common.model) {
    case 0: e = ramppi::launch_batch_rollout<0>(b->dp, a, b->warps, b->ilp, b->is, smem, grid, s); break;
    case 1: e = ramppi::launch_batch_rollout<1>(b->dp, a, b->warps, b->ilp, b->is, smem, grid, s); break;
    default: e = ramppi::launch_batch_rollout<2>(b->dp, a, b->warps, b->ilp, b->is, smem, grid, s); break;
  }
  if (e != cudaSuccess) return e;
  if (timed && b->ev_end != nullptr) {
    e = cudaEventRecord(b->ev_end, s);
    if (e != cudaSuccess) return e;
  }
  BatchUpdateArgs u{};
  u.desc = b->desc;
  u.B = b->B;
  u.st = b->st;
  u.S = b->S;
  u.cvar = b->cvar;
  u.U = b->U;
  u.S_tilde = b->S_tilde;
  u.V_out = b->V_out;
  u.partials = b->partials;
  return ramppi::launch_batch_update(b->dp, u, b->upd_blocks, s);
}

cudaError_t capture(ra_mppi_batch* b) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const cudaError_t e_enq = enqueue(b, b->cap);
  e = cudaStreamEndCapture(b->cap, &b->graph);
  if (e_enq != cudaSuccess) return e_enq;
  if (e != cudaSuccess) return e;
  return cudaGraphInstantiate(&b->exec, b->graph, 0);
}

}  // namespace

extern "C" {

int ra_mppi_batch_create(const ra_mppi_problem* common, const ra_mppi_instance* inst, int32_t B, int32_t device,
                         ra_mppi_batch_t** out) {
  if (common == nullptr || inst == nullptr || out == nullptr || B < 1 || B > 65536) return RA_MPPI_EINVAL;
  // every problem must be valid as a single problem
  for (int i = 0; i < B; ++i) {
    ra_mppi_problem p = *common;
    p.K = inst[i].K;
    p.M = inst[i].M;
    p.T = inst[i].T;
    p.max_obstacles = inst[i].max_obstacles;
    const std::string why = ramppi_api::validate_problem(p);
    if (!why.empty()) {
      std::fprintf(stderr, "ra_mppi_batch_create: problem %d: %s\n", i, why.c_str());
      return RA_MPPI_EINVAL;
    }
  }
  int dev = 0;
  {
    cudaError_t e0 = cudaSuccess;
    if (!ramppi_api::resolve_device(device, &dev, &e0)) {
      if (e0 == cudaSuccess) return RA_MPPI_EINVAL;
      std::fprintf(stderr, "ra_mppi_batch_create: %s\n", cudaGetErrorString(e0));
      return RA_MPPI_ECUDA;
    }
  }
  ramppi_api::DeviceScope scope(dev);
  if (!scope.ok()) return RA_MPPI_ECUDA;
  ra_mppi_batch* b = new (std::nothrow) ra_mppi_batch();
  if (b == nullptr) return RA_MPPI_ENOMEM;
  b->device = dev;
  b->common = *common;
  b->dp = ramppi_api::make_params(*common);
  b->is = common->is_scale != 1.0f && common->is_frac > 0.0f;
  b->B = B;
  b->nx = common->model == RA_MPPI_KIN_BICYCLE ? 4 : common->model == RA_MPPI_DYN_SINGLE_TRACK ? 6 : 1;
  b->nu = common->model == RA_MPPI_LINEAR_TEST ? 1 : 2;
  // descriptors and packed offsets
  b->desc_h.resize(B);
  std::vector<double> cost(B);
  long long x0o = 0, Vo = 0, Uo = 0, ko = 0, oo = 0, po = 0;
  int ub = 0;
  for (int i = 0; i < B; ++i) {
    ra_mppi_problem p = *common;
    p.K = inst[i].K;
    p.M = inst[i].M;
    p.T = inst[i].T;
    p.seed = inst[i].seed;
    p.instance_id = inst[i].instance_id;
    const DevParams d = ramppi_api::make_params(p);
    InstDesc& q = b->desc_h[i];
    q.K = d.K;
    q.M = d.M;
    q.T = d.T;
    q.n_warm = d.n_warm;
    q.j_var = d.j_var;
    q.frac_j = d.frac_j;
    q.tail_denom = d.tail_denom;
    q.instance = d.instance;
    q.seed_lo = d.seed_lo;
    q.seed_hi = d.seed_hi;
    q.obs_cap = inst[i].max_obstacles;
    q.is_m0 = d.is_m0;
    q.is_b = d.is_b;
    q.is_base = d.is_base;
    q.nb_upd = ramppi::update_blocks(q.K);
    q.upd_block_base = ub;
    q.x0_off = x0o;
    q.V_off = Vo;
    q.U_off = Uo;
    q.k_off = ko;
    q.obs_off = oo;
    q.part_off = po;
    const long long TN = (long long)q.T * b->nu;
    x0o += b->nx;
    Vo += TN;
    Uo += (long long)q.K * TN;
    ko += q.K;
    oo += q.obs_cap;
    po += (long long)q.nb_upd * (2 + TN);
    ub += q.nb_upd;
    b->obs_cap_max = std::max(b->obs_cap_max, q.obs_cap);
    b->T_max = std::max(b->T_max, q.T);
    b->M_max = std::max(b->M_max, q.M);
    // relative cost of one disturbed sample: rollouts per lane x steps x per-step work
    cost[i] = (double)((q.M + 31) / 32) * q.T * (40.0 + 6.0 * q.obs_cap) * (common->substeps);
  }
  b->n_x0 = x0o;
  b->n_V = Vo;
  b->n_U = Uo;
  b->n_k = ko;
  b->n_obs = oo;
  b->n_part = po;
  b->upd_blocks = ub;
  // work list: nominal segments in problem order, then disturbed segments
  // in decreasing per-sample cost
  std::vector<int> order(B);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<long long> seg_base(2 * B + 1);
  std::vector<int> seg_inst(2 * B);
  long long items = 0;
  for (int s = 0; s < 2 * B; ++s) {
    const int i = s < B ? s : order[s - B];
    seg_inst[s] = i;
    seg_base[s] = items;
    items += s < B ? (b->desc_h[i].K + 31) / 32 : b->desc_h[i].K;
  }
  seg_base[2 * B] = items;
  b->n_items = items;

  cudaError_t e = cudaDeviceGetAttribute(&b->n_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = balloc(&b->desc, B);
  if (e == cudaSuccess) e = balloc(&b->st, B);
  if (e == cudaSuccess) e = balloc(&b->x0, b->n_x0);
  if (e == cudaSuccess) e = balloc(&b->V, b->n_V);
  if (e == cudaSuccess) e = balloc(&b->V_out, b->n_V);
  if (e == cudaSuccess) e = balloc(&b->obs, b->n_obs);
  if (e == cudaSuccess) e = balloc(&b->U, b->n_U);
  if (e == cudaSuccess) e = balloc(&b->S, b->n_k);
  if (e == cudaSuccess) e = balloc(&b->cvar, b->n_k);
  if (e == cudaSuccess) e = balloc(&b->S_tilde, b->n_k);
  if (e == cudaSuccess) e = balloc(&b->partials, b->n_part);
  if (e == cudaSuccess) e = balloc(&b->seg_base, 2 * B + 1);
  if (e == cudaSuccess) e = balloc(&b->seg_inst, 2 * B);
  if (e == cudaSuccess) e = balloc(&b->queue, 1);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->desc, b->desc_h.data(), sizeof(InstDesc) * B, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->seg_base, seg_base.data(), sizeof(long long) * (2 * B + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->seg_inst, seg_inst.data(), sizeof(int) * 2 * B, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->st, 0, sizeof(DevState) * B);
  if (e == cudaSuccess) e = cudaMemset(b->x0, 0, sizeof(float) * b->n_x0);
  if (e == cudaSuccess) e = cudaMemset(b->V, 0, sizeof(float) * b->n_V);
  if (e == cudaSuccess) e = cudaMemset(b->V_out, 0, sizeof(float) * b->n_V);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  // default launch shape: 4 warps per block; the kinematic model interleaves 2 rollouts
  b->warps = 4;
  b->ilp = common->model == RA_MPPI_KIN_BICYCLE ? 2 : 1;
  if (e == cudaSuccess) e = prepare(b);
  if (e == cudaSuccess) e = capture(b);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "ra_mppi_batch_create: %s\n", cudaGetErrorString(e));
    const int code = e == cudaErrorMemoryAllocation ? RA_MPPI_ENOMEM : RA_MPPI_ECUDA;
    release(b);
    delete b;
    return code;
  }
  *out = b;
  return RA_MPPI_OK;
}

void ra_mppi_batch_destroy(ra_mppi_batch_t* b) {
  if (b == nullptr) return;
  ramppi_api::DeviceScope scope(b->device);
  release(b);
  delete b;
}

int ra_mppi_batch_layout(ra_mppi_batch_t* b, int64_t* offsets) {
  if (b == nullptr || offsets == nullptr) return RA_MPPI_EINVAL;
  for (int i = 0; i < b->B; ++i) {
    const InstDesc& q = b->desc_h[i];
    offsets[4 * i + 0] = q.x0_off;
    offsets[4 * i + 1] = q.V_off;
    offsets[4 * i + 2] = q.k_off;
    offsets[4 * i + 3] = q.U_off;
  }
  return RA_MPPI_OK;
}

int ra_mppi_batch_buffers(ra_mppi_batch_t* b, float** x0, float** V, float** V_out, float** S_tilde) {
  if (b == nullptr) return RA_MPPI_EINVAL;
  if (x0) *x0 = b->x0;
  if (V) *V = b->V;
  if (V_out) *V_out = b->V_out;
  if (S_tilde) *S_tilde = b->S_tilde;
  return RA_MPPI_OK;
}

int ra_mppi_batch_io(ra_mppi_batch_t* b, float** x0_packed, float** V_packed, int64_t* offsets) {
  if (b == nullptr) return RA_MPPI_EINVAL;
  if (x0_packed) *x0_packed = b->x0;
  if (V_packed) *V_packed = b->V;
  return offsets != nullptr ? ra_mppi_batch_layout(b, offsets) : RA_MPPI_OK;
}

int ra_mppi_batch_set_obstacles(ra_mppi_batch_t* b, int32_t i, const float* xyr, int32_t n_obs, void* stream) {
  if (b == nullptr || i < 0 || i >= b->B) return RA_MPPI_EINVAL;
  RA_BATCH_DEVICE_SCOPE(b);
  const InstDesc& q = b->desc_h[i];
  if (n_obs < 0 || n_obs > q.obs_cap) return bfail(b, RA_MPPI_EINVAL, "n_obs exceeds the problem's max_obstacles");
  if (n_obs > 0 && xyr == nullptr) return bfail(b, RA_MPPI_EINVAL, "xyr is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<float> tmp(3 * (size_t)n_obs);
  std::vector<float4> packed(n_obs);
  cudaError_t e = cudaSuccess;
  if (n_obs > 0) e = cudaMemcpy(tmp.data(), xyr, sizeof(float) * 3 * n_obs, cudaMemcpyDefault);
  if (e != cudaSuccess) return bcuda(b, e, "batch_set_obstacles copy");
  for (int o = 0; o < n_obs; ++o) {
    const float r = tmp[3 * o + 2];
    if (!(r >= 0.0f) || !std::isfinite(tmp[3 * o]) || !std::isfinite(tmp[3 * o + 1]))
      return bfail(b, RA_MPPI_EINVAL, "obstacle radius must be >= 0 and centres finite");
    if (!ramppi_api::obstacle_in_extent(tmp[3 * o], tmp[3 * o + 1], r))
      return bfail(b, RA_MPPI_EINVAL, "obstacle disc outside |x|, |y| <= RA_MPPI_OBSTACLE_EXTENT");
    packed[o] = make_float4(tmp[3 * o], tmp[3 * o + 1], r, r * r);
  }
  // stored sorted by x: the kernels' obstacle cull narrows to an x window
  std::stable_sort(packed.begin(), packed.end(), [](const float4& u, const float4& v) { return u.x < v.x; });
  if (n_obs > 0)
    e = cudaMemcpyAsync(b->obs + q.obs_off, packed.data(), sizeof(float4) * n_obs, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&b->st[i].n_obs, &n_obs, sizeof(int32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bcuda(b, e, "batch_set_obstacles upload");
  return RA_MPPI_OK;
}

int ra_mppi_batch_write_inputs(ra_mppi_batch_t* b, const float* x0, const float* V, void* stream) {
  if (b == nullptr) return RA_MPPI_EINVAL;
  RA_BATCH_DEVICE_SCOPE(b);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (x0) e = cudaMemcpyAsync(b->x0, x0, sizeof(float) * b->n_x0, cudaMemcpyDefault, s);
  if (e == cudaSuccess && V) e = cudaMemcpyAsync(b->V, V, sizeof(float) * b->n_V, cudaMemcpyDefault, s);
  if (e != cudaSuccess) return bcuda(b, e, "batch_write_inputs");
  return RA_MPPI_OK;
}

int ra_mppi_batch_read_outputs(ra_mppi_batch_t* b, float* V_out, float* S_tilde, void* stream) {
  if (b == nullptr) return RA_MPPI_EINVAL;
  RA_BATCH_DEVICE_SCOPE(b);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (V_out) e = cudaMemcpyAsync(V_out, b->V_out, sizeof(float) * b->n_V, cudaMemcpyDefault, s);
  if (e == cudaSuccess && S_tilde)
    e = cudaMemcpyAsync(S_tilde, b->S_tilde, sizeof(float) * b->n_k, cudaMemcpyDefault, s);
  if (e != cudaSuccess) return bcuda(b, e, "batch_read_outputs");
  return RA_MPPI_OK;
}

int ra_mppi_step_batched(ra_mppi_batch_t* b, void* stream) {
  if (b == nullptr) return RA_MPPI_EINVAL;
  RA_BATCH_DEVICE_SCOPE(b);
  const cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return bcuda(b, e, "graph launch");
  return RA_MPPI_OK;
}

int ra_mppi_step_batched_eager(ra_mppi_batch_t* b, void* stream) {
  if (b == nullptr) return RA_MPPI_EINVAL;
  RA_BATCH_DEVICE_SCOPE(b);
  const cudaError_t e = enqueue(b, static_cast<cudaStream_t>(stream), true);
  if (e != cudaSuccess) return bcuda(b, e, "batched launch");
  return RA_MPPI_OK;
}

int ra_mppi_batch_set_timing_events(ra_mppi_batch_t* b, void* rollout_begin, void* rollout_end) {
  if (b == nullptr) return RA_MPPI_EINVAL;
  if ((rollout_begin == nullptr) != (rollout_end == nullptr))
    return bfail(b, RA_MPPI_EINVAL, "set both timing events or neither");
  b->ev_begin = static_cast<cudaEvent_t>(rollout_begin);
  b->ev_end = static_cast<cudaEvent_t>(rollout_end);
  return RA_MPPI_OK;
}

int ra_mppi_batch_set_diagnostics(ra_mppi_batch_t* b, unsigned long long* candidates) {
  if (b == nullptr) return RA_MPPI_EINVAL;
  RA_BATCH_DEVICE_SCOPE(b);
  b->dp.diag = candidates;
  const cudaError_t e = capture(b);
  if (e != cudaSuccess) return bcuda(b, e, "batch_set_diagnostics");
  return RA_MPPI_OK;
}

int ra_mppi_batch_copy_workspace(ra_mppi_batch_t* b, float* U, float* S, float* cvar, void* stream) {
  if (b == nullptr) return RA_MPPI_EINVAL;
  RA_BATCH_DEVICE_SCOPE(b);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (U) e = cudaMemcpyAsync(U, b->U, sizeof(float) * b->n_U, cudaMemcpyDefault, s);
  if (e == cudaSuccess && S) e = cudaMemcpyAsync(S, b->S, sizeof(float) * b->n_k, cudaMemcpyDefault, s);
  if (e == cudaSuccess && cvar) e = cudaMemcpyAsync(cvar, b->cvar, sizeof(float) * b->n_k, cudaMemcpyDefault, s);
  if (e != cudaSuccess) return bcuda(b, e, "batch_copy_workspace");
  return RA_MPPI_OK;
}

int ra_mppi_batch_set_iteration(ra_mppi_batch_t* b, uint64_t iteration) {
  if (b == nullptr) return RA_MPPI_EINVAL;
  RA_BATCH_DEVICE_SCOPE(b);
  cudaError_t e = cudaDeviceSynchronize();
  const unsigned long long it = iteration;
  for (int i = 0; e == cudaSuccess && i < b->B; ++i)
    e = cudaMemcpy(&b->st[i].iteration, &it, sizeof(it), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bcuda(b, e, "batch_set_iteration");
  return RA_MPPI_OK;
}

int ra_mppi_batch_get_status(ra_mppi_batch_t* b) {
  if (b == nullptr) return RA_MPPI_EINVAL;
  RA_BATCH_DEVICE_SCOPE(b);
  std::vector<DevState> st(b->B);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(st.data(), b->st, sizeof(DevState) * b->B, cudaMemcpyDeviceToHost);
  int any = 0;
  for (int i = 0; i < b->B; ++i) {
    any |= st[i].status;
    st[i].status = 0;
  }
  if (e == cudaSuccess) e = cudaMemcpy(b->st, st.data(), sizeof(DevState) * b->B, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bcuda(b, e, "batch_get_status");
  return any == 0 ? RA_MPPI_OK : RA_MPPI_ENONFINITE;
}

int ra_mppi_batch_set_launch(ra_mppi_batch_t* b, int32_t warps_per_block, int32_t ilp) {
  if (b == nullptr) return RA_MPPI_EINVAL;
  RA_BATCH_DEVICE_SCOPE(b);
  if (warps_per_block < 1 || warps_per_block > 8) return bfail(b, RA_MPPI_EINVAL, "warps_per_block in [1, 8]");
  if (ilp != 1 && ilp != 2) return bfail(b, RA_MPPI_EINVAL, "ilp must be 1 or 2");
  const int ow = b->warps, oi = b->ilp;
  b->warps = warps_per_block;
  b->ilp = ilp;
  cudaError_t e = prepare(b);
  if (e == cudaSuccess) e = capture(b);
  if (e != cudaSuccess) {
    b->warps = ow;
    b->ilp = oi;
    prepare(b);
    capture(b);
    return bcuda(b, e, "batch_set_launch");
  }
  return RA_MPPI_OK;
}

int ra_mppi_batch_get_launch(ra_mppi_batch_t* b, int32_t* warps_per_block, int32_t* ilp, int32_t* grid) {
  if (b == nullptr) return RA_MPPI_EINVAL;
  if (warps_per_block) *warps_per_block = b->warps;
  if (ilp) *ilp = b->ilp;
  if (grid) *grid = b->blocks_per_sm * b->n_sms;
  return RA_MPPI_OK;
}

int ra_mppi_batch_tune(ra_mppi_batch_t* b, int32_t replays, float* best_ms) {
  if (b == nullptr) return RA_MPPI_EINVAL;
  RA_BATCH_DEVICE_SCOPE(b);
  if (replays < 1) replays = 3;
  // the tuner advances the update counters; put them back afterwards
  std::vector<DevState> saved(b->B);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(saved.data(), b->st, sizeof(DevState) * b->B, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return bcuda(b, e, "batch_tune");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bw = b->warps, bi = b->ilp;
  const int warps_c[] = {2, 4, 8};
  const int ilp_c[] = {1, 2};
  for (int w : warps_c) {
    for (int il : ilp_c) {
      b->warps = w;
      b->ilp = il;
      if (prepare(b) != cudaSuccess || capture(b) != cudaSuccess) continue;
      cudaGraphLaunch(b->exec, b->cap);
      cudaEventRecord(e0, b->cap);
      for (int r = 0; r < replays; ++r) cudaGraphLaunch(b->exec, b->cap);
      cudaEventRecord(e1, b->cap);
      if (cudaEventSynchronize(e1) != cudaSuccess) continue;
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= (float)replays;
      if (ms < best) {
        best = ms;
        bw = w;
        bi = il;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->warps = bw;
  b->ilp = bi;
  e = prepare(b);
  if (e == cudaSuccess) e = capture(b);
  if (e == cudaSuccess) e = cudaMemcpy(b->st, saved.data(), sizeof(DevState) * b->B, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bcuda(b, e, "batch_tune");
  if (best_ms) *best_ms = best;
  return RA_MPPI_OK;
}

const char* ra_mppi_batch_last_error(const ra_mppi_batch_t* b) { return b == nullptr ? "null handle" : b->err.c_str(); }

}  // extern "C"
