// Pipe-throughput probes: the peak rates that the rollout kernel's roofline
// divides by, measured on the device that runs it.  Each probe kernel runs
// eight independent dependency chains per thread of one instruction kind
// (FP32 fused multiply-add, its paired form, one special-function unit
// operation, an integer-to-float conversion, an integer multiply-add), on
// enough warps to cover every latency, so its time is set by the throughput
// of that instruction's pipe.  The special-function operations are written
// as single PTX instructions (rsqrt, cos, ex2, lg2, sin approximations),
// so each counts exactly one operation.  Nothing here is part of the
// RA-MPPI update.
#include <cuda_runtime.h>

#include "ra_host.h"
#include "ra_mppi.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSM = 4;
constexpr int kChains = 8;

// keeps the chains' results alive without writing them out
static __device__ float g_probe_sink[1];

template <int KIND>
__device__ __forceinline__ float probe_op(float x) {
  float y;
  if constexpr (KIND == 0) {
    y = __fmaf_rn(x, 0.999f, 1e-3f);
  } else if constexpr (KIND == 2) {
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  } else if constexpr (KIND == 3) {
    asm volatile("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  } else if constexpr (KIND == 4) {
    asm volatile("{ .reg .f32 t; neg.f32 t, %1; ex2.approx.ftz.f32 %0, t; }" : "=f"(y) : "f"(x));
  } else if constexpr (KIND == 5) {
    asm volatile("{ .reg .f32 t; abs.f32 t, %1; lg2.approx.ftz.f32 %0, t; }" : "=f"(y) : "f"(x));
  } else if constexpr (KIND == 6) {
    asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  } else if constexpr (KIND == 7) {
    asm volatile("{ .reg .u32 t; mov.b32 t, %1; cvt.rn.f32.u32 %0, t; }" : "=f"(y) : "f"(x));
  } else {
    unsigned u = __float_as_uint(x);
    asm volatile("mad.lo.u32 %0, %0, 1664525, 1013904223;" : "+r"(u));
    y = __uint_as_float(u);
  }
  return y;
}

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) pipe_probe_kernel(int iters, float seed) {
  if constexpr (KIND == 1) {
    float2 v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = make_float2(seed + c + threadIdx.x * 1e-3f, seed - c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) v[c] = __ffma2_rn(v[c], make_float2(0.999f, 0.999f), make_float2(1e-3f, 1e-3f));
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c].x + v[c].y;
    if (s == 1234.5678f) g_probe_sink[0] = s;
  } else {
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = seed + 0.37f * c + threadIdx.x * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) v[c] = probe_op<KIND>(v[c]);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == 1234.5678f) g_probe_sink[0] = s;
  }
}

template <int KIND>
cudaError_t run_probe(int grid, int iters, cudaStream_t s) {
  pipe_probe_kernel<KIND><<<grid, kProbeThreads, 0, s>>>(iters, 0.5f);
  return cudaGetLastError();
}

cudaError_t launch_probe(int kind, int grid, int iters, cudaStream_t s) {
  switch (kind) {
    case 0: return run_probe<0>(grid, iters, s);
    case 1: return run_probe<1>(grid, iters, s);
    case 2: return run_probe<2>(grid, iters, s);
    case 3: return run_probe<3>(grid, iters, s);
    case 4: return run_probe<4>(grid, iters, s);
    case 5: return run_probe<5>(grid, iters, s);
    case 6: return run_probe<6>(grid, iters, s);
    case 7: return run_probe<7>(grid, iters, s);
    default: return run_probe<8>(grid, iters, s);
  }
}

}  // namespace

extern "C" int ra_mppi_pipe_probe(int32_t kind, int32_t iters, int32_t device, float* ms, double* lane_ops) {
  if (kind < 0 || kind > 8 || iters < 1 || ms == nullptr || lane_ops == nullptr) return RA_MPPI_EINVAL;
  int dev = 0;
  cudaError_t e = cudaSuccess;
  if (!ramppi_api::resolve_device(device, &dev, &e)) return e == cudaSuccess ? RA_MPPI_EINVAL : RA_MPPI_ECUDA;
  ramppi_api::DeviceScope scope(dev);
  if (!scope.ok()) return RA_MPPI_ECUDA;
  int n_sms = 0;
  e = cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return RA_MPPI_ECUDA;
  const int grid = n_sms * kProbeBlocksPerSM;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = launch_probe(kind, grid, iters / 8 + 1, s);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) e = launch_probe(kind, grid, iters, s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (e != cudaSuccess) return RA_MPPI_ECUDA;
  *ms = t;
  *lane_ops = (double)grid * kProbeThreads * (double)iters * kChains * (kind == 1 ? 2.0 : 1.0);
  return RA_MPPI_OK;
}
