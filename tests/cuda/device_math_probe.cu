// Test-only: evaluates the library's own device math next to CUDA's on a
// grid of arguments (compiled and loaded by tests/test_device_math_gpu.py).
#include <cuda_runtime.h>

#include "ra_device.cuh"

namespace {

constexpr int kOut = 10;

__global__ void probe(const float* z, int n, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = z[i];
  float* o = out + kOut * i;
  o[0] = ramppi::atan_poly(v);
  o[1] = atanf(v);
  ramppi::DevParams p{};
  p.pacejka_c15 = 1;
  p.mp[4] = 10.0f;  // B
  // 1/sqrt(2): the factor the host folds into the axle constants
  o[2] = __fmul_rn(ramppi::Model<1>::pacejka(p, v), 0.70710678118654752f);
  o[3] = sinf(1.5f * atanf(v));
  // the paired arctangent: the general path whenever a lane of the warp has
  // an argument above 1, the fast one when the whole warp is within [-1, 1]
  float a, b;
  ramppi::atan_pair(v, 0.5f, &a, &b);
  o[4] = a;
  const float w = fminf(fmaxf(v, -1.0f), 1.0f);
  ramppi::atan_pair(w, w, &a, &b);
  o[5] = a;
  o[6] = ramppi::atan_poly(w);
  o[7] = b;
  // both axles' Pacejka arguments at B = 10, B steer = 0.25
  float zf, zr;
  ramppi::pacejka_args(p, v, 0.5f, 0.25f, &zf, &zr);
  o[8] = zf;
  o[9] = zr;
}

}  // namespace

extern "C" int device_math_probe(const float* z, int n, float* out) {
  probe<<<(n + 255) / 256, 256>>>(z, n, out);
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : -1;
}
