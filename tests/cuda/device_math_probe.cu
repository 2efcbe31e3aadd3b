// Test-only: evaluates the library's own device math next to CUDA's on a
// grid of arguments (compiled and loaded by tests/test_device_math_gpu.py).
#include <cuda_runtime.h>

#include "ra_device.cuh"

namespace {

__global__ void probe(const float* z, int n, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = z[i];
  out[4 * i + 0] = ramppi::atan_poly(v);
  out[4 * i + 1] = atanf(v);
  ramppi::DevParams p{};
  p.pacejka_c15 = 1;
  out[4 * i + 2] = ramppi::Model<1>::pacejka_shape(p, v);
  out[4 * i + 3] = sinf(1.5f * atanf(v));
}

}  // namespace

extern "C" int device_math_probe(const float* z, int n, float* out) {
  probe<<<(n + 255) / 256, 256>>>(z, n, out);
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : -1;
}
