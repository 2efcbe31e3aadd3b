// Test-only: one step of the dynamic model on a pair of states (float2,
// paired instructions) against two scalar steps (compiled and loaded by
// tests/test_device_math_gpu.py).  Each thread draws two states and a control
// from its random words and writes the scalar results next to the pair
// results; the test asserts equal bits.
#include <cuda_runtime.h>

#include "ra_device.cuh"
#include "ra_mppi.h"

// the library's own host-side parameter setup (libramppi.so)
namespace ramppi_api {
ramppi::DevParams make_params(const ra_mppi_problem& p);
}

namespace {

__global__ void pair_probe(const uint32_t* words, int n, ramppi::DevParams p, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t* w = words + 8 * i;
  float* o = out + 40 * i;
  using Md = ramppi::Model<1>;
  float xa[6], xb[6];
  float2 xx[6];
  for (int j = 0; j < 6; ++j) {
    xa[j] = 2.0f * ramppi::u01(w[j] ^ 0x9E3779B9u) - 1.0f;
    xb[j] = 2.0f * ramppi::u01(w[j] ^ 0x7F4A7C15u) - 1.0f;
  }
  // speeds from 0 to 4 m/s, some below the slip-angle floor; large slips in some lanes
  xa[3] = 4.0f * ramppi::u01(w[6]);
  xb[3] = 4.0f * ramppi::u01(w[7]);
  for (int j = 0; j < 6; ++j) xx[j] = make_float2(xa[j], xb[j]);
  const float4 c = Md::ctl(p, 0.4f * (2.0f * ramppi::u01(w[6] ^ w[7]) - 1.0f), 2.0f * ramppi::u01(w[7]) - 1.0f);
  Md::step(p, xa, c);
  Md::step(p, xb, c);
  Md::step2(p, xx, c);
  for (int j = 0; j < 6; ++j) {
    o[j] = xa[j];
    o[6 + j] = xb[j];
    o[12 + j] = xx[j].x;
    o[18 + j] = xx[j].y;
  }
  // the Pacejka shape and one derivative evaluation, scalar and paired
  {
    const float za = 60.0f * ramppi::u01(w[0]) - 30.0f, zb = 60.0f * ramppi::u01(w[1]) - 30.0f;
    o[24] = Md::pacejka<float>(p, za);
    o[25] = Md::pacejka<float>(p, zb);
    const float2 pz = Md::pacejka<float2>(p, make_float2(za, zb));
    o[26] = pz.x;
    o[27] = pz.y;
    float da[6], db[6];
    float2 d2[6];
    float ya[6], yb[6];
    float2 y2[6];
    for (int j = 0; j < 6; ++j) {
      ya[j] = 2.0f * ramppi::u01(w[j] ^ 0x12345678u) - 1.0f;
      yb[j] = 2.0f * ramppi::u01(w[j] ^ 0x0badf00du) - 1.0f;
    }
    ya[3] += 2.0f;
    yb[3] += 2.0f;
    for (int j = 0; j < 6; ++j) y2[j] = make_float2(ya[j], yb[j]);
    Md::deriv<float>(p, ya, c, da);
    Md::deriv<float>(p, yb, c, db);
    Md::deriv<float2>(p, y2, c, d2);
    for (int j = 0; j < 6; ++j) {
      o[32 + j] = (__float_as_uint(da[j]) == __float_as_uint(d2[j].x)) ? 0.0f : 1.0f;
    }
  }
}

}  // namespace

extern "C" int pair_probe_run(const uint32_t* words, int n, const ra_mppi_problem* prob, float* out) {
  const ramppi::DevParams p = ramppi_api::make_params(*prob);
  pair_probe<<<(n + 127) / 128, 128>>>(words, n, p, out);
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : -1;
}
