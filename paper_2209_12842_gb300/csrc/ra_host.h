// Host-side helpers shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>

namespace ramppi_api {

// Makes a handle's device current for the scope of an entry point and puts
// the caller's device back afterwards, so a handle can be driven from any
// current device.
class DeviceScope {
 public:
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev_) != cudaSuccess) {
      ok_ = false;
      return;
    }
    if (prev_ != dev) ok_ = cudaSetDevice(dev) == cudaSuccess;
    else prev_ = -1;
  }
  ~DeviceScope() {
    if (prev_ >= 0) cudaSetDevice(prev_);
  }
  DeviceScope(const DeviceScope&) = delete;
  DeviceScope& operator=(const DeviceScope&) = delete;
  bool ok() const { return ok_; }

 private:
  int prev_ = -1;
  bool ok_ = true;
};

// The device a create call binds a handle to: `device` itself, or the
// current device for -1.  EINVAL-worthy requests return false with *err 0;
// CUDA failures return false with *err set.
inline bool resolve_device(int device, int* dev, cudaError_t* err) {
  *err = cudaSuccess;
  if (device < -1) return false;
  int n = 0;
  *err = cudaGetDeviceCount(&n);
  if (*err == cudaSuccess && device < 0) *err = cudaGetDevice(&device);
  if (*err != cudaSuccess) return false;
  if (device >= n) return false;
  *dev = device;
  return true;
}

}  // namespace ramppi_api
