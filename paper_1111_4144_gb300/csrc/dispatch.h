// Entry points of the per-dtype translation units, called by api.cu.
#pragma once

#include <cuda_runtime.h>

namespace cholinv {

struct BatchParams;

struct DeviceInfo {
    int sms = 0;
};
DeviceInfo device_info();  // defined in api.cu

// Launch the kernel of size class `cls` (matrices of order cls; at most
// `upper` of them) on stream s.  dry = true only performs the kernel's
// one-time set-up (before a stream capture) and launches nothing.
cudaError_t launch_class_f32(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_class_f64(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_class_c64(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);
cudaError_t launch_class_c128(const BatchParams& p, int cls, int upper, cudaStream_t s, bool dry);

}  // namespace cholinv
