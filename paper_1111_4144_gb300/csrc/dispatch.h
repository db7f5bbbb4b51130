// Entry points of the per-dtype translation units, called by api.cu.
#pragma once

#include <cuda_runtime.h>

namespace cholinv {

struct BatchParams;

struct DeviceInfo {
    int sms = 0;
};
DeviceInfo device_info();  // defined in api.cu

cudaError_t launch_batched_f32(const BatchParams& p, cudaStream_t s, bool dry);
cudaError_t launch_batched_f64(const BatchParams& p, cudaStream_t s, bool dry);
cudaError_t launch_batched_c64(const BatchParams& p, cudaStream_t s, bool dry);
cudaError_t launch_batched_c128(const BatchParams& p, cudaStream_t s, bool dry);

}  // namespace cholinv
