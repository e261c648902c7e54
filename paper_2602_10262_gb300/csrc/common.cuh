// Shared host/device helpers of libgb300fp8: status codes, the per-device
// error word, device properties.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gb300fp8.h"

namespace gb300 {

// Record the first device-side error in the error word (later errors keep
// the first one).
__device__ __forceinline__ void report_device_error(int* err_word, int code)
{
    if (err_word != nullptr)
        atomicCAS(err_word, 0, code);
}

// Address of the current device's error word (a __device__ variable of the
// library; resolved once per device with cudaGetSymbolAddress).  nullptr if
// the lookup failed.
int* device_error_word();

// SM count of the current device (cached per device).
int sm_count();

// True when the current device is an sm_103 part this library was built for.
bool device_supported();

inline bool aligned16(const void* p)
{
    return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

}  // namespace gb300

#define GB_CUDA_OK(expr)                       \
    do {                                       \
        cudaError_t e_ = (expr);               \
        if (e_ != cudaSuccess)                 \
            return FP8_ERR_CUDA;               \
    } while (0)
