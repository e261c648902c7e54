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

// Address of a device float holding 1.0 on the current device (scale
// operand of products that carry no per-row scales); nullptr if the lookup
// failed.
const float* device_one();

// SM count of the current device (cached per device).
int sm_count();

// L2 capacity of the current device in bytes (0 if unknown).
long long l2_bytes();

// True when the current device is an sm_103 part this library was built for.
bool device_supported();

// Re-zero the split-K tile counters of every persistent workspace on the
// current device (per-stream caches and grouped graphs).  Called after the
// device error word was found set: a launch that stopped early may have left
// a counter part-way.  Synchronises the device.
void reset_split_counters();

// Programmatic dependent launch.  A grid launched with programmatic stream
// serialization may start before the previous grid on its stream ends; it
// must pass grid_dependency_wait (which returns once those grids have
// completed and their memory is visible; at once for a grid launched
// without the attribute) before it reads or writes global memory they use.
__device__ __forceinline__ void grid_dependency_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Lets grids launched after this one with programmatic serialization begin
// (their setup overlaps this grid's tail) once every CTA of this grid has
// executed it or exited.  It does not release them past their
// grid_dependency_wait.
__device__ __forceinline__ void grid_launch_dependents()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

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
