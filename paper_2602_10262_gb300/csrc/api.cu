// Status strings, the device error word and device queries of the C ABI.
#include <mutex>

#include "common.cuh"

namespace gb300 {

namespace {
constexpr int kMaxDevices = 64;

__device__ int g_error_word;
__device__ float g_one = 1.0f;

struct DeviceInfo {
    std::once_flag once;
    int* err = nullptr;
    float* one = nullptr;
    int sms = 0;
    int l2_bytes = 0;
    int major = 0, minor = 0;
};
DeviceInfo g_dev[kMaxDevices];

DeviceInfo* info()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return nullptr;
    DeviceInfo* d = &g_dev[dev];
    std::call_once(d->once, [d, dev] {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_error_word) == cudaSuccess)
            d->err = static_cast<int*>(p);
        if (cudaGetSymbolAddress(&p, g_one) == cudaSuccess)
            d->one = static_cast<float*>(p);
        cudaDeviceGetAttribute(&d->sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&d->l2_bytes, cudaDevAttrL2CacheSize, dev);
        cudaDeviceGetAttribute(&d->major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&d->minor, cudaDevAttrComputeCapabilityMinor, dev);
    });
    return d;
}
}  // namespace

int* device_error_word()
{
    DeviceInfo* d = info();
    return d ? d->err : nullptr;
}

const float* device_one()
{
    DeviceInfo* d = info();
    return d ? d->one : nullptr;
}

int sm_count()
{
    DeviceInfo* d = info();
    return d ? d->sms : 0;
}

long long l2_bytes()
{
    DeviceInfo* d = info();
    return d ? d->l2_bytes : 0;
}

bool device_supported()
{
    DeviceInfo* d = info();
    return d && d->err && d->major == 10 && d->minor == 3;
}

}  // namespace gb300

extern "C" const char* fp8_status_string(int status)
{
    switch (status) {
    case FP8_OK: return "ok";
    case FP8_PENDING: return "pending";
    case FP8_ERR_INVALID: return "invalid argument";
    case FP8_ERR_SHAPE: return "unsupported or inconsistent shape";
    case FP8_ERR_ALIGN: return "alignment requirement violated";
    case FP8_ERR_NONFINITE: return "non-finite input";
    case FP8_ERR_OOM: return "not enough free device memory";
    case FP8_ERR_CUDA: return "CUDA runtime error";
    case FP8_ERR_TIMEOUT: return "device pipeline wait timed out";
    case FP8_ERR_UNSUPPORTED: return "unsupported device or feature";
    default: return "unknown status";
    }
}

extern "C" int fp8_last_device_error(fp8_stream_t stream)
{
    int* w = gb300::device_error_word();
    if (!w)
        return FP8_ERR_UNSUPPORTED;
    GB_CUDA_OK(cudaStreamSynchronize(stream));
    int v = 0;
    GB_CUDA_OK(cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost));
    if (v != 0) {
        const int zero = 0;
        GB_CUDA_OK(cudaMemcpy(w, &zero, sizeof(int), cudaMemcpyHostToDevice));
        gb300::reset_split_counters();
    }
    return v;
}

extern "C" int fp8_device_sm_count(void)
{
    return gb300::sm_count();
}
