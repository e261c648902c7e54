// 2:4 prune + compress (prune24_compress) and its inverse.
//
// Vector path: a thread takes pieces of 16 input bytes (four groups of four
// codes): one 16-byte load, a branch-free rank selection for two groups at
// a time (packed 16-bit scores), an 8-byte store of the kept codes and a
// 2-byte store of the four metadata nibbles.  Rows whose length or
// alignment does not allow it fall back to one metadata byte per
// iteration.  Bandwidth-bound: 1 byte read, 0.625 bytes written per
// element; no allocation, one launch.
#include "common.cuh"
#include "prune_select.cuh"

namespace gb300 {
namespace {

constexpr int kThreads = 256;

// Vector path: K % 16 == 0, a 16-aligned with lda % 16 == 0, vals 8-aligned,
// meta 2-aligned.  blockIdx.y walks rows.  A thread takes kPieces pieces of
// 16 codes (four groups) spaced kThreads apart, so each load instruction of
// a warp reads 512 contiguous bytes; all loads are issued before any
// selection.  Per piece: 8 bytes of kept codes and 16 bits of metadata.
constexpr int kPieces = 4;

__global__ void __launch_bounds__(kThreads) prune24_vec_kernel(const uint8_t* __restrict__ a,
                                                               int64_t M, int64_t K, int64_t lda,
                                                               uint8_t* __restrict__ vals,
                                                               uint8_t* __restrict__ meta)
{
    grid_launch_dependents();
    const int pieces = static_cast<int>(K / 16);
    const int64_t ldv = K / 2, ldm = K / 8;
    const int p_first = blockIdx.x * (kThreads * kPieces) + threadIdx.x;
    for (int64_t r = blockIdx.y; r < M; r += gridDim.y) {
        const uint4* src = reinterpret_cast<const uint4*>(a + r * lda);
        uint4 x[kPieces];
#pragma unroll
        for (int u = 0; u < kPieces; ++u) {
            const int p = p_first + u * kThreads;
            if (p < pieces)
                x[u] = __ldg(src + p);
        }
#pragma unroll
        for (int u = 0; u < kPieces; ++u) {
            const int p = p_first + u * kThreads;
            if (p >= pieces)
                continue;
            uint32_t v01, v23;
            const uint32_t n01 = select_group_pair(x[u].x, x[u].y, &v01);
            const uint32_t n23 = select_group_pair(x[u].z, x[u].w, &v23);
            const uint2 v = make_uint2(v01, v23);
            const uint32_t nib = n01 | (n23 << 8);
            *reinterpret_cast<uint2*>(vals + r * ldv + p * 8) = v;
            *reinterpret_cast<uint16_t*>(meta + r * ldm + p * 2) = static_cast<uint16_t>(nib);
        }
    }
}

// Scalar path (any K % 4 == 0 and any alignment): one metadata byte (two
// groups, or one at an odd tail) per iteration so that no two threads write
// the same byte.
__global__ void __launch_bounds__(kThreads) prune24_kernel(const uint8_t* __restrict__ a,
                                                           int64_t M, int64_t K, int64_t lda,
                                                           uint8_t* __restrict__ vals,
                                                           uint8_t* __restrict__ meta)
{
    grid_launch_dependents();
    const int64_t ldv = K / 2, ldm = (K + 7) / 8;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kThreads;
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x;
    for (int64_t i = tid; i < M * ldm; i += stride) {
        const int64_t r = i / ldm, b = i - r * ldm;
        uint8_t out = 0;
        for (int h = 0; h < 2; ++h) {
            const int64_t g = 2 * b + h;
            if (4 * g >= K)
                break;
            const uint8_t* p = a + r * lda + 4 * g;
            const uint32_t w = p[0] | (p[1] << 8) | (p[2] << 16) | (static_cast<uint32_t>(p[3]) << 24);
            const uint32_t sel = select_group(w);
            vals[r * ldv + 2 * g] = static_cast<uint8_t>(sel & 0xFFu);
            vals[r * ldv + 2 * g + 1] = static_cast<uint8_t>((sel >> 8) & 0xFFu);
            out |= static_cast<uint8_t>(((sel >> 16) & 0xFu) << (4 * h));
        }
        meta[r * ldm + b] = out;
    }
}

__global__ void __launch_bounds__(kThreads) decompress24_kernel(const uint8_t* __restrict__ vals,
                                                                const uint8_t* __restrict__ meta,
                                                                int64_t M, int64_t K,
                                                                uint8_t* __restrict__ out)
{
    grid_launch_dependents();
    const int64_t ldv = K / 2, ldm = (K + 7) / 8, groups = K / 4;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kThreads;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; i < M * groups;
         i += stride) {
        const int64_t r = i / groups, g = i - r * groups;
        const uint32_t nib = (meta[r * ldm + g / 2] >> (4 * (g % 2))) & 0xFu;
        const uint32_t i0 = nib & 3u, i1 = nib >> 2;
        uint32_t w = 0;
        w |= static_cast<uint32_t>(vals[r * ldv + 2 * g]) << (8 * i0);
        w |= static_cast<uint32_t>(vals[r * ldv + 2 * g + 1]) << (8 * i1);
        uint8_t* o = out + r * K + 4 * g;
        o[0] = w & 0xFFu;
        o[1] = (w >> 8) & 0xFFu;
        o[2] = (w >> 16) & 0xFFu;
        o[3] = (w >> 24) & 0xFFu;
    }
}

int grid_for(int64_t items)
{
    const int64_t blocks = (items + kThreads - 1) / kThreads;
    const int64_t cap = static_cast<int64_t>(sm_count()) * 16;
    return static_cast<int>(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

}  // namespace
}  // namespace gb300

extern "C" int prune24_compress(const uint8_t* a, int64_t M, int64_t K, int64_t lda,
                                uint8_t* a_vals, uint8_t* a_meta, fp8_stream_t stream)
{
    using namespace gb300;
    if (M < 0 || K < 0)
        return FP8_ERR_INVALID;
    if (K % 4 != 0)
        return FP8_ERR_SHAPE;
    if (M == 0 || K == 0)
        return FP8_OK;
    if (!a || !a_vals || !a_meta)
        return FP8_ERR_INVALID;
    if (lda < K)
        return FP8_ERR_SHAPE;
    if (!device_supported())
        return FP8_ERR_UNSUPPORTED;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const bool vec = (K % 16 == 0) && aligned16(a) && (lda % 16 == 0) &&
                     (reinterpret_cast<uintptr_t>(a_vals) % 8 == 0) &&
                     (reinterpret_cast<uintptr_t>(a_meta) % 2 == 0);
    if (vec) {
        const int64_t pieces = K / 16;
        const unsigned gx = static_cast<unsigned>((pieces + kThreads * kPieces - 1) / (kThreads * kPieces));
        const unsigned gy = static_cast<unsigned>(M < 65535 ? M : 65535);
        prune24_vec_kernel<<<dim3(gx, gy), kThreads, 0, st>>>(a, M, K, lda, a_vals, a_meta);
    } else {
        prune24_kernel<<<grid_for(M * ((K + 7) / 8)), kThreads, 0, st>>>(a, M, K, lda, a_vals, a_meta);
    }
    GB_CUDA_OK(cudaGetLastError());
    return FP8_OK;
}

extern "C" int prune24_decompress(const uint8_t* a_vals, const uint8_t* a_meta, int64_t M,
                                  int64_t K, uint8_t* out, fp8_stream_t stream)
{
    using namespace gb300;
    if (M < 0 || K < 0)
        return FP8_ERR_INVALID;
    if (K % 4 != 0)
        return FP8_ERR_SHAPE;
    if (M == 0 || K == 0)
        return FP8_OK;
    if (!a_vals || !a_meta || !out)
        return FP8_ERR_INVALID;
    if (!device_supported())
        return FP8_ERR_UNSUPPORTED;
    decompress24_kernel<<<grid_for(M * (K / 4)), kThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        a_vals, a_meta, M, K, out);
    GB_CUDA_OK(cudaGetLastError());
    return FP8_OK;
}
