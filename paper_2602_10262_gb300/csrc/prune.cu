// 2:4 prune + compress (prune24_compress) and its inverse.
//
// Vector path: a thread takes chunks of 32 input bytes (eight groups of four
// codes): two 16-byte loads, a branch-free rank selection per group, one
// 16-byte store of the kept codes and one 4-byte store of the eight metadata
// nibbles.  Rows whose length or alignment does not allow it fall back to one
// metadata byte per iteration.  Bandwidth-bound: 1 byte read, 0.625 bytes written per
// element; no allocation, one launch.
#include "common.cuh"

namespace gb300 {
namespace {

constexpr int kThreads = 256;

// One group of four codes (byte i of w = element i).  Element j outranks
// element i when key_j > key_i, or key_j == key_i and j < i (key = code &
// 0x7F).  The two elements outranked by fewer than two others are kept.
// Byte-parallel: rotating the keys by d = 1, 2, 3 places key_{(i+d)%4} in
// byte i; (i + d) % 4 < i exactly for the bytes of tie_d.  Returns the two
// kept codes in the low 16 bits (lower index first) and the nibble
// i0 | i1 << 2 in bits 16..19.
__device__ __forceinline__ uint32_t select_group(uint32_t w)
{
    const uint32_t k = w & 0x7F7F7F7Fu;
    const uint32_t r1 = __byte_perm(k, 0u, 0x0321);
    const uint32_t r2 = __byte_perm(k, 0u, 0x1032);
    const uint32_t r3 = __byte_perm(k, 0u, 0x2103);
    const uint32_t o1 = __vcmpgtu4(r1, k) | (__vcmpeq4(r1, k) & 0xFF000000u);
    const uint32_t o2 = __vcmpgtu4(r2, k) | (__vcmpeq4(r2, k) & 0xFFFF0000u);
    const uint32_t o3 = __vcmpgtu4(r3, k) | (__vcmpeq4(r3, k) & 0xFFFFFF00u);
    const uint32_t rank = (o1 & 0x01010101u) + (o2 & 0x01010101u) + (o3 & 0x01010101u);
    const uint32_t keep = __vcmpltu4(rank, 0x02020202u);               // 0xFF per kept byte
    const uint32_t bits = ((keep & 0x08040201u) * 0x01010101u) >> 24;  // kept byte i -> bit i
    const uint32_t i0 = __ffs(bits) - 1;
    const uint32_t i1 = 31 - __clz(bits);
    const uint32_t vals = __byte_perm(w, 0u, i0 | (i1 << 4)) & 0xFFFFu;
    return vals | ((i0 | (i1 << 2)) << 16);
}

// Vector path: K % 32 == 0, a 16-aligned, lda % 16 == 0, outputs 16-aligned.
// blockIdx.y walks rows; each thread takes kChunks chunks of 32 codes spaced
// kThreads apart in the row, issues all loads first, then selects and
// stores (16 bytes of kept codes + 4 bytes of metadata per chunk).
constexpr int kChunks = 4;

__global__ void __launch_bounds__(kThreads) prune24_vec_kernel(const uint8_t* __restrict__ a,
                                                               int64_t M, int64_t K, int64_t lda,
                                                               uint8_t* __restrict__ vals,
                                                               uint8_t* __restrict__ meta)
{
    const int chunks = static_cast<int>(K / 32);
    const int64_t ldv = K / 2, ldm = K / 8;
    const int c_first = blockIdx.x * (kThreads * kChunks) + threadIdx.x;
    for (int64_t r = blockIdx.y; r < M; r += gridDim.y) {
        const uint4* src = reinterpret_cast<const uint4*>(a + r * lda);
        uint4 x[kChunks][2];
#pragma unroll
        for (int u = 0; u < kChunks; ++u) {
            const int c = c_first + u * kThreads;
            if (c < chunks) {
                x[u][0] = __ldg(src + 2 * c);
                x[u][1] = __ldg(src + 2 * c + 1);
            }
        }
#pragma unroll
        for (int u = 0; u < kChunks; ++u) {
            const int c = c_first + u * kThreads;
            if (c >= chunks)
                continue;
            const uint32_t w[8] = {x[u][0].x, x[u][0].y, x[u][0].z, x[u][0].w,
                                   x[u][1].x, x[u][1].y, x[u][1].z, x[u][1].w};
            uint32_t v[4] = {0, 0, 0, 0};
            uint32_t nib = 0;
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                const uint32_t sel = select_group(w[g]);
                v[g / 2] |= (sel & 0xFFFFu) << (16 * (g % 2));
                nib |= (sel >> 16) << (4 * g);
            }
            *reinterpret_cast<uint4*>(vals + r * ldv + c * 16) = make_uint4(v[0], v[1], v[2], v[3]);
            *reinterpret_cast<uint32_t*>(meta + r * ldm + c * 4) = nib;
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
    const bool vec = (K % 32 == 0) && aligned16(a) && (lda % 16 == 0) && aligned16(a_vals) &&
                     aligned16(a_meta);
    if (vec) {
        const int64_t chunks = K / 32;
        const unsigned gx = static_cast<unsigned>((chunks + kThreads * kChunks - 1) / (kThreads * kChunks));
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
