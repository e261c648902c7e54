// Scale selection + FP8 quantisation (fp8_quantize_e4m3, fp8_quantize_e5m2).
//
// Per row (scale_mode 1): one CTA per row.  Pass 1 takes amax of the row with
// 16-byte loads and a warp/CTA max reduction on the fp32 bit patterns of |x|
// (monotone for non-negative floats; Inf and NaN compare above every finite
// value, which is how non-finite input is detected).  Pass 2 re-reads the
// row (an L2 hit: the rows in flight are far smaller than L2) and writes the
// codes.  HBM traffic: 4 bytes read + 1 byte written per element.
//
// fp8_quantize_e4m3_rows_grouped runs the per-row path for up to 32
// independent matrices in one launch (job table in the kernel parameters).
//
// Per tensor (scale_mode 0): a grid-stride amax kernel folds into the
// dequant_scale[0] slot with atomicMax, an encode kernel reads it, and a
// one-thread kernel turns the slot into d = amax / 448.
//
// The scale is s = T / amax with an IEEE-rounded division (__fdiv_rn), T the
// format's largest finite value (448 for E4M3, 57344 for E5M2), and each code
// is cvt.rn.satfinite of the IEEE product x * s (__fmul_rn) to that format.
// Every kernel is a template on the format (FMT 0: E4M3, 1: E5M2).
#include <cuda_fp8.h>

#include "common.cuh"
#include "prune_select.cuh"

namespace gb300 {
namespace {

constexpr int kThreads = 256;
constexpr uint32_t kInfBits = 0x7F800000u;

__device__ __forceinline__ uint32_t abs_bits(float v)
{
    return __float_as_uint(v) & 0x7FFFFFFFu;
}

// Largest finite value of the format: the target of amax.
template <int FMT>
__device__ __forceinline__ float fmt_max()
{
    return FMT == 1 ? 57344.0f : 448.0f;
}

// Two fp32 values -> two codes (a in the low byte), round to nearest even,
// saturating to the largest finite value.
template <int FMT>
__device__ __forceinline__ uint32_t enc2(float a, float b)
{
    return static_cast<uint32_t>(__nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE,
                                                          FMT == 1 ? __NV_E5M2 : __NV_E4M3));
}

template <int FMT>
__device__ __forceinline__ uint32_t enc4(float4 v, float s)
{
    return enc2<FMT>(__fmul_rn(v.x, s), __fmul_rn(v.y, s)) |
           (enc2<FMT>(__fmul_rn(v.z, s), __fmul_rn(v.w, s)) << 16);
}

__device__ __forceinline__ uint32_t block_max_u32(uint32_t v, uint32_t* red)
{
    v = __reduce_max_sync(0xFFFFFFFFu, v);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < (blockDim.x >> 5) ? red[lane] : 0u;
        w = __reduce_max_sync(0xFFFFFFFFu, w);
        if (lane == 0)
            red[0] = w;
    }
    __syncthreads();
    uint32_t r = red[0];
    __syncthreads();
    return r;
}

// scale and dequant factor from the amax bit pattern
template <int FMT>
__device__ __forceinline__ void scale_from_amax(uint32_t amax_bits, float& s, float& d)
{
    const float amax = __uint_as_float(amax_bits);
    if (amax_bits == 0u) {
        s = 1.0f;
        d = 1.0f;
    } else {
        s = __fdiv_rn(fmt_max<FMT>(), amax);
        d = __fdiv_rn(amax, fmt_max<FMT>());
    }
}

// One row: amax (CTA reduction), scale, codes.  vec: the row allows 16-byte
// loads and 4-byte stores (x 16-aligned, q 4-aligned).
template <int FMT>
__device__ __forceinline__ void quantize_row(const float* __restrict__ xr, int64_t cols,
                                             uint8_t* __restrict__ qr, float* __restrict__ d_out,
                                             int vec, int* err, uint32_t* red)
{
    const int64_t nvec = vec ? cols / 4 : 0;
    uint32_t m = 0;
    for (int64_t i = threadIdx.x; i < nvec; i += kThreads) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(xr) + i);
        m = max(m, max(max(abs_bits(v.x), abs_bits(v.y)), max(abs_bits(v.z), abs_bits(v.w))));
    }
    for (int64_t c = nvec * 4 + threadIdx.x; c < cols; c += kThreads)
        m = max(m, abs_bits(xr[c]));
    m = block_max_u32(m, red);
    if (m >= kInfBits && threadIdx.x == 0)
        report_device_error(err, FP8_ERR_NONFINITE);
    float s, dq;
    scale_from_amax<FMT>(m, s, dq);
    if (threadIdx.x == 0)
        *d_out = dq;
    for (int64_t i = threadIdx.x; i < nvec; i += kThreads) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(xr) + i);
        reinterpret_cast<uint32_t*>(qr)[i] = enc4<FMT>(v, s);
    }
    for (int64_t c = nvec * 4 + threadIdx.x; c < cols; c += kThreads)
        qr[c] = static_cast<uint8_t>(enc2<FMT>(__fmul_rn(xr[c], s), 0.0f) & 0xFFu);
}

// vec: x rows and q rows allow 16-byte loads / 4-byte stores (x 16-aligned,
// ldx % 4 == 0, q 4-aligned, ldq % 4 == 0).
template <int FMT>
__global__ void __launch_bounds__(kThreads) quant_row_kernel(const float* __restrict__ x,
                                                             int64_t rows, int64_t cols,
                                                             int64_t ldx, uint8_t* __restrict__ q,
                                                             int64_t ldq, float* __restrict__ d,
                                                             int vec, int* err)
{
    grid_launch_dependents();
    __shared__ uint32_t red[kThreads / 32];
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x)
        quantize_row<FMT>(x + r * ldx, cols, q + r * ldq, d + r, vec, err, red);
}

// Per-row E4M3 quantisation and 2:4 compression of the codes in one pass
// (fp8_quantize_e4m3_prune24).  Pass 1 takes the row's amax as quantize_row
// does; pass 2 re-reads the row (from L2) and encodes four elements (one 2:4
// group) per lane and step, with coalesced 16-byte loads and 4-byte code
// stores, and selects the group's two kept codes and index nibble from its
// codes exactly as prune24_compress does (prune_select.cuh); lanes 2i and
// 2i + 1 hold consecutive groups and combine their nibbles into one
// metadata byte.  Measured against fp8_quantize_e4m3 followed by
// prune24_compress: 252 against 275 us at 16384 x 16384, 68 against 79 us
// at 8192 x 8192.  Staging each row in shared memory (no second read from
// L2 or DRAM, but three CTAs per SM at 16384 columns) and persistent grids
// of four or eight CTAs per SM were slower.  Needs cols % 128 == 0 (so
// every warp runs the same number of steps), x 16-aligned with ldx % 4 ==
// 0, q 4-aligned with ldq % 4 == 0, a_vals 2-aligned (checked by the host).
__global__ void __launch_bounds__(kThreads) quant_row_prune_kernel(const float* __restrict__ x, int64_t rows,
                                                                   int64_t cols, int64_t ldx,
                                                                   uint8_t* __restrict__ q, int64_t ldq,
                                                                   float* __restrict__ d,
                                                                   uint8_t* __restrict__ vals,
                                                                   uint8_t* __restrict__ meta, int* err)
{
    grid_launch_dependents();
    __shared__ uint32_t red[kThreads / 32];
    const int64_t n4 = cols / 4;
    const int64_t ldv = cols / 2, ldm = cols / 8;
    const int lane = threadIdx.x & 31;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const float4* xr = reinterpret_cast<const float4*>(x + r * ldx);
        uint32_t m = 0;
        for (int64_t i = threadIdx.x; i < n4; i += kThreads) {
            const float4 v = __ldg(xr + i);
            m = max(m, max(max(abs_bits(v.x), abs_bits(v.y)), max(abs_bits(v.z), abs_bits(v.w))));
        }
        m = block_max_u32(m, red);
        if (m >= kInfBits && threadIdx.x == 0)
            report_device_error(err, FP8_ERR_NONFINITE);
        float s, dq;
        scale_from_amax<0>(m, s, dq);
        if (threadIdx.x == 0)
            d[r] = dq;
        uint8_t* qr = q + r * ldq;
        uint8_t* vr = vals + r * ldv;
        uint8_t* mr = meta + r * ldm;
        for (int64_t i = threadIdx.x; i < n4; i += kThreads) {
            const uint32_t w = enc4<0>(__ldg(xr + i), s);
            reinterpret_cast<uint32_t*>(qr)[i] = w;
            const uint32_t sel = select_group(w);
            reinterpret_cast<uint16_t*>(vr)[i] = static_cast<uint16_t>(sel & 0xFFFFu);
            const uint32_t nib = sel >> 16;
            const uint32_t next = __shfl_down_sync(0xFFFFFFFFu, nib, 1);
            if ((lane & 1) == 0)
                mr[i >> 1] = static_cast<uint8_t>(nib | (next << 4));
        }
    }
}

// Many independent per-row quantisations in one launch: the job table is
// passed by value; CTA b takes global row b (rows of job j follow those of
// job j - 1).
struct RowJobs {
    fp8_quant_job job[FP8_QUANT_GROUPED_MAX];
    int64_t row_start[FP8_QUANT_GROUPED_MAX + 1];
    int vec[FP8_QUANT_GROUPED_MAX];
    int n;
};

__global__ void __launch_bounds__(kThreads) quant_rows_grouped_kernel(const __grid_constant__ RowJobs jobs,
                                                                      int* err)
{
    grid_launch_dependents();
    __shared__ uint32_t red[kThreads / 32];
    const int64_t total = jobs.row_start[jobs.n];
    for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
        int j = 0;
        while (j + 1 < jobs.n && jobs.row_start[j + 1] <= g)
            ++j;
        const fp8_quant_job& J = jobs.job[j];
        const int64_t r = g - jobs.row_start[j];
        quantize_row<0>(J.x + r * J.ldx, J.cols, J.q + r * J.ldq, J.dequant_scale + r, jobs.vec[j], err,
                     red);
    }
}

__global__ void __launch_bounds__(kThreads) quant_amax_kernel(const float* __restrict__ x,
                                                              int64_t rows, int64_t cols,
                                                              int64_t ldx, int vec,
                                                              uint32_t* __restrict__ slot)
{
    __shared__ uint32_t red[kThreads / 32];
    uint32_t m = 0;
    const int64_t per_row = vec ? cols / 4 : 0;
    const int64_t total_vec = per_row * rows;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kThreads;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; i < total_vec;
         i += stride) {
        const int64_t r = i / per_row, c4 = i - r * per_row;
        const float4 v = __ldg(reinterpret_cast<const float4*>(x + r * ldx) + c4);
        m = max(m, max(max(abs_bits(v.x), abs_bits(v.y)), max(abs_bits(v.z), abs_bits(v.w))));
    }
    const int64_t tail = cols - per_row * 4;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; i < tail * rows;
         i += stride) {
        const int64_t r = i / tail, c = per_row * 4 + (i - r * tail);
        m = max(m, abs_bits(x[r * ldx + c]));
    }
    m = block_max_u32(m, red);
    if (threadIdx.x == 0 && m != 0u)
        atomicMax(slot, m);
}

template <int FMT>
__global__ void __launch_bounds__(kThreads) quant_encode_kernel(const float* __restrict__ x,
                                                                int64_t rows, int64_t cols,
                                                                int64_t ldx, uint8_t* __restrict__ q,
                                                                int64_t ldq, int vec,
                                                                const uint32_t* __restrict__ slot)
{
    float s, dq;
    scale_from_amax<FMT>(*slot, s, dq);
    const int64_t per_row = vec ? cols / 4 : 0;
    const int64_t total_vec = per_row * rows;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kThreads;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; i < total_vec;
         i += stride) {
        const int64_t r = i / per_row, c4 = i - r * per_row;
        const float4 v = __ldg(reinterpret_cast<const float4*>(x + r * ldx) + c4);
        reinterpret_cast<uint32_t*>(q + r * ldq)[c4] = enc4<FMT>(v, s);
    }
    const int64_t tail = cols - per_row * 4;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; i < tail * rows;
         i += stride) {
        const int64_t r = i / tail, c = per_row * 4 + (i - r * tail);
        q[r * ldq + c] = static_cast<uint8_t>(enc2<FMT>(__fmul_rn(x[r * ldx + c], s), 0.0f) & 0xFFu);
    }
}

template <int FMT>
__global__ void quant_finalize_kernel(uint32_t* slot, int* err)
{
    grid_launch_dependents();
    const uint32_t m = *slot;
    if (m >= kInfBits)
        report_device_error(err, FP8_ERR_NONFINITE);
    float s, dq;
    scale_from_amax<FMT>(m, s, dq);
    *reinterpret_cast<float*>(slot) = dq;
}

template <int FMT>
int quantize(const float* x, int64_t rows, int64_t cols, int64_t ldx, int scale_mode, uint8_t* q,
             int64_t ldq, float* dequant_scale, cudaStream_t st)
{
    if (rows < 0 || cols < 0 || (scale_mode != 0 && scale_mode != 1))
        return FP8_ERR_INVALID;
    if (rows == 0 || cols == 0)
        return FP8_OK;
    if (!x || !q || !dequant_scale)
        return FP8_ERR_INVALID;
    if (ldx < cols || ldq < cols)
        return FP8_ERR_SHAPE;
    if ((reinterpret_cast<uintptr_t>(x) & 3u) || (reinterpret_cast<uintptr_t>(dequant_scale) & 3u))
        return FP8_ERR_ALIGN;
    if (!device_supported())
        return FP8_ERR_UNSUPPORTED;
    int* err = device_error_word();
    const int vec = aligned16(x) && (ldx % 4 == 0) &&
                    (reinterpret_cast<uintptr_t>(q) % 4 == 0) && (ldq % 4 == 0);
    const int sms = sm_count();
    if (scale_mode == 1) {
        const int64_t grid = rows < 65535LL * 8 ? rows : 65535LL * 8;
        quant_row_kernel<FMT><<<static_cast<unsigned>(grid), kThreads, 0, st>>>(
            x, rows, cols, ldx, q, ldq, dequant_scale, vec, err);
        GB_CUDA_OK(cudaGetLastError());
        return FP8_OK;
    }
    uint32_t* slot = reinterpret_cast<uint32_t*>(dequant_scale);
    GB_CUDA_OK(cudaMemsetAsync(slot, 0, sizeof(uint32_t), st));
    const int64_t work = (rows * cols + 4 * kThreads - 1) / (4 * kThreads);
    const int64_t grid = work < static_cast<int64_t>(sms) * 8 ? (work > 0 ? work : 1) : sms * 8;
    quant_amax_kernel<<<static_cast<unsigned>(grid), kThreads, 0, st>>>(x, rows, cols, ldx, vec,
                                                                        slot);
    GB_CUDA_OK(cudaGetLastError());
    quant_encode_kernel<FMT><<<static_cast<unsigned>(grid), kThreads, 0, st>>>(x, rows, cols, ldx,
                                                                               q, ldq, vec, slot);
    GB_CUDA_OK(cudaGetLastError());
    quant_finalize_kernel<FMT><<<1, 1, 0, st>>>(slot, err);
    GB_CUDA_OK(cudaGetLastError());
    return FP8_OK;
}

// ---------------------------------------------------------------- block-scaled (MX)

// Byte offset of the scale of row r, 32-element block b, in the tiled layout
// (include/gb300fp8.h): 512-byte chunks per 128 rows x 128 columns, chunk
// (r / 128, b / 4) at (r / 128) * kb + b / 4, and within a chunk row r % 32
// at 16-byte row r % 32, 4-byte word (r % 128) / 32, byte b % 4.
__device__ __forceinline__ int64_t mx_tiled_offset(int64_t r, int64_t b, int64_t kb)
{
    return 512 * ((r >> 7) * kb + (b >> 2)) + 16 * (r & 31) + 4 * ((r & 127) >> 5) + (b & 3);
}

// One warp quantises a 128-column window of one row at a time: lane l
// holds columns 4l .. 4l + 3, so the 32-element block j (of four) is lanes
// 8j .. 8j + 7, and its amax is an 8-lane max reduction.  For a non-zero
// block, e = floor(log2 amax) - emax (emax 8 for E4M3, 15 for E5M2) read
// from amax's exponent field (a subnormal amax gives the floor -127), so
// amax * 2^-e lies in [2^emax, 2^(emax+1)); the scale code is e + 127 and the
// codes are the format's round-to-nearest-even, saturating encoding of the
// IEEE product x * 2^-e (exact unless it falls below 2^-126).  An all-zero
// block gets scale code 0 and the codes of its (signed) zeros.
// Grid: blockIdx.y walks rows (with a stride past 65535), blockIdx.x takes
// mx_windows<TILED>() consecutive windows of the row: warp w of the block
// handles windows x * that + w + 8 u (u < mx_unroll<TILED>()), all loads
// issued before any arithmetic.  Measured: eight loads in flight per lane
// suit the tiled scale layout, four the row-major one (eight made it 25 %
// slower).
template <int TILED>
__host__ __device__ constexpr int mx_unroll()
{
    return TILED ? 8 : 4;
}

template <int TILED>
__host__ __device__ constexpr int mx_windows()
{
    return (kThreads / 32) * mx_unroll<TILED>();   // windows per block and row
}

template <int FMT, int TILED>
__global__ void __launch_bounds__(kThreads) quant_mx_kernel(const float* __restrict__ x, int64_t rows,
                                                            int64_t cols, int64_t ldx, uint8_t* __restrict__ q,
                                                            int64_t ldq, uint8_t* __restrict__ sc, int vec,
                                                            int qvec, int* err)
{
    grid_launch_dependents();
    constexpr int kEmax = FMT == 1 ? 15 : 8;
    constexpr int kMxU = mx_unroll<TILED>();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t kb = (cols + 127) / 128;
    const int64_t win0 = static_cast<int64_t>(blockIdx.x) * mx_windows<TILED>() + warp;
    for (int64_t r = blockIdx.y; r < rows; r += gridDim.y) {
        const float* xr = x + r * ldx;
        float4 v[kMxU];
        bool in[kMxU];
#pragma unroll
        for (int u = 0; u < kMxU; ++u) {
            const int64_t c0 = (win0 + u * (kThreads / 32)) * 128 + 4 * lane;
            in[u] = c0 < cols;                                // cols % 32 == 0: whole blocks in or out
            v[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (in[u]) {
                if (vec)
                    v[u] = __ldg(reinterpret_cast<const float4*>(xr + c0));
                else
                    v[u] = make_float4(xr[c0], xr[c0 + 1], xr[c0 + 2], xr[c0 + 3]);
            }
        }
#pragma unroll
        for (int u = 0; u < kMxU; ++u) {
            const int64_t w = win0 + u * (kThreads / 32);
            if (w >= kb)
                break;                                        // the whole warp leaves together
            const int64_t c0 = w * 128 + 4 * lane;
            uint32_t m = max(max(abs_bits(v[u].x), abs_bits(v[u].y)), max(abs_bits(v[u].z), abs_bits(v[u].w)));
            m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, 1));
            m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, 2));
            m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, 4));
            if (m >= kInfBits && (lane & 7) == 0)
                report_device_error(err, FP8_ERR_NONFINITE);
            uint32_t code = 0;
            float s = 1.0f;
            if (m != 0u && m < kInfBits) {
                const int E = static_cast<int>(m >> 23);  // biased exponent of amax
                const int e = E == 0 ? -127 : max(E - 127 - kEmax, -127);
                code = static_cast<uint32_t>(e + 127);
                s = __uint_as_float(static_cast<uint32_t>(127 - e) << 23);     // 2^-e, normal
            }
            if (in[u]) {
                const uint32_t word = enc4<FMT>(v[u], s);
                uint8_t* qd = q + r * ldq + c0;
                if (qvec) {
                    *reinterpret_cast<uint32_t*>(qd) = word;
                } else {
                    qd[0] = word & 0xFFu;
                    qd[1] = (word >> 8) & 0xFFu;
                    qd[2] = (word >> 16) & 0xFFu;
                    qd[3] = word >> 24;
                }
            }
            // the four blocks' scale codes, from lanes 0, 8, 16, 24
            const uint32_t s0 = __shfl_sync(0xFFFFFFFFu, code, 0), s1 = __shfl_sync(0xFFFFFFFFu, code, 8);
            const uint32_t s2 = __shfl_sync(0xFFFFFFFFu, code, 16), s3 = __shfl_sync(0xFFFFFFFFu, code, 24);
            if (lane == 0) {
                const int64_t b0 = w * 4;                         // first block of the window
                const int nb = static_cast<int>(min(static_cast<int64_t>(4), cols / 32 - b0));
                const uint32_t sj[4] = {s0, s1, s2, s3};
                if (TILED) {
                    uint32_t word = 0;
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        word |= (j < nb ? sj[j] : 127u) << (8 * j);     // blocks past cols: scale 1
                    *reinterpret_cast<uint32_t*>(sc + mx_tiled_offset(r, b0, kb)) = word;
                } else {
                    uint8_t* sr = sc + r * (cols / 32) + b0;
                    if (nb == 4 && (reinterpret_cast<uintptr_t>(sr) & 3u) == 0) {
                        *reinterpret_cast<uint32_t*>(sr) = s0 | (s1 << 8) | (s2 << 16) | (s3 << 24);
                    } else {
                        for (int j = 0; j < nb; ++j)
                            sr[j] = static_cast<uint8_t>(sj[j]);
                    }
                }
            }
        }
    }
}

// Row-major scales [rows, cols / 32] -> the tiled layout (one 4-byte word,
// four blocks of one row, per thread; padding rows and blocks get 127).
__global__ void __launch_bounds__(kThreads) mx_scales_tile_kernel(const uint8_t* __restrict__ src, int64_t rows,
                                                                  int64_t cols, uint8_t* __restrict__ dst)
{
    grid_launch_dependents();
    const int64_t kb = (cols + 127) / 128;
    const int64_t nbr = cols / 32;
    const int64_t total = (rows + 127) / 128 * 128 * kb;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kThreads;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; i < total; i += stride) {
        const int64_t r = i / kb, k = i - r * kb;
        uint32_t word = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t b = 4 * k + j;
            const uint32_t v = (r < rows && b < nbr) ? src[r * nbr + b] : 127u;
            word |= v << (8 * j);
        }
        *reinterpret_cast<uint32_t*>(dst + mx_tiled_offset(r, 4 * k, kb)) = word;
    }
}

int grid_for_items(int64_t items)
{
    const int64_t blocks = (items + kThreads - 1) / kThreads;
    const int64_t cap = static_cast<int64_t>(sm_count()) * 8;
    return static_cast<int>(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

template <int FMT>
int quantize_mx(const float* x, int64_t rows, int64_t cols, int64_t ldx, uint8_t* q, int64_t ldq,
                uint8_t* scales, int layout, cudaStream_t st)
{
    if (rows < 0 || cols < 0 || (layout != 0 && layout != 1))
        return FP8_ERR_INVALID;
    if (cols % 32 != 0)
        return FP8_ERR_SHAPE;
    if (rows == 0 || cols == 0)
        return FP8_OK;
    if (!x || !q || !scales)
        return FP8_ERR_INVALID;
    if (ldx < cols || ldq < cols)
        return FP8_ERR_SHAPE;
    if ((reinterpret_cast<uintptr_t>(x) & 3u) || (layout == 1 && !aligned16(scales)))
        return FP8_ERR_ALIGN;
    if (!device_supported())
        return FP8_ERR_UNSUPPORTED;
    const int vec = aligned16(x) && (ldx % 4 == 0);
    const int qvec = (reinterpret_cast<uintptr_t>(q) % 4 == 0) && (ldq % 4 == 0);
    // a few blocks per SM, each walking rows (short-lived blocks cost more
    // in launch and tail than they save)
    const int64_t kb = (cols + 127) / 128;
    const int64_t win = layout == 1 ? mx_windows<1>() : mx_windows<0>();
    const int64_t gx = (kb + win - 1) / win;
    int64_t gy = std::min<int64_t>(rows, static_cast<int64_t>(sm_count()) * 16 / gx);
    gy = std::max<int64_t>(1, std::min<int64_t>(gy, 65535));
    const dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
    if (layout == 1) {
        if (rows % 128 != 0)                     // padding rows of the last tile: scale 1
            GB_CUDA_OK(cudaMemsetAsync(scales, 127, fp8_mx_scale_tiled_bytes(rows, cols), st));
        quant_mx_kernel<FMT, 1><<<grid, kThreads, 0, st>>>(x, rows, cols, ldx, q, ldq, scales, vec, qvec,
                                                          device_error_word());
    } else {
        quant_mx_kernel<FMT, 0><<<grid, kThreads, 0, st>>>(x, rows, cols, ldx, q, ldq, scales, vec, qvec,
                                                          device_error_word());
    }
    GB_CUDA_OK(cudaGetLastError());
    return FP8_OK;
}

}  // namespace
}  // namespace gb300

extern "C" size_t fp8_mx_scale_tiled_bytes(int64_t rows, int64_t cols)
{
    if (rows <= 0 || cols <= 0)
        return 0;
    return static_cast<size_t>((rows + 127) / 128) * static_cast<size_t>((cols + 127) / 128) * 512;
}

extern "C" int fp8_quantize_mx(const float* x, int64_t rows, int64_t cols, int64_t ldx, int format,
                               uint8_t* q, int64_t ldq, uint8_t* scales, int scale_layout,
                               fp8_stream_t stream)
{
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (format == FP8_E4M3)
        return gb300::quantize_mx<0>(x, rows, cols, ldx, q, ldq, scales, scale_layout, st);
    if (format == FP8_E5M2)
        return gb300::quantize_mx<1>(x, rows, cols, ldx, q, ldq, scales, scale_layout, st);
    return FP8_ERR_INVALID;
}

extern "C" int fp8_mx_scales_to_tiled(const uint8_t* scales, int64_t rows, int64_t cols, uint8_t* tiled,
                                      fp8_stream_t stream)
{
    using namespace gb300;
    if (rows < 0 || cols < 0)
        return FP8_ERR_INVALID;
    if (cols % 32 != 0)
        return FP8_ERR_SHAPE;
    if (rows == 0 || cols == 0)
        return FP8_OK;
    if (!scales || !tiled)
        return FP8_ERR_INVALID;
    if (!aligned16(tiled))
        return FP8_ERR_ALIGN;
    if (!device_supported())
        return FP8_ERR_UNSUPPORTED;
    const int64_t words = (rows + 127) / 128 * 128 * ((cols + 127) / 128);
    mx_scales_tile_kernel<<<grid_for_items(words), kThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        scales, rows, cols, tiled);
    GB_CUDA_OK(cudaGetLastError());
    return FP8_OK;
}

extern "C" int fp8_quantize_e4m3(const float* x, int64_t rows, int64_t cols, int64_t ldx,
                                 int scale_mode, uint8_t* q, int64_t ldq, float* dequant_scale,
                                 fp8_stream_t stream)
{
    return gb300::quantize<0>(x, rows, cols, ldx, scale_mode, q, ldq, dequant_scale,
                              reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int fp8_quantize_e4m3_prune24(const float* x, int64_t rows, int64_t cols, int64_t ldx, uint8_t* q,
                                         int64_t ldq, float* dequant_scale, uint8_t* a_vals, uint8_t* a_meta,
                                         fp8_stream_t stream)
{
    using namespace gb300;
    if (rows < 0 || cols < 0)
        return FP8_ERR_INVALID;
    if (rows == 0 || cols == 0)
        return FP8_OK;
    if (!x || !q || !dequant_scale || !a_vals || !a_meta)
        return FP8_ERR_INVALID;
    if (cols % 128 != 0 || ldx < cols || ldq < cols)
        return FP8_ERR_SHAPE;
    if (!aligned16(x) || ldx % 4 != 0 || reinterpret_cast<uintptr_t>(q) % 4 != 0 || ldq % 4 != 0 ||
        reinterpret_cast<uintptr_t>(a_vals) % 2 != 0 || reinterpret_cast<uintptr_t>(dequant_scale) % 4 != 0)
        return FP8_ERR_ALIGN;
    if (!device_supported())
        return FP8_ERR_UNSUPPORTED;
    const int64_t grid = rows < 65535LL * 8 ? rows : 65535LL * 8;
    quant_row_prune_kernel<<<static_cast<unsigned>(grid), kThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        x, rows, cols, ldx, q, ldq, dequant_scale, a_vals, a_meta, device_error_word());
    GB_CUDA_OK(cudaGetLastError());
    return FP8_OK;
}

extern "C" int fp8_quantize_e5m2(const float* x, int64_t rows, int64_t cols, int64_t ldx,
                                 int scale_mode, uint8_t* q, int64_t ldq, float* dequant_scale,
                                 fp8_stream_t stream)
{
    return gb300::quantize<1>(x, rows, cols, ldx, scale_mode, q, ldq, dequant_scale,
                              reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int fp8_quantize_e4m3_rows_grouped(const fp8_quant_job* jobs, int num_jobs,
                                              fp8_stream_t stream)
{
    using namespace gb300;
    if (num_jobs < 0 || (num_jobs > 0 && !jobs))
        return FP8_ERR_INVALID;
    if (num_jobs > FP8_QUANT_GROUPED_MAX)
        return FP8_ERR_SHAPE;
    RowJobs rj;
    memset(&rj, 0, sizeof(rj));
    int64_t rows = 0;
    for (int i = 0; i < num_jobs; ++i) {
        const fp8_quant_job& J = jobs[i];
        if (J.rows < 0 || J.cols < 0)
            return FP8_ERR_INVALID;
        if (J.rows == 0 || J.cols == 0)
            continue;
        if (!J.x || !J.q || !J.dequant_scale)
            return FP8_ERR_INVALID;
        if (J.ldx < J.cols || J.ldq < J.cols)
            return FP8_ERR_SHAPE;
        if ((reinterpret_cast<uintptr_t>(J.x) & 3u) ||
            (reinterpret_cast<uintptr_t>(J.dequant_scale) & 3u))
            return FP8_ERR_ALIGN;
        const int k = rj.n++;
        rj.job[k] = J;
        rj.row_start[k] = rows;
        rj.vec[k] = aligned16(J.x) && (J.ldx % 4 == 0) &&
                    (reinterpret_cast<uintptr_t>(J.q) % 4 == 0) && (J.ldq % 4 == 0);
        rows += J.rows;
    }
    rj.row_start[rj.n] = rows;
    if (rows == 0)
        return FP8_OK;
    if (!device_supported())
        return FP8_ERR_UNSUPPORTED;
    const int64_t grid = rows < 65535LL * 8 ? rows : 65535LL * 8;
    quant_rows_grouped_kernel<<<static_cast<unsigned>(grid), kThreads, 0,
                                reinterpret_cast<cudaStream_t>(stream)>>>(rj, device_error_word());
    GB_CUDA_OK(cudaGetLastError());
    return FP8_OK;
}
