/*
 * gb300fp8 — FP8 (E4M3) dense and 2:4-sparse GEMM for one NVIDIA GB300 GPU.
 *
 * C ABI of libgb300fp8.so.  The operation is the one arXiv 2602.10262
 * characterises on FP8 matrix cores (section 2 "FP8 Matrix Cores", section 4):
 * FP8 x FP8 operands with FP32 accumulation,
 *
 *     C[m,n] = alpha * dA[m] * dB[n] * sum_k dec(A[m,k]) * dec(B[n,k]),
 *
 * dense, or with A in 2:4 structured sparsity (section 2 "Structured
 * Sparsity", section 6: two of every four consecutive elements along K are
 * zero).  dec() is the OCP E4M3 decoding the paper cites; dA, dB are the
 * dequantisation factors written by fp8_quantize_e4m3.
 *
 * Conventions for every entry point:
 *   - Pointers named as device pointers must point to device memory of the
 *     current CUDA device; the caller owns every buffer and the library never
 *     frees caller memory.
 *   - All work is enqueued on `stream` (a cudaStream_t; NULL = the legacy
 *     default stream) and the call returns after enqueueing.  Outputs are
 *     valid once the stream has reached that point.
 *   - Matrices are row-major with a row stride ("ld") in elements.  FP8 code
 *     matrices are bytes; A is [M, K] and B is stored [N, K] (K contiguous
 *     in both, i.e. the product is A * B^T of the stored arrays).
 *   - Return value: FP8_OK, or a negative fp8_status for rejected arguments
 *     (nothing is enqueued then) or a CUDA launch error.  Errors detected on
 *     the device (non-finite input, a pipeline wait that timed out) are
 *     recorded in a per-device error word read by fp8_last_device_error.
 */
#ifndef GB300FP8_H
#define GB300FP8_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *fp8_stream_t; /* identical to cudaStream_t */

typedef enum {
    FP8_OK = 0,
    FP8_PENDING = 1,          /* server: request not finished yet */
    FP8_ERR_INVALID = -1,     /* bad argument (null pointer, bad mode, ...) */
    FP8_ERR_SHAPE = -2,       /* unsupported or inconsistent sizes */
    FP8_ERR_ALIGN = -3,       /* pointer / stride alignment requirement violated */
    FP8_ERR_NONFINITE = -4,   /* quantisation input held NaN or Inf */
    FP8_ERR_OOM = -5,         /* server: admission refused for lack of free HBM */
    FP8_ERR_CUDA = -6,        /* a CUDA runtime call failed */
    FP8_ERR_TIMEOUT = -7,     /* a device pipeline wait ran past its limit */
    FP8_ERR_UNSUPPORTED = -8  /* no sm_103a device, or feature not built */
} fp8_status;

/* FP8 operand formats (the OCP 8-bit floating point variants; paper section
 * 2 lists both as FP8 matrix-core operand types, "fp8" = E4M3 and "bf8" =
 * E5M2, and Table 3 pairs them in all four combinations). */
typedef enum {
    FP8_E4M3 = 0,   /* sign, 4 exponent bits (bias 7), 3 mantissa bits; no
                       infinities, S.1111.111 NaN; largest finite 448 */
    FP8_E5M2 = 1    /* sign, 5 exponent bits (bias 15), 2 mantissa bits;
                       IEEE-style infinities and NaNs; largest finite 57344 */
} fp8_format;

/* Static English text for a status code. */
const char *fp8_status_string(int status);

/* Synchronises `stream`, then returns and clears the device error word of the
 * current device (FP8_OK if no kernel reported an error since the last call).
 * Kernels record FP8_ERR_NONFINITE (quantisation saw NaN/Inf) and
 * FP8_ERR_TIMEOUT (an mbarrier wait exceeded its ~2 s limit; the kernel then
 * stops its pipeline, releases tensor memory and exits).  When the word was
 * set, the call also synchronises the device and re-zeroes the split-K tile
 * counters of the library's persistent workspaces (a GEMM that stopped early
 * may have left one part-way); results of GEMMs launched between the failed
 * one and this call are unspecified. */
int fp8_last_device_error(fp8_stream_t stream);

/* Number of SMs of the current device (persistent grids are sized from it). */
int fp8_device_sm_count(void);

/* Failure-path testing (the paper has no counterpart; this exercises the
 * device error handling above without faulting the GPU).  The next
 * `launches` eager GEMM kernel launches of the process (any entry point, any
 * thread; CUDA-graph nodes made by gemm_fp8_grouped_graph_create are not
 * affected) run with their TMA producer issuing no operand loads: the MMA
 * warp's wait for the first stage then runs past the wait limit, the kernel
 * records FP8_ERR_TIMEOUT, stops every role, waits for its own outstanding
 * tensor-core work, frees its tensor memory and exits, leaving C unwritten
 * (split-K counters untouched).  wait_limit_ms > 0 sets the limit of every
 * bounded wait of eager GEMM launches from now on (the default is 2 s);
 * 0 restores the default.  launches = 0 cancels pending stalls.
 * FP8_ERR_INVALID for launches < 0 or a limit outside [0, 60000] ms. */
int fp8_test_stall_gemm_loads(int launches, double wait_limit_ms);

/* ---------------------------------------------------------------------------
 * Scale selection + E4M3 quantisation (rows a1, a2 of the path).
 * Paper: section 2 "FP8 Matrix Cores" (OCP E4M3 format).
 *
 * x:  device fp32 [rows, cols], row stride ldx elements (ldx >= cols).
 * scale_mode 0: one scale for the tensor; 1: one scale per row.
 * For each scaling group: amax = max|x|;  s = fl32(448 / amax);
 * d = fl32(amax / 448)  (both IEEE-rounded divisions; amax == 0 gives
 * s = d = 1);  q = E4M3(fl32(x * s)) rounded to nearest even and saturated to
 * +-448.
 * q:  device uint8 [rows, cols], row stride ldq bytes (ldq >= cols).
 * dequant_scale: device fp32, [1] (mode 0) or [rows] (mode 1), receives d.
 * Mode 0 uses dequant_scale[0] as its reduction slot while it runs.
 * NaN/Inf in x: FP8_ERR_NONFINITE in the device error word; q and d are then
 * unspecified.  rows == 0 or cols == 0: nothing to do, FP8_OK.
 * ------------------------------------------------------------------------- */
int fp8_quantize_e4m3(const float *x, int64_t rows, int64_t cols, int64_t ldx, int scale_mode,
                      uint8_t *q, int64_t ldq, float *dequant_scale, fp8_stream_t stream);

/* E5M2 quantisation: fp8_quantize_e4m3 with 57344, the largest finite E5M2
 * value, in place of 448.  s = fl32(57344 / amax), d = fl32(amax / 57344),
 * q = E5M2(fl32(x * s)) rounded to nearest even and saturated to +-57344,
 * so no code is ever an infinity or NaN.  Arguments, layouts, ownership
 * and errors as fp8_quantize_e4m3. */
int fp8_quantize_e5m2(const float *x, int64_t rows, int64_t cols, int64_t ldx, int scale_mode,
                      uint8_t *q, int64_t ldq, float *dequant_scale, fp8_stream_t stream);

/* Per-row quantisation (scale_mode 1 above) of up to FP8_QUANT_GROUPED_MAX
 * independent fp32 matrices in one launch; each job follows the conventions
 * of fp8_quantize_e4m3 (FP8_ERR_SHAPE for more jobs).  Used by the request
 * server to quantise a whole batch of activations at once. */
#define FP8_QUANT_GROUPED_MAX 32

typedef struct {
    const float *x;          /* device fp32 [rows, cols], row stride ldx */
    int64_t rows, cols, ldx;
    uint8_t *q;              /* device codes [rows, cols], row stride ldq */
    int64_t ldq;
    float *dequant_scale;    /* device fp32 [rows] */
} fp8_quant_job;

int fp8_quantize_e4m3_rows_grouped(const fp8_quant_job *jobs, int num_jobs, fp8_stream_t stream);

/* ---------------------------------------------------------------------------
 * Block-scaled FP8 (the OCP Microscaling "MX" formats MXFP8 E4M3 / E5M2).
 * The paper measures FP8 with one scale per tensor or channel; this is the
 * next precision step on the same tensor cores (tcgen05 kind::mxf8f6f4),
 * with one power-of-two scale per 32 consecutive elements along K.
 *
 * fp8_quantize_mx: x device fp32 [rows, cols], row stride ldx, cols % 32 == 0
 * (FP8_ERR_SHAPE otherwise).  For each row and block b of 32 columns:
 * amax = max|x| over the block; amax == 0 gives scale code 0 and the codes
 * of the block's signed zeros; otherwise e = floor(log2 amax) - emax (emax 8
 * for E4M3, 15 for E5M2) clamped to [-127, 127], scale code e + 127 (E8M0:
 * the scale 2^(code - 127)), and codes = the format's round-to-nearest-even,
 * saturating encoding of fl32(x * 2^-e).  So amax * 2^-e lies in
 * [2^emax, 2^(emax+1)) and a block maximum above the format's largest value
 * saturates to it.  format: an fp8_format.  q: device [rows, cols], row
 * stride ldq.  scales: device bytes, in one of two layouts:
 *   scale_layout 0, row-major: [rows, cols / 32], scale of (r, b) at
 *     r * (cols / 32) + b;
 *   scale_layout 1, tiled (what gemm_fp8_mx reads; 16-byte aligned,
 *     fp8_mx_scale_tiled_bytes(rows, cols) bytes): 512-byte chunks, one per
 *     128 rows x 128 columns, chunk (r / 128) * ceil(cols / 128) + b / 4;
 *     within it the scale of (r, b) at 16 * (r % 32) + 4 * ((r % 128) / 32)
 *     + b % 4 (the order in which the tensor core takes a 128 x 4 block of
 *     scales).  Entries of rows >= rows or blocks >= cols / 32 hold 127 (1.0).
 * NaN/Inf in x: FP8_ERR_NONFINITE in the device error word.
 *
 * fp8_mx_scales_to_tiled: row-major scales [rows, cols / 32] (contiguous)
 * -> the tiled layout above (for scales produced elsewhere).
 *
 * gemm_fp8_mx: C[m,n] = alpha * sum over blocks b of 2^(SA[m,b] - 127) *
 * 2^(SB[n,b] - 127) * sum_{k in b} decA(A[m,k]) decB(B[n,k]), accumulated in
 * FP32 on the tensor cores, which apply the block scales.  A [M, K] (lda),
 * B [N, K] (ldb) codes as in gemm_fp8_dense (16-byte aligned, strides
 * multiples of 16); a_scales / b_scales: the tiled layout of A's and B's
 * scales (16-byte aligned).  K % 32 == 0 (FP8_ERR_SHAPE otherwise).  C, ldc,
 * out_dtype, formats and stream as gemm_fp8_dense_fmt.  Needs no workspace.
 * ------------------------------------------------------------------------- */
size_t fp8_mx_scale_tiled_bytes(int64_t rows, int64_t cols);

int fp8_quantize_mx(const float *x, int64_t rows, int64_t cols, int64_t ldx, int format,
                    uint8_t *q, int64_t ldq, uint8_t *scales, int scale_layout, fp8_stream_t stream);

int fp8_mx_scales_to_tiled(const uint8_t *scales, int64_t rows, int64_t cols, uint8_t *tiled,
                           fp8_stream_t stream);

int gemm_fp8_mx(int64_t M, int64_t N, int64_t K, const uint8_t *A, int64_t lda,
                const uint8_t *a_scales, const uint8_t *B, int64_t ldb, const uint8_t *b_scales,
                float alpha, void *C, int64_t ldc, int out_dtype, int a_format, int b_format,
                fp8_stream_t stream);

/* ---------------------------------------------------------------------------
 * 2:4 prune + compress (row a3).  Paper: section 2 "Structured Sparsity",
 * section 6 (2 of every 4 consecutive elements along K are zero; the paper
 * blames a fixed conversion + allocation + dispatch cost in section 6.1.1 —
 * this call allocates nothing and is one bandwidth-bound kernel).
 *
 * a: device FP8 codes [M, K] (E4M3 or E5M2), row stride lda bytes;
 * K % 4 == 0 (else FP8_ERR_SHAPE).  For each row and each group g of four
 * codes a[4g..4g+3]: key = code & 0x7F (monotone in |value| over the finite
 * codes of either format); the two positions
 * first in (key descending, index ascending) order are kept.
 * a_vals: device [M, K/2] (row stride K/2): the kept codes of group g at
 *         2g, 2g+1 in increasing index order.
 * a_meta: device [M, ceil(K/8)] (row stride ceil(K/8)): for group g the
 *         nibble i0 | (i1 << 2) (i0 < i1 the kept indices) in byte g/2,
 *         low nibble for even g.
 * ------------------------------------------------------------------------- */
int prune24_compress(const uint8_t *a, int64_t M, int64_t K, int64_t lda, uint8_t *a_vals,
                     uint8_t *a_meta, fp8_stream_t stream);

/* Per-row E4M3 quantisation (fp8_quantize_e4m3, scale_mode 1) and the 2:4
 * compression of its codes (prune24_compress) in one pass over x: q,
 * dequant_scale, a_vals and a_meta are bitwise what the two calls in turn
 * write, with one read of x and no read of q.  Paper: sections 2 and 6 (the
 * quantised operand of a 2:4-sparse GEMM; section 6.1.1's conversion cost
 * becomes part of the quantiser's own HBM pass).
 * x: device fp32 [rows, cols], row stride ldx (elements); q: device
 * [rows, cols], row stride ldq bytes; dequant_scale: device fp32 [rows];
 * a_vals [rows, cols/2] and a_meta [rows, cols/8] packed, as
 * prune24_compress writes them.  cols % 128 == 0 (the 2:4 GEMM's K rule),
 * ldx >= cols, ldq >= cols (else FP8_ERR_SHAPE); x 16-byte aligned with
 * ldx % 4 == 0, q 4-byte aligned with ldq % 4 == 0, a_vals 2-byte and
 * dequant_scale 4-byte aligned (else FP8_ERR_ALIGN).  Non-finite input:
 * as fp8_quantize_e4m3. */
int fp8_quantize_e4m3_prune24(const float *x, int64_t rows, int64_t cols, int64_t ldx, uint8_t *q,
                              int64_t ldq, float *dequant_scale, uint8_t *a_vals, uint8_t *a_meta,
                              fp8_stream_t stream);

/* Inverse of prune24_compress: out [M, K] (row stride K) gets the kept codes
 * at their positions and 0x00 elsewhere. */
int prune24_decompress(const uint8_t *a_vals, const uint8_t *a_meta, int64_t M, int64_t K,
                       uint8_t *out, fp8_stream_t stream);

/* ---------------------------------------------------------------------------
 * Dense FP8 GEMM (rows a4, a6).  Paper: section 4 (FP8 x FP8 -> FP32 matrix
 * operation).
 *
 * C[m,n] = alpha * sa(m) * sb(n) * sum_k dec(A[m,k]) dec(B[n,k]), where
 * sa(m) = a_scale[a_mode ? m : 0] and sb(n) = b_scale[b_mode ? n : 0].
 * A: device E4M3 [M, K], row stride lda bytes; B: device E4M3 [N, K], row
 * stride ldb bytes.  A, B 16-byte aligned, lda and ldb multiples of 16
 * (FP8_ERR_ALIGN otherwise).  M, N, K >= 0 arbitrary (ragged edges are
 * zero-filled on load and masked on store; K == 0 writes zeros).
 * Products are accumulated in FP32 on the tensor cores (tcgen05, tensor
 * memory accumulators); the epilogue applies the scales in FP32.
 * C: device [M, N], row stride ldc elements, out_dtype 0 = fp32,
 * 1 = bf16 (round to nearest even).
 * Skinny products whose N-side tiles are too few to occupy the GPU (and
 * whose K is at least 4096) are split along K over several CTAs; their FP32
 * partial sums are added in a fixed order, so results are deterministic and
 * do not depend on how the problem is launched.  When the slices of a tile
 * fit one thread-block cluster (and all clusters can be resident at once)
 * they add up through distributed shared memory and need no workspace.
 * Otherwise the partials go through a workspace: a buffer kept per stream
 * (allocated with cudaMallocAsync on `stream` at the first split launch,
 * grown the same way, kept for the life of the process; at most 64 streams
 * get one; calls on further streams allocate and free one per call, ordered
 * on `stream`).  A
 * call made while `stream` is being captured gives the captured graph a
 * workspace of its own: allocated at capture time outside the capture, freed
 * once the graph and every executable graph made from it are destroyed, so
 * replays allocate nothing.  Replays of one executable graph are ordered by
 * CUDA; two executable graphs instantiated from the same captured graph must
 * not be replayed at the same time.  FP8_ERR_OOM if an allocation fails.
 * ------------------------------------------------------------------------- */
int gemm_fp8_dense(int64_t M, int64_t N, int64_t K, const uint8_t *A, int64_t lda,
                   const uint8_t *B, int64_t ldb, const float *a_scale, int a_mode,
                   const float *b_scale, int b_mode, float alpha, void *C, int64_t ldc,
                   int out_dtype, fp8_stream_t stream);

/* gemm_fp8_dense with a format for each operand: A's codes decode as
 * a_format and B's as b_format, each an fp8_format (FP8_ERR_INVALID
 * otherwise), so the four pairings of paper Table 3 (E4M3 x E4M3,
 * E4M3 x E5M2, E5M2 x E4M3, E5M2 x E5M2) run on the same kernel; only the
 * tensor-core instruction descriptor changes.  gemm_fp8_dense is this call
 * with FP8_E4M3 for both.  Everything else as gemm_fp8_dense. */
int gemm_fp8_dense_fmt(int64_t M, int64_t N, int64_t K, const uint8_t *A, int64_t lda,
                       const uint8_t *B, int64_t ldb, const float *a_scale, int a_mode,
                       const float *b_scale, int b_mode, float alpha, void *C, int64_t ldc,
                       int out_dtype, int a_format, int b_format, fp8_stream_t stream);

/* ---------------------------------------------------------------------------
 * gemm_fp8_dense without any device allocation.  (The paper has no
 * counterpart: this serves callers of the library.)
 *
 * Same arguments, results and errors as gemm_fp8_dense.  That call may
 * allocate the scratch of a split-K launch (partial sums of skinny products,
 * see above) with cudaMallocAsync; this one uses a fixed 4 MiB array that
 * the library keeps in every device's global memory instead, so it never
 * calls cudaMalloc, cudaMallocAsync or any other allocating routine.  It is
 * meant for callers that must not allocate while serving a request: systems
 * that plan their whole device memory budget up front (a failed or blocking
 * allocation mid-request is not acceptable there), and code that runs inside
 * an allocator's own callbacks or out-of-memory handling, where allocating
 * again would re-enter the allocator.
 *
 * Limits and caveats:
 *   - a problem whose split-K scratch exceeds 4 MiB is rejected with
 *     FP8_ERR_SHAPE and nothing is launched.  Only products with M <= 128
 *     (or N <= 128) and K >= 4096 split; when the slices of each tile add
 *     up within a thread-block cluster (the other slices' partial sums fit
 *     in a CTA's shared-memory ring) they need no scratch.  Otherwise the
 *     scratch is 256 bytes of counters plus tiles x slices x 128 x (N-tile
 *     width) floats, tiles x slices at most the SM count: skinny products
 *     with M <= 32 always fit; M = 64 with a long side of 2432 rows and
 *     K = 8192, split in eight, needs 4.98 MB and is rejected.  Problems
 *     that do not split need none and always run;
 *   - all calls on a device share the array, which keeps the previous call's
 *     contents; each call zeroes the counters it needs (cudaMemsetAsync, not
 *     an allocation).  Calls whose kernels overlap on the GPU (for example on
 *     two streams at once) race on the array: serialise them;
 *   - the first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress); make it before any stream capture.  A lookup
 *     that fails is not remembered: the next call tries again.  Separately,
 *     under CUDA's lazy module loading (the default) the driver loads a
 *     kernel's code, and the array, on a device the first time they are
 *     used there, which can take device memory once.  Callers for whom no
 *     call may allocate set CUDA_MODULE_LOADING=EAGER (everything is loaded
 *     with the library) or make a warm-up call per device and shape class
 *     at start-up.
 * ------------------------------------------------------------------------- */
int gemm_fp8_dense_noalloc(int64_t M, int64_t N, int64_t K, const uint8_t *A, int64_t lda,
                           const uint8_t *B, int64_t ldb, const float *a_scale, int a_mode,
                           const float *b_scale, int b_mode, float alpha, void *C, int64_t ldc,
                           int out_dtype, fp8_stream_t stream);

/* ---------------------------------------------------------------------------
 * 2:4-sparse FP8 GEMM (rows a5, a6).  Paper: section 6 (sparse GEMM against
 * dense GEMM on the same operands).
 *
 * Same product as gemm_fp8_dense with A given in the compressed form written
 * by prune24_compress (a_vals [M, K/2], a_meta [M, K/8], both contiguous);
 * the result equals the dense product of the decompressed A.  K % 128 == 0
 * (FP8_ERR_SHAPE otherwise).  Sparsity is on the M-side operand; for sparse
 * weights pass the weight as A and the activations as B, and set
 * out_transposed = 1 to receive C^T, i.e. out[n, m] with row stride ldc.
 * ------------------------------------------------------------------------- */
int gemm_fp8_sparse24(int64_t M, int64_t N, int64_t K, const uint8_t *a_vals,
                      const uint8_t *a_meta, const uint8_t *B, int64_t ldb, const float *a_scale,
                      int a_mode, const float *b_scale, int b_mode, float alpha, void *C,
                      int64_t ldc, int out_dtype, int out_transposed, fp8_stream_t stream);

/* gemm_fp8_sparse24 with a format for each operand (a_format for the kept
 * codes of A, b_format for B; fp8_format values, FP8_ERR_INVALID otherwise).
 * prune24_compress serves both formats: its key (code & 0x7F) orders the
 * finite codes of either by magnitude. */
int gemm_fp8_sparse24_fmt(int64_t M, int64_t N, int64_t K, const uint8_t *a_vals,
                          const uint8_t *a_meta, const uint8_t *B, int64_t ldb,
                          const float *a_scale, int a_mode, const float *b_scale, int b_mode,
                          float alpha, void *C, int64_t ldc, int out_dtype, int out_transposed,
                          int a_format, int b_format, fp8_stream_t stream);

/* ---------------------------------------------------------------------------
 * Grouped GEMM (row a7): many independent problems in one persistent launch.
 * Paper: section 7.1 (a transformer-style sequence of FP8 GEMMs) and the
 * section 8 guidance to batch small or fragmented work.
 *
 * Each problem is a dense (A_meta == NULL) or 2:4-sparse (A = a_vals,
 * A_meta = a_meta) GEMM with the conventions above; out_transposed as in
 * gemm_fp8_sparse24 (dense problems may use it too).  The problem table is
 * passed by value in the kernel parameters (no device workspace), so one
 * launch holds at most FP8_GROUPED_MAX_PROBLEMS problems; a longer list is
 * checked as a whole and then run as consecutive launches of up to that
 * many problems each, in list order, on `stream` (the autotuner and the
 * CUDA-graph form take at most FP8_GROUPED_MAX_PROBLEMS: FP8_ERR_SHAPE).
 * One launch runs one tile kind, so (unless fp8_gemm_set_tile_config forces
 * a kind, or the autotuner has tuned this exact list) the problems that
 * would run on CTA-pair tiles alone are launched apart from the rest, one
 * launch for the dense ones and one for the 2:4 ones, after a launch of the
 * rest; the CUDA-graph form keeps the whole list in one launch.  A list
 * of one problem runs as the single call would (the same kernel variant
 * and, without a CTA cap, split-K slices added within clusters).
 * Results are bitwise identical to issuing each problem alone.
 * ------------------------------------------------------------------------- */
#define FP8_GROUPED_MAX_PROBLEMS 32

typedef struct {
    int64_t M, N, K;
    const uint8_t *A;       /* dense [M,K] codes, or a_vals [M,K/2] */
    const uint8_t *A_meta;  /* NULL for dense; a_meta [M,K/8] for 2:4 */
    int64_t lda;            /* dense only: row stride of A in bytes */
    const uint8_t *B;       /* [N,K] codes */
    int64_t ldb;
    const float *a_scale;
    int a_mode;
    const float *b_scale;
    int b_mode;
    float alpha;
    void *C;
    int64_t ldc;
    int out_dtype;
    int out_transposed;
    int a_format;           /* fp8_format of A (a zero-initialised problem is */
    int b_format;           /* E4M3 x E4M3) and of B */
} fp8_gemm_problem;

int gemm_fp8_grouped(const fp8_gemm_problem *problems, int num_problems, fp8_stream_t stream);

/* As gemm_fp8_grouped, with the grid capped at max_ctas CTAs (max_ctas <= 0:
 * one CTA per SM).  Below the SM count, SMs are left free so work on another
 * stream (a latency-sensitive tenant) runs beside this launch — the
 * occupancy-aware co-scheduling the paper recommends in section 8.2.  Above
 * it, the launch has more CTAs than SMs, each taking a few tiles and
 * running in waves, so SMs are handed back between tiles (higher-priority
 * streams get them then) instead of being held to the launch's last tile.
 * A cap of 1 never uses CTA-pair tiles (a pair needs two CTAs).  The
 * results do not depend on max_ctas. */
int gemm_fp8_grouped_ex(const fp8_gemm_problem *problems, int num_problems, int max_ctas,
                        fp8_stream_t stream);

/* Process-wide tile configuration of the GEMM kernels, for tuning and tests.
 * mt: 1 (128 x N tiles of one CTA, double-buffered accumulators), 2 (256 x N
 * tiles of one CTA: two MMAs share each B tile, a third fewer operand bytes
 * per FLOP), 3 (256 x 256 tiles of a CTA pair, tcgen05 cta_group::2: each
 * CTA of a two-CTA cluster loads 128 rows of A and 128 rows of B and holds
 * its half of the accumulator; 2:4 launches take 256 x 224 pair tiles,
 * each CTA loading the kept codes and metadata of its 128 rows of A and
 * 112 rows of B; dense launches whose N tiles are 256 wide and 2:4 launches
 * whose N tiles are at least 224 wide, otherwise as 0), 0 = chosen per
 * launch (256-row tiles when every problem fills them with N tiles >= 128
 * wide and those tiles number at least half the SMs, or, for CTA pairs
 * with K >= 4096, occupy as many SMs as 128-row tiles would: 3 when pairs
 * apply as above, else 2; a launch mixing dense and sparse problems always
 * uses 1).
 * group_m: M-blocks per raster band (0 = 16, or 8 for dense CTA-pair
 * launches whose operands exceed the L2 cache).  Results do not depend on
 * either.  Affects launches enqueued after the call, from any thread. */
int fp8_gemm_set_tile_config(int mt, int group_m);

/* B-block multicast for 128-row-tile launches.  mode 1: a single dense
 * problem that is not split along K runs as clusters of 4 (else 2) CTAs on
 * consecutive row blocks of one N column where the tiles, the grid and the
 * raster divide into such clusters: each CTA loads its own A rows (MMA-M
 * side) and a quarter (half) of the shared B block (MMA-N side), multicast
 * to the cluster by TMA, which cuts the bytes each SM reads per k-block.
 * mode 0 (default): never; measured 2-9 % slower on mid-size and skinny
 * products on GB300.  Results do not depend on it.  FP8_ERR_INVALID for any
 * other mode.  Affects launches planned after the call, from any thread. */
int fp8_gemm_set_multicast(int mode);

/* How gemm_fp8_dense would run a problem now (tile shape, split, grid),
 * without launching anything; for tuning, tests and callers of
 * gemm_fp8_dense_noalloc that size their problems against its scratch. */
typedef struct {
    int mt;                 /* tile kind as in fp8_gemm_set_tile_config (1, 2 or 3) */
    int bn;                 /* N width of a tile */
    int k_blocks_per_stage; /* 128-wide K chunks per pipeline stage */
    int splits;             /* K slices per tile (1: no split) */
    int cluster;            /* CTAs per thread-block cluster (0: no clusters) */
    int grid;               /* CTAs launched */
    int swapped;            /* 1: run as C^T = B A^T (small M on the MMA N side) */
    int group_m;            /* raster band height in tiles (fp8_gemm_set_tile_config) */
    int multicast;          /* CTAs sharing one B block by TMA multicast
                               (fp8_gemm_set_multicast; 0: none) */
    size_t workspace_bytes; /* split-K scratch the launch needs (0: none) */
} fp8_gemm_plan_info;

int gemm_fp8_dense_plan(int64_t M, int64_t N, int64_t K, int out_dtype, fp8_gemm_plan_info *info);

/* How gemm_fp8_mx would run a block-scaled problem now: mt 3 (CTA pairs,
 * 256 x 256 tiles, one accumulator per CTA, scale chunks loaded by TMA) or
 * mt 1 with bn 256 or 128 (128-row tiles).  FP8_ERR_SHAPE unless K % 32 == 0. */
int gemm_fp8_mx_plan(int64_t M, int64_t N, int64_t K, int out_dtype, fp8_gemm_plan_info *info);

/* How gemm_fp8_sparse24 would run an M x N x K 2:4 problem now: mt 3 (CTA
 * pairs, 256 x 224 tiles, two accumulators per CTA), mt 2 (256-row tiles of
 * one CTA, N <= 224) or mt 1 (128-row tiles).  A is always the sparse side
 * (swapped = 0).  FP8_ERR_SHAPE unless K % 128 == 0.  Paper: section 6 (2:4
 * sparse GEMM against dense on the same operands). */
int gemm_fp8_sparse24_plan(int64_t M, int64_t N, int64_t K, int out_dtype, fp8_gemm_plan_info *info);

/* Autotuner: times every candidate tile configuration of this exact problem
 * list on `stream` (iters timed launches each, after one warm-up; the
 * problems' outputs are written each time): tile kind mt in {1, 2, 3} (3 only
 * for dense lists whose N tiles are 256 wide and 2:4 lists whose N tiles are
 * at least 224 wide), raster band group_m in {2, 4,
 * 8, 16, 32}, and for 128-row tiles a cap of 128 or 64 on the N tile width
 * (which also selects the pipeline ring: two k-blocks per stage up to 128
 * wide).  K splits stay as the problems fix them, so no candidate changes a
 * result.  Records the fastest in the process-wide tile cache under the
 * list's shape signature (sizes, dense/sparse, output type and layout,
 * max_ctas) and returns it.  Later launches with the same signature
 * (grouped or single calls) use the cached choice unless
 * fp8_gemm_set_tile_config forces one.  Synchronises `stream`. */
typedef struct {
    int mt;
    int group_m;
    float ms_per_launch;
    int bn_max;               /* N tile cap of the choice (0: the problems' own widths) */
} fp8_tile_config;

int gemm_fp8_grouped_autotune(const fp8_gemm_problem *problems, int num_problems, int max_ctas,
                              int iters, fp8_stream_t stream, fp8_tile_config *best);

/* Persist / restore / empty the tile cache (a text file, one signature per
 * line: the signature, mt, group_m and the N tile cap; lines without the
 * cap read as 0).  Loading merges into the current cache; a malformed file
 * changes nothing and returns FP8_ERR_INVALID. */
int gemm_fp8_tune_cache_save(const char *path);
int gemm_fp8_tune_cache_load(const char *path);
int gemm_fp8_tune_cache_clear(void);

/* CUDA-graph form of a grouped launch.  create builds a one-node graph for
 * the problem list (every problem needs K > 0; FP8_ERR_SHAPE otherwise);
 * update swaps in a list with the same shape signature (new pointers,
 * scales, alpha) by rewriting the kernel node's parameters, without
 * re-capturing (FP8_ERR_SHAPE if the signature differs); launch replays it
 * on a stream.  The graph holds no pointer to the caller's problem array. */
typedef struct fp8_grouped_graph fp8_grouped_graph;

int gemm_fp8_grouped_graph_create(const fp8_gemm_problem *problems, int num_problems, int max_ctas,
                                  fp8_grouped_graph **out);
int gemm_fp8_grouped_graph_update(fp8_grouped_graph *graph, const fp8_gemm_problem *problems,
                                  int num_problems);
int gemm_fp8_grouped_graph_launch(fp8_grouped_graph *graph, fp8_stream_t stream);
int gemm_fp8_grouped_graph_destroy(fp8_grouped_graph *graph);

/* ---------------------------------------------------------------------------
 * Request server (row a8): continuous batching of FP8 GEMM requests.
 * Paper: sections 5 and 6.2 (concurrent GEMMs on separate hardware queues:
 * overlap, fairness, per-stream latency) and the section 8.2 guidance
 * (continuous batching, occupancy-aware co-scheduling, sparsity under
 * concurrency).
 *
 * A request multiplies activations x (device fp32 [M, K], quantised per row
 * by the server) with a registered resident weight W (E4M3 [N, K], dense or
 * 2:4-compressed, with its dequantisation factors) into out (device [M, N],
 * fp32 or bf16): out = alpha * dX[m] * dW[n] * dec(X) dec(W)^T.
 *
 * A scheduler thread owns the GPU work.  Each tenant has its own CUDA stream;
 * the latency tenant's stream has the highest priority.  Whenever one of a
 * bulk tenant's in-flight slots frees, the requests that arrived meanwhile
 * (FIFO, up to max_batch) are admitted if their workspace (M x K codes + M
 * scales) fits in the server's device pool, quantised by one grouped launch
 * and multiplied by one grouped persistent GEMM launch.  The latency tenant
 * is not held to an in-flight limit: its requests go out as soon as they are
 * admitted, in batches of at most latency_max_batch.  Bulk tenants' GEMMs may
 * be capped at bulk_max_ctas CTAs so latency work finds free SMs beside
 * them (a persistent GEMM keeps its SMs until its last tile).  The
 * scheduler builds each batch under the server's lock and enqueues it
 * without holding it, so submit, poll and wait never wait on a launch.  With
 * batching = 0 every request is launched on its own as soon as it is
 * admitted (one quantise + one GEMM launch per request: the per-call
 * baseline).  A request's result does not depend on what it was batched
 * with.
 *
 * Thread safety: submit, poll, wait and stats may be called from any
 * threads; register_weight must not race with submit; destroy must not race
 * with anything.  The caller owns x, out and the weight buffers and keeps
 * them alive until the request (or the server) is done.
 * ------------------------------------------------------------------------- */
#define FP8_SERVER_MAX_TENANTS 8

typedef struct {
    int num_tenants;          /* 1..FP8_SERVER_MAX_TENANTS */
    int latency_tenant;       /* tenant given the high-priority stream (-1: none) */
    int batching;             /* 1: continuous batching; 0: one launch per request */
    int max_batch;            /* requests per batch, 1..FP8_GROUPED_MAX_PROBLEMS (0: max) */
    int max_inflight;         /* in-flight batches per bulk tenant (0: 4) */
    int bulk_max_ctas;        /* grid cap for non-latency tenants' GEMMs (0: one CTA
                                 per SM; above the SM count: CTAs in waves, see
                                 gemm_fp8_grouped_ex) */
    size_t pool_bytes;        /* workspace pool; 0: free HBM minus reserve_bytes */
    size_t reserve_bytes;     /* HBM left untouched when sizing the pool (0: 1 GiB) */
    int latency_max_batch;    /* with batching: requests per batch of the latency
                                 tenant (0: 1, i.e. each of its requests is
                                 launched on its own as soon as it is admitted) */
    int latency_max_ctas;     /* CTA cap for the latency tenant's GEMMs (0: all
                                 SMs); set to the SMs bulk_max_ctas leaves free,
                                 its work never waits for SMs held by bulk GEMMs */
    size_t latency_pool_bytes; /* pool bytes that bulk tenants may not take, kept
                                 for the latency tenant's workspace (0: none) */
} fp8_server_config;

typedef struct fp8_server fp8_server;

typedef struct {
    int tenant;
    uint64_t weight;          /* handle from fp8_server_register_weight */
    int64_t M;                /* rows of x and out */
    const float *x;           /* device fp32 [M, K], row stride ldx */
    int64_t ldx;
    void *out;                /* device [M, N], row stride ldo elements */
    int64_t ldo;
    int out_dtype;            /* 0 fp32, 1 bf16 */
    float alpha;
} fp8_request;

typedef struct {
    int status;               /* FP8_OK or the error that ended the request */
    int batch_size;           /* requests in the launch that carried it */
    double t_submit_us;       /* host clock, microseconds since server creation */
    double t_launch_us;       /* when its batch was enqueued */
    double t_end_us;          /* when the GPU finished its batch */
    double t_start_us;        /* when the batch's stream reached it (the work
                                 queued before it on that stream was done):
                                 its kernels ran within [t_start_us, t_end_us] */
} fp8_result;

typedef struct {
    uint64_t submitted, completed, failed, rejected;
    uint64_t batches, kernel_launches, max_batch_seen;
    size_t pool_bytes, pool_in_use, pool_high_water;
} fp8_server_stats;

/* Creates the server on the current device.  FP8_ERR_OOM if the pool cannot
 * be allocated. */
int fp8_server_create(const fp8_server_config *cfg, fp8_server **out);

/* Host-only server for capacity planning and tests: no device work; a batch
 * takes launch_us + us_per_gflop * (its GFLOP) of simulated time, and with
 * fail_every > 0 every fail_every-th launch fails with FP8_ERR_CUDA (the
 * failure is reported on each request of that batch). */
int fp8_server_create_simulated(const fp8_server_config *cfg, double launch_us,
                                double us_per_gflop, int fail_every, fp8_server **out);

/* Finishes in-flight batches, fails queued requests with FP8_ERR_INVALID,
 * frees the pool and streams. */
int fp8_server_destroy(fp8_server *srv);

/* Registers a resident E4M3 weight: W [N, K] (row stride ldw) for dense, or
 * the 2:4 pair (W = kept codes [N, K/2], W_meta = metadata [N, K/8], K %
 * 128 == 0) when W_meta != NULL; w_scale fp32 [1] (w_mode 0) or [N]
 * (w_mode 1).  K % 16 == 0. */
int fp8_server_register_weight(fp8_server *srv, int64_t N, int64_t K, const uint8_t *W, int64_t ldw,
                               const uint8_t *W_meta, const float *w_scale, int w_mode,
                               uint64_t *handle);

/* fp8_server_register_weight for weights stored as w_format (an
 * fp8_format; FP8_ERR_INVALID otherwise).  Requests against it quantise
 * their activations to E4M3 as always, so an E5M2 weight runs the E4M3 x
 * E5M2 pairing (paper Table 3's FP8 x BF8) on the same kernels. */
int fp8_server_register_weight_fmt(fp8_server *srv, int64_t N, int64_t K, const uint8_t *W,
                                   int64_t ldw, const uint8_t *W_meta, const float *w_scale,
                                   int w_mode, int w_format, uint64_t *handle);

/* Queues a request; *ticket identifies it.  FP8_ERR_OOM if its workspace
 * can never fit in the pool; FP8_ERR_INVALID / FP8_ERR_SHAPE for bad
 * arguments. */
int fp8_server_submit(fp8_server *srv, const fp8_request *req, uint64_t *ticket);

/* FP8_PENDING while the request runs; otherwise fills *res, forgets the
 * ticket and returns the request's status (FP8_ERR_INVALID for an unknown
 * ticket). */
int fp8_server_poll(fp8_server *srv, uint64_t ticket, fp8_result *res);

/* As poll, blocking up to timeout_s seconds (FP8_PENDING on expiry). */
int fp8_server_wait(fp8_server *srv, uint64_t ticket, fp8_result *res, double timeout_s);

int fp8_server_get_stats(fp8_server *srv, fp8_server_stats *stats);

/* Microseconds since the server was created (the clock of fp8_result). */
double fp8_server_now_us(fp8_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* GB300FP8_H */
