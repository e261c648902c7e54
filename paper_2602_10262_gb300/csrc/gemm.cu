// FP8 GEMM on tcgen05 tensor cores: gemm_fp8_dense(_fmt), gemm_fp8_sparse24(_fmt)
// and gemm_fp8_grouped all run the kernel below.  Each operand is E4M3 or
// E5M2; the format only sets two fields of the MMA instruction descriptor.
//
// Roles of one CTA (192 threads, one CTA per SM, persistent over tiles):
//   warp 0, lane 0   TMA producer: for each (tile, k-block) waits for a free
//                    ring slot, arms the slot's "full" mbarrier with the
//                    expected bytes and issues two 2-D TMA loads (128B swizzle).
//   warp 1           allocates 512 TMEM columns (two accumulators of up to
//                    256 fp32 columns); lane 0 then issues the MMAs: per
//                    k-block 4 x tcgen05.mma.kind::f8f6f4 (K = 32 each) into
//                    the tile's accumulator, tcgen05.commit -> "empty" slot
//                    barrier, and after the last k-block commit -> "tmem_full".
//   warps 2..5       epilogue: tcgen05.ld of the accumulator (warp w reads
//                    TMEM lanes 32*(w%4)..), scale by alpha*sa*sb in fp32,
//                    convert, store to global; then release the accumulator.
// Two accumulators let the epilogue of tile i overlap the MMAs of tile i+1.
//
// Tile = 128 rows of P (the MMA M side) x bn rows of Q (MMA N side), bn in
// {16,...,256} per problem; K-block = 128 codes (one 128-byte swizzle row).
// P/Q are the two stored operands; for skinny products the host swaps them
// (P = B, Q = A) so that the long side fills the 128-row MMA and the output
// is written transposed.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "ptx.cuh"

namespace gb300 {
namespace {

constexpr int BM = 128;                   // rows of one MMA (M = 128, cta_group::1)
constexpr int BK = 128;                   // codes per k-block (one 128-byte swizzle row)
constexpr int BN_MAX = 256;
constexpr int TMEM_COLS = 512;
constexpr int GROUP_M_DEFAULT = 16;       // raster: M-blocks per band
constexpr int GROUP_M_PAIR_LARGE = 8;     // dense CTA-pair launches whose operands exceed L2
constexpr int PREFETCH_STAGES = 2;        // first-tile stages prefetched into L2 at kernel entry
// 2:4-sparse tiles: per stage the kept A codes (rows x 64 bytes, 64-byte
// swizzle) and the metadata (rows x 16 bytes) fill the A region; the metadata
// of each 128-row half is copied into a ring of TMEM columns beside that
// half's accumulator (4 columns per stage).
constexpr int SPARSE_BN_MAX = 240;
constexpr int SPARSE_BN_MAX_MT2 = 224;

// MT = 128-row MMA halves per CTA tile.
//  MT = 1: tile 128 x bn (dense and sparse problems alike), two accumulators
//          (cols 0 / 256) so the epilogue of tile i overlaps the MMAs of tile
//          i + 1.  BNC caps bn for the launch and sizes the ring: BNC = 256,
//          4 stages of 48 KB (metadata ring at cols 240..255, bn <= 240 for
//          sparse problems); BNC = 128, 6 stages of 32 KB; BNC = 64 / 32 /
//          16: 8 / 9 / 11 stages of 24 / 20 / 18 KB (narrow N, e.g. skinny
//          products whose small M is the MMA N: more loads in flight per SM
//          where few tiles exist);
//  MT = 2: tile 256 x bn; two MMAs per k-step share the B tile (a third fewer
//          operand bytes per FLOP); one accumulator spanning all 512 columns
//          (rows 0-127 in cols 0-255, rows 128-255 in cols 256-511).  Dense
//          launches (SP = false): 3 stages of 64 KB.  Sparse launches
//          (SP = true): 4 stages of 48 KB (20 KB kept codes + metadata, 28 KB
//          B with bn <= 224), metadata rings at cols 224..239 of each half.
// KC = k-blocks (128-wide K chunks) per stage.  A CTA's TMA loads complete
// at about one stage barrier per ~0.36 us whatever the bytes behind it, so
// a stage must carry enough bytes for the tile's MMA rate (or, for skinny
// products, for its share of HBM bandwidth).  Dense launches of 128-row
// tiles with bn <= 128 use KC = 2: stage = KC x (A chunk + B chunk), chunk c
// of each operand at its own 1024-aligned offset (A chunks 16 KB apart, B
// chunks bn x 128 bytes apart); BNC = 128 / 64 / 32 / 16 then run 3 / 4 / 5
// / 5 stages of 64 / 48 / 40 / 36 KB.  When K % 128 == 0 one 3-D TMA box per
// operand (x: byte in a 128-byte chunk, y: row, z: chunk) brings all KC
// chunks of a stage, else one 2-D box per chunk.  Launches whose problems
// are all 2:4-sparse (SP = true, KC = 2) hold per stage the kept codes of
// both k-blocks (8 KB each, 64-byte swizzle), then both metadata blocks
// (2 KB each), then the B chunks: 4 / 5 / 7 / 8 stages for BNC = 128 / 64 /
// 32 / 16, each k-block's metadata in its own 4 TMEM columns.  Launches
// mixing dense and sparse problems, BNC = 256 and MT = 2 keep KC = 1.
// MX: block-scaled launches (kind::mxf8f6f4): 128 x 128 or 128 x 256 tiles
// or CTA pairs, dense codes as above, and per k-block 512-byte chunks of
// E8M0 scales after the B chunks (A's 128 rows, then B's, 128 rows per
// chunk; a pair's CTA holds all 256 rows of B's), copied into a ring of
// TMEM columns (per k-block A's 4, then 4 per 128 rows of B): columns
// 128..255 beside the first of two accumulators for 128-wide tiles, from
// column 256 after the single accumulator for 256-wide ones and pairs.
// PAIR: CTA-pair launches (cta_group::2, clusters of two): a 256 x 256 tile
// per pair, each CTA loading its 128 rows of A and 128 rows of B (two
// k-blocks per stage, three 64 KB stages) and holding its 128 x 256 half of
// the accumulator; the even CTA issues the MMAs.  Per SM that is MT = 2's
// bytes per FLOP with half of MT = 2's tensor memory per accumulator.
// 2:4 pairs (SP): 256 x 224 tiles, each CTA loading the kept codes and
// metadata of its 128 rows of A and 112 rows of B per k-block (four 48 KB
// stages of two k-blocks); two 224-column accumulators at columns 0 and 256
// and the metadata ring between them (columns 224..255, each CTA holding its
// own rows' metadata).
constexpr int PAIR_TMEM_COLS = 512;       // columns per CTA: two accumulators (the epilogue of
                                          // one tile overlaps the MMAs of the next)

template <int MT, bool SP = false, int BNC = BN_MAX, int KC = 1, bool MX = false, bool PAIR = false>
struct Cfg {
    static constexpr bool kSparse2 = MT == 2 && SP;
    static constexpr int kStages =
        PAIR ? (SP ? 4 : 3) :
        KC == 2 ? (SP ? (BNC == 128 ? 4 : (BNC == 64 ? 5 : (BNC == 32 ? 7 : 8)))
                      : (BNC == 128 ? 3 : (BNC == 64 ? 4 : 5)))
                : MT == 2 ? (SP ? 4 : 3)
                          : (BNC == 256 ? 4 : (BNC == 128 ? 6 : (BNC == 64 ? 8 : (BNC == 32 ? 9 : 11))));
    static constexpr int kSpChunk = MT * BM * BK / 2;            // kept codes of one k-block
    static constexpr int kMetaChunk = MT * BM * BK / 8;          // metadata of one k-block
    // A bytes of one k-block: dense codes, or (SP launches) kept codes +
    // metadata; 128-row dense-capable tiles also hold a sparse k-block there
    static constexpr int kAChunk = SP ? kSpChunk + kMetaChunk : MT * BM * BK;
    static constexpr int kBChunk = PAIR ? (BNC / 2) * BK : kSparse2 ? SPARSE_BN_MAX_MT2 * BK : BNC * BK;
    static constexpr int kABytes = KC * kAChunk;
    static constexpr int kBBytes = KC * kBChunk;
    static constexpr int kSfChunk = 512;                        // scales of 128 rows x one k-block
    // MX: 128-row scale chunks of B per k-block (a pair's MMA reads all 256
    // rows' scales from each CTA's tensor memory, so each CTA holds both)
    static constexpr int kSfQ = MX ? BNC / 128 : 0;
    // MX: A's chunk and B's chunks of each k-block, rounded up to whole
    // swizzle atoms
    static constexpr int kSfBytes = MX ? (KC * (1 + kSfQ) * kSfChunk + 1023) / 1024 * 1024 : 0;
    // MX: the scale ring's TMEM columns (per k-block 4 for A, 4 per 128 rows
    // of B): beside the first accumulator for 128-wide tiles, after the
    // single accumulator for 256-wide ones
    static constexpr int kSfCols = 4 * (1 + kSfQ);
    static constexpr int kSfCol0 = (MX && BNC == BN_MAX) ? BN_MAX : BNC;
    static constexpr int kStageBytes = kABytes + kBBytes + kSfBytes;
    static constexpr int kMetaCol0 = kSparse2 ? SPARSE_BN_MAX_MT2 : (BNC == 256 ? SPARSE_BN_MAX : BNC);
    static constexpr int kTmemCols = PAIR ? PAIR_TMEM_COLS : TMEM_COLS;
    static constexpr int kAcc = (PAIR && !MX) ? PAIR_TMEM_COLS / BN_MAX
                                              : ((MT == 2 || (MX && BNC == BN_MAX)) ? 1 : 2);   // accumulators
    // epilogue warps: 4 per 128 rows (one per TMEM lane quarter); 256-wide
    // 128-row tiles (and pairs) use 8, two per lane quarter splitting the
    // columns, so each SM sub-partition has a second warp to hide latencies
    static constexpr int kEpiSplit = (MT == 1 && (BNC == BN_MAX || PAIR) && !MX) ? 2 : 1;
    static constexpr int kEpiWarps = 4 * MT * kEpiSplit;
    static constexpr int kThreads = 64 + 32 * kEpiWarps;         // producer, MMA, epilogue warps
    // staging buffers of 32 rows x 128 B per epilogue warp: two where they
    // fit, so a chunk is packed while the previous chunk's TMA store still
    // reads its buffer
    static constexpr int kSmemBase = 1024 + kStages * kStageBytes + 256;
    static constexpr int kEpiBufs = kSmemBase + 2 * kEpiWarps * 32 * 128 <= 232448 ? 2 : 1;
    static constexpr int kEpiBytes = kEpiBufs * kEpiWarps * 32 * 128;
    static constexpr int kSmem = kSmemBase + kEpiBytes;
    static_assert((PAIR && !SP) || kMetaCol0 + 4 * kStages * KC <= BN_MAX,
                  "metadata ring must fit beside the accumulator");
    static_assert(KC * (kSpChunk + kMetaChunk) <= kABytes || (MT == 2 && !SP),
                  "sparse A + metadata fit the A region");
    static_assert(kStageBytes % 1024 == 0 && kABytes % 1024 == 0, "swizzle atoms stay aligned");
    static_assert(kSmem <= 232448, "shared memory per CTA");
    static_assert((2 * kStages + 2 * kAcc + 3) * 8 + 12 <= 256, "barriers and flags fit their 256-byte region");
    static_assert(MT == 1 || BNC == BN_MAX, "narrow rings are for 128-row tiles");
    static_assert(KC == 1 || (KC == 2 && MT == 1 && (BNC <= 128 || PAIR)), "two-chunk stages: 128-row tiles");
    static_assert(!PAIR || (MT == 1 && KC == 2 && BNC == (SP ? SPARSE_BN_MAX_MT2 : BN_MAX)),
                  "CTA pairs: dense 256 x 256 or 2:4 256 x 224 tiles");
    static_assert(kBChunk % 1024 == 0, "B chunks stay swizzle-atom aligned");
    static_assert(!MX || (MT == 1 && !SP && (BNC == 128 || (BNC == BN_MAX && (KC == 1 || PAIR)))),
                  "block-scaled launches: 128-row dense tiles, 128 or 256 wide, or CTA pairs");
    static_assert(!MX || kSfCol0 + kSfCols * kStages * KC <= (kAcc == 1 ? TMEM_COLS : BN_MAX),
                  "scale ring fits beside the accumulators");
};

// Everything of a problem but its tensor maps.  Each role thread copies this
// part into registers once per tile, so its inner loops read no kernel
// parameter memory.
struct ProblemScalars {
    const float* sp;        // scale of P rows (mode sp_mode)
    const float* sq;        // scale of Q rows
    void* C;
    long long ldc;
    int rows_p, rows_q, K;
    int sp_mode, sq_mode;
    float alpha;
    int out_bf16;
    int trans_out;          // 0: C[i * ldc + j]; 1: C[j * ldc + i]  (i: P row, j: Q row)
    int vec_store;          // 16-byte stores allowed in the non-transposed path
    int bn;
    int sparse;             // P holds kept codes [rows_p, K/2] + metadata in tmE
    int tma3d;              // tmP / tmQ are 3-D chunk views (one box per operand per stage)
    int tma_store;          // tmC is a map of C: full output chunks leave through TMA stores
    int m_blocks, n_blocks, k_blocks;
    int splits;             // k-slices per tile (split-K); 1 = none
    int kb_per_split;       // k-blocks per slice
    long long ws_off;       // split-K: first partial (floats) of this problem in the workspace
    int ctr_off;            // split-K: first tile counter of this problem
    int tile_start;         // first work unit (tile x slice) of this problem
    uint32_t idesc;
    const uint8_t* sfp;     // block-scaled only: tiled E8M0 scales of P and Q (512-byte
    const uint8_t* sfq;     // chunks, sf_kb per 128-row tile)
    int sf_kb;
};

struct Problem : ProblemScalars {
    CUtensorMap tmP;        // P [rows_p, K] codes, box {128, 128 * MT}
    CUtensorMap tmQ;        // Q [rows_q, K] codes, box {128, bn}
    CUtensorMap tmE;        // sparse: metadata [rows_p, K/8], box {16, 128 * MT}; block-scaled CTA
                            // pairs: P's scale chunks [chunks][32][16 bytes], box {16, 32, KC}
    CUtensorMap tmSFQ;      // block-scaled CTA pairs: Q's scale chunks, as tmE
    CUtensorMap tmC;        // C [rows_p, rows_q] (row stride ldc), box {128 bytes, 32 rows}, 128-byte swizzle
};

template <int MAXP>
struct Params {
    Problem prob[MAXP];
    int num_problems;
    int total_tiles;
    int group_m;
    int* err;
    float* ws;              // split-K partial sums (nullptr when no problem splits)
    unsigned* ctr;          // split-K arrival counters, zero between launches
    int cluster_split;      // > 0: one problem whose split tiles run as clusters of this many CTAs
    int mc;                 // > 0: clusters of this many CTAs take consecutive tiles of one N column;
                            // each loads 1/mc of the shared Q block and multicasts it to all
    unsigned long long wait_ns;   // limit of every bounded wait (kWaitLimitNs unless a test sets another)
    int withhold_loads;     // failure-path test: the producer issues no loads, so the MMA warp's
                            // first wait runs past wait_ns and the launch ends with FP8_ERR_TIMEOUT
};

struct TileCoord {
    int p, m_blk, n_blk;
    int tile;               // tile index within its problem
    int slice;              // k-slice of the unit
};

template <int MAXP>
__device__ __forceinline__ TileCoord tile_coord(const Params<MAXP>& prm, int tile)
{
    int p = 0;
#pragma unroll 1
    while (p + 1 < MAXP && p + 1 < prm.num_problems && prm.prob[p + 1].tile_start <= tile)
        ++p;
    const Problem& P = prm.prob[p];
    const int unit = tile - P.tile_start;
    const int lt = unit / P.splits;
    const int gm = prm.group_m;
    const int per_band = gm * P.n_blocks;
    const int band = lt / per_band;
    const int first_m = band * gm;
    const int rows_in_band = min(P.m_blocks - first_m, gm);
    const int r = lt - band * per_band;
    return {p, first_m + r % rows_in_band, r / rows_in_band, lt, unit - lt * P.splits};
}

__device__ __forceinline__ void abort_pipeline(volatile int* flag, int* err)
{
    report_device_error(err, FP8_ERR_TIMEOUT);
    *flag = 1;
}

// ---------------------------------------------------------------- epilogue

// Column scales of the tile, 32 columns (one window) at a time: lane l
// holds the scale of column 32 w + l of window w (0 past the last column).
// Two windows are kept loaded ahead of use, and the first two are loaded
// before the epilogue waits for the accumulator, so the scale loads do not
// add their latency to the epilogue.
struct ScaleWindows {
    float w0, w1;           // the next two windows to hand out
    int next;               // column (from the first) of the window after w1
    int width;              // columns this warp covers

    __device__ __forceinline__ static float load(const ProblemScalars& P, int j, int lane)
    {
        j += lane;
        return j < P.rows_q ? __ldg(P.sq + (P.sq_mode ? j : 0)) : 0.0f;
    }
    __device__ __forceinline__ void init(const ProblemScalars& P, int jbase, int lane, int cols)
    {
        width = cols;
        w0 = load(P, jbase, lane);
        w1 = cols > 32 ? load(P, jbase + 32, lane) : 0.0f;
        next = 64;
    }
    // The window at tile columns 32 k .. 32 k + 31 for k = 0, 1, 2, ... in turn.
    __device__ __forceinline__ float take(const ProblemScalars& P, int jbase, int lane)
    {
        const float s = w0;
        w0 = w1;
        w1 = next < width ? load(P, jbase + next, lane) : 0.0f;
        next += 32;
        return s;
    }
};

// Scale 16 accumulator values (columns j0 .. j0+15 of row i) and store them.
// sw: the scale window holding those columns, at lane offset j_off.
__device__ __forceinline__ void store_vals16(const ProblemScalars& P, int i, bool row_ok, float fi, int j0,
                                             const float (&acc)[16], float sw, int j_off)
{
    float v[16];
    const int rows_q = P.rows_q;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        const float sj = __shfl_sync(0xFFFFFFFFu, sw, j_off + t);
        v[t] = __fmul_rn(__fmul_rn(acc[t], fi), sj);
    }
    if (!row_ok)
        return;
    if (!P.trans_out) {
        if (P.out_bf16) {
            __nv_bfloat16* c = static_cast<__nv_bfloat16*>(P.C) + static_cast<long long>(i) * P.ldc + j0;
            if (P.vec_store && j0 + 16 <= rows_q) {
                uint32_t w[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * t], v[2 * t + 1]);
                    w[t] = *reinterpret_cast<uint32_t*>(&h);
                }
                reinterpret_cast<uint4*>(c)[0] = make_uint4(w[0], w[1], w[2], w[3]);
                reinterpret_cast<uint4*>(c)[1] = make_uint4(w[4], w[5], w[6], w[7]);
            } else {
#pragma unroll
                for (int t = 0; t < 16; ++t)
                    if (j0 + t < rows_q)
                        c[t] = __float2bfloat16_rn(v[t]);
            }
        } else {
            float* c = static_cast<float*>(P.C) + static_cast<long long>(i) * P.ldc + j0;
            if (P.vec_store && j0 + 16 <= rows_q) {
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    reinterpret_cast<float4*>(c)[t] =
                        make_float4(v[4 * t], v[4 * t + 1], v[4 * t + 2], v[4 * t + 3]);
            } else {
#pragma unroll
                for (int t = 0; t < 16; ++t)
                    if (j0 + t < rows_q)
                        c[t] = v[t];
            }
        }
    } else {
        // C[j, i]: for a fixed j the 32 lanes write 32 consecutive i
        if (P.out_bf16) {
            __nv_bfloat16* c = static_cast<__nv_bfloat16*>(P.C) + i;
#pragma unroll
            for (int t = 0; t < 16; ++t)
                if (j0 + t < rows_q)
                    c[static_cast<long long>(j0 + t) * P.ldc] = __float2bfloat16_rn(v[t]);
        } else {
            float* c = static_cast<float*>(P.C) + i;
#pragma unroll
            for (int t = 0; t < 16; ++t)
                if (j0 + t < rows_q)
                    c[static_cast<long long>(j0 + t) * P.ldc] = v[t];
        }
    }
}

__device__ __forceinline__ void store_chunk16(const ProblemScalars& P, int i, bool row_ok, float fi,
                                              int j0, const uint32_t (&r)[16], float sw, int j_off)
{
    float acc[16];
#pragma unroll
    for (int t = 0; t < 16; ++t)
        acc[t] = __uint_as_float(r[t]);
    store_vals16(P, i, row_ok, fi, j0, acc, sw, j_off);
}

// Split-K, part 1: this unit's partial sums (row `row` of the tile, straight
// from TMEM) go to its slot of the workspace.  A slot holds the tile column
// by column (element (row, col) at col * rows_per_tile + row), so the 32
// lanes of a warp, which own 32 consecutive rows, store 128 contiguous bytes
// per column.
__device__ __forceinline__ void split_write_partial(const ProblemScalars& P, float* ws, int rows_per_tile,
                                                    int tile, int slice, int row, uint32_t taddr, int c_lo,
                                                    int c_hi)
{
    float* dst = ws + P.ws_off + (static_cast<long long>(tile) * P.splits + slice) * rows_per_tile * P.bn + row;
    for (int c0 = c_lo; c0 < c_hi; c0 += 16) {
        uint32_t r[16];
        tmem_ld_32x32b_x16(taddr + c0, r);
        tmem_ld_wait();
#pragma unroll
        for (int t = 0; t < 16; ++t)
            __stcg(dst + static_cast<long long>(c0 + t) * rows_per_tile, __uint_as_float(r[t]));
    }
}

// Split-K, part 2 (the tile's last unit only): add the partials of every
// slice in slice order and store the scaled result.
__device__ __forceinline__ void split_reduce_store(const ProblemScalars& P, const float* ws, int rows_per_tile,
                                                   int tile, int row, int i, bool row_ok, float fi, int jbase,
                                                   ScaleWindows& sw, int lane, int c_lo, int c_hi)
{
    const float* src = ws + P.ws_off + static_cast<long long>(tile) * P.splits * rows_per_tile * P.bn + row;
    const long long slot = static_cast<long long>(rows_per_tile) * P.bn;
    float s_cur = 0.0f;
    for (int c0 = c_lo; c0 < c_hi; c0 += 16) {
        if ((c0 & 31) == 0)
            s_cur = sw.take(P, jbase + c_lo, lane);
        float acc[16];
#pragma unroll
        for (int t = 0; t < 16; ++t)
            acc[t] = 0.0f;
        for (int sl = 0; sl < P.splits; ++sl) {
            const float* col = src + sl * slot + static_cast<long long>(c0) * rows_per_tile;
#pragma unroll
            for (int t = 0; t < 16; ++t)
                acc[t] = __fadd_rn(acc[t], __ldcg(col + static_cast<long long>(t) * rows_per_tile));
        }
        store_vals16(P, i, row_ok, fi, jbase + c0, acc, s_cur, c0 & 31);
    }
}

// Split-K within a cluster (one unit per CTA, the slices of a tile as the
// CTAs of one cluster, rank = slice).  Slice r > 0 writes its partial sums
// into the idle TMA ring of the cluster's rank-0 CTA, column by column
// (element (row, col) of slice r at ((r - 1) * bn + col) * rows_per_tile +
// row floats from the ring's start).
__device__ __forceinline__ void cluster_send_partial(const ProblemScalars& P, uint32_t leader_ring,
                                                     int rows_per_tile, int slice, int row, uint32_t taddr,
                                                     int c_lo, int c_hi)
{
    const uint32_t base = leader_ring + 4u * static_cast<uint32_t>((slice - 1) * P.bn * rows_per_tile + row);
    for (int c0 = c_lo; c0 < c_hi; c0 += 16) {
        uint32_t r[16];
        tmem_ld_32x32b_x16(taddr + c0, r);
        tmem_ld_wait();
#pragma unroll
        for (int t = 0; t < 16; ++t)
            st_cluster_f32(base + 4u * static_cast<uint32_t>((c0 + t) * rows_per_tile), __uint_as_float(r[t]));
    }
}

// The rank-0 CTA: its own partial from TMEM, then the other slices' from its
// ring, added in slice order (the same sums as the global split path), then
// scaled and stored.
__device__ __forceinline__ void cluster_reduce_store(const ProblemScalars& P, const uint8_t* ring,
                                                     int rows_per_tile, int row, uint32_t taddr, int i,
                                                     bool row_ok, float fi, int jbase, ScaleWindows& sw,
                                                     int lane, int c_lo, int c_hi)
{
    const float* recv = reinterpret_cast<const float*>(ring) + row;
    float s_cur = 0.0f;
    for (int c0 = c_lo; c0 < c_hi; c0 += 16) {
        if ((c0 & 31) == 0)
            s_cur = sw.take(P, jbase + c_lo, lane);
        uint32_t r[16];
        tmem_ld_32x32b_x16(taddr + c0, r);
        tmem_ld_wait();
        float acc[16];
#pragma unroll
        for (int t = 0; t < 16; ++t)
            acc[t] = __fadd_rn(0.0f, __uint_as_float(r[t]));
        for (int sl = 1; sl < P.splits; ++sl) {
            const float* col = recv + ((sl - 1) * P.bn + c0) * rows_per_tile;
#pragma unroll
            for (int t = 0; t < 16; ++t)
                acc[t] = __fadd_rn(acc[t], col[t * rows_per_tile]);
        }
        store_vals16(P, i, row_ok, fi, jbase + c0, acc, s_cur, c0 & 31);
    }
}

// Coalesced epilogue for a row-major output (trans_out == 0, 16-byte stores
// allowed).  The warp owns 32 tile rows (TMEM lanes); per chunk of 128 bytes
// of output columns (64 bf16 or 32 fp32) each thread scales its row's
// accumulators, packs them and writes the 128 bytes into the warp's staging
// buffer (16-byte pieces XOR-swizzled by row: conflict-free on both sides);
// then 8 lanes per row copy 4 rows x 128 contiguous bytes per instruction.
// The staging buffer of a warp is 32 rows x 128 bytes, 1024-aligned, with
// 16-byte piece k of row r at (k ^ (r & 7)) * 16: the layout of a TMA box
// {128 bytes, 32 rows} with 128-byte swizzle.  Full-width chunks leave
// through one TMA store issued by lane 0 (which clips rows and columns
// outside C); lane 0 waits until that store has read the buffer before the
// buffer is written again.  A partial last chunk (bn not a multiple of the
// chunk width) is copied out by the lanes, masked, so no store reaches the
// next tile's columns.
template <int ESZ, int LB, int NB>  // LB: 16-column TMEM loads in flight per wait (1 or 2); NB: staging buffers
__device__ __forceinline__ void epilogue_rows_coalesced(const ProblemScalars& P, uint32_t taddr, int row0,
                                                        float fi, int jbase, uint8_t* bufs, int lane,
                                                        ScaleWindows& sw, const CUtensorMap* tmC, int c_lo,
                                                        int c_hi)
{
    constexpr int CW = 128 / ESZ;                     // columns per chunk
    const int rows_q = P.rows_q;
    int nb = 0;                                       // staging buffer of this chunk
    for (int c0 = c_lo; c0 < c_hi; c0 += CW) {
        uint8_t* buf = bufs + nb * (32 * 128);
        nb = NB == 2 ? nb ^ 1 : 0;
        const int cw = min(CW, c_hi - c0);           // multiple of 16
        // column scales of the chunk: lane l holds columns c0 + l and c0 + 32 + l
        const float s_lo = sw.take(P, jbase + c_lo, lane);
        const float s_hi = (CW > 32 && c0 + 32 < c_hi) ? sw.take(P, jbase + c_lo, lane) : 0.0f;
        uint32_t packed[32];
        // scale + convert 16 columns starting at column c of the chunk
        auto convert16 = [&](const uint32_t (&r)[16], int q) {
#pragma unroll
            for (int t = 0; t < 16; t += 2) {
                const int c = q + t;                          // compile-time column in chunk
                const float s0 = __shfl_sync(0xFFFFFFFFu, c < 32 ? s_lo : s_hi, c & 31);
                const float s1 = __shfl_sync(0xFFFFFFFFu, c + 1 < 32 ? s_lo : s_hi, (c + 1) & 31);
                const float v0 = __fmul_rn(__fmul_rn(__uint_as_float(r[t]), fi), s0);
                const float v1 = __fmul_rn(__fmul_rn(__uint_as_float(r[t + 1]), fi), s1);
                if (ESZ == 2) {
                    __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
                    packed[c / 2] = *reinterpret_cast<uint32_t*>(&h);
                } else {
                    packed[c] = __float_as_uint(v0);
                    packed[c + 1] = __float_as_uint(v1);
                }
            }
        };
        if constexpr (LB == 2) {
#pragma unroll
            for (int q = 0; q < CW; q += 32) {
                uint32_t ra[16], rb[16];
                if (q < cw)
                    tmem_ld_32x32b_x16(taddr + c0 + q, ra);
                if (q + 16 < cw)
                    tmem_ld_32x32b_x16(taddr + c0 + q + 16, rb);
                tmem_ld_wait();
                if (q < cw)
                    convert16(ra, q);
                if (q + 16 < cw)
                    convert16(rb, q + 16);
            }
        } else {
#pragma unroll
            for (int q = 0; q < CW; q += 16) {
                if (q < cw) {
                    uint32_t r[16];
                    tmem_ld_32x32b_x16(taddr + c0 + q, r);
                    tmem_ld_wait();
                    convert16(r, q);
                }
            }
        }
        const int nck = cw * ESZ / 16;                   // 16-byte pieces per row
        const bool via_tma = tmC != nullptr && cw == CW;
        if (tmC != nullptr) {
            // the store that last used this buffer (NB chunks ago) must have read it
            if (lane == 0) {
                if (NB == 2)
                    bulk_wait_read_1();
                else
                    bulk_wait_read_all();
            }
            __syncwarp();
        }
        uint8_t* my_row = buf + lane * 128;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k < nck)
                *reinterpret_cast<uint4*>(my_row + ((k ^ (lane & 7)) << 4)) =
                    make_uint4(packed[4 * k], packed[4 * k + 1], packed[4 * k + 2], packed[4 * k + 3]);
        if (via_tma) {
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                tma_store_2d(tmC, smem_u32(buf), jbase + c0, row0);
                bulk_commit();
            }
            continue;
        }
        __syncwarp();
        const int k = lane & 7;
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int r = it * 4 + (lane >> 3);
            const int gi = row0 + r;
            if (k < nck && gi < P.rows_p) {
                const uint4 val = *reinterpret_cast<const uint4*>(buf + r * 128 + ((k ^ (r & 7)) << 4));
                const int gj = jbase + c0 + k * (16 / ESZ);
                uint8_t* dst = static_cast<uint8_t*>(P.C) + (static_cast<long long>(gi) * P.ldc + gj) * ESZ;
                if (gj + 16 / ESZ <= rows_q) {
                    *reinterpret_cast<uint4*>(dst) = val;
                } else {
                    const uint8_t* src = reinterpret_cast<const uint8_t*>(&val);
                    for (int e = 0; e < 16 / ESZ && gj + e < rows_q; ++e)
                        for (int b = 0; b < ESZ; ++b)
                            dst[e * ESZ + b] = src[e * ESZ + b];
                }
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- kernel

template <int MAXP, int MT, bool SP, int BNC, int KC, bool MX = false, bool PAIR = false>
__global__ void __launch_bounds__(Cfg<MT, SP, BNC, KC, MX, PAIR>::kThreads, 1)
    gemm_fp8_kernel(const __grid_constant__ Params<MAXP> prm)
{
    using C = Cfg<MT, SP, BNC, KC, MX, PAIR>;
    constexpr int S = C::kStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~static_cast<uintptr_t>(1023));
    // ring | epilogue staging (1024-aligned, per warp 32 x 128 bytes) | barriers
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + S * C::kStageBytes + C::kEpiBytes);
    // bar[0..S) full, bar[S..2S) empty, then kAcc tmem_full, kAcc tmem_empty,
    // then drain, split-K "partials written", split-K "verdict ready"
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2 * S + 2 * C::kAcc + 3);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    uint8_t* epi_smem = smem + S * C::kStageBytes;            // epilogue staging, per warp
    volatile int* split_flag = reinterpret_cast<volatile int*>(tmem_slot + 2);

    const uint32_t smem_base = smem_u32(smem);
    const uint32_t bar_base = smem_u32(bar);
    auto full_bar = [&](int s) { return bar_base + 8u * s; };
    auto empty_bar = [&](int s) { return bar_base + 8u * (S + s); };
    auto tfull_bar = [&](int b) { return bar_base + 8u * (2 * S + b); };
    auto tempty_bar = [&](int b) { return bar_base + 8u * (2 * S + C::kAcc + b); };
    const uint32_t drain_bar = bar_base + 8u * (2 * S + 2 * C::kAcc);
    const uint32_t split_written_bar = drain_bar + 8u;
    const uint32_t split_verdict_bar = drain_bar + 16u;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    grid_launch_dependents();
    // a launch whose cluster shape does not match its plan (pairs need
    // clusters of two, cluster split-K one CTA per slice, B multicast its
    // group) does nothing: no CTA addresses a peer that is not there
    const int mc = PAIR || MX || SP || MT != 1 ? 0 : prm.mc;
    if ((PAIR ? 2u
              : (prm.cluster_split > 0 ? static_cast<uint32_t>(prm.cluster_split)
                                       : (mc > 0 ? static_cast<uint32_t>(mc) : 1u))) != cluster_nctarank()) {
        if (threadIdx.x == 0)
            report_device_error(prm.err, FP8_ERR_UNSUPPORTED);
        return;
    }
    // Loop-invariant parameters, the first tile's coordinates and problem
    // scalars are read into registers before the setup below, so their
    // parameter loads overlap it (indexed parameter reads are memory loads,
    // and the asm statements below would otherwise make the compiler repeat
    // them on the critical path).
    const int total_tiles = prm.total_tiles;
    const int cluster_split = prm.cluster_split;
    int* const err = prm.err;
    const unsigned long long wlim = prm.wait_ns;
    float* const ws = prm.ws;
    unsigned* const ctr = prm.ctr;
    // CTA pairs walk the tiles pair by pair (both CTAs of a pair take the
    // same tiles); other launches CTA by CTA
    const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
    const int qrank = mc > 0 ? static_cast<int>(cluster_ctarank()) : 0;
    const uint16_t mc_mask = static_cast<uint16_t>((1u << (mc > 0 ? mc : 1)) - 1u);
    const int tile0 = PAIR ? static_cast<int>(blockIdx.x >> 1) : static_cast<int>(blockIdx.x);
    const int tile_step = PAIR ? static_cast<int>(gridDim.x >> 1) : static_cast<int>(gridDim.x);
    const TileCoord tc_first = tile_coord(prm, tile0);
    const ProblemScalars P_first = prm.prob[tc_first.p];
    if (threadIdx.x == 0) {
        tma_prefetch_desc(&prm.prob[tc_first.p].tmP);
        tma_prefetch_desc(&prm.prob[tc_first.p].tmQ);
    }
    // The operand boxes of the first tile's first stages are prefetched into
    // L2 now, by an epilogue warp (idle until the first accumulator is
    // ready), so that the setup below and the dependency wait overlap their
    // DRAM latency.  A prefetch only warms L2, which every later load reads
    // through and which the hardware keeps coherent, so data the previous
    // kernel writes after it is still what the loads return.  Coordinates
    // are those of the producer's loads below (block scales are not
    // prefetched).
    if (warp == 2 && lane == 0 && tile0 < total_tiles && !prm.withhold_loads) {
        const int bn = P_first.bn;
        const int prow0 = PAIR ? tc_first.m_blk * 2 * BM + BM * static_cast<int>(rank) : tc_first.m_blk * BM * MT;
        const int pcol0 = tc_first.n_blk * bn + (PAIR ? (BNC / 2) * static_cast<int>(rank) : 0) +
                          (mc > 0 ? qrank * (bn / (mc > 0 ? mc : 1)) : 0);
        const int kb0 = tc_first.slice * P_first.kb_per_split;
        const int kb1 = min(min(P_first.k_blocks, kb0 + P_first.kb_per_split), kb0 + PREFETCH_STAGES * KC);
        const CUtensorMap* map_p = &prm.prob[tc_first.p].tmP;
        const CUtensorMap* map_q = &prm.prob[tc_first.p].tmQ;
        const CUtensorMap* map_e = &prm.prob[tc_first.p].tmE;
        const bool box3d = KC > 1 && P_first.tma3d;
        for (int kb = kb0; kb < kb1; kb += KC) {
            if (P_first.sparse) {
                if (KC > 1) {
                    tma_prefetch_l2_3d(map_p, 0, prow0, kb);
                    tma_prefetch_l2_3d(map_e, 0, prow0, kb);
                } else {
                    tma_prefetch_l2_2d(map_p, kb * (BK / 2), prow0);
                    tma_prefetch_l2_2d(map_e, kb * (BK / 8), prow0);
                }
            } else if (box3d) {
                tma_prefetch_l2_3d(map_p, 0, prow0, kb);
            } else {
                for (int c = 0; c < KC && kb + c < kb1; ++c)
                    tma_prefetch_l2_2d(map_p, (kb + c) * BK, prow0);
            }
            if (box3d && mc == 0) {
                tma_prefetch_l2_3d(map_q, 0, pcol0, kb);
            } else {
                for (int c = 0; c < KC && kb + c < kb1; ++c)
                    tma_prefetch_l2_2d(map_q, (kb + c) * BK, pcol0);
            }
        }
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full_bar(s), 1);
            // Q multicast: a slot is free once every CTA of the cluster has
            // finished with it (their commits all arrive here)
            mbar_init(empty_bar(s), mc > 0 ? mc : 1);
        }
        for (int b = 0; b < C::kAcc; ++b) {
            mbar_init(tfull_bar(b), 1);
            // pairs: the even CTA's barrier counts both CTAs' epilogue threads
            mbar_init(tempty_bar(b), (PAIR ? 2 : 1) * 32 * C::kEpiWarps);
        }
        mbar_init(drain_bar, 1);
        // cluster split-K: "written" counts the other slices' epilogue
        // threads, "verdict" is the rank-0 CTA's "ring free" signal
        mbar_init(split_written_bar, cluster_split ? (cluster_split - 1) * 32 * C::kEpiWarps : 32 * C::kEpiWarps);
        mbar_init(split_verdict_bar, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncwarp();
    if (warp == 1) {
        if constexpr (PAIR) {
            tmem_alloc_pair(smem_u32(tmem_slot), C::kTmemCols);
            tmem_relinquish_pair();
        } else {
            tmem_alloc(smem_u32(tmem_slot), C::kTmemCols);
            tmem_relinquish();
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    int my_tiles = total_tiles;                 // tiles this CTA walks (0: it takes none)
    if constexpr (PAIR) {
        // both CTAs' barriers and tensor memory exist before either touches
        // the other's; a collective allocation gives both the same columns
        // (checked: a pair that disagrees does no work and reports an error)
        cluster_sync();
        const uint32_t peer_base = ld_shared_cluster_u32(cluster_map(smem_u32(tmem_slot), rank ^ 1u));
        if (peer_base != tmem_base) {
            my_tiles = 0;
            if (threadIdx.x == 0)
                report_device_error(err, FP8_ERR_UNSUPPORTED);
        }
    }
    // Q multicast: every CTA's barriers exist before a peer's copies or
    // commits reach them
    if (!PAIR && mc > 0)
        cluster_sync();
    // Everything above reads only the kernel parameters and shared memory;
    // from here on the previous kernel's outputs (operands, scales, the
    // split-K workspace) are read and written.
    grid_dependency_wait();

    // Roles are chosen per warp; inside warps 0 and 1 only lane 0 works.
    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------ TMA producer
            int stage = 0;
            uint32_t phase = 0;
            uint32_t armed = 0;                 // bit s: slot s armed at least once
            bool ok = true;
            const int producer_tiles = prm.withhold_loads ? 0 : my_tiles;
            // pairs: the even CTA arms its "full" barrier for both CTAs' bytes
            // and both CTAs' loads complete on it
            const uint32_t full_rank = PAIR ? 0u : rank;
            for (int tile = tile0; ok && tile < producer_tiles; tile += tile_step) {
                const TileCoord tc = tile == tile0 ? tc_first : tile_coord(prm, tile);
                const bool first = tile == tile0;
                const ProblemScalars P = first ? P_first : prm.prob[tc.p];
                const int sf_q_tiles = MX ? (P.rows_q + BM - 1) / BM : 0;     // B's 128-row scale tiles
                if (!first || P.sparse || (PAIR && MX)) {
                    tma_prefetch_desc(&prm.prob[tc.p].tmP);
                    tma_prefetch_desc(&prm.prob[tc.p].tmQ);
                    if (P.sparse || (PAIR && MX))
                        tma_prefetch_desc(&prm.prob[tc.p].tmE);
                    if (PAIR && MX)
                        tma_prefetch_desc(&prm.prob[tc.p].tmSFQ);
                }
                const CUtensorMap* map_p = &prm.prob[tc.p].tmP;
                const CUtensorMap* map_q = &prm.prob[tc.p].tmQ;
                const CUtensorMap* map_e = &prm.prob[tc.p].tmE;
                const bool sparse = P.sparse != 0;
                const uint32_t a_bytes = sparse ? C::kSpChunk + C::kMetaChunk : C::kAChunk;
                const uint32_t b_chunk = static_cast<uint32_t>(P.bn) * BK;      // B chunks bn x 128 B apart
                const int row0 = tc.m_blk * BM * MT;
                const int col0 = tc.n_blk * P.bn;
                const int kb0 = tc.slice * P.kb_per_split;
                const int kb1 = min(P.k_blocks, kb0 + P.kb_per_split);
                for (int kb = kb0; kb < kb1; kb += KC) {
                    const int nck = min(KC, kb1 - kb);          // k-blocks in this stage
                    // a slot never armed is free: no wait on its first use
                    if (((armed >> stage) & 1u) && !mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, wlim)) {
                        ok = false;
                        abort_pipeline(abort_flag, err);
                        break;
                    }
                    const uint32_t sa = smem_base + stage * C::kStageBytes;
                    if constexpr (PAIR) {
                        // this CTA's 128 rows of A and half of the tile's B rows
                        // (2:4: kept codes and metadata of its 128 rows of A); both
                        // CTAs' copies complete on the even CTA's barrier
                        const uint32_t fb = rank == 0 ? full_bar(stage) : cluster_map(full_bar(stage), 0u);
                        const int prow0 = tc.m_blk * 2 * BM + BM * static_cast<int>(rank);
                        const int pcol0 = tc.n_blk * P.bn + (BNC / 2) * static_cast<int>(rank);
                        // block-scaled: by TMA, completing on the same barrier, each
                        // CTA's scale chunks of its 128 rows of A and of both 128-row
                        // halves of the tile's B (KC k-blocks each)
                        if (rank == 0)
                            mbar_arrive_expect_tx(fb, 2u * static_cast<uint32_t>(C::kAChunk + C::kBChunk) *
                                                              static_cast<uint32_t>(P.tma3d ? KC : nck) +
                                                          (MX ? 2u * (1 + C::kSfQ) * KC * C::kSfChunk : 0u));
                        if constexpr (MX) {
                            const uint32_t sf = sa + C::kABytes + C::kBBytes;
                            const int chunk_p = (tc.m_blk * 2 + static_cast<int>(rank)) * P.sf_kb + kb;
                            tma_load_3d_pair(sf, &prm.prob[tc.p].tmE, fb, 0, 0, chunk_p);
#pragma unroll
                            for (int h = 0; h < C::kSfQ; ++h)
                                tma_load_3d_pair(sf + (1 + h) * KC * C::kSfChunk, &prm.prob[tc.p].tmSFQ, fb, 0, 0,
                                                 (tc.n_blk * C::kSfQ + h) * P.sf_kb + kb);
                        }
                        if constexpr (SP) {
                            // kept codes of the KC k-blocks, then their metadata
                            tma_load_3d_pair(sa, map_p, fb, 0, prow0, kb);
                            tma_load_3d_pair(sa + KC * C::kSpChunk, map_e, fb, 0, prow0, kb);
                            tma_load_3d_pair(sa + C::kABytes, map_q, fb, 0, pcol0, kb);
                        } else if (P.tma3d) {
                            tma_load_3d_pair(sa, map_p, fb, 0, prow0, kb);
                            tma_load_3d_pair(sa + C::kABytes, map_q, fb, 0, pcol0, kb);
                        } else {
#pragma unroll
                            for (int c = 0; c < KC; ++c) {
                                if (c < nck) {
                                    tma_load_2d_pair(sa + c * C::kAChunk, map_p, fb, (kb + c) * BK, prow0);
                                    tma_load_2d_pair(sa + C::kABytes + c * C::kBChunk, map_q, fb, (kb + c) * BK,
                                                     pcol0);
                                }
                            }
                        }
                        armed |= 1u << stage;
                        if (++stage == S) {
                            stage = 0;
                            phase ^= 1u;
                        }
                        continue;
                    }
                    // a 3-D box always lands all KC chunks (those past K as zeros);
                    // multicast Q slices and block scales come for the nck
                    // k-blocks of the stage only
                    const uint32_t p_chunks = static_cast<uint32_t>(KC > 1 && P.tma3d ? KC : nck);
                    const uint32_t q_chunks = static_cast<uint32_t>(KC > 1 && P.tma3d && mc == 0 ? KC : nck);
                    uint32_t sf_chunks = 0;
                    if constexpr (MX) {
                        sf_chunks = 1;
                        for (int h = 0; h < C::kSfQ; ++h)
                            sf_chunks += (tc.n_blk * C::kSfQ + h < sf_q_tiles) ? 1u : 0u;
                    }
                    mbar_arrive_expect_tx(full_bar(stage),
                                          a_bytes * p_chunks + b_chunk * q_chunks +
                                              sf_chunks * C::kSfChunk * static_cast<uint32_t>(nck));
                    if (sparse && KC > 1) {
                        // kept codes then metadata of all KC k-blocks (3-D chunk boxes)
                        tma_load_3d(sa, map_p, full_bar(stage), 0, row0, kb);
                        tma_load_3d(sa + KC * C::kSpChunk, map_e, full_bar(stage), 0, row0, kb);
                    } else if (sparse) {
                        tma_load_2d(sa, map_p, full_bar(stage), kb * (BK / 2), row0);
                        tma_load_2d(sa + C::kSpChunk, map_e, full_bar(stage), kb * (BK / 8), row0);
                    } else if (KC > 1 && P.tma3d) {
                        tma_load_3d(sa, map_p, full_bar(stage), 0, row0, kb);
                    } else {
#pragma unroll
                        for (int c = 0; c < KC; ++c)
                            if (c < nck)
                                tma_load_2d(sa + c * C::kAChunk, map_p, full_bar(stage), (kb + c) * BK, row0);
                    }
                    if (mc > 0) {
                        // this CTA's 1/mc of the Q rows, into every CTA of the cluster
                        const int qrows = P.bn / (mc > 0 ? mc : 1);
                        const uint32_t qoff = static_cast<uint32_t>(qrank * qrows * BK);
#pragma unroll
                        for (int c = 0; c < KC; ++c)
                            if (c < nck)
                                tma_load_2d_multicast(sa + C::kABytes + c * b_chunk + qoff, map_q, full_bar(stage),
                                                      (kb + c) * BK, col0 + qrank * qrows, mc_mask);
                    } else if (KC > 1 && P.tma3d) {
                        tma_load_3d(sa + C::kABytes, map_q, full_bar(stage), 0, col0, kb);
                    } else {
#pragma unroll
                        for (int c = 0; c < KC; ++c)
                            if (c < nck)
                                tma_load_2d(sa + C::kABytes + c * b_chunk, map_q, full_bar(stage), (kb + c) * BK,
                                            col0);
                    }
                    if constexpr (MX) {
                        // the k-blocks of one 128-row tile are consecutive chunks;
                        // B's 128-row halves past its last row tile are not loaded
                        // (their columns are never stored)
                        const uint32_t sf = sa + C::kABytes + C::kBBytes;
                        const size_t chunk_p = static_cast<size_t>(tc.m_blk) * P.sf_kb + kb;
                        bulk_load(sf, P.sfp + chunk_p * C::kSfChunk, C::kSfChunk * nck, full_bar(stage));
#pragma unroll
                        for (int h = 0; h < C::kSfQ; ++h) {
                            const int q_tile = tc.n_blk * C::kSfQ + h;
                            if (q_tile < sf_q_tiles) {
                                const size_t chunk_q = static_cast<size_t>(q_tile) * P.sf_kb + kb;
                                bulk_load(sf + (1 + h) * KC * C::kSfChunk, P.sfq + chunk_q * C::kSfChunk,
                                          C::kSfChunk * nck, full_bar(stage));
                            }
                        }
                    }
                    armed |= 1u << stage;
                    if (++stage == S) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok && full_rank == rank) {
                // let the copies already in flight land before the CTA exits:
                // the latest arming of slot s has parity `phase` if s < stage
                // (armed in the current round), else `phase ^ 1`
                const volatile int never = 0;
                for (int s = 0; s < S; ++s) {
                    if (!(armed >> s & 1u))
                        continue;
                    const uint32_t last_parity = (s < stage) ? phase : (phase ^ 1u);
                    mbar_wait(full_bar(s), last_parity, &never, wlim);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------------------------ MMA issuer
            int stage = 0;
            uint32_t phase = 0;
            int local = 0;
            bool ok = true;
            // pairs: the even CTA issues the pair's MMAs
            const int mma_tiles = (PAIR && rank != 0) ? 0 : my_tiles;
            for (int tile = tile0; ok && tile < mma_tiles; tile += tile_step, ++local) {
                const TileCoord tc = tile == tile0 ? tc_first : tile_coord(prm, tile);
                const ProblemScalars P = tile == tile0 ? P_first : prm.prob[tc.p];
                const bool sparse = P.sparse != 0;
                const uint32_t idesc = P.idesc;
                const uint32_t b_chunk = PAIR ? static_cast<uint32_t>(C::kBChunk)
                                              : static_cast<uint32_t>(P.bn) * BK;   // B chunks bn x 128 B apart
                const int acc = local % C::kAcc;
                const uint32_t acc_phase = (local / C::kAcc) & 1;
                // an accumulator not used yet is free: no wait on its first use
                // (pairs: both CTAs' epilogues release it, the odd one remotely)
                if (local >= C::kAcc &&
                    !(PAIR ? mbar_wait_cluster(tempty_bar(acc), acc_phase ^ 1u, abort_flag, wlim)
                           : mbar_wait(tempty_bar(acc), acc_phase ^ 1u, abort_flag, wlim))) {
                    abort_pipeline(abort_flag, err);
                    break;
                }
                tc_fence_after();
                // half h of the tile accumulates into columns d_tmem + 256 h
                const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(acc * BN_MAX);
                const int kb0 = tc.slice * P.kb_per_split;
                const int kb1 = min(P.k_blocks, kb0 + P.kb_per_split);
                for (int kb = kb0; kb < kb1; kb += KC) {
                    const int nck = min(KC, kb1 - kb);          // k-blocks in this stage
                    const uint32_t first = kb == kb0 ? 0u : 1u;     // 0: overwrite the accumulator
                    if (!(PAIR ? mbar_wait_cluster(full_bar(stage), phase, abort_flag, wlim)
                               : mbar_wait(full_bar(stage), phase, abort_flag, wlim))) {
                        ok = false;
                        abort_pipeline(abort_flag, err);
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_base + stage * C::kStageBytes;
                    if constexpr (PAIR) {
#pragma unroll
                        for (int c = 0; c < KC; ++c) {
                            if (c >= nck)
                                break;
                            // each CTA's 128 rows of A and of B sit at these offsets
                            const uint64_t adesc = sdesc_kmajor_sw128(sa + c * C::kAChunk);
                            const uint64_t bdesc_c = sdesc_kmajor_sw128(sa + C::kABytes + c * b_chunk);
                            if constexpr (SP) {
                                // both CTAs' metadata of k-block c -> their own
                                // tensor memory (each CTA's 128 rows), then the
                                // M = 256 MMAs over logical K = 64 steps
                                const uint32_t sm_meta = sa + KC * C::kSpChunk + c * C::kMetaChunk;
                                const uint32_t mcol = static_cast<uint32_t>(C::kMetaCol0 + 4 * (stage * KC + c));
                                tmem_cp_128x128b_pair(tmem_base + mcol, sdesc_rows16_noswizzle(sm_meta));
                                const uint64_t sp_desc = sdesc_kmajor_sw64(sa + c * C::kSpChunk);
#pragma unroll
                                for (int k = 0; k < BK / 64; ++k)
                                    mma_sp_f8f6f4_pair(d_tmem, sp_desc + 2u * k, bdesc_c + 4u * k,
                                                       tmem_base + mcol + 2u * k, idesc,
                                                       (first | c | k) != 0 ? 1u : 0u);
                            } else if constexpr (MX) {
                                // both CTAs' scale chunks of k-block c -> their own
                                // tensor memory: A's 4 ring columns (the CTA's rows),
                                // then B's 8 (all 256 rows of the tile)
                                const uint32_t sf_col =
                                    static_cast<uint32_t>(C::kSfCol0 + C::kSfCols * (stage * KC + c));
                                const uint32_t sm_sf = sa + C::kABytes + C::kBBytes + c * C::kSfChunk;
                                tmem_cp_32x128b_warpx4_pair(tmem_base + sf_col, sdesc_rows16_noswizzle(sm_sf));
#pragma unroll
                                for (int h = 0; h < C::kSfQ; ++h)
                                    tmem_cp_32x128b_warpx4_pair(
                                        tmem_base + sf_col + 4u * (1 + h),
                                        sdesc_rows16_noswizzle(sm_sf + (1 + h) * KC * C::kSfChunk));
#pragma unroll
                                for (int k = 0; k < BK / 32; ++k)
                                    mma_mx_f8f6f4_pair(d_tmem, adesc + 2u * k, bdesc_c + 2u * k,
                                                       mx_sf_ids(idesc, static_cast<uint32_t>(k)), tmem_base + sf_col,
                                                       tmem_base + sf_col + 4u, (first | c | k) != 0 ? 1u : 0u);
                            } else {
#pragma unroll
                                for (int k = 0; k < BK / 32; ++k)
                                    mma_f8f6f4_pair(d_tmem, adesc + 2u * k, bdesc_c + 2u * k, idesc,
                                                    (first | c | k) != 0 ? 1u : 0u);
                            }
                        }
                        // the stage is free in both CTAs once these MMAs are done
                        mma_commit_pair_multicast(empty_bar(stage), 0x3);
                        if (++stage == S) {
                            stage = 0;
                            phase ^= 1u;
                        }
                        continue;
                    }
                    if constexpr (MX) {
#pragma unroll
                        for (int c = 0; c < KC; ++c) {
                            if (c >= nck)
                                break;
                            // scales of k-block c (A's 128 rows, then B's rows 128 at a
                            // time) -> their ring columns, each 32-row group to every
                            // lane quarter: B row r in column 4 + r / 32
                            const uint32_t sf_col =
                                static_cast<uint32_t>(C::kSfCol0 + C::kSfCols * (stage * KC + c));
                            const uint32_t sm_sf = sa + C::kABytes + C::kBBytes + c * C::kSfChunk;
                            tmem_cp_32x128b_warpx4(tmem_base + sf_col, sdesc_rows16_noswizzle(sm_sf));
#pragma unroll
                            for (int h = 0; h < C::kSfQ; ++h)
                                tmem_cp_32x128b_warpx4(tmem_base + sf_col + 4u * (1 + h),
                                                       sdesc_rows16_noswizzle(sm_sf + (1 + h) * KC * C::kSfChunk));
                            const uint64_t adesc = sdesc_kmajor_sw128(sa + c * C::kAChunk);
                            const uint64_t bdesc_c = sdesc_kmajor_sw128(sa + C::kABytes + c * b_chunk);
#pragma unroll
                            for (int k = 0; k < BK / 32; ++k)
                                mma_mx_f8f6f4(d_tmem, adesc + 2u * k, bdesc_c + 2u * k,
                                              mx_sf_ids(idesc, static_cast<uint32_t>(k)), tmem_base + sf_col,
                                              tmem_base + sf_col + 4u, (first | c | k) != 0 ? 1u : 0u);
                        }
                    } else if (sparse) {
#pragma unroll
                        for (int c = 0; c < KC; ++c) {
                            if (c >= nck)
                                break;
                            // metadata of k-block c -> its TMEM columns (tcgen05.cp
                            // and the MMAs below execute in issue order)
                            const uint32_t sm_meta = sa + KC * C::kSpChunk + c * C::kMetaChunk;
                            const uint32_t mcol = static_cast<uint32_t>(C::kMetaCol0 + 4 * (stage * KC + c));
#pragma unroll
                            for (int h = 0; h < MT; ++h)
                                tmem_cp_128x128b(tmem_base + h * BN_MAX + mcol,
                                                 sdesc_rows16_noswizzle(sm_meta + h * BM * 16));
                            const uint64_t bdesc_c = sdesc_kmajor_sw128(sa + C::kABytes + c * b_chunk);
#pragma unroll
                            for (int k = 0; k < BK / 64; ++k) {
#pragma unroll
                                for (int h = 0; h < MT; ++h) {
                                    // logical K = 64 per MMA: 32 kept A bytes, 64 B
                                    // bytes, 64 metadata bits (two TMEM columns)
                                    const uint64_t adesc = sdesc_kmajor_sw64(sa + c * C::kSpChunk + h * BM * 64);
                                    mma_sp_f8f6f4(d_tmem + h * BN_MAX, adesc + 2u * k, bdesc_c + 4u * k,
                                                  tmem_base + h * BN_MAX + mcol + 2u * k, idesc,
                                                  (first | c | k) != 0 ? 1u : 0u);
                                }
                            }
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < KC; ++c) {
                            if (c >= nck)
                                break;
                            const uint64_t bdesc_c = sdesc_kmajor_sw128(sa + C::kABytes + c * b_chunk);
#pragma unroll
                            for (int k = 0; k < BK / 32; ++k) {
#pragma unroll
                                for (int h = 0; h < MT; ++h) {
                                    // advance the start address by 32 bytes (K = 32 codes)
                                    const uint64_t adesc = sdesc_kmajor_sw128(sa + c * C::kAChunk + h * BM * BK);
                                    mma_f8f6f4(d_tmem + h * BN_MAX, adesc + 2u * k, bdesc_c + 2u * k, idesc,
                                               (first | c | k) != 0 ? 1u : 0u);
                                }
                            }
                        }
                    }
                    if (mc > 0)
                        mma_commit_multicast(empty_bar(stage), mc_mask);
                    else
                        mma_commit(empty_bar(stage));
                    if (++stage == S) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (ok) {
                    if constexpr (PAIR)
                        mma_commit_pair_multicast(tfull_bar(acc), 0x3);     // both CTAs' epilogues
                    else
                        mma_commit(tfull_bar(acc));
                }
            }
            // every MMA this thread issued has finished before TMEM is freed
            const volatile int never = 0;
            if constexpr (PAIR) {
                if (rank == 0) {
                    mma_commit_pair_multicast(drain_bar, 0x1);
                    mbar_wait(drain_bar, 0u, &never, wlim);
                }
            } else {
                mma_commit(drain_bar);
                mbar_wait(drain_bar, 0u, &never, wlim);
            }
        }
    } else {
        // ---------------------------------------------------- epilogue
        // warp w reads TMEM lanes 32 (w % 4) ..; with 256-row tiles of half
        // (w - 2) / 4, with two warps per lane quarter of columns [0, mid) or
        // [mid, bn) (mid: half the tile rounded up to 64 columns)
        const int quarter = warp & 3;
        const int half = MT == 2 ? (warp - 2) >> 2 : 0;
        const int cpart = C::kEpiSplit == 2 ? (warp - 2) >> 2 : 0;
        const int row = half * BM + quarter * 32 + lane;
        int local = 0;
        uint32_t split_phase = 0;
        for (int tile = tile0; tile < my_tiles; tile += tile_step, ++local) {
            const TileCoord tc = tile == tile0 ? tc_first : tile_coord(prm, tile);
            const ProblemScalars P = tile == tile0 ? P_first : prm.prob[tc.p];
            const int acc = local % C::kAcc;
            const uint32_t acc_phase = (local / C::kAcc) & 1;
            // the scales do not depend on the accumulator: load them first
            // (pairs: CTA r holds rows 128 r .. of the 256-row tile)
            const int i = PAIR ? tc.m_blk * 2 * BM + BM * static_cast<int>(rank) + row : tc.m_blk * BM * MT + row;
            const bool row_ok = i < P.rows_p;
            const float fi = row_ok ? __fmul_rn(P.alpha, __ldg(P.sp + (P.sp_mode ? i : 0))) : 0.0f;
            const int jbase = tc.n_blk * P.bn;
            // every column scale of the tile reaches L1 while its MMAs run:
            // read window by window during the epilogue, each would
            // otherwise wait a memory round trip (one line per 32 columns)
            if (warp == 2 && P.sq_mode && lane < (P.bn + 31) / 32 && jbase + 32 * lane < P.rows_q)
                prefetch_l1(P.sq + jbase + 32 * lane);
            int c_lo = 0, c_hi = P.bn;
            if (C::kEpiSplit == 2) {
                const int mid = min(P.bn, (P.bn / 2 + 63) & ~63);
                c_lo = cpart ? mid : 0;
                c_hi = cpart ? P.bn : mid;
            }
            ScaleWindows sw;
            sw.init(P, jbase + c_lo, lane, c_hi - c_lo);
            // the whole warp takes the same branch (tcgen05.ld is warp-collective)
            const bool got = mbar_wait(tfull_bar(acc), acc_phase, abort_flag, wlim);
            if (!__all_sync(0xFFFFFFFFu, got)) {
                abort_pipeline(abort_flag, err);
                break;
            }
            tc_fence_after();
            const uint32_t taddr = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) +
                                   static_cast<uint32_t>((acc + half) * BN_MAX);
            if (P.splits > 1 && cluster_split) {
                const int crank = static_cast<int>(cluster_ctarank());
                if (crank != tc.slice) {                // launch shape broken: never expected
                    abort_pipeline(abort_flag, err);
                    break;
                }
                if (crank == 0) {
                    // every MMA of this unit has completed: the ring is free
                    if (threadIdx.x == 64)
                        for (int r = 1; r < P.splits; ++r)
                            mbar_arrive_remote(cluster_map(split_verdict_bar, static_cast<uint32_t>(r)));
                    const bool got = mbar_wait_cluster(split_written_bar, 0u, abort_flag, wlim);
                    if (!__all_sync(0xFFFFFFFFu, got)) {
                        abort_pipeline(abort_flag, err);
                        break;
                    }
                    cluster_reduce_store(P, smem, BM * MT, row, taddr, i, row_ok, fi, jbase, sw, lane, c_lo, c_hi);
                } else {
                    const bool got = mbar_wait_cluster(split_verdict_bar, 0u, abort_flag, wlim);
                    if (!__all_sync(0xFFFFFFFFu, got)) {
                        abort_pipeline(abort_flag, err);
                        break;
                    }
                    cluster_send_partial(P, cluster_map(smem_base, 0u), BM * MT, crank, row, taddr, c_lo, c_hi);
                    mbar_arrive_remote(cluster_map(split_written_bar, 0u));
                }
                tc_fence_before();
                mbar_arrive(tempty_bar(acc));
                continue;
            }
            if (P.splits > 1) {
                // every epilogue thread stores its row's partials, then one
                // thread counts this unit in; the tile's last unit reduces.
                // (The verdict slot is rewritten only after every thread has
                // arrived for the next split tile, i.e. after it was read.)
                split_write_partial(P, ws, BM * MT, tc.tile, tc.slice, row, taddr, c_lo, c_hi);
                tc_fence_before();
                mbar_arrive(tempty_bar(acc));          // TMEM is free; the reduction reads global memory
                __threadfence();
                mbar_arrive(split_written_bar);
                if (threadIdx.x == 64) {
                    if (mbar_wait(split_written_bar, split_phase, abort_flag, wlim)) {
                        const unsigned prev = atomicAdd(ctr + P.ctr_off + tc.tile, 1u);
                        *split_flag = (prev == static_cast<unsigned>(P.splits - 1)) ? 1 : 0;
                    } else {
                        *split_flag = 0;
                        abort_pipeline(abort_flag, err);
                    }
                    mbar_arrive(split_verdict_bar);
                }
                const bool got_verdict = mbar_wait(split_verdict_bar, split_phase, abort_flag, wlim);
                split_phase ^= 1u;
                if (!__all_sync(0xFFFFFFFFu, got_verdict)) {
                    abort_pipeline(abort_flag, err);
                    break;
                }
                if (*split_flag) {
                    __threadfence();
                    split_reduce_store(P, ws, BM * MT, tc.tile, row, i, row_ok, fi, jbase, sw, lane, c_lo, c_hi);
                    if (threadIdx.x == 64)
                        ctr[P.ctr_off + tc.tile] = 0u;         // ready for the next launch
                }
                continue;
            }
            if (!P.trans_out && P.vec_store) {
                uint8_t* buf = epi_smem + (warp - 2) * C::kEpiBufs * 32 * 128;
                const int row0 = i - lane;
                const CUtensorMap* tmC = P.tma_store ? &prm.prob[tc.p].tmC : nullptr;
                // (kernels with 8 epilogue warps have the smaller register
                // budget: one load per wait)
                constexpr int LB = C::kEpiWarps == 4 ? 2 : 1;
                if (P.out_bf16)
                    epilogue_rows_coalesced<2, LB, C::kEpiBufs>(P, taddr, row0, fi, jbase, buf, lane, sw, tmC, c_lo,
                                                               c_hi);
                else
                    epilogue_rows_coalesced<4, LB, C::kEpiBufs>(P, taddr, row0, fi, jbase, buf, lane, sw, tmC, c_lo,
                                                               c_hi);
            } else {
                float s_cur = 0.0f;
                for (int c0 = c_lo; c0 < c_hi; c0 += 16) {
                    if ((c0 & 31) == 0)
                        s_cur = sw.take(P, jbase + c_lo, lane);
                    uint32_t r[16];
                    tmem_ld_32x32b_x16(taddr + c0, r);
                    tmem_ld_wait();
                    store_chunk16(P, i, row_ok, fi, jbase + c0, r, s_cur, c0 & 31);
                }
            }
            tc_fence_before();
            if (PAIR && rank != 0)
                mbar_arrive_remote(cluster_map(tempty_bar(acc), 0u));     // the even CTA's barrier
            else
                mbar_arrive(tempty_bar(acc));
        }
        // TMA stores issued by this warp are complete before the CTA ends
        if (lane == 0)
            bulk_wait_all();
    }

    // In warps 0 and 1 only lane 0 ran a role loop: reconverge every warp
    // before the CTA-wide barrier (bar.sync is warp-aligned).
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    // cluster split-K: no CTA leaves while a peer may still write to its
    // shared memory; pairs: neither CTA frees the pair's tensor memory (or
    // its barriers) while the other may still use them (every wait above is
    // bounded, so all threads get here)
    if (PAIR || cluster_split || mc > 0)
        cluster_sync();
    if (warp == 1) {
        tc_fence_after();
        if constexpr (PAIR)
            tmem_dealloc_pair(tmem_base, C::kTmemCols);
        else
            tmem_dealloc(tmem_base, C::kTmemCols);
    }
}

// ---------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 2-D map over a byte matrix [rows, cols] with row stride ld bytes; box
// {box_cols bytes, box_rows}; out-of-range elements read as 0.
bool make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld,
              int box_cols, int box_rows, CUtensorMapSwizzle swizzle)
{
    auto fn = encode_fn();
    if (!fn)
        return false;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld)};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(box_cols), static_cast<cuuint32_t>(box_rows)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Map of an output matrix C [rows, cols] (row stride ld elements of esz
// bytes): box {128 bytes of a row, 32 rows}, 128-byte swizzle, the layout
// of the epilogue's per-warp staging buffer.
bool make_out_map(CUtensorMap* map, void* base, int64_t rows, int64_t cols, int64_t ld, int esz)
{
    auto fn = encode_fn();
    if (!fn)
        return false;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld * esz)};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(128 / esz), 32};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base,
                    dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// 3-D view of a byte matrix [rows, cols] (cols % chunk == 0, row stride ld
// bytes) as x = byte within a chunk of K, y = row, z = chunk; box {chunk,
// box_rows, chunks}: one copy lands `chunks` tiles of box_rows x chunk bytes
// back to back in shared memory, each swizzled as a 2-D box would be.
bool make_map3(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int chunk,
               int box_rows, int chunks, CUtensorMapSwizzle swizzle)
{
    auto fn = encode_fn();
    if (!fn)
        return false;
    cuuint64_t dims[3] = {static_cast<cuuint64_t>(chunk), static_cast<cuuint64_t>(rows),
                          static_cast<cuuint64_t>(cols / chunk)};
    cuuint64_t strides[2] = {static_cast<cuuint64_t>(ld), static_cast<cuuint64_t>(chunk)};
    cuuint32_t box[3] = {static_cast<cuuint32_t>(chunk), static_cast<cuuint32_t>(box_rows),
                         static_cast<cuuint32_t>(chunks)};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// 3-D map over block-scale chunks viewed as [chunks][32][16 bytes] (the
// tiled layout: 512 bytes per 128 rows x one k-block); box {16, 32, kc}
// lands kc consecutive chunks as the contiguous bytes a bulk copy would.
bool make_sf_map(CUtensorMap* map, const void* base, int64_t chunks, int kc)
{
    auto fn = encode_fn();
    if (!fn)
        return false;
    cuuint64_t dims[3] = {16, 32, static_cast<cuuint64_t>(chunks)};
    cuuint64_t strides[2] = {16, 512};
    cuuint32_t box[3] = {16, 32, static_cast<cuuint32_t>(kc)};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// N of the MMA tile for a problem of rows_p x rows_q: the smallest of
// {16, 32, 64, 128, 256} covering rows_q, then halved (down to 64) while the
// problem has fewer 128-row tiles than half the SMs, so small problems still
// occupy the GPU.  (Halving further, to a full wave, costs more than it
// gains: every extra column block reads the P operand again, and the tiles
// run at a lower ratio of MMA work to loaded bytes.)  Depends on the problem
// only (not on what it is launched with).
int pick_bn(int64_t rows_p, int64_t rows_q, int64_t K, int bn_max)
{
    (void)K;
    int bn = 256;
    if (rows_q <= 16) bn = 16;
    else if (rows_q <= 32) bn = 32;
    else if (rows_q <= 64) bn = 64;
    else if (rows_q <= 128) bn = 128;
    const int64_t m_blocks = (rows_p + BM - 1) / BM;
    while (bn > 64 && 2 * m_blocks * ((rows_q + bn - 1) / bn) < sm_count())
        bn /= 2;
    return bn < bn_max ? bn : bn_max;
}

// Tiles of a problem at its pick_bn width.
int64_t problem_tiles(int64_t rows_p, int64_t rows_q, int64_t K)
{
    const int64_t bn = pick_bn(rows_p, rows_q, K, BN_MAX);
    return ((rows_p + BM - 1) / BM) * ((rows_q + bn - 1) / bn);
}

// True when a problem is split along K (see split_count): K spans at least
// 32 k-blocks, its Q side is at most 128 rows and its tiles fill at most
// half the SMs.  Measured on L2-cold skinny products (single calls, slices
// added within a cluster): below K = 4096, or with more tiles, the extra
// pass over the partial sums costs more than the shorter K loop saves.
bool splits_k(int64_t rows_p, int64_t rows_q, int64_t K)
{
    if ((K + BK - 1) / BK < 32 || rows_q > 128 || rows_p <= 0 || rows_q <= 0)
        return false;
    return 2 * problem_tiles(rows_p, rows_q, K) <= sm_count();
}

// One GEMM in the kernel's (P, Q) roles.
struct Job {
    int64_t rows_p, rows_q, K;
    const uint8_t* P;       // dense codes, or kept codes [rows_p, K/2] when E != nullptr
    const uint8_t* E;       // 2:4 metadata [rows_p, K/8], or nullptr for dense
    int64_t ldp;
    const uint8_t* Q;
    int64_t ldq;
    const float* sp;
    int sp_mode;
    const float* sq;
    int sq_mode;
    float alpha;
    void* C;
    int64_t ldc;
    int out_bf16;
    int trans_out;
    int fmt_p, fmt_q;       // fp8_format of P and Q (instruction-descriptor A / B format)
    const uint8_t* sfp;     // block-scaled problems: tiled E8M0 scales of P and Q
    const uint8_t* sfq;     // (nullptr otherwise)
};

bool valid_format(int f)
{
    return f == FP8_E4M3 || f == FP8_E5M2;
}

uint32_t mma_format(int f)
{
    return f == FP8_E5M2 ? kMmaFmtE5M2 : kMmaFmtE4M3;
}

// Argument checks shared by every entry point.  `sparse`: A is the kept-code
// array [M, K/2] (contiguous) and A_meta the metadata [M, K/8] (contiguous).
int validate(int64_t M, int64_t N, int64_t K, const uint8_t* A, int64_t lda, const uint8_t* A_meta,
             bool sparse, const uint8_t* B, int64_t ldb, const float* a_scale, int a_mode,
             const float* b_scale, int b_mode, void* C, int64_t ldc, int out_dtype,
             int out_transposed)
{
    if (M < 0 || N < 0 || K < 0)
        return FP8_ERR_INVALID;
    if ((a_mode != 0 && a_mode != 1) || (b_mode != 0 && b_mode != 1) ||
        (out_dtype != 0 && out_dtype != 1) || (out_transposed != 0 && out_transposed != 1))
        return FP8_ERR_INVALID;
    if (M == 0 || N == 0)
        return FP8_OK;
    if (!C || !a_scale || !b_scale)
        return FP8_ERR_INVALID;
    if (ldc < (out_transposed ? M : N))
        return FP8_ERR_SHAPE;
    if (M > INT32_MAX / 2 || N > INT32_MAX / 2 || K > INT32_MAX / 2)
        return FP8_ERR_SHAPE;
    if (K == 0)
        return FP8_OK;
    if (!A || !B || (sparse && !A_meta))
        return FP8_ERR_INVALID;
    if (sparse) {
        if (K % BK != 0)
            return FP8_ERR_SHAPE;
        if (ldb < K)
            return FP8_ERR_SHAPE;
        if (!aligned16(A) || !aligned16(A_meta) || !aligned16(B) || ldb % 16)
            return FP8_ERR_ALIGN;
        return FP8_OK;
    }
    if (lda < K || ldb < K)
        return FP8_ERR_SHAPE;
    if (!aligned16(A) || !aligned16(B) || lda % 16 || ldb % 16)
        return FP8_ERR_ALIGN;
    return FP8_OK;
}

// Split-K: k-slices for a skinny problem (Q side <= 128 rows) with too few
// tiles to occupy the GPU: each SM streams operands at a fraction of HBM
// bandwidth, so more SMs must share the long operand.  Decided from the
// problem alone (its tile count, the SM count and K), never from what it is
// launched with, so a problem sums its K range the same way alone, grouped
// or under any tile configuration.  Every slice gets at least eight k-blocks
// (K >= 1024): below that the extra pass over the partials costs more than
// the shorter K loop saves.  No slice is empty.
// k-blocks per slice when K is cut into s slices: a multiple of 4, so
// slices start on stage boundaries whatever the k-blocks per stage of the
// launch.
int slice_kblocks(int k_blocks, int s)
{
    return ((k_blocks + s - 1) / s + 3) / 4 * 4;
}

int split_count(const Job& j)
{
    const int sms = sm_count();
    if (j.sfp != nullptr || !splits_k(j.rows_p, j.rows_q, j.K))
        return 1;
    const int64_t tiles = problem_tiles(j.rows_p, j.rows_q, j.K);
    const int k_blocks = static_cast<int>((j.K + BK - 1) / BK);
    int s = std::min<int64_t>(8, sms / tiles);
    s = std::min(s, k_blocks / 8);
    if (s <= 1)
        return 1;
    const int kbs = slice_kblocks(k_blocks, s);
    return (k_blocks + kbs - 1) / kbs;
}

// Fill one problem entry for a launch with MT row-halves per tile.
int fill_problem(Problem& pr, const Job& j, int bn, int mt, int kc)
{
    memset(&pr, 0, sizeof(pr));
    pr.sparse = j.E != nullptr;
    // mt 3: a CTA pair per 256-row tile; each CTA's boxes are 128 rows of P
    // and bn / 2 rows of Q
    const bool pair = mt == 3;
    const int box_p = pair ? BM : BM * mt;
    const int box_q = pair ? bn / 2 : bn;
    const int tile_p = pair ? 2 * BM : box_p;
    if (kc > 1 && pr.sparse) {
        // sparse K is a multiple of 128: kept codes in 64-byte chunks,
        // metadata in 16-byte chunks, B in 128-byte chunks
        if (!make_map3(&pr.tmP, j.P, j.rows_p, j.K / 2, j.K / 2, BK / 2, box_p, kc, CU_TENSOR_MAP_SWIZZLE_64B) ||
            !make_map3(&pr.tmE, j.E, j.rows_p, j.K / 8, j.K / 8, BK / 8, box_p, kc, CU_TENSOR_MAP_SWIZZLE_NONE) ||
            !make_map3(&pr.tmQ, j.Q, j.rows_q, j.K, j.ldq, BK, box_q, kc, CU_TENSOR_MAP_SWIZZLE_128B))
            return FP8_ERR_CUDA;
        pr.tma3d = 1;
    } else {
        pr.tma3d = kc > 1 && j.K % BK == 0 &&
                   make_map3(&pr.tmP, j.P, j.rows_p, j.K, j.ldp, BK, box_p, kc, CU_TENSOR_MAP_SWIZZLE_128B) &&
                   make_map3(&pr.tmQ, j.Q, j.rows_q, j.K, j.ldq, BK, box_q, kc, CU_TENSOR_MAP_SWIZZLE_128B);
    }
    if (pr.tma3d) {
        // maps made above
    } else if (pr.sparse) {
        if (!make_map(&pr.tmP, j.P, j.rows_p, j.K / 2, j.K / 2, BK / 2, box_p, CU_TENSOR_MAP_SWIZZLE_64B) ||
            !make_map(&pr.tmE, j.E, j.rows_p, j.K / 8, j.K / 8, BK / 8, box_p, CU_TENSOR_MAP_SWIZZLE_NONE))
            return FP8_ERR_CUDA;
    } else if (!make_map(&pr.tmP, j.P, j.rows_p, j.K, j.ldp, BK, box_p, CU_TENSOR_MAP_SWIZZLE_128B)) {
        return FP8_ERR_CUDA;
    }
    if (!pr.tma3d && !make_map(&pr.tmQ, j.Q, j.rows_q, j.K, j.ldq, BK, box_q, CU_TENSOR_MAP_SWIZZLE_128B))
        return FP8_ERR_CUDA;
    pr.sp = j.sp;
    pr.sq = j.sq;
    pr.C = j.C;
    pr.ldc = j.ldc;
    pr.rows_p = static_cast<int>(j.rows_p);
    pr.rows_q = static_cast<int>(j.rows_q);
    pr.K = static_cast<int>(j.K);
    pr.sp_mode = j.sp_mode;
    pr.sq_mode = j.sq_mode;
    pr.alpha = j.alpha;
    pr.out_bf16 = j.out_bf16;
    pr.trans_out = j.trans_out;
    const int esz = j.out_bf16 ? 2 : 4;
    pr.vec_store = aligned16(j.C) && ((j.ldc * esz) % 16 == 0);
    pr.tma_store = pr.vec_store && !pr.trans_out && make_out_map(&pr.tmC, j.C, j.rows_p, j.rows_q, j.ldc, esz);
    pr.bn = bn;
    pr.m_blocks = static_cast<int>((j.rows_p + tile_p - 1) / tile_p);
    pr.n_blocks = static_cast<int>((j.rows_q + bn - 1) / bn);
    pr.k_blocks = static_cast<int>((j.K + BK - 1) / BK);
    pr.splits = split_count(j);
    pr.kb_per_split = pr.splits > 1 ? slice_kblocks(pr.k_blocks, pr.splits) : pr.k_blocks;
    pr.splits = (pr.k_blocks + pr.kb_per_split - 1) / pr.kb_per_split;     // no empty slice
    pr.idesc = idesc_f8_f32(pair ? 2 * BM : BM, bn, pr.sparse != 0, 0, mma_format(j.fmt_p), mma_format(j.fmt_q));
    if (j.sfp) {
        pr.idesc = idesc_mx_f8(pair ? 2 * BM : BM, bn, mma_format(j.fmt_p), mma_format(j.fmt_q));
        pr.sfp = j.sfp;
        pr.sfq = j.sfq;
        pr.sf_kb = pr.k_blocks;
        // pairs load the scale chunks by TMA (their copies complete on the
        // even CTA's barrier); chunks past the arrays read as zeros
        if (pair && (!make_sf_map(&pr.tmE, j.sfp, ((j.rows_p + BM - 1) / BM) * pr.sf_kb, kc) ||
                     !make_sf_map(&pr.tmSFQ, j.sfq, ((j.rows_q + BM - 1) / BM) * pr.sf_kb, kc)))
            return FP8_ERR_CUDA;
    }
    return FP8_OK;
}

// Zero C for K == 0 (the sum over an empty K range).
int write_zeros(void* C, int64_t ldc, int64_t rows, int64_t cols, int out_bf16, cudaStream_t st)
{
    const size_t esz = out_bf16 ? 2 : 4;
    GB_CUDA_OK(cudaMemset2DAsync(C, ldc * esz, 0, cols * esz, rows, st));
    return FP8_OK;
}

// Kernel variant, grid and shared memory of one launch.
struct Plan {
    const void* func = nullptr;
    int grid = 0, threads = 0, smem = 0;
    int cluster = 0;            // > 1: launched as clusters of this many CTAs (split-K in the
                                // cluster, or 2: CTA pairs)
    int kc = 1;                 // k-blocks per pipeline stage
    int rows_per_tile = BM;     // P rows of a CTA's tile (128 or 256)
    size_t ring_bytes = 0;      // bytes of the kernel's TMA ring
    size_t ws_floats = 0;       // split-K partials
    size_t ctr_count = 0;       // split-K tile counters
};

// Workspace of a split-K launch: the tile counters (a region rounded up to
// 256 bytes), then the partial sums.  The counters come first so that their
// slots stay put whatever the size of the partials: in a buffer reused by
// launches of different shapes a counter slot is only ever a counter.
size_t ctr_region_bytes(size_t ctr_count)
{
    return (ctr_count * sizeof(unsigned) + 255) / 256 * 256;
}

size_t workspace_bytes(const Plan& pl)
{
    if (pl.ctr_count == 0)
        return 0;
    return ctr_region_bytes(pl.ctr_count) + pl.ws_floats * sizeof(float);
}

// Point the launch at a workspace whose counter region holds ctr_cap counters.
template <int MAXP>
void bind_workspace(Params<MAXP>& prm, void* base, size_t ctr_cap)
{
    prm.ctr = static_cast<unsigned*>(base);
    prm.ws = base ? reinterpret_cast<float*>(static_cast<uint8_t*>(base) + ctr_region_bytes(ctr_cap))
                  : nullptr;
}

template <int MAXP>
void bind_workspace(Params<MAXP>& prm, const Plan& pl, void* base)
{
    bind_workspace(prm, base, pl.ctr_count);
}

template <int MAXP, int MT, bool SP, int BNC = BN_MAX, int KC = 1, bool MX = false, bool PAIR = false>
int plan(Params<MAXP>& prm, int max_ctas, Plan* out)
{
    using C = Cfg<MT, SP, BNC, KC, MX, PAIR>;
    static std::once_flag attr_once[64];
    int dev = 0;
    GB_CUDA_OK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64)
        return FP8_ERR_UNSUPPORTED;
    cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once[dev], [&] {
        attr_err = cudaFuncSetAttribute(gemm_fp8_kernel<MAXP, MT, SP, BNC, KC, MX, PAIR>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
    });
    GB_CUDA_OK(attr_err);
    int tiles = 0;
    long long ws = 0;
    int ctrs = 0;
    for (int p = 0; p < prm.num_problems; ++p) {
        Problem& P = prm.prob[p];
        P.tile_start = tiles;
        tiles += P.m_blocks * P.n_blocks * P.splits;
        if (P.splits > 1) {
            P.ws_off = ws;
            P.ctr_off = ctrs;
            ws += static_cast<long long>(P.m_blocks) * P.n_blocks * P.splits * (BM * MT) * P.bn;
            ctrs += P.m_blocks * P.n_blocks;
        }
    }
    prm.total_tiles = tiles;
    out->ws_floats = static_cast<size_t>(ws);
    out->ctr_count = static_cast<size_t>(ctrs);
    prm.err = device_error_word();
    prm.wait_ns = kWaitLimitNs;
    prm.withhold_loads = 0;
    // persistent: one CTA per SM; a cap above the SM count launches more
    // CTAs than SMs, which then run in waves of a few tiles each
    const int cap = max_ctas > 0 ? max_ctas : sm_count();
    int grid = std::min(tiles, cap);
    if (PAIR) {
        // one pair of CTAs per tile at most (build_plan trims a persistent
        // launch to the pairs that can be resident at once)
        grid = 2 * std::min(tiles, std::max(1, cap / 2));
    }
    out->cluster = PAIR ? 2 : 0;
    out->kc = KC;
    out->rows_per_tile = BM * MT;
    out->func = reinterpret_cast<const void*>(gemm_fp8_kernel<MAXP, MT, SP, BNC, KC, MX, PAIR>);
    out->ring_bytes = static_cast<size_t>(C::kStages) * C::kStageBytes;
    out->grid = grid;
    out->threads = C::kThreads;
    out->smem = C::kSmem;
    return FP8_OK;
}

// Failure-path test switch (fp8_test_stall_gemm_loads): eager launches still
// to be stalled, and the wait limit eager launches get.
std::atomic<int> g_stall_launches{0};
std::atomic<unsigned long long> g_test_wait_ns{0};

template <int MAXP>
int launch_plan(Params<MAXP>& prm, const Plan& pl, cudaStream_t st)
{
    if (pl.grid == 0)
        return FP8_OK;
    const unsigned long long test_wait = g_test_wait_ns.load(std::memory_order_relaxed);
    if (test_wait)
        prm.wait_ns = test_wait;
    int n = g_stall_launches.load(std::memory_order_relaxed);
    while (n > 0 && !g_stall_launches.compare_exchange_weak(n, n - 1)) {
    }
    prm.withhold_loads = n > 0 ? 1 : 0;
    void* args[] = {&prm};
    // programmatic stream serialization: the kernel's setup may overlap the
    // tail of the previous kernel on `st` (it waits for it before touching
    // global memory)
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = static_cast<unsigned>(pl.cluster);
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(pl.grid);
    cfg.blockDim = dim3(pl.threads);
    cfg.dynamicSmemBytes = static_cast<size_t>(pl.smem);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = pl.cluster > 1 ? 2 : 1;
    GB_CUDA_OK(cudaLaunchKernelExC(&cfg, pl.func, args));
    return FP8_OK;
}

// Clusters of `size` CTAs of the plan's kernel that can be resident at once
// (each CTA needs an SM to itself; clusters must fit in one GPC).  Cached per
// kernel variant and size.
int max_clusters(const Plan& pl, int size)
{
    static std::mutex mu;
    static std::map<std::tuple<int, const void*, int>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return 0;
    const auto key = std::make_tuple(dev, pl.func, size);
    int active = -1;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end())
            active = it->second;
    }
    if (active < 0) {
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = static_cast<unsigned>(size);
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(static_cast<unsigned>(size * std::max(1, sm_count() / size)));
        cfg.blockDim = dim3(pl.threads);
        cfg.dynamicSmemBytes = static_cast<size_t>(pl.smem);
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaOccupancyMaxActiveClusters(&active, pl.func, &cfg) != cudaSuccess) {
            cudaGetLastError();
            active = 0;
        }
        std::lock_guard<std::mutex> lk(mu);
        cache[key] = active;
    }
    return active;
}

bool clusters_fit(const Plan& pl, int size, int clusters)
{
    return max_clusters(pl, size) >= clusters;
}

// ---------------------------------------------------------------- tile choice

std::atomic<int> g_force_mt{0};
std::atomic<int> g_force_group_m{0};

struct TileChoice {
    int mt = 0;        // 0: not set
    int group_m = 0;
    int bn_cap = 0;    // > 0: N tiles at most this wide (and the ring that width selects)
};

// Shape signature of a launch: what the best tile choice depends on.
std::vector<int64_t> signature(const Job* jobs, const int* bns, int n, int max_ctas)
{
    std::vector<int64_t> k;
    k.reserve(2 + 7 * n);
    k.push_back(n);
    k.push_back(max_ctas);
    for (int i = 0; i < n; ++i) {
        const Job& j = jobs[i];
        k.insert(k.end(), {j.rows_p, j.rows_q, j.K, j.E != nullptr, bns[i], j.out_bf16, j.trans_out});
    }
    return k;
}

std::mutex g_tune_mu;
std::map<std::vector<int64_t>, TileChoice> g_tuned;

bool mixed_kinds(const Job* jobs, int n)
{
    for (int i = 1; i < n; ++i)
        if ((jobs[i].E != nullptr) != (jobs[0].E != nullptr))
            return true;
    return false;
}

// CTA pairs (mt 3) take launches allowed two CTAs or more whose problems are
// all dense with 256-wide N tiles, or all 2:4-sparse with N tiles of at least
// 224 (run 224 wide), and block-scaled launches of one problem.
bool pairs_allowed(const Job* jobs, const int* bns, int n, int max_ctas, int bn_cap)
{
    if (n <= 0 || (jobs[0].sfp != nullptr && n != 1) || (max_ctas > 0 && max_ctas < 2))
        return false;
    bool dense = true, sparse = jobs[0].sfp == nullptr;
    for (int i = 0; i < n; ++i) {
        dense = dense && jobs[i].E == nullptr && bns[i] == BN_MAX;
        sparse = sparse && jobs[i].E != nullptr && bns[i] >= SPARSE_BN_MAX_MT2;
    }
    if (dense)
        return bn_cap == 0 || bn_cap >= BN_MAX;
    return sparse && (bn_cap == 0 || bn_cap >= SPARSE_BN_MAX_MT2);
}

// Tile shape of a launch, in order of precedence: an explicit choice (the
// autotuner's candidates), the process-wide override, the autotuner's cached
// winner for this shape signature, the heuristic.  Heuristic: 256-row tiles
// (a third fewer operand bytes per FLOP) when every problem fills them with
// a wide N tile, they give at least half the SMs a tile and the problems are
// all dense or all sparse: as CTA pairs (mt 3) when every problem is dense
// with 256-wide N tiles, else on one CTA (mt 2); otherwise 128-row tiles
// (more, smaller tiles keep every SM busy on skinny and small problems).
// Dense and sparse problems share only the 128-row layout.
TileChoice choose(const Job* jobs, const int* bns, int n, int max_ctas, const TileChoice* expl)
{
    TileChoice c;
    if (expl && expl->mt) {
        c = *expl;
        const bool pair_ok = pairs_allowed(jobs, bns, n, max_ctas, c.bn_cap);
        if (c.mt == 3 && !pair_ok)
            c.mt = 1;
    } else {
        c.mt = g_force_mt.load(std::memory_order_relaxed);
        c.group_m = g_force_group_m.load(std::memory_order_relaxed);
        if (c.mt == 0) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tuned.find(signature(jobs, bns, n, max_ctas));
            if (it != g_tuned.end()) {
                c.mt = it->second.mt;
                c.bn_cap = it->second.bn_cap;
                if (c.group_m == 0)
                    c.group_m = it->second.group_m;
            }
        }
        const bool pair_ok = pairs_allowed(jobs, bns, n, max_ctas, c.bn_cap);
        if (c.mt == 3 && !pair_ok)
            c.mt = 0;
        if (c.mt == 0) {
            int64_t tiles1 = 0, tiles2 = 0;
            bool ok2 = true, long_k = n > 0;
            for (int i = 0; i < n && ok2; ++i) {
                if (jobs[i].rows_p <= BM || bns[i] < 128)
                    ok2 = false;
                const int64_t nb = (jobs[i].rows_q + bns[i] - 1) / bns[i];
                tiles1 += ((jobs[i].rows_p + BM - 1) / BM) * nb;
                tiles2 += ((jobs[i].rows_p + 2 * BM - 1) / (2 * BM)) * nb;
                long_k = long_k && jobs[i].K >= 32 * BK;
            }
            // 256-row tiles load a third fewer bytes per MMA; take them
            // while they still give at least half the SMs a tile, on CTA
            // pairs where the launch allows them (measured: the tensor pipe
            // 88 % busy at 8192^3 against 75 % for one-CTA 256-row tiles).
            // Pairs also where they occupy as many SMs as 128-row tiles
            // would and K is long enough for the k-loop to dominate
            // (512 x 8192 x 8192: 29.4 us against 32.5 us; at K = 2048 the
            // two run level).
            const int sms = sm_count();
            const bool pair_fill = pair_ok && long_k && 2 * tiles2 >= std::min<int64_t>(tiles1, sms);
            c.mt = ok2 && (2 * tiles2 >= sms || pair_fill) ? (pair_ok ? 3 : 2) : 1;
        }
    }
    // block-scaled launches: CTA pairs or 128-row tiles
    if (mixed_kinds(jobs, n) || (n > 0 && jobs[0].sfp != nullptr && c.mt != 3))
        c.mt = 1;
    if (c.group_m <= 0) {
        // Each wave of concurrent tiles re-reads its band's P rows and its Q
        // columns from HBM once operands exceed L2 (the band is gone from L2
        // by the time the raster returns to it), so the traffic per wave
        // grows with band + tiles per wave / band, least near the square
        // root of the tiles per wave.  Pairs run half as many tiles at once
        // as one-CTA tiles: measured at 16384^3, 8-row bands read 4.09 GB
        // from HBM per launch against 4.95 GB for 16-row ones, in the same
        // time (one-CTA 256-row tiles: 3.13 GB at 16, 3.25 at 8).  2:4 pairs
        // read 0.625 of the dense A bytes per row, which moves the best band
        // up: 16-row bands ran 2.5 % faster than 8-row ones at 16384^3 and
        // 16384 x 4096 x 14336, and level on smaller shapes.
        bool beyond_l2 = false;
        for (int i = 0; i < n; ++i)
            beyond_l2 = beyond_l2 || (jobs[i].rows_p + jobs[i].rows_q) * jobs[i].K > l2_bytes();
        const bool sparse_list = n > 0 && jobs[0].E != nullptr;
        c.group_m = c.mt == 3 && beyond_l2 && !sparse_list ? GROUP_M_PAIR_LARGE : GROUP_M_DEFAULT;
    }
    return c;
}

// Fill the table for `n` jobs and plan the kernel variant that fits them.
template <int MAXP>
int build_plan_tiles(Params<MAXP>& prm, const Job* jobs, const int* bns_in, int n, int max_ctas,
                     const TileChoice* expl, Plan* pl)
{
    const TileChoice c = choose(jobs, bns_in, n, max_ctas, expl);
    const bool sparse = n > 0 && jobs[0].E != nullptr;     // all alike when mt == 2
    // N tile widths: the problems' own, under the tuned cap if any (block-
    // scaled launches: 128 or 256, as gemm_fp8_mx chose)
    int bns[MAXP > 0 ? MAXP : 1];
    for (int i = 0; i < n; ++i)
        bns[i] = (c.bn_cap > 0 && jobs[i].sfp == nullptr) ? std::min(bns_in[i], c.bn_cap) : bns_in[i];
    int max_bn = 0;
    bool any_sparse = false, all_sparse = n > 0;
    for (int i = 0; i < n; ++i) {
        max_bn = std::max(max_bn, bns[i]);
        any_sparse = any_sparse || jobs[i].E != nullptr;
        all_sparse = all_sparse && jobs[i].E != nullptr;
    }
    // two k-blocks per stage for 128-row tiles up to 128 wide, unless the
    // launch mixes dense and sparse problems, and for CTA pairs
    const int kc = ((c.mt == 1 && max_bn <= 128 && (!any_sparse || all_sparse)) || c.mt == 3) ? 2 : 1;
    for (int i = 0; i < n; ++i) {
        int bn = bns[i];
        if ((c.mt == 2 || c.mt == 3) && sparse)
            bn = std::min(bn, SPARSE_BN_MAX_MT2);
        int rc = fill_problem(prm.prob[i], jobs[i], bn, c.mt, kc);
        if (rc != FP8_OK)
            return rc;
    }
    prm.num_problems = n;
    prm.group_m = c.group_m;
    if (n > 0 && jobs[0].sfp != nullptr) {
        // block-scaled launches (single problems): CTA pairs or 128 x 256
        // tiles (one accumulator, the scale ring after it) or 128 x 128
        // tiles (two)
        if constexpr (MAXP == 1) {
            if (c.mt == 3)
                return plan<MAXP, 1, false, BN_MAX, 2, true, true>(prm, max_ctas, pl);
            if (max_bn > 128)
                return plan<MAXP, 1, false, BN_MAX, 1, true>(prm, max_ctas, pl);
            return kc == 2 ? plan<MAXP, 1, false, 128, 2, true>(prm, max_ctas, pl)
                           : plan<MAXP, 1, false, 128, 1, true>(prm, max_ctas, pl);
        }
        return FP8_ERR_UNSUPPORTED;
    }
    if (c.mt == 3)
        return sparse ? plan<MAXP, 1, true, SPARSE_BN_MAX_MT2, 2, false, true>(prm, max_ctas, pl)
                      : plan<MAXP, 1, false, BN_MAX, 2, false, true>(prm, max_ctas, pl);
    if (c.mt == 1) {
        if (kc == 2 && all_sparse) {
            if (max_bn <= 16)
                return plan<MAXP, 1, true, 16, 2>(prm, max_ctas, pl);
            if (max_bn <= 32)
                return plan<MAXP, 1, true, 32, 2>(prm, max_ctas, pl);
            if (max_bn <= 64)
                return plan<MAXP, 1, true, 64, 2>(prm, max_ctas, pl);
            return plan<MAXP, 1, true, 128, 2>(prm, max_ctas, pl);
        }
        if (kc == 2) {
            if (max_bn <= 16)
                return plan<MAXP, 1, false, 16, 2>(prm, max_ctas, pl);
            if (max_bn <= 32)
                return plan<MAXP, 1, false, 32, 2>(prm, max_ctas, pl);
            if (max_bn <= 64)
                return plan<MAXP, 1, false, 64, 2>(prm, max_ctas, pl);
            return plan<MAXP, 1, false, 128, 2>(prm, max_ctas, pl);
        }
        if (max_bn <= 16)
            return plan<MAXP, 1, false, 16>(prm, max_ctas, pl);
        if (max_bn <= 32)
            return plan<MAXP, 1, false, 32>(prm, max_ctas, pl);
        if (max_bn <= 64)
            return plan<MAXP, 1, false, 64>(prm, max_ctas, pl);
        if (max_bn <= 128)
            return plan<MAXP, 1, false, 128>(prm, max_ctas, pl);
        return plan<MAXP, 1, false, 256>(prm, max_ctas, pl);
    }
    return sparse ? plan<MAXP, 2, true>(prm, max_ctas, pl) : plan<MAXP, 2, false>(prm, max_ctas, pl);
}

// Q multicast (fp8_gemm_set_multicast): 1 = where plan_multicast finds it
// applies, 0 = never (default: measured slower, see plan_multicast).
std::atomic<int> g_multicast_mode{0};

// Q multicast for a launch of 128-row tiles of one dense problem that is not
// split along K: clusters of mc CTAs (4, else 2) take mc consecutive tiles of
// the raster, i.e. mc row blocks of one N column, and each loads 1/mc of the
// column's Q block per stage, multicast to the whole cluster.  Every CTA
// still reads its own P rows.  Applies when the tiles, the grid, the raster
// band and the row blocks divide into clusters (so every CTA of a cluster
// walks the same columns in lockstep), the Q slices stay whole swizzle atoms
// (8 rows), and every cluster can be resident at once.  Remakes the Q map
// for the slice box; the MMAs and their order do not change, so neither do
// the results.  Off unless enabled: on GB300 it made every shape it applies
// to slower (1024^3 by 9 %, 2048^3 by 7 %, 128 x 8192 x 8192 by 2 %, one
// box, interleaved replays): each SM reads fewer B bytes, but the k-loops
// here are not bound by them, and the clusters' lockstep ring and launch
// cost more than that saves.
template <int MAXP>
bool plan_multicast(Params<MAXP>& prm, const Job* jobs, int n, Plan* pl)
{
    if (g_multicast_mode.load(std::memory_order_relaxed) != 1 || n != 1 || pl->rows_per_tile != BM ||
        jobs[0].E != nullptr || jobs[0].sfp != nullptr)
        return false;
    Problem& P = prm.prob[0];
    if (P.splits != 1)
        return false;
    const int tiles = P.m_blocks * P.n_blocks;
    for (int mc : {4, 2}) {
        if (P.bn % (8 * mc) != 0 || P.m_blocks % mc != 0 || prm.group_m % mc != 0 || tiles % mc != 0 ||
            pl->grid % mc != 0 || max_clusters(*pl, mc) < pl->grid / mc)
            continue;
        const Job& j = jobs[0];
        if (!make_map(&P.tmQ, j.Q, j.rows_q, j.K, j.ldq, BK, P.bn / mc, CU_TENSOR_MAP_SWIZZLE_128B))
            return false;
        prm.mc = mc;
        pl->cluster = mc;
        return true;
    }
    return false;
}

// Plan a launch.  With allow_cluster, a single problem that splits along K
// runs its tiles' slices as thread-block clusters (the slices add up through
// distributed shared memory, no workspace) when one unit per CTA covers the
// problem, the other slices' partial sums fit in a CTA's TMA ring, and all
// clusters can be resident at once; otherwise the global split path.
template <int MAXP>
int build_plan(Params<MAXP>& prm, const Job* jobs, const int* bns_in, int n, int max_ctas,
               const TileChoice* expl, Plan* pl, bool allow_cluster = false)
{
    const int rc = build_plan_tiles(prm, jobs, bns_in, n, max_ctas, expl, pl);
    prm.cluster_split = 0;
    prm.mc = 0;
    if (rc == FP8_OK && pl->cluster == 0 && plan_multicast(prm, jobs, n, pl))
        return rc;
    if (rc == FP8_OK && pl->cluster == 2) {
        // CTA pairs: a persistent launch takes no more pairs than can be
        // resident at once (a launch in waves may take more)
        const int fit = max_clusters(*pl, 2);
        if (fit < 1)
            return FP8_ERR_UNSUPPORTED;
        if (max_ctas <= sm_count())
            pl->grid = 2 * std::min(pl->grid / 2, fit);
        return rc;
    }
    pl->cluster = 0;
    if (rc != FP8_OK || !allow_cluster || n != 1 || max_ctas != 0)
        return rc;
    const ProblemScalars& P = prm.prob[0];
    const int s = P.splits;
    const size_t rows_per_tile = static_cast<size_t>(pl->rows_per_tile);
    if (s < 2 || s > 8 || pl->grid != prm.total_tiles || prm.total_tiles % s != 0 ||
        static_cast<size_t>(s - 1) * P.bn * rows_per_tile * sizeof(float) > pl->ring_bytes ||
        !clusters_fit(*pl, s, prm.total_tiles / s))
        return rc;
    prm.cluster_split = s;
    pl->cluster = s;
    pl->ws_floats = 0;
    pl->ctr_count = 0;
    return rc;
}

// Split-K workspaces of eager (not captured) launches, one per device and
// stream.  Launches on one stream run in order, so they can share a buffer:
// the last unit of every split tile re-zeroes its counter, hence the counters
// are zero between launches and only a new buffer is cleared.  A launch that
// needs more grows the buffer (the new one allocated and cleared, the old one
// freed, all ordered on the stream).  Entries are keyed by the stream's id,
// which unlike its handle is never given to a later stream, and live as long
// as the process; past kMaxStreamWorkspaces streams, launches on further
// streams allocate per call.  The entry's mutex is held from binding to the
// end of the launch call, so threads sharing a stream never free a buffer
// that a launch was just bound to.
struct StreamWorkspace {
    std::mutex mu;
    void* buf = nullptr;
    size_t ctr_cap = 0;         // counters in the counter region
    size_t floats_cap = 0;      // partial sums after it
};
constexpr size_t kMaxStreamWorkspaces = 64;
std::mutex g_sws_mu;
std::map<std::pair<int, unsigned long long>, std::unique_ptr<StreamWorkspace>> g_sws;

StreamWorkspace* stream_workspace(int dev, cudaStream_t st)
{
    unsigned long long id = 0;
    if (cudaStreamGetId(st, &id) != cudaSuccess)
        return nullptr;
    std::lock_guard<std::mutex> lk(g_sws_mu);
    const auto key = std::make_pair(dev, id);
    auto it = g_sws.find(key);
    if (it != g_sws.end())
        return it->second.get();
    if (g_sws.size() >= kMaxStreamWorkspaces)
        return nullptr;
    return g_sws.emplace(key, std::make_unique<StreamWorkspace>()).first->second.get();
}

// Split-K workspaces of captured launches.  Each captured split launch gets
// a buffer of its own, allocated and cleared outside the capture (on a
// private non-blocking stream, with this thread in relaxed capture mode) and
// tied to the captured graph by a CUDA user object: replays then run with no
// allocation nodes, and the buffer lives until the graph and every
// executable graph made from it are gone.  CUDA orders the replays of one
// executable graph; two executables instantiated from the same graph and
// replayed at the same time would share the buffer.  A user object's
// destructor may not call CUDA, so it only queues the buffer; the next
// split launch on that device frees it.
struct CapturedWorkspace {
    int dev;
    void* buf;
    size_t ctr_bytes;
};
std::mutex g_cap_mu;
std::set<CapturedWorkspace*> g_cap_live;          // counters re-zeroed after a device error
std::vector<CapturedWorkspace*> g_cap_dead;       // released by their graphs, not yet freed

void CUDART_CB release_captured_workspace(void* p)
{
    auto* w = static_cast<CapturedWorkspace*>(p);
    std::lock_guard<std::mutex> lk(g_cap_mu);
    g_cap_live.erase(w);
    g_cap_dead.push_back(w);
}

cudaStream_t side_stream(int dev)
{
    static std::once_flag once[64];
    static cudaStream_t streams[64];
    if (dev < 0 || dev >= 64)
        return nullptr;
    std::call_once(once[dev], [dev] {
        if (cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
            streams[dev] = nullptr;
    });
    return streams[dev];
}

// Runs fn with this thread in relaxed capture mode (allocation calls are
// then allowed while a stream of this or another thread is being captured).
template <typename F>
int relaxed_capture_mode(F fn)
{
    cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
    GB_CUDA_OK(cudaThreadExchangeStreamCaptureMode(&mode));
    const int rc = fn();
    cudaThreadExchangeStreamCaptureMode(&mode);
    return rc;
}

void free_released_workspaces(int dev)
{
    std::vector<CapturedWorkspace*> mine;
    {
        std::lock_guard<std::mutex> lk(g_cap_mu);
        if (g_cap_dead.empty())
            return;
        auto keep = std::partition(g_cap_dead.begin(), g_cap_dead.end(),
                                   [dev](CapturedWorkspace* w) { return w->dev != dev; });
        mine.assign(keep, g_cap_dead.end());
        g_cap_dead.erase(keep, g_cap_dead.end());
    }
    cudaStream_t side = side_stream(dev);
    relaxed_capture_mode([&] {
        for (CapturedWorkspace* w : mine) {
            if (side)
                cudaFreeAsync(w->buf, side);
            delete w;
        }
        return FP8_OK;
    });
}

int captured_workspace(int dev, cudaGraph_t graph, const Plan& pl, void** out)
{
    cudaStream_t side = side_stream(dev);
    if (!side)
        return FP8_ERR_CUDA;
    const size_t ctr_bytes = ctr_region_bytes(pl.ctr_count);
    return relaxed_capture_mode([&] {
        void* buf = nullptr;
        if (cudaMallocAsync(&buf, workspace_bytes(pl), side) != cudaSuccess)
            return FP8_ERR_OOM;
        if (cudaMemsetAsync(buf, 0, ctr_bytes, side) != cudaSuccess ||
            cudaStreamSynchronize(side) != cudaSuccess) {
            cudaFreeAsync(buf, side);
            return FP8_ERR_CUDA;
        }
        auto* w = new CapturedWorkspace{dev, buf, ctr_bytes};
        cudaUserObject_t obj = nullptr;
        if (cudaUserObjectCreate(&obj, w, release_captured_workspace, 1,
                                 cudaUserObjectNoDestructorSync) != cudaSuccess) {
            cudaFreeAsync(buf, side);
            delete w;
            return FP8_ERR_CUDA;
        }
        {
            std::lock_guard<std::mutex> lk(g_cap_mu);
            g_cap_live.insert(w);
        }
        if (cudaGraphRetainUserObject(graph, obj, 1, cudaGraphUserObjectMove) != cudaSuccess) {
            cudaUserObjectRelease(obj, 1);            // the destructor queues the buffer
            return FP8_ERR_CUDA;
        }
        *out = buf;
        return FP8_OK;
    });
}

// Launch a split-K plan: on the graph's own workspace under capture, else on
// the stream's persistent one, else (past the stream limit) on a workspace
// from the stream-ordered allocator for this call only (cudaMallocAsync,
// counters cleared, cudaFreeAsync after the kernel, all on `st`).
template <int MAXP>
int launch_split(Params<MAXP>& prm, const Plan& pl, cudaStream_t st)
{
    int dev = 0;
    GB_CUDA_OK(cudaGetDevice(&dev));
    free_released_workspaces(dev);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaGraph_t graph = nullptr;
    GB_CUDA_OK(cudaStreamGetCaptureInfo(st, &cap, nullptr, &graph));
    if (cap == cudaStreamCaptureStatusActive) {
        void* buf = nullptr;
        const int rc = captured_workspace(dev, graph, pl, &buf);
        if (rc != FP8_OK)
            return rc;
        bind_workspace(prm, pl, buf);
        return launch_plan(prm, pl, st);
    }
    if (cap != cudaStreamCaptureStatusNone)
        return FP8_ERR_CUDA;                      // a capture that was invalidated
    if (StreamWorkspace* w = stream_workspace(dev, st)) {
        std::lock_guard<std::mutex> lk(w->mu);
        if (pl.ctr_count > w->ctr_cap || pl.ws_floats > w->floats_cap) {
            const size_t ctr_cap = std::max(pl.ctr_count, w->ctr_cap);
            const size_t floats_cap = std::max(pl.ws_floats, w->floats_cap);
            void* nb = nullptr;
            if (cudaMallocAsync(&nb, ctr_region_bytes(ctr_cap) + floats_cap * sizeof(float), st) !=
                cudaSuccess)
                return FP8_ERR_OOM;
            if (cudaMemsetAsync(nb, 0, ctr_region_bytes(ctr_cap), st) != cudaSuccess ||
                (w->buf && cudaFreeAsync(w->buf, st) != cudaSuccess)) {
                cudaFreeAsync(nb, st);
                return FP8_ERR_CUDA;
            }
            w->buf = nb;
            w->ctr_cap = ctr_cap;
            w->floats_cap = floats_cap;
        }
        bind_workspace(prm, w->buf, w->ctr_cap);
        return launch_plan(prm, pl, st);
    }
    void* buf = nullptr;
    if (cudaMallocAsync(&buf, workspace_bytes(pl), st) != cudaSuccess)
        return FP8_ERR_OOM;
    bind_workspace(prm, pl, buf);
    int rc = cudaMemsetAsync(prm.ctr, 0, pl.ctr_count * sizeof(unsigned), st) == cudaSuccess
                 ? launch_plan(prm, pl, st)
                 : FP8_ERR_CUDA;
    if (cudaFreeAsync(buf, st) != cudaSuccess && rc == FP8_OK)
        rc = FP8_ERR_CUDA;
    return rc;
}

// Plan and launch (split-K plans through launch_split).
template <int MAXP>
int run_jobs(Params<MAXP>& prm, const Job* jobs, const int* bns, int n, int max_ctas,
             cudaStream_t st, const TileChoice* expl = nullptr, bool allow_cluster = false)
{
    Plan pl;
    int rc = build_plan(prm, jobs, bns, n, max_ctas, expl, &pl, allow_cluster);
    if (rc != FP8_OK)
        return rc;
    if (workspace_bytes(pl) == 0) {
        bind_workspace(prm, pl, nullptr);
        return launch_plan(prm, pl, st);
    }
    return launch_split(prm, pl, st);
}

// N width of a block-scaled launch: 256 (CTA pairs, or 128 x 256 tiles with
// two 128-row scale chunks of B per k-block) where the problem has enough
// tiles for it, else 128.
int mx_tile_width(const Job& j)
{
    return pick_bn(j.rows_p, j.rows_q, j.K, BN_MAX) == BN_MAX ? BN_MAX : 128;
}

// Map a user-level GEMM (A [M,K], B [N,K], C [M,N] or C^T) onto (P, Q)
// roles.  A dense product with small M puts A on the MMA N side (Q = A,
// P = B) and writes the output transposed back; a sparse A always stays on
// the MMA M side (the tensor core takes sparsity on that operand only).
Job make_job(int64_t M, int64_t N, int64_t K, const uint8_t* A, int64_t lda,
             const uint8_t* A_meta, const uint8_t* B, int64_t ldb, const float* a_scale, int a_mode,
             const float* b_scale, int b_mode, float alpha, void* C, int64_t ldc, int out_dtype,
             int out_transposed, int a_fmt, int b_fmt)
{
    Job j{};
    const bool swap = A_meta == nullptr && M <= 128 && N > M;
    j.K = K;
    j.alpha = alpha;
    j.C = C;
    j.ldc = ldc;
    j.out_bf16 = out_dtype;
    if (!swap) {
        j.rows_p = M, j.P = A, j.E = A_meta, j.ldp = lda, j.sp = a_scale, j.sp_mode = a_mode;
        j.rows_q = N, j.Q = B, j.ldq = ldb, j.sq = b_scale, j.sq_mode = b_mode;
        j.fmt_p = a_fmt, j.fmt_q = b_fmt;
        j.trans_out = out_transposed;
    } else {
        j.rows_p = N, j.P = B, j.E = nullptr, j.ldp = ldb, j.sp = b_scale, j.sp_mode = b_mode;
        j.rows_q = M, j.Q = A, j.ldq = lda, j.sq = a_scale, j.sq_mode = a_mode;
        j.fmt_p = b_fmt, j.fmt_q = a_fmt;
        j.trans_out = !out_transposed;
    }
    return j;
}

}  // namespace
}  // namespace gb300

extern "C" int gemm_fp8_dense(int64_t M, int64_t N, int64_t K, const uint8_t* A, int64_t lda,
                              const uint8_t* B, int64_t ldb, const float* a_scale, int a_mode,
                              const float* b_scale, int b_mode, float alpha, void* C, int64_t ldc,
                              int out_dtype, fp8_stream_t stream)
{
    return gemm_fp8_dense_fmt(M, N, K, A, lda, B, ldb, a_scale, a_mode, b_scale, b_mode, alpha, C,
                              ldc, out_dtype, FP8_E4M3, FP8_E4M3, stream);
}

extern "C" int gemm_fp8_dense_fmt(int64_t M, int64_t N, int64_t K, const uint8_t* A, int64_t lda,
                                  const uint8_t* B, int64_t ldb, const float* a_scale, int a_mode,
                                  const float* b_scale, int b_mode, float alpha, void* C,
                                  int64_t ldc, int out_dtype, int a_format, int b_format,
                                  fp8_stream_t stream)
{
    using namespace gb300;
    if (!valid_format(a_format) || !valid_format(b_format))
        return FP8_ERR_INVALID;
    int rc = validate(M, N, K, A, lda, nullptr, false, B, ldb, a_scale, a_mode, b_scale, b_mode, C,
                      ldc, out_dtype, 0);
    if (rc != FP8_OK || M == 0 || N == 0)
        return rc;
    if (!device_supported())
        return FP8_ERR_UNSUPPORTED;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (K == 0)
        return write_zeros(C, ldc, M, N, out_dtype, st);
    Job j = make_job(M, N, K, A, lda, nullptr, B, ldb, a_scale, a_mode, b_scale, b_mode, alpha, C,
                     ldc, out_dtype, 0, a_format, b_format);
    const int bn = pick_bn(j.rows_p, j.rows_q, j.K, BN_MAX);
    Params<1> prm;
    memset(&prm, 0, sizeof(prm));
    return run_jobs(prm, &j, &bn, 1, 0, st, nullptr, true);
}

namespace gb300 {
namespace {

// The plan of one job, as its entry point would launch it, into `info`.
int describe_plan(const Job& j, int bn, bool allow_cluster, int64_t M, int64_t N, fp8_gemm_plan_info* info)
{
    Params<1> prm;
    memset(&prm, 0, sizeof(prm));
    Plan pl;
    const int rc = build_plan(prm, &j, &bn, 1, 0, nullptr, &pl, allow_cluster);
    if (rc != FP8_OK)
        return rc;
    const ProblemScalars& P = prm.prob[0];
    info->mt = pl.cluster == 2 && !prm.cluster_split && !prm.mc ? 3 : pl.rows_per_tile / BM;
    info->bn = P.bn;
    info->k_blocks_per_stage = pl.kc;
    info->splits = P.splits;
    info->cluster = pl.cluster > 1 ? pl.cluster : 0;
    info->grid = pl.grid;
    info->swapped = M <= 128 && N > M ? 1 : 0;          // make_job's rule for dense products
    info->multicast = prm.mc;
    info->group_m = prm.group_m;
    info->workspace_bytes = workspace_bytes(pl);
    return FP8_OK;
}

int check_plan_args(int64_t M, int64_t N, int64_t K, int out_dtype, const fp8_gemm_plan_info* info)
{
    if (!info || M <= 0 || N <= 0 || K <= 0 || (out_dtype != 0 && out_dtype != 1))
        return FP8_ERR_INVALID;
    if (M > INT32_MAX / 2 || N > INT32_MAX / 2 || K > INT32_MAX / 2)
        return FP8_ERR_SHAPE;
    if (!device_supported() || !device_one())
        return FP8_ERR_UNSUPPORTED;
    return FP8_OK;
}

}  // namespace
}  // namespace gb300

extern "C" int gemm_fp8_dense_plan(int64_t M, int64_t N, int64_t K, int out_dtype, fp8_gemm_plan_info* info)
{
    using namespace gb300;
    const int rc = check_plan_args(M, N, K, out_dtype, info);
    if (rc != FP8_OK)
        return rc;
    // tensor maps are encoded (never dereferenced) for an aligned stand-in
    // address; the plan depends on the sizes only
    const uint8_t* fake = reinterpret_cast<const uint8_t*>(uintptr_t(1) << 20);
    const int64_t ld = (K + 15) / 16 * 16;
    const float* one = device_one();
    Job j = make_job(M, N, K, fake, ld, nullptr, fake, ld, one, 0, one, 0, 1.0f, const_cast<uint8_t*>(fake),
                     N, out_dtype, 0, FP8_E4M3, FP8_E4M3);
    return describe_plan(j, pick_bn(j.rows_p, j.rows_q, j.K, BN_MAX), true, M, N, info);
}

extern "C" int gemm_fp8_sparse24_plan(int64_t M, int64_t N, int64_t K, int out_dtype, fp8_gemm_plan_info* info)
{
    using namespace gb300;
    const int rc = check_plan_args(M, N, K, out_dtype, info);
    if (rc != FP8_OK)
        return rc;
    if (K % 128 != 0)
        return FP8_ERR_SHAPE;
    const uint8_t* fake = reinterpret_cast<const uint8_t*>(uintptr_t(1) << 20);
    const float* one = device_one();
    Job j = make_job(M, N, K, fake, K / 2, fake, fake, K, one, 0, one, 0, 1.0f, const_cast<uint8_t*>(fake), N,
                     out_dtype, 0, FP8_E4M3, FP8_E4M3);
    const int prc = describe_plan(j, pick_bn(j.rows_p, j.rows_q, j.K, SPARSE_BN_MAX), true, M, N, info);
    info->swapped = 0;                                  // A is always the sparse P side
    return prc;
}

extern "C" int gemm_fp8_mx_plan(int64_t M, int64_t N, int64_t K, int out_dtype, fp8_gemm_plan_info* info)
{
    using namespace gb300;
    int rc = check_plan_args(M, N, K, out_dtype, info);
    if (rc != FP8_OK)
        return rc;
    if (K % 32 != 0)
        return FP8_ERR_SHAPE;
    const uint8_t* fake = reinterpret_cast<const uint8_t*>(uintptr_t(1) << 20);
    const int64_t ld = (K + 15) / 16 * 16;
    const float* one = device_one();
    Job j = make_job(M, N, K, fake, ld, nullptr, fake, ld, one, 0, one, 0, 1.0f, const_cast<uint8_t*>(fake),
                     N, out_dtype, 0, FP8_E4M3, FP8_E4M3);
    j.sfp = fake;
    j.sfq = fake;
    return describe_plan(j, mx_tile_width(j), false, M, N, info);
}

// ---------------------------------------------------------------- no-allocation variant

namespace gb300 {
namespace {

// Device scratch of gemm_fp8_dense_noalloc: the split-K partial sums and tile
// counters live here instead of in memory allocated per call.  Every device
// that loads the library holds this array until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch on the current device (host code only
// has a stand-in for the symbol).  A successful lookup is kept for the rest
// of the process; a failed one (a transient error, or a first call made
// while a stream is being captured in global mode) is not, so the next call
// tries again instead of failing for good.
int noalloc_scratch(void** out)
{
    static std::mutex mu;
    static void* addr[64];
    int dev = 0;
    GB_CUDA_OK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64)
        return FP8_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();                 // leave no sticky error behind
            return FP8_ERR_CUDA;
        }
        addr[dev] = p;
    }
    *out = addr[dev];
    return FP8_OK;
}

}  // namespace
}  // namespace gb300

extern "C" int gemm_fp8_dense_noalloc(int64_t M, int64_t N, int64_t K, const uint8_t* A, int64_t lda,
                                      const uint8_t* B, int64_t ldb, const float* a_scale,
                                      int a_mode, const float* b_scale, int b_mode, float alpha,
                                      void* C, int64_t ldc, int out_dtype, fp8_stream_t stream)
{
    using namespace gb300;
    int rc = validate(M, N, K, A, lda, nullptr, false, B, ldb, a_scale, a_mode, b_scale, b_mode, C,
                      ldc, out_dtype, 0);
    if (rc != FP8_OK || M == 0 || N == 0)
        return rc;
    if (!device_supported())
        return FP8_ERR_UNSUPPORTED;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (K == 0)
        return write_zeros(C, ldc, M, N, out_dtype, st);
    Job j = make_job(M, N, K, A, lda, nullptr, B, ldb, a_scale, a_mode, b_scale, b_mode, alpha, C,
                     ldc, out_dtype, 0, FP8_E4M3, FP8_E4M3);
    const int bn = pick_bn(j.rows_p, j.rows_q, j.K, BN_MAX);
    Params<1> prm;
    memset(&prm, 0, sizeof(prm));
    Plan pl;
    // slices that add up within a cluster need no scratch at all
    rc = build_plan(prm, &j, &bn, 1, 0, nullptr, &pl, true);
    if (rc != FP8_OK)
        return rc;
    const size_t bytes = workspace_bytes(pl);
    if (bytes > kNoAllocScratchBytes)
        return FP8_ERR_SHAPE;                    // needs more scratch than the fixed array holds
    // resolved on every call (a cached pointer after the first), so any
    // first call on a device does the lookup
    void* scratch = nullptr;
    rc = noalloc_scratch(&scratch);
    if (rc != FP8_OK)
        return rc;
    bind_workspace(prm, pl, bytes ? scratch : nullptr);
    if (bytes)
        GB_CUDA_OK(cudaMemsetAsync(prm.ctr, 0, pl.ctr_count * sizeof(unsigned), st));
    return launch_plan(prm, pl, st);
}

extern "C" int gemm_fp8_mx(int64_t M, int64_t N, int64_t K, const uint8_t* A, int64_t lda,
                           const uint8_t* a_scales, const uint8_t* B, int64_t ldb, const uint8_t* b_scales,
                           float alpha, void* C, int64_t ldc, int out_dtype, int a_format, int b_format,
                           fp8_stream_t stream)
{
    using namespace gb300;
    if (!valid_format(a_format) || !valid_format(b_format))
        return FP8_ERR_INVALID;
    if (M < 0 || N < 0 || K < 0 || (out_dtype != 0 && out_dtype != 1))
        return FP8_ERR_INVALID;
    if (M == 0 || N == 0)
        return FP8_OK;
    if (!C)
        return FP8_ERR_INVALID;
    if (ldc < N || K % 32 != 0 || M > INT32_MAX / 2 || N > INT32_MAX / 2 || K > INT32_MAX / 2)
        return FP8_ERR_SHAPE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (K == 0) {
        if (!device_supported())
            return FP8_ERR_UNSUPPORTED;
        return write_zeros(C, ldc, M, N, out_dtype, st);
    }
    if (!A || !B || !a_scales || !b_scales)
        return FP8_ERR_INVALID;
    if (lda < K || ldb < K)
        return FP8_ERR_SHAPE;
    if (!aligned16(A) || !aligned16(B) || lda % 16 || ldb % 16 || !aligned16(a_scales) || !aligned16(b_scales))
        return FP8_ERR_ALIGN;
    if (!device_supported() || !device_one())
        return FP8_ERR_UNSUPPORTED;
    // no per-row scales: both scale operands read a device 1.0, so the
    // epilogue stores alpha * acc
    const float* one = device_one();
    Job j = make_job(M, N, K, A, lda, nullptr, B, ldb, one, 0, one, 0, alpha, C, ldc, out_dtype, 0, a_format,
                     b_format);
    const bool swapped = M <= 128 && N > M;          // make_job's rule for small-M dense products
    j.sfp = swapped ? b_scales : a_scales;
    j.sfq = swapped ? a_scales : b_scales;
    const int bn = mx_tile_width(j);
    Params<1> prm;
    memset(&prm, 0, sizeof(prm));
    return run_jobs(prm, &j, &bn, 1, 0, st);
}

extern "C" int gemm_fp8_sparse24(int64_t M, int64_t N, int64_t K, const uint8_t* a_vals,
                                 const uint8_t* a_meta, const uint8_t* B, int64_t ldb,
                                 const float* a_scale, int a_mode, const float* b_scale, int b_mode,
                                 float alpha, void* C, int64_t ldc, int out_dtype,
                                 int out_transposed, fp8_stream_t stream)
{
    return gemm_fp8_sparse24_fmt(M, N, K, a_vals, a_meta, B, ldb, a_scale, a_mode, b_scale, b_mode,
                                 alpha, C, ldc, out_dtype, out_transposed, FP8_E4M3, FP8_E4M3,
                                 stream);
}

extern "C" int gemm_fp8_sparse24_fmt(int64_t M, int64_t N, int64_t K, const uint8_t* a_vals,
                                     const uint8_t* a_meta, const uint8_t* B, int64_t ldb,
                                     const float* a_scale, int a_mode, const float* b_scale,
                                     int b_mode, float alpha, void* C, int64_t ldc, int out_dtype,
                                     int out_transposed, int a_format, int b_format,
                                     fp8_stream_t stream)
{
    using namespace gb300;
    if (!valid_format(a_format) || !valid_format(b_format))
        return FP8_ERR_INVALID;
    int rc = validate(M, N, K, a_vals, K / 2, a_meta, true, B, ldb, a_scale, a_mode, b_scale,
                      b_mode, C, ldc, out_dtype, out_transposed);
    if (rc != FP8_OK || M == 0 || N == 0)
        return rc;
    if (!device_supported())
        return FP8_ERR_UNSUPPORTED;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (K == 0)
        return out_transposed ? write_zeros(C, ldc, N, M, out_dtype, st)
                              : write_zeros(C, ldc, M, N, out_dtype, st);
    Job j = make_job(M, N, K, a_vals, K / 2, a_meta, B, ldb, a_scale, a_mode, b_scale, b_mode,
                     alpha, C, ldc, out_dtype, out_transposed, a_format, b_format);
    const int bn = pick_bn(j.rows_p, j.rows_q, j.K, SPARSE_BN_MAX);
    Params<1> prm;
    memset(&prm, 0, sizeof(prm));
    return run_jobs(prm, &j, &bn, 1, 0, st, nullptr, true);
}

extern "C" int gemm_fp8_grouped(const fp8_gemm_problem* problems, int num_problems,
                                fp8_stream_t stream)
{
    return gemm_fp8_grouped_ex(problems, num_problems, 0, stream);
}

namespace gb300 {
namespace {

// Validate a problem list and turn it into jobs.  K == 0 problems are written
// as zeros on `st` (when `zeros_ok`) or rejected.  *n_out: jobs produced.
int grouped_jobs(const fp8_gemm_problem* problems, int num_problems, cudaStream_t st,
                 bool zeros_ok, Job* jobs, int* bns, int* n_out, bool check_only = false)
{
    *n_out = 0;
    if (num_problems < 0 || (num_problems > 0 && !problems))
        return FP8_ERR_INVALID;
    if (num_problems > FP8_GROUPED_MAX_PROBLEMS)
        return FP8_ERR_SHAPE;
    bool any_sparse = false;
    for (int i = 0; i < num_problems; ++i) {
        const fp8_gemm_problem& g = problems[i];
        const bool sp = g.A_meta != nullptr;
        int rc = validate(g.M, g.N, g.K, g.A, sp ? g.K / 2 : g.lda, g.A_meta, sp, g.B, g.ldb,
                          g.a_scale, g.a_mode, g.b_scale, g.b_mode, g.C, g.ldc, g.out_dtype,
                          g.out_transposed);
        if (rc != FP8_OK)
            return rc;
        if (!valid_format(g.a_format) || !valid_format(g.b_format))
            return FP8_ERR_INVALID;
        if (!zeros_ok && g.M > 0 && g.N > 0 && g.K == 0)
            return FP8_ERR_SHAPE;
        any_sparse |= sp && g.M > 0 && g.N > 0 && g.K > 0;
    }
    if (num_problems == 0 || check_only)
        return FP8_OK;
    if (!device_supported())
        return FP8_ERR_UNSUPPORTED;
    // a launch holding a sparse problem keeps TMEM columns beside the
    // accumulators for the metadata ring, so every tile in it has N <= 240
    const int bn_max = any_sparse ? SPARSE_BN_MAX : BN_MAX;
    int n = 0;
    for (int i = 0; i < num_problems; ++i) {
        const fp8_gemm_problem& g = problems[i];
        if (g.M == 0 || g.N == 0)
            continue;
        if (g.K == 0) {
            int rc = g.out_transposed ? write_zeros(g.C, g.ldc, g.N, g.M, g.out_dtype, st)
                                      : write_zeros(g.C, g.ldc, g.M, g.N, g.out_dtype, st);
            if (rc != FP8_OK)
                return rc;
            continue;
        }
        const bool sp = g.A_meta != nullptr;
        jobs[n] = make_job(g.M, g.N, g.K, g.A, sp ? g.K / 2 : g.lda, g.A_meta, g.B, g.ldb,
                           g.a_scale, g.a_mode, g.b_scale, g.b_mode, g.alpha, g.C, g.ldc,
                           g.out_dtype, g.out_transposed, g.a_format, g.b_format);
        bns[n] = pick_bn(jobs[n].rows_p, jobs[n].rows_q, jobs[n].K, bn_max);
        ++n;
    }
    *n_out = n;
    return FP8_OK;
}

}  // namespace
}  // namespace gb300

extern "C" int gemm_fp8_grouped_ex(const fp8_gemm_problem* problems, int num_problems,
                                   int max_ctas, fp8_stream_t stream)
{
    using namespace gb300;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (num_problems > FP8_GROUPED_MAX_PROBLEMS && problems) {
        // longer lists: every problem checked first (nothing is launched for
        // a bad list), then consecutive launches of up to
        // FP8_GROUPED_MAX_PROBLEMS problems each, in list order
        Job unused[FP8_GROUPED_MAX_PROBLEMS];
        int ub[FP8_GROUPED_MAX_PROBLEMS], un = 0;
        for (int b = 0; b < num_problems; b += FP8_GROUPED_MAX_PROBLEMS) {
            const int rc = grouped_jobs(problems + b, std::min(FP8_GROUPED_MAX_PROBLEMS, num_problems - b), st, true,
                                        unused, ub, &un, true);
            if (rc != FP8_OK)
                return rc;
        }
        for (int b = 0; b < num_problems; b += FP8_GROUPED_MAX_PROBLEMS) {
            const int rc = gemm_fp8_grouped_ex(problems + b, std::min(FP8_GROUPED_MAX_PROBLEMS, num_problems - b),
                                               max_ctas, stream);
            if (rc != FP8_OK)
                return rc;
        }
        return FP8_OK;
    }
    Job jobs[FP8_GROUPED_MAX_PROBLEMS];
    int bns[FP8_GROUPED_MAX_PROBLEMS];
    int n = 0;
    int rc = grouped_jobs(problems, num_problems, st, true, jobs, bns, &n);
    if (rc != FP8_OK || n == 0)
        return rc;
    static thread_local Params<FP8_GROUPED_MAX_PROBLEMS> prm;
    static thread_local Params<1> prm1;
    // a one-problem launch runs as a single call does: the one-problem
    // kernel variant (the same tiles and arithmetic, a 32nd of the kernel
    // parameters to upload: 6.05 against 6.78 us for a 1024^3 launch) and,
    // uncapped, split-K slices added within clusters (64 x 8192 x 8192:
    // 19.7 against 21.6 us through the workspace; bitwise the same sums)
    auto run = [&](const Job* js, const int* bs, int m) -> int {
        if (m == 1) {
            memset(&prm1, 0, sizeof(prm1));
            return run_jobs(prm1, js, bs, 1, max_ctas, st, nullptr, true);
        }
        memset(&prm, 0, sizeof(prm));
        return run_jobs(prm, js, bs, m, max_ctas, st);
    };
    // A launch takes one tile kind, and one small or mixed-kind problem puts
    // the whole list on 128-row tiles.  So problems that would run on CTA
    // pairs alone (the large ones) are launched apart from the rest, one
    // launch per kind (dense, 2:4), after the rest; a list whose tile kind
    // is forced or tuned as a whole keeps its one launch.
    int group[FP8_GROUPED_MAX_PROBLEMS];
    int count[3] = {0, 0, 0};
    bool whole = n == 1 || g_force_mt.load(std::memory_order_relaxed) != 0;
    if (!whole) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        whole = g_tuned.count(signature(jobs, bns, n, max_ctas)) != 0;
    }
    for (int i = 0; i < n; ++i) {
        group[i] = 0;
        if (!whole && choose(&jobs[i], &bns[i], 1, max_ctas, nullptr).mt == 3)
            group[i] = jobs[i].E ? 2 : 1;
        ++count[group[i]];
    }
    if (count[0] == n || count[1] == n || count[2] == n)
        return run(jobs, bns, n);
    for (int g = 0; g < 3; ++g) {
        Job gj[FP8_GROUPED_MAX_PROBLEMS];
        int gbn[FP8_GROUPED_MAX_PROBLEMS];
        int m = 0;
        for (int i = 0; i < n; ++i) {
            if (group[i] == g) {
                gj[m] = jobs[i];
                gbn[m] = bns[i];
                ++m;
            }
        }
        if (m == 0)
            continue;
        rc = run(gj, gbn, m);
        if (rc != FP8_OK)
            return rc;
    }
    return FP8_OK;
}

extern "C" int gemm_fp8_grouped_autotune(const fp8_gemm_problem* problems, int num_problems,
                                         int max_ctas, int iters, fp8_stream_t stream,
                                         fp8_tile_config* best)
{
    using namespace gb300;
    if (iters <= 0)
        return FP8_ERR_INVALID;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Job jobs[FP8_GROUPED_MAX_PROBLEMS];
    int bns[FP8_GROUPED_MAX_PROBLEMS];
    int n = 0;
    int rc = grouped_jobs(problems, num_problems, st, true, jobs, bns, &n);
    if (rc != FP8_OK)
        return rc;
    if (n == 0)
        return FP8_OK;
    static thread_local Params<FP8_GROUPED_MAX_PROBLEMS> prm;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GB_CUDA_OK(cudaEventCreate(&e0));
    GB_CUDA_OK(cudaEventCreate(&e1));
    TileChoice winner;
    float best_ms = 0.0f;
    // candidates: tile kind (128-row, 256-row, CTA pair), raster band height,
    // and for 128-row tiles a cap on the N width (which also picks the ring:
    // two k-blocks per stage up to 128 wide); split counts stay fixed per
    // problem, so no candidate changes a result
    int max_bn = 0;
    const bool pair_ok = jobs[0].sfp == nullptr && pairs_allowed(jobs, bns, n, max_ctas, 0);
    for (int i = 0; i < n; ++i)
        max_bn = std::max(max_bn, bns[i]);
    std::vector<TileChoice> cands;
    const int gms[5] = {2, 4, 8, 16, 32};
    for (int mt = 1; mt <= 3; ++mt) {
        if ((mt == 2 && mixed_kinds(jobs, n)) || (mt == 3 && !pair_ok))
            continue;
        for (int cap : {0, 128, 64}) {
            if (cap && (mt != 1 || cap >= max_bn))
                continue;
            for (int gm : gms) {
                TileChoice c;
                c.mt = mt;
                c.group_m = gm;
                c.bn_cap = cap;
                cands.push_back(c);
            }
        }
    }
    for (const TileChoice& c : cands) {
        memset(&prm, 0, sizeof(prm));
        rc = run_jobs(prm, jobs, bns, n, max_ctas, st, &c);                // warm-up
        for (int it = 0; rc == FP8_OK && it < iters; ++it) {
            if (it == 0 && cudaEventRecord(e0, st) != cudaSuccess)
                rc = FP8_ERR_CUDA;
            if (rc == FP8_OK)
                rc = run_jobs(prm, jobs, bns, n, max_ctas, st, &c);
        }
        float ms = 0.0f;
        if (rc == FP8_OK && (cudaEventRecord(e1, st) != cudaSuccess ||
                             cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = FP8_ERR_CUDA;
        if (rc != FP8_OK)
            break;
        if (winner.mt == 0 || ms < best_ms) {
            winner = c;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != FP8_OK)
        return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[signature(jobs, bns, n, max_ctas)] = winner;
    }
    if (best) {
        best->mt = winner.mt;
        best->group_m = winner.group_m;
        best->ms_per_launch = best_ms / static_cast<float>(iters);
        best->bn_max = winner.bn_cap;
    }
    return FP8_OK;
}

extern "C" int gemm_fp8_tune_cache_save(const char* path)
{
    using namespace gb300;
    if (!path)
        return FP8_ERR_INVALID;
    FILE* f = fopen(path, "w");
    if (!f)
        return FP8_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    fprintf(f, "# gb300fp8 tile cache v2: <signature length> <signature...> <mt> <group_m> <bn cap>\n");
    for (const auto& kv : g_tuned) {
        fprintf(f, "%zu", kv.first.size());
        for (int64_t v : kv.first)
            fprintf(f, " %lld", static_cast<long long>(v));
        fprintf(f, " %d %d %d\n", kv.second.mt, kv.second.group_m, kv.second.bn_cap);
    }
    fclose(f);
    return FP8_OK;
}

extern "C" int gemm_fp8_tune_cache_load(const char* path)
{
    using namespace gb300;
    if (!path)
        return FP8_ERR_INVALID;
    FILE* f = fopen(path, "r");
    if (!f)
        return FP8_ERR_INVALID;
    std::map<std::vector<int64_t>, TileChoice> loaded;
    char line[8192];
    int rc = FP8_OK;
    while (fgets(line, sizeof(line), f)) {
        if (line[0] == '#' || line[0] == '\n')
            continue;
        char* p = line;
        char* end = nullptr;
        const long long len = strtoll(p, &end, 10);
        if (end == p || len <= 0 || len > 2 + 7 * FP8_GROUPED_MAX_PROBLEMS) {
            rc = FP8_ERR_INVALID;
            break;
        }
        std::vector<int64_t> key;
        for (long long i = 0; i < len && rc == FP8_OK; ++i) {
            p = end;
            const long long v = strtoll(p, &end, 10);
            if (end == p)
                rc = FP8_ERR_INVALID;
            key.push_back(v);
        }
        TileChoice c;
        p = end;
        c.mt = static_cast<int>(strtol(p, &end, 10));
        p = end;
        c.group_m = static_cast<int>(strtol(p, &end, 10));
        p = end;                                  // optional bn cap (v2 lines)
        c.bn_cap = static_cast<int>(strtol(p, &end, 10));
        if (end == p)
            c.bn_cap = 0;
        if (rc != FP8_OK || c.mt < 1 || c.mt > 3 || c.group_m <= 0 || c.group_m > 4096 ||
            (c.bn_cap != 0 && c.bn_cap != 64 && c.bn_cap != 128)) {
            rc = FP8_ERR_INVALID;
            break;
        }
        loaded[key] = c;
    }
    fclose(f);
    if (rc != FP8_OK)
        return rc;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto& kv : loaded)
        g_tuned[kv.first] = kv.second;
    return FP8_OK;
}

extern "C" int gemm_fp8_tune_cache_clear(void)
{
    std::lock_guard<std::mutex> lk(gb300::g_tune_mu);
    gb300::g_tuned.clear();
    return FP8_OK;
}

// ---------------------------------------------------------------- CUDA graphs

struct fp8_grouped_graph {
    gb300::Params<FP8_GROUPED_MAX_PROBLEMS> prm;
    gb300::Plan plan;
    std::vector<int64_t> sig;
    int max_ctas = 0;
    int dev = 0;
    void* ws = nullptr;         // split-K workspace owned by the graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t node = nullptr;
};

namespace {

// Graphs that own a split-K workspace (their counters are re-zeroed after a
// device error).
std::mutex g_graphs_mu;
std::set<fp8_grouped_graph*> g_graphs;

int graph_params(fp8_grouped_graph* g, const fp8_gemm_problem* problems, int num_problems,
                 std::vector<int64_t>* sig)
{
    using namespace gb300;
    Job jobs[FP8_GROUPED_MAX_PROBLEMS];
    int bns[FP8_GROUPED_MAX_PROBLEMS];
    int n = 0;
    int rc = grouped_jobs(problems, num_problems, nullptr, false, jobs, bns, &n);
    if (rc != FP8_OK)
        return rc;
    if (n == 0)
        return FP8_ERR_SHAPE;
    *sig = signature(jobs, bns, n, g->max_ctas);
    memset(&g->prm, 0, sizeof(g->prm));
    rc = build_plan(g->prm, jobs, bns, n, g->max_ctas, nullptr, &g->plan);
    if (rc == FP8_OK)
        bind_workspace(g->prm, g->plan, g->ws);
    return rc;
}

cudaKernelNodeParams node_params(fp8_grouped_graph* g, void** args)
{
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(g->plan.func);
    kp.gridDim = dim3(g->plan.grid);
    kp.blockDim = dim3(g->plan.threads);
    kp.sharedMemBytes = static_cast<unsigned>(g->plan.smem);
    args[0] = &g->prm;
    kp.kernelParams = args;
    return kp;
}

}  // namespace

extern "C" int gemm_fp8_grouped_graph_create(const fp8_gemm_problem* problems, int num_problems,
                                             int max_ctas, fp8_grouped_graph** out)
{
    if (!out)
        return FP8_ERR_INVALID;
    auto* g = new fp8_grouped_graph;
    g->max_ctas = max_ctas;
    if (cudaGetDevice(&g->dev) != cudaSuccess) {
        delete g;
        return FP8_ERR_CUDA;
    }
    int rc = graph_params(g, problems, num_problems, &g->sig);
    const size_t bytes = rc == FP8_OK ? gb300::workspace_bytes(g->plan) : 0;
    if (bytes) {
        // a persistent split-K workspace; its counters start (and stay) zero
        if (cudaMalloc(&g->ws, bytes) != cudaSuccess)
            rc = FP8_ERR_OOM;
        else if (cudaMemset(g->ws, 0, bytes) != cudaSuccess)
            rc = FP8_ERR_CUDA;
        else
            gb300::bind_workspace(g->prm, g->plan, g->ws);
    }
    void* args[1];
    if (rc == FP8_OK) {
        cudaKernelNodeParams kp = node_params(g, args);
        // CTA-pair launches: the node carries the cluster shape
        cudaKernelNodeAttrValue cv{};
        cv.clusterDim.x = static_cast<unsigned>(g->plan.cluster > 1 ? g->plan.cluster : 1);
        cv.clusterDim.y = 1;
        cv.clusterDim.z = 1;
        if (cudaGraphCreate(&g->graph, 0) != cudaSuccess ||
            cudaGraphAddKernelNode(&g->node, g->graph, nullptr, 0, &kp) != cudaSuccess ||
            (g->plan.cluster > 1 &&
             cudaGraphKernelNodeSetAttribute(g->node, cudaKernelNodeAttributeClusterDimension, &cv) !=
                 cudaSuccess) ||
            cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess)
            rc = FP8_ERR_CUDA;
    }
    if (rc != FP8_OK) {
        if (g->exec)
            cudaGraphExecDestroy(g->exec);
        if (g->graph)
            cudaGraphDestroy(g->graph);
        if (g->ws)
            cudaFree(g->ws);
        delete g;
        return rc;
    }
    if (g->ws) {
        std::lock_guard<std::mutex> lk(g_graphs_mu);
        g_graphs.insert(g);
    }
    *out = g;
    return FP8_OK;
}

extern "C" int gemm_fp8_grouped_graph_update(fp8_grouped_graph* g,
                                             const fp8_gemm_problem* problems, int num_problems)
{
    if (!g)
        return FP8_ERR_INVALID;
    std::vector<int64_t> sig;
    const gb300::Plan old = g->plan;
    int rc = graph_params(g, problems, num_problems, &sig);
    if (rc != FP8_OK)
        return rc;
    if (sig != g->sig || g->plan.func != old.func || g->plan.grid != old.grid)
        return FP8_ERR_SHAPE;
    void* args[1];
    cudaKernelNodeParams kp = node_params(g, args);
    if (cudaGraphExecKernelNodeSetParams(g->exec, g->node, &kp) != cudaSuccess)
        return FP8_ERR_CUDA;
    return FP8_OK;
}

extern "C" int gemm_fp8_grouped_graph_launch(fp8_grouped_graph* g, fp8_stream_t stream)
{
    if (!g)
        return FP8_ERR_INVALID;
    GB_CUDA_OK(cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream)));
    return FP8_OK;
}

extern "C" int gemm_fp8_grouped_graph_destroy(fp8_grouped_graph* g)
{
    if (!g)
        return FP8_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(g_graphs_mu);
        g_graphs.erase(g);
    }
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    if (g->ws)
        cudaFree(g->ws);
    delete g;
    return FP8_OK;
}

void gb300::reset_split_counters()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return;
    cudaDeviceSynchronize();
    {
        std::lock_guard<std::mutex> lk(g_sws_mu);
        for (auto& kv : g_sws) {
            if (kv.first.first != dev)
                continue;
            std::lock_guard<std::mutex> lk2(kv.second->mu);
            if (kv.second->buf)
                cudaMemset(kv.second->buf, 0, ctr_region_bytes(kv.second->ctr_cap));
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_graphs_mu);
        for (fp8_grouped_graph* g : g_graphs)
            if (g->dev == dev && g->ws)
                cudaMemset(g->ws, 0, ctr_region_bytes(g->plan.ctr_count));
    }
    {
        std::lock_guard<std::mutex> lk(g_cap_mu);
        for (CapturedWorkspace* w : g_cap_live)
            if (w->dev == dev)
                cudaMemset(w->buf, 0, w->ctr_bytes);
    }
    cudaDeviceSynchronize();
}

extern "C" int fp8_gemm_set_tile_config(int mt, int group_m)
{
    if (mt < 0 || mt > 3 || group_m < 0 || group_m > 4096)
        return FP8_ERR_INVALID;
    gb300::g_force_mt.store(mt);
    gb300::g_force_group_m.store(group_m);
    return FP8_OK;
}

extern "C" int fp8_gemm_set_multicast(int mode)
{
    if (mode != 0 && mode != 1)
        return FP8_ERR_INVALID;
    gb300::g_multicast_mode.store(mode);
    return FP8_OK;
}

extern "C" int fp8_test_stall_gemm_loads(int launches, double wait_limit_ms)
{
    if (launches < 0 || !(wait_limit_ms >= 0.0) || wait_limit_ms > 60000.0)
        return FP8_ERR_INVALID;
    gb300::g_test_wait_ns.store(static_cast<unsigned long long>(wait_limit_ms * 1e6));
    gb300::g_stall_launches.store(launches);
    return FP8_OK;
}
