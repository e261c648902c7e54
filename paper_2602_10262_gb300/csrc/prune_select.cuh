// 2:4 selection of one or two groups of four E4M3/E5M2 codes, shared by
// prune24_compress (prune.cu) and the fused quantise + compress
// (fp8_quantize_e4m3_prune24, quant.cu): both keep the two codes of largest
// magnitude (code & 0x7F, the lower index on a tie) and write the same
// kept-code and index layout.
#pragma once
#include <cstdint>

namespace gb300 {

// One group of four codes (byte i of w = element i).  Element j outranks
// element i when key_j > key_i, or key_j == key_i and j < i (key = code &
// 0x7F); the two highest-ranked elements are kept.  score_i = key_i * 4 +
// (3 - i) orders the elements exactly that way and makes every score
// distinct, so the kept pair is the top two of four scores: a two-round
// max/min tournament.  Returns the two kept codes in the low 16 bits (lower
// index first) and the nibble i0 | i1 << 2 in bits 16..19.
__device__ __forceinline__ uint32_t select_group(uint32_t w)
{
    const uint32_t s0 = ((w << 2) & 0x1FCu) | 3u;
    const uint32_t s1 = ((w >> 6) & 0x1FCu) | 2u;
    const uint32_t s2 = ((w >> 14) & 0x1FCu) | 1u;
    const uint32_t s3 = (w >> 22) & 0x1FCu;
    const uint32_t a = max(s0, s1), b = min(s0, s1), c = max(s2, s3), d = min(s2, s3);
    const uint32_t t1 = max(a, c);
    const uint32_t t2 = max(min(a, c), max(b, d));
    const uint32_t i0 = 3u - max(t1 & 3u, t2 & 3u);
    const uint32_t i1 = 3u - min(t1 & 3u, t2 & 3u);
    const uint32_t vals = __byte_perm(w, 0u, i0 | (i1 << 4)) & 0xFFFFu;
    return vals | ((i0 | (i1 << 2)) << 16);
}

// Two groups at once (group a = word wa, group b = word wb): the same scores
// and tournament as select_group, with the scores of element j of both
// groups side by side in the two 16-bit halves of a register, so one
// packed max / min does the work of two.  Returns the kept codes of a in
// bits 0-15 and of b in bits 16-31 of *vals, and the nibble of a in bits
// 0-3 and of b in bits 4-7 of the result.
__device__ __forceinline__ uint32_t select_group_pair(uint32_t wa, uint32_t wb, uint32_t* vals)
{
    // element j of a in bytes 0-1, of b in bytes 2-3; keep its key, * 4, | (3 - j)
    const uint32_t s0 = ((__byte_perm(wa, wb, 0x4400u) << 2) & 0x01FC01FCu) | 0x00030003u;
    const uint32_t s1 = ((__byte_perm(wa, wb, 0x5511u) << 2) & 0x01FC01FCu) | 0x00020002u;
    const uint32_t s2 = ((__byte_perm(wa, wb, 0x6622u) << 2) & 0x01FC01FCu) | 0x00010001u;
    const uint32_t s3 = (__byte_perm(wa, wb, 0x7733u) << 2) & 0x01FC01FCu;
    const uint32_t a = __vmaxu2(s0, s1), b = __vminu2(s0, s1);
    const uint32_t c = __vmaxu2(s2, s3), d = __vminu2(s2, s3);
    const uint32_t t1 = __vmaxu2(a, c);
    const uint32_t t2 = __vmaxu2(__vminu2(a, c), __vmaxu2(b, d));
    const uint32_t x1 = t1 & 0x00030003u, x2 = t2 & 0x00030003u;
    const uint32_t i0 = __vmaxu2(x1, x2) ^ 0x00030003u;       // 3 - (larger low bits)
    const uint32_t i1 = __vminu2(x1, x2) ^ 0x00030003u;
    const uint32_t sel = i0 | (i1 << 4);                       // byte selectors, per half
    const uint32_t va = __byte_perm(wa, 0u, sel & 0xFFFFu);
    const uint32_t vb = __byte_perm(wb, 0u, sel >> 16);
    *vals = __byte_perm(va, vb, 0x5410u);
    const uint32_t nib = i0 | (i1 << 2);
    return (nib & 0xFu) | ((nib >> 12) & 0xF0u);
}

}  // namespace gb300
