/*
 * CPU oracle for the FP8 (E4M3 / E5M2) GEMM path: plain, slow, obviously correct.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant generator
 * with the CUDA path.
 *
 * What it computes (Jarmusch, Vitz, Chandrasekaran, "Execution-Centric
 * Characterization of FP8 Matrix Cores, Asynchronous Execution, and Structured
 * Sparsity on AMD MI300A", arXiv 2602.10262):
 *   - E4M3 decode / encode: the OCP 8-bit floating point format the paper
 *     names for its FP8 matrix cores (section 2, "FP8 Matrix Cores").  The
 *     paper gives no bit layout; the OCP E4M3 definition is used: 1 sign bit,
 *     4 exponent bits (bias 7), 3 mantissa bits, no infinities, S.1111.111 is
 *     NaN, largest finite 448.
 *   - E5M2 decode / encode: the other OCP variant the paper lists ("bf8",
 *     section 2; mixed E4M3 x E5M2 operands in Table 3): 1 sign bit, 5
 *     exponent bits (bias 15), 2 mantissa bits, infinities and NaNs as in
 *     IEEE-754, largest finite 57344.
 *   - Quantisation: per-tensor or per-row amax scaling so that amax maps to
 *     the format's largest finite value (448 or 57344), one fp32 multiply,
 *     round-to-nearest-even with saturation to the finite range.
 *   - 2:4 structured sparsity (section 2 "Structured Sparsity" and section 6):
 *     in every group of four consecutive elements along K two are zero; the
 *     pruning keeps the two largest magnitudes.
 *   - Block-scaled FP8 (OCP MX, not in the paper): 32-element blocks along K
 *     sharing an E8M0 power-of-two scale, and the GEMM over such operands.
 *   - GEMM: C = alpha * dA[m] * dB[n] * sum_k decA(A[m,k]) * decB(B[n,k]),
 *     FP8 x FP8 products accumulated (here in FP64), as the FP8 matrix-core
 *     operation of section 4 (FP8 x FP8 operands, wide accumulation).
 *
 * Every function states the reading it follows where the paper is silent.
 * Floating point: compile with -ffp-contract=off so that no multiply-add is
 * fused; fp32 products and quotients below are single IEEE operations.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* E4M3 decode (OCP FP8, E4M3 variant; paper section 2).                     */
/* ------------------------------------------------------------------------ */

/* Value of code c.  s = bit 7, e = bits 6..3, m = bits 2..0.
 *   e == 15 and m == 7      -> NaN (codes 0x7F, 0xFF)
 *   e == 0                  -> (-1)^s * m * 2^-9          (subnormal)
 *   otherwise               -> (-1)^s * (1 + m/8) * 2^(e-7)               */
double orc_e4m3_decode(uint8_t c)
{
    int s = (c >> 7) & 1;
    int e = (c >> 3) & 15;
    int m = c & 7;
    double v;
    if (e == 15 && m == 7)
        return NAN;
    if (e == 0)
        v = ldexp((double)m, -9);
    else
        v = ldexp(1.0 + (double)m / 8.0, e - 7);
    return s ? -v : v;
}

void orc_e4m3_decode_array(const uint8_t *c, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; ++i)
        out[i] = orc_e4m3_decode(c[i]);
}

/* ------------------------------------------------------------------------ */
/* E4M3 encode: round to nearest, ties to even, saturate to +-448.           */
/* ------------------------------------------------------------------------ */

/* Round a non-negative double that holds an exact fp32-derived quotient to the
 * nearest integer, ties to even.  (Operands here are fp32 values scaled by a
 * power of two, so the quotient is exact in double.) */
static double rne_int(double q)
{
    double f = floor(q);
    double r = q - f;
    if (r > 0.5)
        return f + 1.0;
    if (r < 0.5)
        return f;
    return (fmod(f, 2.0) == 0.0) ? f : f + 1.0;
}

/* Arithmetic encoder.  Readings where the paper is silent:
 *   - overflow saturates to the largest finite magnitude (448), including
 *     +-inf ("satfinite"); the workloads scale amax to 448 so finite inputs
 *     are in range anyway;
 *   - NaN -> 0x7F with the sign bit of the input;
 *   - ties go to the even code (mantissa LSB 0); the code sequence is
 *     continuous across the subnormal/normal and binade edges, so "even
 *     mantissa" and "even code" coincide;
 *   - the sign is kept for results that round to zero (-tiny -> 0x80).      */
uint8_t orc_e4m3_encode(float xf)
{
    uint8_t sign = signbit(xf) ? 0x80 : 0x00;
    double a = fabs((double)xf);
    if (isnan(xf))
        return (uint8_t)(sign | 0x7F);
    if (a >= 448.0)                       /* includes +-inf */
        return (uint8_t)(sign | 0x7E);
    if (a < ldexp(1.0, -6)) {
        /* subnormal range: quantum 2^-9, code = number of quanta (0..8);
         * 8 quanta is 2^-6, whose code 0x08 is the first normal code.       */
        double q = rne_int(a / ldexp(1.0, -9));
        return (uint8_t)(sign | (uint8_t)q);
    }
    int e;
    frexp(a, &e);                         /* a = f * 2^e, f in [0.5, 1)      */
    e -= 1;                               /* a in [2^e, 2^(e+1))             */
    double q = rne_int(a / ldexp(1.0, e - 3));   /* in [8, 16]               */
    if (q == 16.0) {                      /* carried into the next binade    */
        q = 8.0;
        e += 1;
    }
    if (e + 7 > 15 || (e + 7 == 15 && q - 8.0 > 6.0))
        return (uint8_t)(sign | 0x7E);    /* cannot happen below 448         */
    return (uint8_t)(sign | (uint8_t)(((e + 7) << 3) | (int)(q - 8.0)));
}

void orc_e4m3_encode_array(const float *x, int64_t n, uint8_t *q)
{
    for (int64_t i = 0; i < n; ++i)
        q[i] = orc_e4m3_encode(x[i]);
}

/* Brute-force encoder straight from "nearest representable value": scan all
 * finite codes of the input's sign, keep the one at the smallest distance,
 * and on an exact tie the one with the even code.  For |x| <= 1024 every
 * distance |x - v| is exact in double (x is fp32 with exponent <= 10, every
 * v is a multiple of 2^-9 below 2^9).                                     */
uint8_t orc_e4m3_encode_bruteforce(float xf)
{
    uint8_t sign = signbit(xf) ? 0x80 : 0x00;
    if (isnan(xf))
        return (uint8_t)(sign | 0x7F);
    /* Beyond 1024 every candidate lies below x and the largest finite value
     * is trivially the nearest; there the double differences x - v would no
     * longer be exact (x's ulp exceeds 2^-9), so take it directly.  From 448
     * to 1024 the scan itself decides.                                    */
    if (isinf(xf) || fabs((double)xf) > 1024.0)
        return (uint8_t)(sign | 0x7E);
    double x = (double)xf;
    int best = -1;
    double bestd = INFINITY;
    for (int c = 0; c < 0x7F; ++c) {
        uint8_t code = (uint8_t)(sign | c);
        double d = fabs(x - orc_e4m3_decode(code));
        if (d < bestd || (d == bestd && (code & 1) == 0 && (best & 1) == 1)) {
            bestd = d;
            best = code;
        }
    }
    return (uint8_t)best;
}

/* Same definition, located by bisection over the (monotone) positive codes
 * 0x00..0x7E instead of a linear scan; used for the exhaustive 2^32 sweep. */
uint8_t orc_e4m3_encode_search(float xf)
{
    uint8_t sign = signbit(xf) ? 0x80 : 0x00;
    if (isnan(xf))
        return (uint8_t)(sign | 0x7F);
    double a = fabs((double)xf);
    if (isinf(xf) || a >= 448.0)
        return (uint8_t)(sign | 0x7E);
    /* largest c with dec(c) <= a */
    int lo = 0, hi = 0x7E;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (orc_e4m3_decode((uint8_t)mid) <= a)
            lo = mid;
        else
            hi = mid - 1;
    }
    int c = lo;
    if (c == 0x7E)
        return (uint8_t)(sign | c);
    double dl = a - orc_e4m3_decode((uint8_t)c);
    double du = orc_e4m3_decode((uint8_t)(c + 1)) - a;
    int pick;
    if (dl < du)
        pick = c;
    else if (du < dl)
        pick = c + 1;
    else
        pick = (c % 2 == 0) ? c : c + 1;
    return (uint8_t)(sign | pick);
}

/* Exhaustive comparison of the arithmetic encoder with the search encoder over
 * fp32 bit patterns [lo, hi).  Returns the number of mismatches and stores the
 * first mismatching pattern (or 0xFFFFFFFF).                              */
int64_t orc_check_encoder_range(uint64_t lo, uint64_t hi, uint32_t *first_bad)
{
    int64_t bad = 0;
    uint32_t first = 0xFFFFFFFFu;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t i = (int64_t)lo; i < (int64_t)hi; ++i) {
        uint32_t u = (uint32_t)i;
        float x;
        memcpy(&x, &u, 4);
        uint8_t a = orc_e4m3_encode(x);
        uint8_t b = orc_e4m3_encode_search(x);
        /* both NaN encodings carry the sign; compare bytes exactly */
        if (a != b) {
            bad += 1;
#pragma omp critical
            if (u < first)
                first = u;
        }
    }
    *first_bad = first;
    return bad;
}

/* Encode every fp32 bit pattern in [lo, hi) (for the device encoder sweep). */
void orc_encode_pattern_range(uint64_t lo, uint64_t hi, uint8_t *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = (int64_t)lo; i < (int64_t)hi; ++i) {
        uint32_t u = (uint32_t)i;
        float x;
        memcpy(&x, &u, 4);
        out[i - (int64_t)lo] = orc_e4m3_encode(x);
    }
}

/* ------------------------------------------------------------------------ */
/* E5M2 decode / encode (OCP FP8, E5M2 variant; paper section 2 lists both  */
/* FP8 variants, E5M2 ("bf8") beside E4M3 ("fp8"), as MFMA operand types).  */
/* ------------------------------------------------------------------------ */

/* Value of code c.  s = bit 7, e = bits 6..2, m = bits 1..0 (bias 15, the
 * IEEE-754 binary16 layout with the low eight mantissa bits dropped).
 *   e == 31, m == 0          -> (-1)^s * inf
 *   e == 31, m != 0          -> NaN (codes 0x7D..0x7F, 0xFD..0xFF)
 *   e == 0                   -> (-1)^s * m * 2^-16            (subnormal)
 *   otherwise                -> (-1)^s * (1 + m/4) * 2^(e-15)
 * Largest finite magnitude: (1 + 3/4) * 2^15 = 57344 (code 0x7B).         */
double orc_e5m2_decode(uint8_t c)
{
    int s = (c >> 7) & 1;
    int e = (c >> 2) & 31;
    int m = c & 3;
    double v;
    if (e == 31)
        v = (m == 0) ? INFINITY : NAN;
    else if (e == 0)
        v = ldexp((double)m, -16);
    else
        v = ldexp(1.0 + (double)m / 4.0, e - 15);
    if (isnan(v))
        return v;
    return s ? -v : v;
}

/* Arithmetic encoder, round to nearest, ties to even, saturating.  Readings
 * where the paper is silent (the same as for E4M3):
 *   - finite overflow and +-inf saturate to +-57344 ("satfinite"), so no
 *     quantised operand is ever infinite;
 *   - NaN -> 0x7F with the input's sign bit;
 *   - ties go to the even code; the code sequence is continuous across the
 *     subnormal/normal and binade edges, so "even mantissa" = "even code";
 *   - the sign is kept for results that round to zero.                     */
uint8_t orc_e5m2_encode(float xf)
{
    uint8_t sign = signbit(xf) ? 0x80 : 0x00;
    double a = fabs((double)xf);
    if (isnan(xf))
        return (uint8_t)(sign | 0x7F);
    if (a >= 57344.0)                     /* includes +-inf */
        return (uint8_t)(sign | 0x7B);
    if (a < ldexp(1.0, -14)) {
        /* subnormal range: quantum 2^-16, code = number of quanta (0..4);
         * 4 quanta is 2^-14, whose code 0x04 is the first normal code.      */
        double q = rne_int(a / ldexp(1.0, -16));
        return (uint8_t)(sign | (uint8_t)q);
    }
    int e;
    frexp(a, &e);                         /* a = f * 2^e, f in [0.5, 1)      */
    e -= 1;                               /* a in [2^e, 2^(e+1))             */
    double q = rne_int(a / ldexp(1.0, e - 2));   /* in [4, 8]                */
    if (q == 8.0) {                       /* carried into the next binade    */
        q = 4.0;
        e += 1;
    }
    if (e + 15 > 30)
        return (uint8_t)(sign | 0x7B);    /* cannot happen below 57344       */
    return (uint8_t)(sign | (uint8_t)(((e + 15) << 2) | (int)(q - 4.0)));
}

void orc_e5m2_decode_array(const uint8_t *c, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; ++i)
        out[i] = orc_e5m2_decode(c[i]);
}

void orc_e5m2_encode_array(const float *x, int64_t n, uint8_t *q)
{
    for (int64_t i = 0; i < n; ++i)
        q[i] = orc_e5m2_encode(x[i]);
}

/* Brute force from "nearest finite value, ties to the even code": a scan of
 * the finite codes of the input's sign.  Where two codes are nearly equally
 * near, x lies between them within a factor of two of the larger, so both
 * differences are exact in double (fp32 x: 24 significant bits; codes:
 * multiples of 2^-16 with 3 significant bits); farther codes may round but
 * rounding is monotone and cannot move them ahead.  Beyond 2^17 every finite
 * code lies below x and the largest is the nearest.                       */
uint8_t orc_e5m2_encode_bruteforce(float xf)
{
    uint8_t sign = signbit(xf) ? 0x80 : 0x00;
    if (isnan(xf))
        return (uint8_t)(sign | 0x7F);
    if (isinf(xf) || fabs((double)xf) > 131072.0)
        return (uint8_t)(sign | 0x7B);
    double x = (double)xf;
    int best = -1;
    double bestd = INFINITY;
    for (int c = 0; c <= 0x7B; ++c) {
        uint8_t code = (uint8_t)(sign | c);
        double d = fabs(x - orc_e5m2_decode(code));
        if (d < bestd || (d == bestd && (code & 1) == 0 && (best & 1) == 1)) {
            bestd = d;
            best = code;
        }
    }
    return (uint8_t)best;
}

/* The same definition located by bisection over the monotone positive finite
 * codes 0x00..0x7B; used for the exhaustive fp32 sweep.                   */
uint8_t orc_e5m2_encode_search(float xf)
{
    uint8_t sign = signbit(xf) ? 0x80 : 0x00;
    if (isnan(xf))
        return (uint8_t)(sign | 0x7F);
    double a = fabs((double)xf);
    if (isinf(xf) || a >= 57344.0)
        return (uint8_t)(sign | 0x7B);
    int lo = 0, hi = 0x7B;                /* largest c with dec(c) <= a */
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (orc_e5m2_decode((uint8_t)mid) <= a)
            lo = mid;
        else
            hi = mid - 1;
    }
    int c = lo;
    if (c == 0x7B)
        return (uint8_t)(sign | c);
    double dl = a - orc_e5m2_decode((uint8_t)c);
    double du = orc_e5m2_decode((uint8_t)(c + 1)) - a;
    int pick;
    if (dl < du)
        pick = c;
    else if (du < dl)
        pick = c + 1;
    else
        pick = (c % 2 == 0) ? c : c + 1;
    return (uint8_t)(sign | pick);
}

/* Format-generic front ends.  fmt 0: E4M3, fmt 1: E5M2.                   */
double orc_fp8_decode(int fmt, uint8_t c)
{
    return fmt == 1 ? orc_e5m2_decode(c) : orc_e4m3_decode(c);
}

uint8_t orc_fp8_encode(int fmt, float x)
{
    return fmt == 1 ? orc_e5m2_encode(x) : orc_e4m3_encode(x);
}

/* Exhaustive arithmetic-vs-search comparison for E5M2 over fp32 patterns
 * [lo, hi); returns mismatches, *first_bad the first (or 0xFFFFFFFF).     */
int64_t orc_check_e5m2_encoder_range(uint64_t lo, uint64_t hi, uint32_t *first_bad)
{
    int64_t bad = 0;
    uint32_t first = 0xFFFFFFFFu;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t i = (int64_t)lo; i < (int64_t)hi; ++i) {
        uint32_t u = (uint32_t)i;
        float x;
        memcpy(&x, &u, 4);
        if (orc_e5m2_encode(x) != orc_e5m2_encode_search(x)) {
            bad += 1;
#pragma omp critical
            if (u < first)
                first = u;
        }
    }
    *first_bad = first;
    return bad;
}

/* E5M2 codes of every fp32 bit pattern in [lo, hi).                       */
void orc_e5m2_encode_pattern_range(uint64_t lo, uint64_t hi, uint8_t *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = (int64_t)lo; i < (int64_t)hi; ++i) {
        uint32_t u = (uint32_t)i;
        float x;
        memcpy(&x, &u, 4);
        out[i - (int64_t)lo] = orc_e5m2_encode(x);
    }
}

/* ------------------------------------------------------------------------ */
/* Quantisation (scale selection + E4M3 / E5M2 encode).                     */
/* ------------------------------------------------------------------------ */

/* x: fp32 [rows, cols] with row stride ld (elements).  mode 0: one scale for
 * the tensor; mode 1: one scale per row.  fmt 0: E4M3, whose largest finite
 * value T is 448; fmt 1: E5M2, T = 57344.  For each scaling group:
 *   amax = max |x|                                   (exact)
 *   s    = fl32(T / amax),  d = fl32(amax / T)       (one IEEE fp32 division
 *                                                     each; amax == 0 gives
 *                                                     s = d = 1)
 *   q    = enc(fl32(x * s))                          (one fp32 multiply)
 * d (the dequantisation factor) is written to d[0] (mode 0) or d[r].
 * q has row stride ldq bytes.  Returns 0, or -4 if any input is not finite
 * (outputs are then unspecified).                                        */
int orc_quantize_fmt(const float *x, int64_t rows, int64_t cols, int64_t ld,
                     int mode, int fmt, uint8_t *q, int64_t ldq, float *d)
{
    int64_t groups = (mode == 0) ? 1 : rows;
    for (int64_t g = 0; g < groups; ++g) {
        int64_t r0 = (mode == 0) ? 0 : g;
        int64_t r1 = (mode == 0) ? rows : g + 1;
        float amax = 0.0f;
        for (int64_t r = r0; r < r1; ++r)
            for (int64_t c = 0; c < cols; ++c) {
                float v = x[r * ld + c];
                if (!isfinite(v))
                    return -4;
                float av = fabsf(v);
                if (av > amax)
                    amax = av;
            }
        float s, dq;
        if (amax == 0.0f) {
            s = 1.0f;
            dq = 1.0f;
        } else {
            volatile float num = 448.0f;   /* keep both divisions in fp32 */
            if (fmt == 1)
                num = 57344.0f;
            s = num / amax;
            dq = amax / num;
        }
        d[g] = dq;
        for (int64_t r = r0; r < r1; ++r)
            for (int64_t c = 0; c < cols; ++c) {
                volatile float y = x[r * ld + c] * s;
                q[r * ldq + c] = orc_fp8_encode(fmt, y);
            }
    }
    return 0;
}

/* E4M3 quantisation: orc_quantize_fmt with fmt 0. */
int orc_quantize(const float *x, int64_t rows, int64_t cols, int64_t ld,
                 int mode, uint8_t *q, int64_t ldq, float *d)
{
    return orc_quantize_fmt(x, rows, cols, ld, mode, 0, q, ldq, d);
}

/* ------------------------------------------------------------------------ */
/* 2:4 pruning and compression (paper section 2 "Structured Sparsity",      */
/* section 6: two of every four consecutive elements along K are zero).     */
/* ------------------------------------------------------------------------ */

/* a: codes [M, K], row stride lda.  K % 4 == 0.
 * For row m and group g (elements 4g..4g+3):
 *   key(c) = c & 0x7F (monotone in |value| over the finite codes of either
 *            FP8 variant, so the same pruning serves E4M3 and E5M2);
 *   the kept pair is the first two positions when the four are ordered by
 *   key descending, then index ascending (ties keep the lower index);
 *   vals[m, 2g], vals[m, 2g+1] = the kept codes in increasing index order;
 *   nibble(g) = i0 | (i1 << 2)   (i0 < i1 are the kept indices in 0..3),
 *   stored in meta[m, g/2]: low nibble for even g, high nibble for odd g.
 * vals has row stride K/2, meta has row stride (K+7)/8.  Returns 0 or -2. */
int orc_prune24(const uint8_t *a, int64_t M, int64_t K, int64_t lda,
                uint8_t *vals, uint8_t *meta)
{
    if (K % 4 != 0)
        return -2;
    int64_t ldv = K / 2, ldm = (K + 7) / 8;
    memset(meta, 0, (size_t)(M * ldm));
    for (int64_t m = 0; m < M; ++m)
        for (int64_t g = 0; g < K / 4; ++g) {
            const uint8_t *grp = a + m * lda + 4 * g;
            int first = -1, second = -1;
            for (int i = 0; i < 4; ++i) {
                int k = grp[i] & 0x7F;
                if (first < 0 || k > (grp[first] & 0x7F)) {
                    second = first;
                    first = i;
                } else if (second < 0 || k > (grp[second] & 0x7F)) {
                    second = i;
                }
            }
            int i0 = first < second ? first : second;
            int i1 = first < second ? second : first;
            vals[m * ldv + 2 * g] = grp[i0];
            vals[m * ldv + 2 * g + 1] = grp[i1];
            uint8_t nib = (uint8_t)(i0 | (i1 << 2));
            meta[m * ldm + g / 2] |= (uint8_t)(nib << (4 * (g % 2)));
        }
    return 0;
}

/* Inverse of the compression: scatter the kept codes back to their positions
 * and write 0x00 elsewhere.  out: [M, K] dense, row stride K.              */
void orc_decompress24(const uint8_t *vals, const uint8_t *meta, int64_t M,
                      int64_t K, uint8_t *out)
{
    int64_t ldv = K / 2, ldm = (K + 7) / 8;
    memset(out, 0, (size_t)(M * K));
    for (int64_t m = 0; m < M; ++m)
        for (int64_t g = 0; g < K / 4; ++g) {
            uint8_t nib = (meta[m * ldm + g / 2] >> (4 * (g % 2))) & 0xF;
            int i0 = nib & 3, i1 = (nib >> 2) & 3;
            out[m * K + 4 * g + i0] = vals[m * ldv + 2 * g];
            out[m * K + 4 * g + i1] = vals[m * ldv + 2 * g + 1];
        }
}

/* ------------------------------------------------------------------------ */
/* GEMM: C[m,n] = alpha * dA[m] * dB[n] * sum_k decA(A[m,k]) * decB(B[n,k])  */
/* A: codes [M, K] (row stride lda), B: codes [N, K] (row stride ldb), both */
/* K-contiguous; a_fmt / b_fmt pick each operand's FP8 variant (0: E4M3,    */
/* 1: E5M2; paper section 2 and Table 3: the FP8 matrix cores take either   */
/* variant for each operand).  a_mode/b_mode 0: one scale dA[0] / dB[0];    */
/* 1: per row of the stored matrix (dA[m], dB[n]).  FP64 everywhere; C is   */
/* [M, N] doubles.                                                          */
/* ------------------------------------------------------------------------ */

static double dot_codes(const uint8_t *a, int fa, const uint8_t *b, int fb, int64_t K)
{
    double s = 0.0;
    for (int64_t k = 0; k < K; ++k)
        s += orc_fp8_decode(fa, a[k]) * orc_fp8_decode(fb, b[k]);
    return s;
}

void orc_gemm(int64_t M, int64_t N, int64_t K, const uint8_t *A, int64_t lda,
              const uint8_t *B, int64_t ldb, const float *dA, int a_mode,
              const float *dB, int b_mode, double alpha, int a_fmt, int b_fmt,
              double *C)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t m = 0; m < M; ++m)
        for (int64_t n = 0; n < N; ++n) {
            double sa = (double)dA[a_mode ? m : 0];
            double sb = (double)dB[b_mode ? n : 0];
            C[m * N + n] = alpha * sa * sb *
                           dot_codes(A + m * lda, a_fmt, B + n * ldb, b_fmt, K);
        }
}

/* The same definition evaluated only at the listed (m, n) pairs; used where
 * the full product is too large for the CPU (each entry is an independent
 * dot product).                                                           */
void orc_gemm_sampled(int64_t K, const uint8_t *A, int64_t lda,
                      const uint8_t *B, int64_t ldb, const float *dA,
                      int a_mode, const float *dB, int b_mode, double alpha,
                      int a_fmt, int b_fmt, int64_t n_samples, const int64_t *ms,
                      const int64_t *ns, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n_samples; ++i) {
        int64_t m = ms[i], n = ns[i];
        double sa = (double)dA[a_mode ? m : 0];
        double sb = (double)dB[b_mode ? n : 0];
        out[i] = alpha * sa * sb * dot_codes(A + m * lda, a_fmt, B + n * ldb, b_fmt, K);
    }
}

/* Sparse GEMM: the dense definition applied to the decompressed pruned A
 * (paper section 6 compares sparse GEMM against dense GEMM on the same
 * operands; the sparse product equals the dense product of the zero-filled
 * matrix).  Code 0x00 is +0 in both FP8 variants.                         */
void orc_gemm_sparse24(int64_t M, int64_t N, int64_t K, const uint8_t *vals,
                       const uint8_t *meta, const uint8_t *B, int64_t ldb,
                       const float *dA, int a_mode, const float *dB,
                       int b_mode, double alpha, int a_fmt, int b_fmt, double *C)
{
    uint8_t *a = (uint8_t *)malloc((size_t)(M * K));
    orc_decompress24(vals, meta, M, K, a);
    orc_gemm(M, N, K, a, K, B, ldb, dA, a_mode, dB, b_mode, alpha, a_fmt, b_fmt, C);
    free(a);
}

/* ------------------------------------------------------------------------ */
/* Block-scaled FP8 (the OCP Microscaling formats MXFP8 E4M3 / E5M2): each  */
/* block of 32 consecutive elements along K shares one power-of-two scale   */
/* stored as E8M0.  Not in the paper; the next precision step after the     */
/* per-row scaling it measures.                                             */
/* ------------------------------------------------------------------------ */

#define ORC_MX_BLOCK 32

/* E8M0 scale code e: 2^(e - 127) for e = 0..254; 0xFF is NaN.  No sign,
 * no zero, no mantissa.                                                   */
double orc_e8m0_decode(uint8_t e)
{
    if (e == 0xFF)
        return NAN;
    return ldexp(1.0, (int)e - 127);
}

void orc_e8m0_decode_array(const uint8_t *c, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; ++i)
        out[i] = orc_e8m0_decode(c[i]);
}

/* x: fp32 [rows, cols], row stride ld; cols % 32 == 0.  For each row and
 * each block of 32 columns:
 *   amax = max |x| over the block;
 *   amax == 0      -> scale code 0 (2^-127) and all codes 0 (reading: the
 *                     spec leaves the exponent free for an all-zero block);
 *   otherwise  e   = floor(log2(amax)) - emax, emax = 8 for E4M3 (448 =
 *                    1.75 * 2^8) and 15 for E5M2 (57344 = 1.75 * 2^15),
 *                    clamped to the E8M0 range [-127, 127];
 *              code = e + 127;  q = enc(x * 2^-e) (round to nearest even,
 *                    saturating; amax * 2^-e lies in [2^emax, 2^(emax+1)),
 *                    so block maxima above the format's largest value
 *                    saturate to it).
 * The scaling by 2^-e is exact in fp32 wherever the result is at least
 * 2^-126, and anything smaller encodes to zero in both formats.
 * q has row stride ldq; scales are [rows, cols / 32] row-major.
 * Returns 0, -2 if cols % 32 != 0, -4 on a non-finite input.             */
int orc_mx_quantize(const float *x, int64_t rows, int64_t cols, int64_t ld,
                    int fmt, uint8_t *q, int64_t ldq, uint8_t *scales)
{
    if (cols % ORC_MX_BLOCK != 0)
        return -2;
    const int emax = (fmt == 1) ? 15 : 8;
    const int64_t nb = cols / ORC_MX_BLOCK;
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t b = 0; b < nb; ++b) {
            const float *xb = x + r * ld + b * ORC_MX_BLOCK;
            uint8_t *qb = q + r * ldq + b * ORC_MX_BLOCK;
            double amax = 0.0;
            for (int i = 0; i < ORC_MX_BLOCK; ++i) {
                if (!isfinite(xb[i]))
                    return -4;
                if (fabs((double)xb[i]) > amax)
                    amax = fabs((double)xb[i]);
            }
            if (amax == 0.0) {
                scales[r * nb + b] = 0;
                for (int i = 0; i < ORC_MX_BLOCK; ++i)
                    qb[i] = orc_fp8_encode(fmt, xb[i]);       /* +-0 keep their sign */
                continue;
            }
            int E;
            frexp(amax, &E);                  /* amax = f * 2^E, f in [0.5, 1) */
            int e = (E - 1) - emax;           /* floor(log2(amax)) - emax      */
            if (e < -127)
                e = -127;
            if (e > 127)
                e = 127;
            scales[r * nb + b] = (uint8_t)(e + 127);
            for (int i = 0; i < ORC_MX_BLOCK; ++i)
                qb[i] = orc_fp8_encode(fmt, (float)ldexp((double)xb[i], -e));
        }
    return 0;
}

/* C[m,n] = alpha * sum over blocks b of SA[m,b] * SB[n,b] *
 *          sum_{k in b} decA(A[m,k]) * decB(B[n,k])   (FP64), with SA, SB
 * the decoded E8M0 scales ([M, K/32] and [N, K/32] row-major), A [M, K]
 * and B [N, K] codes (row strides lda, ldb).  K % 32 == 0.               */
void orc_gemm_mx(int64_t M, int64_t N, int64_t K, const uint8_t *A, int64_t lda,
                 const uint8_t *SA, const uint8_t *B, int64_t ldb, const uint8_t *SB,
                 double alpha, int a_fmt, int b_fmt, double *C)
{
    const int64_t nb = K / ORC_MX_BLOCK;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t m = 0; m < M; ++m)
        for (int64_t n = 0; n < N; ++n) {
            double acc = 0.0;
            for (int64_t b = 0; b < nb; ++b) {
                const double sb = orc_e8m0_decode(SA[m * nb + b]) * orc_e8m0_decode(SB[n * nb + b]);
                const int64_t k0 = b * ORC_MX_BLOCK;
                acc += sb * dot_codes(A + m * lda + k0, a_fmt, B + n * ldb + k0, b_fmt,
                                      ORC_MX_BLOCK);
            }
            C[m * N + n] = alpha * acc;
        }
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n);
#else
    (void)n;
#endif
}
