"""Planted mistakes in the oracle must fail its pins.

Each case copies ``oracle/oracle.c``, applies one plausible mistake (a wrong
bias, a dropped term, a wrong sign or index, a swapped tie-break, a transposed
nibble), compiles the copy into a temporary library and runs the CPU pins of
``test_oracle_*.py`` against it.  At least one pin must fail for every
mutant; the unmodified source must pass them all.
"""
import os

import numpy as np
import pytest

import oracle
from tests import test_oracle_codec as tc
from tests import test_oracle_e5m2 as t5
from tests import test_oracle_mx as tmx
from tests import test_oracle_gemm as tg
from tests import test_oracle_prune as tp
from tests import test_oracle_quant as tq

MUTANTS = {
    "decode_bias_8": ("ldexp(1.0 + (double)m / 8.0, e - 7)", "ldexp(1.0 + (double)m / 8.0, e - 8)"),
    "decode_subnormal_scale": ("v = ldexp((double)m, -9);", "v = ldexp((double)m, -10);"),
    "decode_sign_dropped": ("return s ? -v : v;", "return v;"),
    "encode_ties_away": ("return (fmod(f, 2.0) == 0.0) ? f : f + 1.0;", "return f + 1.0;"),
    "encode_no_saturation": ("    if (a >= 448.0)                       /* includes +-inf */\n"
                             "        return (uint8_t)(sign | 0x7E);",
                             "    if (a >= 448.0)                       /* includes +-inf */\n"
                             "        return (uint8_t)(sign | 0x7F);"),
    "encode_binade_off_by_one": ("double q = rne_int(a / ldexp(1.0, e - 3));",
                                 "double q = rne_int(a / ldexp(1.0, e - 2));"),
    "quant_wrong_target": ("volatile float num = 448.0f;", "volatile float num = 240.0f;"),
    "quant_scale_inverted": ("dq = amax / num;", "dq = num / amax;"),
    "quant_amax_not_abs": ("float av = fabsf(v);", "float av = v;"),
    "prune_tie_high_index": ("if (first < 0 || k > (grp[first] & 0x7F)) {",
                             "if (first < 0 || k >= (grp[first] & 0x7F)) {"),
    "prune_signed_key": ("int k = grp[i] & 0x7F;", "int k = grp[i];"),
    "prune_nibble_swapped": ("uint8_t nib = (uint8_t)(i0 | (i1 << 2));",
                             "uint8_t nib = (uint8_t)(i1 | (i0 << 2));"),
    "prune_nibble_high_first": ("meta[m * ldm + g / 2] |= (uint8_t)(nib << (4 * (g % 2)));",
                                "meta[m * ldm + g / 2] |= (uint8_t)(nib << (4 * (1 - g % 2)));"),
    "gemm_sign": ("s += orc_fp8_decode(fa, a[k]) * orc_fp8_decode(fb, b[k]);",
                  "s -= orc_fp8_decode(fa, a[k]) * orc_fp8_decode(fb, b[k]);"),
    "gemm_b_format_from_a": ("orc_fp8_decode(fb, b[k])", "orc_fp8_decode(fa, b[k])"),
    "gemm_short_k": ("for (int64_t k = 0; k < K; ++k)\n        s +=",
                     "for (int64_t k = 1; k < K; ++k)\n        s +="),
    "gemm_alpha_dropped": ("C[m * N + n] = alpha * sa * sb *", "C[m * N + n] = sa * sb *"),
    "gemm_scale_index": ("            double sa = (double)dA[a_mode ? m : 0];\n"
                         "            double sb = (double)dB[b_mode ? n : 0];\n"
                         "            C[m * N + n]",
                         "            double sa = (double)dA[a_mode ? m : 0];\n"
                         "            double sb = (double)dB[b_mode ? m % 1 : 0];\n"
                         "            C[m * N + n]"),
    "gemm_b_row_stride": ("dot_codes(A + m * lda, a_fmt, B + n * ldb, b_fmt, K);\n        }\n}",
                          "dot_codes(A + m * lda, a_fmt, B + n, b_fmt, K);\n        }\n}"),
    "e5m2_decode_bias_16": ("ldexp(1.0 + (double)m / 4.0, e - 15)", "ldexp(1.0 + (double)m / 4.0, e - 16)"),
    "e5m2_decode_subnormal_scale": ("v = ldexp((double)m, -16);", "v = ldexp((double)m, -15);"),
    "e5m2_decode_inf_as_nan": ("v = (m == 0) ? INFINITY : NAN;", "v = NAN;"),
    "e5m2_encode_saturates_to_inf": ("    if (a >= 57344.0)                     /* includes +-inf */\n"
                                     "        return (uint8_t)(sign | 0x7B);",
                                     "    if (a >= 57344.0)                     /* includes +-inf */\n"
                                     "        return (uint8_t)(sign | 0x7C);"),
    "e5m2_encode_binade_off_by_one": ("double q = rne_int(a / ldexp(1.0, e - 2));   /* in [4, 8]",
                                      "double q = rne_int(a / ldexp(1.0, e - 3));   /* in [4, 8]"),
    "e5m2_encode_subnormal_edge": ("if (a < ldexp(1.0, -14)) {", "if (a < ldexp(1.0, -15)) {"),
    "e5m2_encode_carry_dropped": ("    if (q == 8.0) {                       /* carried into the next binade    */\n"
                                  "        q = 4.0;\n        e += 1;\n    }",
                                  "    if (q == 8.0) {                       /* carried into the next binade    */\n"
                                  "        q = 7.0;\n    }"),
    "fp8_decode_dispatch": ("return fmt == 1 ? orc_e5m2_decode(c) : orc_e4m3_decode(c);",
                            "return fmt == 0 ? orc_e5m2_decode(c) : orc_e4m3_decode(c);"),
    "fp8_encode_dispatch": ("return fmt == 1 ? orc_e5m2_encode(x) : orc_e4m3_encode(x);",
                            "return orc_e4m3_encode(x);"),
    "quant_e5m2_target": ("                num = 57344.0f;", "                num = 65536.0f;"),
    "mx_emax_e4m3": ("const int emax = (fmt == 1) ? 15 : 8;", "const int emax = (fmt == 1) ? 15 : 7;"),
    "mx_ceil_not_floor": ("int e = (E - 1) - emax;", "int e = E - emax;"),
    "mx_scale_code_bias": ("scales[r * nb + b] = (uint8_t)(e + 127);", "scales[r * nb + b] = (uint8_t)(e + 128);"),
    "mx_scale_applied_inverted": ("qb[i] = orc_fp8_encode(fmt, (float)ldexp((double)xb[i], -e));",
                                  "qb[i] = orc_fp8_encode(fmt, (float)ldexp((double)xb[i], e));"),
    "e8m0_bias_128": ("return ldexp(1.0, (int)e - 127);", "return ldexp(1.0, (int)e - 128);"),
    "gemm_mx_b_scale_block": ("orc_e8m0_decode(SB[n * nb + b])", "orc_e8m0_decode(SB[n * nb])"),
    "decompress_swapped": ("out[m * K + 4 * g + i0] = vals[m * ldv + 2 * g];",
                           "out[m * K + 4 * g + i1] = vals[m * ldv + 2 * g];"),
}


def _pins(orc):
    """The CPU pins, bound to their arguments (the exhaustive sweep is left
    out for time; the sampled sweep and the library cross-checks stand in)."""
    return [
        lambda: tc.test_decode_all_256_codes_vs_torch(orc),
        lambda: tc.test_decode_landmarks(orc),
        lambda: tc.test_encode_landmarks_roundtrip(orc),
        lambda: tc.test_encode_vs_torch_in_range(orc),
        lambda: tc.test_encode_saturates(orc),
        lambda: tq.test_closed_form_cases(orc),
        lambda: tq.test_matches_torch_restatement(orc, 1, (64, 256)),
        lambda: tq.test_matches_torch_restatement(orc, 0, (3, 17)),
        lambda: tq.test_amax_maps_to_448(orc),
        lambda: tp.test_golden_groups(orc),
        lambda: tp.test_golden_groups_packed_in_rows(orc),
        lambda: tp.test_matches_sort_restatement(orc, (5, 12)),
        lambda: tp.test_invariants(orc),
        lambda: tg.test_vs_numpy_matmul(orc, 17, 9, 64, 1, 1),
        lambda: tg.test_vs_numpy_matmul(orc, 3, 5, 7, 0, 0),
        lambda: tg.test_small_integers_exact(orc),
        lambda: tg.test_identity(orc),
        lambda: tg.test_sparse_equals_dense_on_pruned(orc),
        lambda: t5.test_decode_all_256_codes_vs_torch(orc),
        lambda: t5.test_decode_landmarks(orc),
        lambda: t5.test_encode_landmarks_roundtrip(orc),
        lambda: t5.test_encode_vs_torch_in_range(orc),
        lambda: t5.test_encode_every_binary16_by_integer_rounding(orc),
        lambda: t5.test_encode_saturates(orc),
        lambda: t5.test_quantize_closed_form(orc),
        lambda: t5.test_quantize_matches_torch_restatement(orc, 1, (64, 256)),
        lambda: t5.test_gemm_formats_vs_numpy(orc, 0, 1, 17, 9, 64, 1, 1),
        lambda: t5.test_gemm_formats_vs_numpy(orc, 1, 0, 3, 5, 7, 0, 0),
        lambda: t5.test_gemm_small_integers_exact_every_pairing(orc),
        lambda: t5.test_gemm_format_is_per_operand(orc),
        lambda: tmx.test_e8m0_decode_all_codes_vs_torch_and_ml_dtypes(orc),
        lambda: tmx.test_hand_worked_blocks(orc),
        lambda: tmx.test_zero_block_and_errors(orc),
        lambda: tmx.test_scale_property_and_codes_vs_torch(orc, 0),
        lambda: tmx.test_power_of_two_invariance(orc, 0),
        lambda: tmx.test_gemm_mx_vs_numpy(orc, 0, 1),
    ]


def _failures(orc):
    n = 0
    for pin in _pins(orc):
        try:
            pin()
        except Exception:
            n += 1
    return n


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    return tmp_path_factory.mktemp("mutants")


def test_unmodified_source_passes_all_pins(orc):
    assert _failures(orc) == 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, mutant_dir):
    old, new = MUTANTS[name]
    src = open(oracle.SOURCE).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mutated = src.replace(old, new, 1)
    path = os.path.join(mutant_dir, f"{name}.c")
    with open(path, "w") as f:
        f.write(mutated)
    lib = oracle.compile_library(path, os.path.join(mutant_dir, f"lib{name}.so"))
    assert _failures(oracle.Oracle(lib)) >= 1, f"mutant {name} passed every pin"
