"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every function that include/gb300fp8.h declares, and rejects bad arguments
on the host before touching a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def _declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            if not m.group(0).lstrip().startswith(("typedef", "#")):
                names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2602_10262_gb300 import _lib
    return _lib.load()


def test_header_declares_the_path():
    names = _declared_functions()
    for n in ("fp8_quantize_e4m3", "fp8_quantize_e5m2", "prune24_compress", "gemm_fp8_dense",
              "gemm_fp8_dense_fmt", "gemm_fp8_sparse24", "gemm_fp8_sparse24_fmt",
              "gemm_fp8_grouped", "fp8_last_device_error", "fp8_status_string"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    assert lib.fp8_status_string(0) == b"ok"
    assert lib.fp8_status_string(-7) == b"device pipeline wait timed out"
    assert lib.fp8_status_string(12345) == b"unknown status"


def test_host_validation_without_gpu(lib):
    P = ctypes.c_void_p
    # negative sizes, bad modes and bad K are rejected before any CUDA call
    assert lib.gemm_fp8_dense(-1, 4, 4, None, 16, None, 16, None, 0, None, 0, 1.0, None, 4, 0, None) == -1
    assert lib.gemm_fp8_dense(4, 4, 4, None, 16, None, 16, None, 2, None, 0, 1.0, None, 4, 0, None) == -1
    assert lib.gemm_fp8_dense(4, 4, 4, P(16), 16, P(16), 16, P(16), 0, P(16), 0, 1.0, P(16), 4, 5, None) == -1
    assert lib.gemm_fp8_dense(4, 4, 32, P(16), 16, P(16), 32, P(16), 0, P(16), 0, 1.0, P(16), 4, 0, None) == -2
    assert lib.gemm_fp8_dense(4, 4, 32, P(16), 40, P(16), 48, P(16), 0, P(16), 0, 1.0, P(16), 4, 0, None) == -3
    assert lib.gemm_fp8_dense(4, 4, 32, P(8), 32, P(16), 32, P(16), 0, P(16), 0, 1.0, P(16), 4, 0, None) == -3
    assert lib.prune24_compress(P(16), 4, 6, 16, P(16), P(16), None) == -2
    assert lib.fp8_quantize_e4m3(P(16), 4, 4, 4, 3, P(16), 4, P(16), None) == -1
    assert lib.fp8_quantize_e4m3(P(16), 4, 8, 4, 0, P(16), 8, P(16), None) == -2
    assert lib.fp8_quantize_e5m2(P(16), 4, 4, 4, 3, P(16), 4, P(16), None) == -1
    assert lib.fp8_quantize_e5m2(P(16), 4, 8, 4, 0, P(16), 8, P(16), None) == -2
    # the fused quantise + 2:4 compress: K % 128, leading dimensions, alignment
    fq = lib.fp8_quantize_e4m3_prune24
    assert fq(None, 4, 128, 128, P(16), 128, P(16), P(16), P(16), None) == -1
    assert fq(P(16), 4, 100, 100, P(16), 100, P(16), P(16), P(16), None) == -2
    assert fq(P(16), 4, 128, 100, P(16), 128, P(16), P(16), P(16), None) == -2
    assert fq(P(20), 4, 128, 128, P(16), 128, P(16), P(16), P(16), None) == -3
    assert fq(P(16), 4, 128, 130, P(16), 128, P(16), P(16), P(16), None) == -3
    assert fq(P(16), 4, 128, 128, P(18), 128, P(16), P(16), P(16), None) == -3
    assert fq(P(16), 4, 128, 128, P(16), 130, P(16), P(16), P(16), None) == -3
    assert fq(None, 0, 128, 128, None, 128, None, None, None, None) == 0
    # operand formats other than E4M3 (0) and E5M2 (1) are rejected
    ok = (4, 4, 32, P(16), 32, P(16), 32, P(16), 0, P(16), 0, 1.0, P(16), 4, 0)
    for af, bf in ((2, 0), (0, -1), (7, 7)):
        assert lib.gemm_fp8_dense_fmt(*ok, af, bf, None) == -1
    sp = (4, 4, 128, P(16), P(16), P(16), 128, P(16), 0, P(16), 0, 1.0, P(16), 4, 0, 0)
    assert lib.gemm_fp8_sparse24_fmt(*sp, 0, 2, None) == -1
    assert lib.gemm_fp8_sparse24_fmt(4, 4, 96, P(16), P(16), P(16), 128, P(16), 0, P(16), 0, 1.0,
                                     P(16), 4, 0, 0, 1, 1, None) == -2
    # empty problems are a no-op
    assert lib.gemm_fp8_dense(0, 4, 4, None, 16, None, 16, None, 0, None, 0, 1.0, None, 4, 0, None) == 0
    assert lib.gemm_fp8_dense_fmt(0, 4, 4, None, 16, None, 16, None, 0, None, 0, 1.0, None, 4, 0,
                                  1, 1, None) == 0
    assert lib.fp8_quantize_e4m3(None, 0, 4, 4, 0, None, 4, None, None) == 0
    assert lib.fp8_quantize_e5m2(None, 0, 4, 4, 0, None, 4, None, None) == 0


def test_stall_switch_validates_and_resets(lib):
    # failure-path test switch: bad counts and limits are refused; 0, 0
    # cancels pending stalls and restores the default limit (no CUDA call)
    assert lib.fp8_test_stall_gemm_loads(-1, 0.0) == -1
    assert lib.fp8_test_stall_gemm_loads(0, -1.0) == -1
    assert lib.fp8_test_stall_gemm_loads(0, float("nan")) == -1
    assert lib.fp8_test_stall_gemm_loads(0, 1e9) == -1
    assert lib.fp8_test_stall_gemm_loads(3, 50.0) == 0
    assert lib.fp8_test_stall_gemm_loads(0, 0.0) == 0


def test_plan_queries_reject_bad_arguments(lib):
    """The plan queries (dense, 2:4, block-scaled) refuse a missing info
    struct, empty or negative sizes and bad output types before any CUDA
    call, and sizes past int32 / 2 as shapes."""
    from paper_2602_10262_gb300 import _lib
    info = _lib.FP8PlanInfo()
    ref = ctypes.byref(info)
    for fn in (lib.gemm_fp8_dense_plan, lib.gemm_fp8_sparse24_plan, lib.gemm_fp8_mx_plan):
        assert fn(256, 256, 256, 0, None) == -1
        assert fn(0, 256, 256, 0, ref) == -1
        assert fn(256, -1, 256, 0, ref) == -1
        assert fn(256, 256, 256, 2, ref) == -1
        assert fn(1 << 31, 256, 256, 0, ref) == -2


def test_tile_and_multicast_switches_validate(lib):
    # launch-shape switches (no CUDA call): out-of-range values are refused,
    # the defaults are restored
    assert lib.fp8_gemm_set_tile_config(4, 0) == -1
    assert lib.fp8_gemm_set_tile_config(-1, 0) == -1
    assert lib.fp8_gemm_set_tile_config(0, -1) == -1
    assert lib.fp8_gemm_set_tile_config(3, 8) == 0
    assert lib.fp8_gemm_set_tile_config(0, 0) == 0
    for bad in (-1, 2, 4):
        assert lib.fp8_gemm_set_multicast(bad) == -1
    assert lib.fp8_gemm_set_multicast(1) == 0
    assert lib.fp8_gemm_set_multicast(0) == 0


def test_mx_host_checks(lib):
    P = ctypes.c_void_p
    # tiled scale bytes: 512 per 128 rows x 128 columns, partial tiles rounded up
    assert lib.fp8_mx_scale_tiled_bytes(128, 128) == 512
    assert lib.fp8_mx_scale_tiled_bytes(129, 160) == 2 * 2 * 512
    assert lib.fp8_mx_scale_tiled_bytes(0, 128) == 0
    # the row length must hold whole 32-element blocks; formats and layouts checked
    assert lib.fp8_quantize_mx(P(16), 4, 48, 48, 0, P(16), 48, P(16), 0, None) == -2
    assert lib.fp8_quantize_mx(P(16), 4, 64, 64, 2, P(16), 64, P(16), 0, None) == -1
    assert lib.fp8_quantize_mx(P(16), 4, 64, 64, 0, P(16), 64, P(16), 2, None) == -1
    assert lib.fp8_quantize_mx(P(16), 4, 64, 64, 0, P(16), 64, P(8), 1, None) == -3
    assert lib.fp8_mx_scales_to_tiled(P(16), 4, 40, P(16), None) == -2
    ok = (P(16), 64, P(16), P(16), 64, P(16), 1.0, P(16), 4, 0)
    assert lib.gemm_fp8_mx(4, 4, 48, *ok, 0, 0, None) == -2        # K % 32
    assert lib.gemm_fp8_mx(4, 4, 64, *ok, 0, 3, None) == -1        # format
    assert lib.gemm_fp8_mx(4, 4, 64, P(16), 64, P(8), P(16), 64, P(16), 1.0, P(16), 4, 0, 0, 0,
                           None) == -3                              # scales 16-byte aligned
    assert lib.gemm_fp8_mx(0, 4, 64, *ok, 0, 0, None) == 0


def test_grouped_rejects_bad_format(lib):
    from paper_2602_10262_gb300 import _lib
    pr = _lib.FP8Problem(4, 4, 32, 16, 0, 32, 16, 32, 16, 0, 16, 0, 1.0, 16, 4, 0, 0, 0, 0)
    good = (_lib.FP8Problem * 1)(pr)
    pr.b_format = 2
    bad = (_lib.FP8Problem * 1)(pr)
    assert lib.gemm_fp8_grouped(bad, 1, None) == -1
    # the same problem with valid formats passes the host checks and stops
    # only where a device is needed (no GPU here)
    assert lib.gemm_fp8_grouped(good, 1, None) == -8


def test_grouped_long_lists(lib):
    from paper_2602_10262_gb300 import _lib
    # more than 32 problems: the whole list is checked before any launch
    arr = (_lib.FP8Problem * 70)()
    assert lib.gemm_fp8_grouped(arr, 70, None) in (0, -8)      # empty problems; -8 without a GPU
    arr[65].a_mode = 7
    assert lib.gemm_fp8_grouped(arr, 70, None) == -1
    assert lib.gemm_fp8_grouped(None, 1, None) == -1
    assert lib.gemm_fp8_grouped(None, 0, None) in (0, -8)
    # the autotuner and graphs keep the one-launch limit
    best = _lib.FP8TileConfig()
    assert lib.gemm_fp8_grouped_autotune((_lib.FP8Problem * 33)(), 33, 0, 1, None, ctypes.byref(best)) == -2


def test_tune_cache_file_round_trip(lib, tmp_path):
    good = tmp_path / "tiles.txt"
    good.write_text("# comment\n9 1 0 8192 4096 4096 0 256 1 0 2 16\n")
    assert lib.gemm_fp8_tune_cache_clear() == 0
    assert lib.gemm_fp8_tune_cache_load(str(good).encode()) == 0
    out = tmp_path / "saved.txt"
    assert lib.gemm_fp8_tune_cache_save(str(out).encode()) == 0
    lines = [l for l in out.read_text().splitlines() if not l.startswith("#")]
    assert lines == ["9 1 0 8192 4096 4096 0 256 1 0 2 16 0"]        # a line without a cap reads as 0
    good.write_text("9 1 0 8192 4096 4096 0 256 1 0 1 8 64\n")
    assert lib.gemm_fp8_tune_cache_clear() == 0
    assert lib.gemm_fp8_tune_cache_load(str(good).encode()) == 0
    assert lib.gemm_fp8_tune_cache_save(str(out).encode()) == 0
    lines = [l for l in out.read_text().splitlines() if not l.startswith("#")]
    assert lines == ["9 1 0 8192 4096 4096 0 256 1 0 1 8 64"]
    for bad in ("3 1 2\n", "9 1 0 8192 4096 4096 0 256 1 0 7 16\n", "x y z\n",
                "9 1 0 8192 4096 4096 0 256 1 0 2 0\n", "9 1 0 8192 4096 4096 0 256 1 0 1 8 96\n"):
        f = tmp_path / "bad.txt"
        f.write_text(bad)
        assert lib.gemm_fp8_tune_cache_load(str(f).encode()) == -1
    assert lib.gemm_fp8_tune_cache_load(str(tmp_path / "missing.txt").encode()) == -1
    assert lib.gemm_fp8_tune_cache_clear() == 0


@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++11")])
def test_header_is_plain_c(lang, std):
    # the boundary is a C ABI: the header compiles on its own as C99 (and as
    # C++), with no torch or CUDA headers needed
    import shutil
    import subprocess
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    for h in HEADERS:
        r = subprocess.run([cc, "-fsyntax-only", std, "-Wall", "-Wextra", "-pedantic", "-Werror",
                            "-x", lang, h], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
