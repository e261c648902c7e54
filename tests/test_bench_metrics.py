"""CPU tests of the benchmark's concurrency metrics (the paper's section
3.2 definitions: speedup over serial execution, per-stream coefficient of
variation, fairness 1 - (t_max - t_min) / t_mean and min / max, overlap
efficiency) on hand-made stream intervals."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_concurrency_stats_two_streams():
    import bench
    # stream 0 busy [0, 4] ms, stream 1 busy [2, 8] ms; alone they take 3 and 5
    st = bench._concurrency_stats([(0.0, 4.0), (2.0, 8.0)], 8.0, [3.0, 5.0])
    assert st["streams"] == 2
    assert st["speedup"] == pytest.approx(8.0 / 8.0)
    assert st["per_stream_ms"] == [4.0, 6.0]
    assert st["per_stream_speedup"] == pytest.approx([0.75, 5.0 / 6.0])
    assert st["cv"] == pytest.approx(1.0 / 5.0)
    assert st["fairness_1_minus_range_over_mean"] == pytest.approx(1.0 - 2.0 / 5.0)
    assert st["fairness_min_over_max"] == pytest.approx(4.0 / 6.0)
    assert st["overlap_efficiency"] == pytest.approx(2.0 / 8.0)


def test_concurrency_stats_serial_and_identical():
    import bench
    st = bench._concurrency_stats([(0.0, 1.0), (1.0, 2.0)], 2.0, [1.0, 1.0])
    assert st["overlap_efficiency"] == 0.0 and st["speedup"] == pytest.approx(1.0)
    st = bench._concurrency_stats([(0.0, 2.0), (0.0, 2.0)], 2.0, [1.0, 1.0])
    assert st["overlap_efficiency"] == pytest.approx(1.0)
    assert st["fairness_1_minus_range_over_mean"] == 1.0 and st["cv"] == 0.0


def test_recorded_traffic_follows_the_kernel_source(tmp_path):
    """The DRAM traffic in the benchmark line comes from the committed ncu
    summary only while the GEMM source is the one it was captured on."""
    import hashlib
    import bench
    src = tmp_path / "gemm.cu"
    src.write_bytes(b"// a kernel source\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "gemm_fp8_kernel_dense_16384.md").write_text(
        f"# record\n\n- source_sha256_16: `{sha}`\n- dram_bytes_per_launch: `3646000000`\n")
    assert bench.recorded_traffic(str(src), "dense_16384", str(prof)) == 3646000000.0
    src.write_bytes(src.read_bytes() + b"// edited\n")
    assert bench.recorded_traffic(str(src), "dense_16384", str(prof)) is None
    assert bench.recorded_traffic(str(src), "no_such_workload", str(prof)) is None
