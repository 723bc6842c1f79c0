"""Host-side logic of bench.py that needs no GPU: the roofline entry of the
dominant stage, the stage notes it carries, and the key that ties a DRAM
traffic figure to the kernel code it was captured on."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_source_digest_ignores_comments_but_not_code(tmp_path):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    c = tmp_path / "c.cu"
    a.write_text("int f(int x) {\n    return x + 1;   // one more\n}\n")
    b.write_text("// a new header comment\nint f(int x) {\n\n    return x + 1;\n}\n")
    c.write_text("int f(int x) {\n    return x + 2;   // one more\n}\n")
    da = bench.source_digest([str(a)])
    assert da == bench.source_digest([str(b)])
    assert da != bench.source_digest([str(c)])
    # the order of the sources is part of the key
    assert bench.source_digest([str(a), str(c)]) != bench.source_digest([str(c), str(a)])


def test_kernel_traffic_is_reported_only_for_the_captured_code(monkeypatch, tmp_path):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    entry = {"sources": [str(src)], "sha1": bench.source_digest([str(src)]), "bytes_per_view": 1000.0}
    monkeypatch.setitem(bench.KERNEL_TRAFFIC, "probe", entry)
    assert bench.kernel_traffic("probe", 8) == 8000
    src.write_text("__global__ void k() { }  // comment only\n")
    assert bench.kernel_traffic("probe", 8) is None   # the code changed ("{}" -> "{ }")
    src.write_text("__global__ void k() {}\n// comment only\n")
    assert bench.kernel_traffic("probe", 8) == 8000
    assert bench.kernel_traffic("no such kernel", 8) is None


def test_roofline_names_the_dominant_stage_and_carries_the_stage_notes():
    per_step = {"entries": 24_000_000, "gaussians": 3_000_000, "attr_bytes": 124, "kept": 23_990_000,
                "depth_passes": 3, "compact_rect": 1, "pairs": 16_000_000, "sort_passes": 2, "tiles": 65280,
                "slices": 6, "evals": 1.4e9, "views": 8}
    stage_ms = {"blend": {"ms": 1.1, "calls": 1}, "emit": {"ms": 0.24, "calls": 1},
                "depth_sort": {"ms": 0.67, "calls": 1}, "frame": {"ms": 3.3, "calls": 1}}
    peaks = {"hbm_gbs": 6510.4, "source": "measured"}
    roof, stages = bench.roofline(stage_ms, per_step, peaks, {"sm_mhz": 2032.0}, 20)
    assert roof["kernel"] == "blend" and roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    # 14 operations per evaluation over the FP32 peak at the sampled clock
    peak = 148 * 128 * 2 * 2032e6 / 1e12
    assert abs(roof["peak"] - peak) < 1e-9
    assert abs(roof["frac"] - (1.4e9 * 14 / 1.1e-3 / 1e12) / peak) < 1e-4
    assert "frame" not in stages
    for name in ("blend", "emit", "depth_sort"):
        assert stages[name]["limit"] == bench.STAGE_LIMITS[name]
    # the depth sort's algorithmic bytes: passes x 24 B per entry with compact rectangles
    assert stages["depth_sort"]["work"] == 24_000_000 * 3 * 24
