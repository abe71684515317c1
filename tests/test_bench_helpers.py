"""bench.py's accounting on CPU: algorithmic bytes, the HBM and FP32 roofline arithmetic, and the
DRAM-traffic record keyed by source digest."""
import os

import bench


def test_algorithmic_bytes_per_kernel():
    ab = bench.algorithmic_bytes(50_000, 981_312, 1297 * 840, 4346)
    # projection: index + 75 FP32 parameters + 64 B of records per active splat (+ tile counts)
    assert ab["project"] == 50_000 * (4 + 300 + 64) + 4 * 4346
    # forward raster: pair ids + records + per pixel frozen sums, target, image, state (64 B)
    assert ab["raster_fwd"] == 4 * 981_312 + 48 * 50_000 + 1297 * 840 * 64
    assert ab["raster_bwd"] == 4 * 981_312 + 48 * 50_000 + 1297 * 840 * 20 + 40 * 50_000
    assert ab["project_bwd"] == 50_000 * (4 + 300 + 40 + 300)
    # more active splats, more bytes, for every kernel
    ab2 = bench.algorithmic_bytes(100_000, 2 * 981_312, 1297 * 840, 4346)
    assert all(ab2[k] > ab[k] for k in ab if k != "scan_tiles")


def test_hbm_report_fractions():
    per = {k: {"avg_ms": 0.1} for k in ("project", "scatter", "raster_fwd", "raster_bwd", "project_bwd")}
    rep = bench.hbm_report(per, 50_000, 981_312, 1297 * 840, 4346, 0.5, {"hbm_gbs": 6000.0}, "measured")
    ab = bench.algorithmic_bytes(50_000, 981_312, 1297 * 840, 4346)
    assert abs(rep["per_kernel"]["raster_fwd"]["gbs"] - ab["raster_fwd"] / 1e-4 / 1e9) < 1e-6
    assert abs(rep["per_kernel"]["raster_fwd"]["frac"] - rep["per_kernel"]["raster_fwd"]["gbs"] / 6000.0) < 1e-12
    assert abs(rep["floor_ms"] - rep["step_bytes"] / 6000e9 * 1e3) < 1e-12
    assert "scan_tiles" not in rep["per_kernel"]  # no time given for it


def test_fp32_peak():
    # 152 SMs x 128 lanes x 2 flops x 2070 MHz
    assert abs(bench.fp32_peak_tflops(2070.0) - 80.54784) < 1e-9


def test_recorded_traffic_follows_the_source_digest(tmp_path, monkeypatch):
    d = bench.kernel_digest("raster_bwd")
    assert d == bench.kernel_digest("raster_bwd") and len(d) == 16
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "dram_traffic.txt").write_text(f"# comment\nraster_bwd 12345 {d} w\nraster_fwd 9 0000000000000000 w\n")
    csrc = tmp_path / "paper_2605_13855_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in set(sum(bench.KERNEL_SOURCES.values(), ())):
        (csrc / f).write_bytes(open(os.path.join(bench.ROOT, "paper_2605_13855_gb300", "csrc", f), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("raster_bwd") == 12345.0
    assert bench.recorded_traffic("raster_fwd") is None  # recorded for other sources
    assert bench.recorded_traffic("project_bwd") is None  # not recorded


def test_digest_ignores_comments_but_not_code():
    src = "// header\nint f(int x) {  /* block\n comment */\n    return x + 1;  // trailing\n}\n\n"
    same = "int f(int x) {\n    return x + 1;\n}\n"
    other = "int f(int x) {\n    return x + 2;\n}\n"
    assert bench._code_only(src) == bench._code_only(same)
    assert bench._code_only(src) != bench._code_only(other)
