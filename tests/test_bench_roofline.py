"""bench.py's bookkeeping on CPU: the algorithmic bytes per shaded texel, the committed
DRAM-traffic record (used only while the shading sources are unchanged), the HBM peak (the
measured file, else the labelled fallback) and the clock-record check that decides whether
a timed region is taken again."""
import json

import pytest

import bench


def test_ssao64_bytes_per_texel():
    # per non-sky texel: depth 4 B + float4 normal 16 B + 64 depth gathers of 4 B + a 4 B
    # store; per sky texel: its depth and the store
    cfg = {"effect": "ssao", "samples": 64}
    assert bench.algorithmic_bytes(cfg, 1, 0) == 280
    assert bench.algorithmic_bytes(cfg, 0, 1) == 8
    # binary16 storage: half4 normals (8 B) and a 2 B store; depth stays FP32
    assert bench.algorithmic_bytes(dict(cfg, precision="fp16"), 1, 0) == 4 + 8 + 256 + 2
    assert bench.algorithmic_bytes(dict(cfg, precision="fp16"), 0, 1) == 6


def test_ssao64_1080p_scene0_total():
    # scene 0 of the 1920x1080 SSAO-64 workload: 308,846 non-sky and 21,360 sky texels
    # in its level lists give 86,647,760 algorithmic bytes per shading launch
    assert bench.algorithmic_bytes({"effect": "ssao", "samples": 64}, 308846, 21360) == 86647760


def test_ssgi_and_ssm_bytes_per_texel():
    # SSGI-32: each sample gathers depth, normal and binary16 direct light (8 B); the
    # sub-image stores float4 (FP32) or half4 (binary16)
    gi = {"effect": "ssgi", "samples": 32}
    assert bench.algorithmic_bytes(gi, 1, 0) == 4 + 16 + 32 * (4 + 16 + 8) + 16
    assert bench.algorithmic_bytes(dict(gi, precision="fp16"), 1, 0) == 4 + 8 + 32 * (4 + 8 + 8) + 8
    # soft shadows: the receiver's depth, every blocker and PCF tap of the FP32 shadow map
    sm = {"effect": "ssm", "blocker_samples": 32, "pcf_samples": 64}
    assert bench.algorithmic_bytes(sm, 1, 0) == 4 + 96 * 4 + 4
    assert bench.algorithmic_bytes(dict(sm, precision="fp16"), 1, 0) == 4 + 96 * 4 + 2


def test_traffic_record_only_for_unchanged_sources(monkeypatch):
    with open(bench.os.path.join(bench.ROOT, "profiles", "traffic_ssao64_4k.json")) as f:
        rec = json.load(f)
    monkeypatch.setattr(bench, "shade_sources_sha", lambda: rec["sources_sha"])
    assert bench.measured_traffic("ssao64_4k") == rec["dram_bytes_per_launch"]
    monkeypatch.setattr(bench, "shade_sources_sha", lambda: "0" * 16)
    assert bench.measured_traffic("ssao64_4k") is None
    assert bench.measured_traffic("no_such_workload") is None


def test_traffic_record_is_per_launch_mean():
    with open(bench.os.path.join(bench.ROOT, "profiles", "traffic_ssao64_4k.json")) as f:
        rec = json.load(f)
    per = [r + w for r, w in zip(rec["dram_read_bytes"], rec["dram_write_bytes"])]
    assert rec["dram_bytes_per_launch"] == pytest.approx(sum(per) / len(per), abs=1)


def test_peak_is_measured_file_else_labelled_fallback(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6793.1, "bf16_tflops": 1900.0}))
    assert bench.measured_peaks() == (6793.1, "measured")


def test_clock_records_rejected_as_the_timing_rules_say():
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 8}
    assert not bench.clocks_rejected(ok)
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_rejected(dict(ok, reasons=[r]))
    # the power cap alone is kept, even with lower clocks
    assert not bench.clocks_rejected(dict(ok, sm_mhz=1650.0, reasons=["sw_power_cap"]))
    # clocks stuck well below the maximum with no reason: a leftover clock lock
    assert bench.clocks_rejected(dict(ok, sm_mhz=1400.0))
    assert not bench.clocks_rejected(dict(ok, sm_mhz=1980.0))
    # no clock record at all (no nvidia-smi): nothing to reject on
    assert not bench.clocks_rejected({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                                      "samples": 0})
