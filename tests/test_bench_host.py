"""Host-side logic of bench.py that needs no GPU: a kernel's ncu counters are used only
while the walk source they were captured on is unchanged; the issue roofline scales
them to the launch; the roofline peak comes from
the measured-peaks file or the stated fallback; the clock sampler cleans up after
itself when nvidia-smi is missing."""
import hashlib
import json
import os

import bench


def _fake_root(tmp_path, src_text, sha=None):
    src = tmp_path / "paper_1902_08083_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "walk.cu").write_text(src_text)
    prof = tmp_path / "profiles"
    prof.mkdir()
    digest = sha or hashlib.sha256(src_text.encode()).hexdigest()
    (prof / "walk_warp_kernel_issue.json").write_text(json.dumps({
        "source": "paper_1902_08083_gb300/csrc/walk.cu", "source_sha256": digest,
        "sinks": 1000, "warp_inst_issued": 4.0e6, "thread_inst_executed": 9.6e7,
        "cells_tested": 300000, "cells_clipped": 600000, "dram_bytes_per_sink": 80.5}))
    return tmp_path


def test_counters_only_for_the_captured_source(tmp_path, monkeypatch):
    root = _fake_root(tmp_path, "kernel v1\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench._kernel_profile("walk_warp_kernel_issue.json")["dram_bytes_per_sink"] == 80.5
    (root / "paper_1902_08083_gb300" / "csrc" / "walk.cu").write_text("kernel v2\n")
    assert bench._kernel_profile("walk_warp_kernel_issue.json") is None


def test_counters_missing_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._kernel_profile("walk_warp_kernel_issue.json") is None


def test_issue_roofline_arithmetic(tmp_path, monkeypatch):
    root = _fake_root(tmp_path, "kernel v1\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    prof = bench._kernel_profile("walk_warp_kernel_issue.json")
    # 4000 warp instructions per sink, 2000 sinks in 10 ms: 0.8 G/s; peak 4 x 2 x 1000 MHz
    r = bench._issue_roofline(prof, 2000, 0.01, 1000.0, 2, 6.4e9, 6400.0, "measured", "k")
    assert r["bound"] == "issue" and abs(r["achieved"] - 0.8) < 1e-12
    assert abs(r["peak"] - 8.0) < 1e-12 and abs(r["frac"] - 0.1) < 1e-12
    assert abs(r["traffic"] - 80.5 * 2000) < 1e-9
    assert abs(r["thread_instructions_per_cell_step"] - 9.6e7 / 9e5) < 1e-9
    assert abs(r["logical_bytes"]["frac"] - 0.1) < 1e-12
    stale = bench._issue_roofline(None, 2000, 0.01, 1000.0, 2, 6.4e6, 6400.0, "m", "k")
    assert stale["achieved"] is None and stale["traffic"] is None


def test_peaks_measured_or_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6759.6}))
    assert bench._peaks() == (6759.6, "measured")


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))  # no nvidia-smi on the path
    c = bench.Clocks(0, str(tmp_path / "keep"))
    c.start()
    r = c.stop()
    assert r["sm_mhz"] is None and r["reasons"]
    assert not os.path.exists(c.path)
