"""Host-side logic of bench.py that needs no GPU: the DRAM-traffic file is used only
while the walk source it was captured on is unchanged; the roofline peak comes from
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
    (prof / "walk_warp_kernel_dram.json").write_text(json.dumps({
        "source": "paper_1902_08083_gb300/csrc/walk.cu", "source_sha256": digest,
        "dram_bytes_per_sink": 80.5}))
    return tmp_path


def test_traffic_only_for_the_captured_source(tmp_path, monkeypatch):
    root = _fake_root(tmp_path, "kernel v1\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench._walk_traffic_per_sink() == 80.5
    (root / "paper_1902_08083_gb300" / "csrc" / "walk.cu").write_text("kernel v2\n")
    assert bench._walk_traffic_per_sink() is None


def test_traffic_missing_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._walk_traffic_per_sink() is None


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
