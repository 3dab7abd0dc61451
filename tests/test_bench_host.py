"""Host logic of bench.py: the measured DRAM traffic is reported only for the
kernel sources and the tuning it was captured with."""
import os
import shutil

import bench

KEY = ("k_seg_pivots/vertex", 24, 3)


def _copy_sources(tmp_path):
    entry = bench.MEASURED_TRAFFIC[KEY]
    for rel in entry["sources"]:
        dst = tmp_path / rel
        os.makedirs(dst.parent, exist_ok=True)
        shutil.copyfile(os.path.join(bench.ROOT, rel), dst)
    return entry


def test_traffic_needs_the_captured_tuning(tmp_path, monkeypatch):
    entry = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic(*KEY, dict(entry["tuning"])) == entry["bytes"]
    other = dict(entry["tuning"], seg_long=entry["tuning"]["seg_long"] * 2)
    assert bench.measured_traffic(*KEY, other) is None
    assert bench.measured_traffic(*KEY, None) is None
    assert bench.measured_traffic("k_cta_pivots/vertex", 24, 3, dict(entry["tuning"])) is None
    assert bench.measured_traffic(KEY[0], 22, 3, dict(entry["tuning"])) is None


def test_traffic_is_dropped_when_a_kernel_source_changes(tmp_path, monkeypatch):
    entry = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rel = next(iter(entry["sources"]))
    with open(tmp_path / rel, "ab") as f:
        f.write(b"\n")
    assert bench.measured_traffic(*KEY, dict(entry["tuning"])) is None
