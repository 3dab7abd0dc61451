"""Host logic of bench.py: a measured DRAM traffic figure is reported only for
the kernel sources and the tuning it was captured with (checked here on
stand-in source files, so the test does not depend on the real kernels)."""
import hashlib

import bench

KEY = ("k_seg_pivots/vertex", 24, 3)
TUNING = {"cta_max_outdeg": 512, "seg_long": 128}


def _entry(tmp_path, monkeypatch):
    sources = {}
    for rel, text in (("src/a.cu", b"kernel a\n"), ("src/b.cuh", b"header b\n")):
        path = tmp_path / rel
        path.parent.mkdir(parents=True, exist_ok=True)
        path.write_bytes(text)
        sources[rel] = hashlib.sha256(text).hexdigest()
    entry = {"bytes": 123456789, "sources": sources, "tuning": dict(TUNING)}
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", {KEY: entry})
    return entry


def test_traffic_needs_the_captured_tuning(tmp_path, monkeypatch):
    entry = _entry(tmp_path, monkeypatch)
    assert bench.measured_traffic(*KEY, dict(TUNING)) == entry["bytes"]
    assert bench.measured_traffic(*KEY, dict(TUNING, seg_long=256)) is None
    assert bench.measured_traffic(*KEY, None) is None
    assert bench.measured_traffic("k_cta_pivots/vertex", 24, 3, dict(TUNING)) is None
    assert bench.measured_traffic(KEY[0], 22, 3, dict(TUNING)) is None


def test_traffic_is_dropped_when_a_kernel_source_changes(tmp_path, monkeypatch):
    _entry(tmp_path, monkeypatch)
    with open(tmp_path / "src/a.cu", "ab") as f:
        f.write(b"\n")
    assert bench.measured_traffic(*KEY, dict(TUNING)) is None


def test_recorded_entry_names_existing_sources():
    for (kernel, scale, seed), e in bench.MEASURED_TRAFFIC.items():
        assert e["bytes"] > 0 and e["tuning"]
        for rel in e["sources"]:
            assert (bench.os.path.exists(bench.os.path.join(bench.ROOT, rel))), rel


def test_recorded_tuning_has_every_tuning_field():
    """A recorded entry can only match the tuning the autotuner returns when
    it names exactly the library's tuning fields."""
    from paper_2006_11494_gb300 import Tuning
    fields = {name for name, _ in Tuning._fields_}
    for e in bench.MEASURED_TRAFFIC.values():
        assert set(e["tuning"]) == fields
