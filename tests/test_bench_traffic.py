"""bench.py's DRAM-traffic record: a capture taken on a smaller launch is
scaled by the entries of A streamed, and is dropped once the kernel's sources
differ from the ones the counters were taken on."""

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _write(tmp_path, entry):
    (tmp_path / "profiles").mkdir(exist_ok=True)
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"tc_apass_kernel": entry}))


def test_traffic_scales_with_the_streamed_entries(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _write(tmp_path, {"source_digest": bench.kernel_digest("tc_apass_kernel"),
                      "dram_bytes_per_launch": 1000, "captured_elements": 10})
    assert bench._traffic_for("tc_apass_kernel", 40) == 4000


def test_traffic_is_dropped_for_other_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _write(tmp_path, {"source_digest": "0" * 64, "dram_bytes_per_launch": 1000, "captured_elements": 10})
    assert bench._traffic_for("tc_apass_kernel", 40) is None


def test_missing_record_gives_no_traffic(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic_for("tc_apass_kernel", 40) is None

