"""Host logic of bench.py that needs no GPU: the committed DRAM-traffic figure of the
dominant kernel is reported only while the capture matches the kernel's sources and the
workload, and the roofline object names the dominant stage's kernel."""
import json
import sys
import types
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))

import bench  # noqa: E402

WORKLOAD = "a test workload"


def _write(path, sha, workload, traffic=123456.0):
    path.write_text(json.dumps({"k_render_bwd": {"workload": workload, "traffic_bytes_per_launch": traffic,
                                                 "source_sha256": sha}}))


def test_recorded_traffic_follows_the_sources_and_the_workload(tmp_path, monkeypatch):
    f = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", f)
    assert bench.recorded_traffic(WORKLOAD) is None                    # no capture on record
    _write(f, bench.raster_bwd_source_hash(), WORKLOAD)
    assert bench.recorded_traffic(WORKLOAD) == 123456.0                # same sources, same workload
    assert bench.recorded_traffic("another workload") is None          # taken on another workload
    _write(f, "0" * 64, WORKLOAD)
    assert bench.recorded_traffic(WORKLOAD) is None                    # the kernel changed since


def test_source_hash_covers_the_backward_kernel_sources():
    h = bench.raster_bwd_source_hash()
    assert len(h) == 64 and int(h, 16) >= 0
    for f in bench.RASTER_BWD_SOURCES:
        assert (ROOT / "paper_2410_00486_gb300" / "csrc" / f).is_file()


def test_roofline_reports_traffic_only_for_the_raster_backward(tmp_path, monkeypatch):
    f = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", f)
    _write(f, bench.raster_bwd_source_hash(), WORKLOAD, traffic=9.0e8)
    pk = types.SimpleNamespace(alu_source="alu peak", hbm_source="hbm peak")
    alu = {"bound": "alu", "achieved": 30.0, "peak": 40.0, "unit": "Top/s", "frac": 0.75}
    hbm = {"bound": "hbm", "achieved": 600.0, "peak": 6800.0, "unit": "GB/s", "frac": 600.0 / 6800.0}
    work = {"workload": WORKLOAD, "pairs_fwd_eval": 1.0, "pairs_bwd_eval": 2.0, "pairs_blend": 3.0}
    roofs = {"raster_bwd": alu, "render_fwd": dict(alu, frac=0.6), "bin_sort": hbm}
    r = bench.roofline({"raster_bwd": 3.2, "render_fwd": 1.6, "bin_sort": 0.7}, work, pk, roofs)
    assert r["kernel"] == "k_render_bwd" and r["bound"] == "alu" and r["frac"] == 0.75
    assert r["traffic"] == 9.0e8 and r["peak_source"] == "alu peak"
    assert r["work"] == {"pairs_fwd_eval": 1.0, "pairs_bwd_eval": 2.0, "pairs_blend": 3.0}
    r = bench.roofline({"raster_bwd": 0.1, "render_fwd": 0.1, "bin_sort": 0.7}, work, pk, roofs)
    assert r["kernel"] == "bin_sort" and r["bound"] == "hbm" and r["traffic"] is None
    assert r["peak_source"] == "hbm peak"
