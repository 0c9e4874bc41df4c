"""Host logic of the benchmark (no GPU): the ncu record of the tile kernel's
DRAM traffic and instructions per hit holds only for the kernel source it
was taken on."""
import json

import bench


def test_traffic_record_matches_the_kernel_source():
    tf = bench._traffic_record()
    assert tf is not None, "profiles/k_tile_traffic.json was taken on another version of the kernel source"
    assert tf["source_hash"] == bench._tile_source_hash()
    for leg in ("batched", "scaled"):
        assert 16.0 <= tf["bytes_per_hit"][leg] < 32.0      # the hits and their halos, read once
        assert tf["warp_inst_per_hit"][leg] > 0
        assert set(tf["shapes"][leg]) == {"cap", "warps", "fill_pct"}


def test_traffic_record_is_dropped_for_another_source(monkeypatch):
    monkeypatch.setattr(bench, "_tile_source_hash", lambda: "0" * 16)
    assert bench._traffic_record() is None


def test_traffic_record_is_dropped_when_unreadable(monkeypatch, tmp_path):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k_tile_traffic.json").write_text("{not json")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_tile_source_hash", lambda: "y" * 16)
    assert bench._traffic_record() is None
    (tmp_path / "profiles" / "k_tile_traffic.json").write_text(json.dumps({"source_hash": "x"}))
    assert bench._traffic_record() is None
