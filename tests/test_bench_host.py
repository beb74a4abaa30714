"""bench.py's host-side arithmetic: the algorithmic bytes of one launch (the numerator of the
roofline's achieved bandwidth) and the lookup of the committed ncu traffic, which applies only
to the kernel sources, workload and storage type it was captured on. CPU only."""

import json

import bench

PAPER = {"w": 1280, "h": 384, "d": 128}
N = 1280 * 384 * 128


def test_algorithmic_bytes_of_the_paper_workload():
    assert N == 62_914_560
    assert bench.algorithmic_bytes("dt_hpair", PAPER, 4) == 503_316_480       # F32 read + write
    assert bench.algorithmic_bytes("dt_vpair", PAPER, 2) == 2 * 2 * N          # F16 read + write
    assert bench.algorithmic_bytes("dt_vpair_wta", PAPER, 4) == 4 * N          # read only
    assert bench.algorithmic_bytes("zncc_cost_hpair", PAPER, 1) == N           # FastDT codes written
    assert bench.algorithmic_bytes("zncc_cost_wta", PAPER, 4) == 4 * 1280 * 384   # images in, map out
    assert bench.algorithmic_bytes("wta_finish", PAPER, 4) is None


def test_traffic_applies_only_to_its_own_sources_workload_and_storage(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    f = tmp_path / "profiles" / "ncu_traffic.json"
    f.write_text(json.dumps({"workload_key": "paper_1280x384", "storage": "f32", "source_digest": "abc",
                             "kernels": {"dt_hpair": {"bytes_per_launch": 482_000_000}}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic("dt_hpair", "abc", "paper_1280x384", "f32") == 482_000_000
    assert bench.load_traffic("dt_hpair", "abd", "paper_1280x384", "f32") is None    # sources changed
    assert bench.load_traffic("dt_hpair", "abc", "plain_320x96", "f32") is None      # other workload
    assert bench.load_traffic("dt_hpair", "abc", "paper_1280x384", "f16") is None    # other storage
    assert bench.load_traffic("dt_vpair", "abc", "paper_1280x384", "f32") is None    # not captured
    f.write_text("{not json")
    assert bench.load_traffic("dt_hpair", "abc", "paper_1280x384", "f32") is None
    f.unlink()
    assert bench.load_traffic("dt_hpair", "abc", "paper_1280x384", "f32") is None
