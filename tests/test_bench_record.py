"""The ncu traffic record bench.py reports as roofline.traffic: used only for
the workload it was taken on and only while the kernel's sources are the ones
it was taken with."""
import json
import os
import shutil

import bench


def _copy_tree(tmp_path):
    rec_name = "reencode_kernel_column-100M-u64-zipf1-delta1M.traffic.json"
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", rec_name)))
    for f in rec["reencode_kernel"]["sources"]:
        dst = tmp_path / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, f), dst)
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(bench.ROOT, "profiles", rec_name), tmp_path / "profiles" / rec_name)
    return rec["reencode_kernel"]


def test_record_matches_current_sources(monkeypatch, tmp_path):
    rec = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    got = bench.recorded_traffic("reencode_kernel", "column-100M-u64-zipf1-delta1M")
    assert got == rec["dram_bytes_read"] + rec["dram_bytes_write"]
    # another workload has no record
    assert bench.recorded_traffic("reencode_kernel", "column-40M-u64-zipf1-delta400k") is None


def test_record_is_dropped_when_a_source_changes(monkeypatch, tmp_path):
    rec = _copy_tree(tmp_path)
    with open(tmp_path / rec["sources"][0], "a") as f:
        f.write("\n// changed\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("reencode_kernel", "column-100M-u64-zipf1-delta1M") is None
