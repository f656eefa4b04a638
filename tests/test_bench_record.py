"""The ncu traffic record bench.py reports as roofline.traffic: used only for
the workload it was taken on and only while the kernel's sources are the ones
it was taken with."""
import hashlib
import json
import os
import shutil

import bench

SOURCES = ["paper_1109_6885_gb300/csrc/dm_reencode.cu", "include/dmerge.h"]
NAME = "reencode_kernel_column-100M-u64-zipf1-delta1M.traffic.json"


def _tree(tmp_path, read=1000, write=500):
    h = hashlib.sha256()
    for f in SOURCES:
        dst = tmp_path / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, f), dst)
        h.update(open(dst, "rb").read())
    (tmp_path / "profiles").mkdir()
    rec = {"reencode_kernel": {"workload": "column-100M-u64-zipf1-delta1M", "dram_bytes_read": read,
                               "dram_bytes_write": write, "sources": SOURCES,
                               "sources_sha256": h.hexdigest()}}
    json.dump(rec, open(tmp_path / "profiles" / NAME, "w"))


def test_record_matches_its_sources(monkeypatch, tmp_path):
    _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("reencode_kernel", "column-100M-u64-zipf1-delta1M") == 1500
    # another workload has no record
    assert bench.recorded_traffic("reencode_kernel", "column-40M-u64-zipf1-delta400k") is None


def test_record_is_dropped_when_a_source_changes(monkeypatch, tmp_path):
    _tree(tmp_path)
    with open(tmp_path / SOURCES[0], "a") as f:
        f.write("\n// changed\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("reencode_kernel", "column-100M-u64-zipf1-delta1M") is None


def test_committed_record_is_well_formed():
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", NAME)))["reencode_kernel"]
    assert rec["workload"] == "column-100M-u64-zipf1-delta1M"
    assert rec["dram_bytes_read"] > 0 and rec["dram_bytes_write"] > 0
    assert all(os.path.exists(os.path.join(bench.ROOT, f)) for f in rec["sources"])
