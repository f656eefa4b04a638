"""The ncu traffic record bench.py reports as roofline.traffic: used only for
the workload it was taken on and only while the kernel's sources are the ones
it was taken with."""
import json
import os
import shutil

import bench

SOURCES = ["paper_1109_6885_gb300/csrc/dm_reencode.cu", "include/dmerge.h"]
NAME = "reencode_kernel_column-100M-u64-zipf1-delta1M.traffic.json"


def _tree(tmp_path, read=1000, write=500):
    for f in SOURCES:
        dst = tmp_path / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, f), dst)
    (tmp_path / "profiles").mkdir()
    rec = {"reencode_kernel": {"workload": "column-100M-u64-zipf1-delta1M", "dram_bytes_read": read,
                               "dram_bytes_write": write, "sources": SOURCES,
                               "sources_sha256": None}}
    root = bench.ROOT
    try:
        bench.ROOT = str(tmp_path)
        rec["reencode_kernel"]["sources_sha256"] = bench.sources_digest(SOURCES)
    finally:
        bench.ROOT = root
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
        f.write("\nstatic int changed_for_the_test;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("reencode_kernel", "column-100M-u64-zipf1-delta1M") is None


def test_record_survives_comment_edits(monkeypatch, tmp_path):
    _tree(tmp_path)
    with open(tmp_path / SOURCES[1], "a") as f:
        f.write("\n/* a new comment */\n// and another one\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("reencode_kernel", "column-100M-u64-zipf1-delta1M") == 1500


def test_strip_comments():
    assert bench.strip_comments("int a;  // x\nint b; /* y\n z */ int c;") == "int a; int b; int c;"
    assert bench.strip_comments('const char* s = "// not a comment"; // a comment') == \
        'const char* s = "// not a comment";'
    assert bench.strip_comments("char q = '\\''; /* c */ x") == "char q = '\\''; x"
    assert bench.strip_comments('asm("mov.u64 %0, %%globaltimer;" : "=l"(t));') == \
        'asm("mov.u64 %0, %%globaltimer;" : "=l"(t));'


def test_committed_record_is_used_only_while_current():
    """The committed record is reported while the kernel's sources are the
    ones it was taken with, and dropped (None) once they change."""
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", NAME)))["reencode_kernel"]
    got = bench.recorded_traffic("reencode_kernel", rec["workload"])
    if bench.sources_digest(rec["sources"]) == rec["sources_sha256"]:
        assert got == rec["dram_bytes_read"] + rec["dram_bytes_write"]
    else:
        assert got is None


def test_committed_record_is_well_formed():
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", NAME)))["reencode_kernel"]
    assert rec["workload"] == "column-100M-u64-zipf1-delta1M"
    assert rec["dram_bytes_read"] > 0 and rec["dram_bytes_write"] > 0
    assert all(os.path.exists(os.path.join(bench.ROOT, f)) for f in rec["sources"])
