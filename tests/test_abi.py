"""The C-ABI library builds, loads, and exports every symbol its header
declares; the host-only helpers answer without a GPU."""
import ctypes
import os
import re

import pytest

from paper_1109_6885_gb300 import build as cuda_build
from paper_1109_6885_gb300 import dmerge as dm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dmerge.h")


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return dm.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dm_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["dm_create", "dm_destroy", "dm_merge_column", "dm_merge_table", "dm_sync_status",
              "dm_packed_bytes", "dm_max_bits", "dm_sort_delta", "dm_merge_dicts", "dm_reencode",
              "dm_merge_column_host"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(cuda_build.LIB)
    for n in declared_functions():
        assert hasattr(raw, n), n
    assert set(declared_functions()) <= set(dm.EXPORTS)


def test_host_helpers(lib):
    assert dm.dm_packed_bytes(0, 17) == 0
    assert dm.dm_packed_bytes(1, 1) == 16
    assert dm.dm_packed_bytes(128, 1) == 16
    assert dm.dm_packed_bytes(129, 1) == 32
    assert dm.dm_packed_bytes(1_000_000, 17) == ((1_000_000 * 17 + 127) // 128) * 16
    for n, b in [(0, 0), (1, 0), (2, 1), (6, 3), (9, 4), (100_000, 17), (2**32, 32)]:
        assert dm.dm_bits_for(n) == b
    cin = dm.ColumnIn(8, None, 1000, None, 10, 0, None, 300, None, 0)
    assert dm.dm_max_bits(cin) == 11
    assert dm.dm_scratch_bytes(cin) > 2 * 300 * 12


def test_status_names(lib):
    assert lib.dm_status_str(dm.DM_ECODE) == b"DM_ECODE"
    assert lib.dm_status_str(dm.DM_OK) == b"DM_OK"


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(cuda_build, "LIB", str(tmp_path / "absent.so"))
    monkeypatch.setattr(dm, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        dm.load()


def test_ingest_scratch_sizes(lib):
    """Ingest scratch: two tables of a power of two of at least 2n slots (4 bytes each),
    one slot index per row, one count per 1024-row tile (256-byte aligned pieces)."""
    r = lambda v: (v + 255) // 256 * 256
    for n in [0, 1, 31, 1024, 1025, 1_000_000, 123_456_789]:
        slots = 64
        while slots < 2 * n:
            slots *= 2
        tiles = (n + 1023) // 1024
        want = 2 * r(slots * 4) + r(n * 4) + r(tiles * 4 + 4)
        for w in (4, 8, 16):
            assert dm.dm_ingest_scratch_bytes(w, n) == want
