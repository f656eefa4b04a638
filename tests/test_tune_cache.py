"""The autotuner's cache through the C ABI, on the host (no GPU needed):
column classes, entries, validation, and the JSON file it persists to."""
import json

import pytest

from paper_1109_6885_gb300 import build as cuda_build
from paper_1109_6885_gb300 import dmerge as dm


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return dm.load()


def col(w=8, m=0, bits=0, n_main=0, d=0, n_delta=0):
    return dm.ColumnIn(w, None, m, None, bits, n_main, None, d, None, n_delta)


def ceil_log2(n):
    return 0 if n <= 1 else (n - 1).bit_length()


def choice(**kw):
    c = dm.TuneChoice()
    for k, v in kw.items():
        setattr(c, k, v)
    return c


@pytest.mark.parametrize("w,m,bits,n_main,d,n_delta", [
    (8, 1_000_000, 20, 100_000_000, 300_000, 1_000_000),
    (16, 100_000, 17, 1_000_000, 9_900, 10_000),
    (4, 0, 0, 0, 5, 7),
    (8, 1, 0, 12, 0, 0),
    (8, 2, 1, 2**20, 2**20 - 1, 2**20 + 1),
    (4, 2**32 - 5, 32, 2**33, 4, 1),
])
def test_key_is_widths_and_bit_lengths(lib, w, m, bits, n_main, d, n_delta):
    k = dm.dm_tune_key_of(col(w, m, bits, n_main, d, n_delta))
    assert k.as_tuple() == (w, bits, ceil_log2(m + d), m.bit_length(), d.bit_length(),
                            n_main.bit_length(), n_delta.bit_length())


def test_same_class_same_key(lib):
    # sizes within one power of two share a class; crossing one does not
    a = dm.dm_tune_key_of(col(8, 600_000, 20, 70_000_000, 1000, 700_000))
    b = dm.dm_tune_key_of(col(8, 700_000, 20, 100_000_000, 1023, 1_000_000))
    c = dm.dm_tune_key_of(col(8, 700_000, 20, 100_000_000, 1024, 1_000_000))
    assert a.as_tuple() == b.as_tuple()
    assert a.as_tuple() != c.as_tuple()


def test_put_get_clear(lib):
    cache = dm.TuneCache()
    k1 = dm.dm_tune_key_of(col(8, 1000, 10, 5000, 10, 20))
    k2 = dm.dm_tune_key_of(col(16, 1000, 10, 5000, 10, 20))
    assert len(cache) == 0 and cache.get(k1) is None
    g0 = cache.generation
    cache.put(k1, choice(reencode_warps=8, reencode_stages=3, x_staging=dm.DM_STAGE_GLOBAL))
    assert len(cache) == 1 and cache.generation > g0
    got = cache.get(k1)
    assert got.as_dict() == {"reencode_warps": 8, "reencode_stages": 3, "reencode_obufs": 0,
                             "x_staging": dm.DM_STAGE_GLOBAL, "x8": 0, "step1_blocks": 0}
    assert cache.get(k2) is None
    cache.put(k1, choice(reencode_obufs=2))   # replaces
    assert len(cache) == 1 and cache.get(k1).reencode_obufs == 2 and cache.get(k1).reencode_warps == 0
    cache.put(k2, choice(step1_blocks=38, x8=dm.DM_X8_OFF))
    assert len(cache) == 2
    g1 = cache.generation
    cache.clear()
    assert len(cache) == 0 and cache.generation > g1 and cache.get(k2) is None


@pytest.mark.parametrize("bad", [
    {"reencode_warps": 17}, {"reencode_stages": 1}, {"reencode_stages": 5}, {"reencode_obufs": 3},
    {"x_staging": 3}, {"x8": 2},
])
def test_out_of_range_choice_is_rejected(lib, bad):
    cache = dm.TuneCache()
    k = dm.dm_tune_key_of(col(8, 10, 4, 100, 1, 1))
    with pytest.raises(dm.DmError) as e:
        cache.put(k, choice(**bad))
    assert e.value.status == dm.DM_EINVAL
    assert len(cache) == 0


def _fill(cache):
    entries = []
    for i, (w, m) in enumerate([(4, 10), (8, 1_000_000), (16, 50_000_000)]):
        k = dm.dm_tune_key_of(col(w, m, ceil_log2(m) + 1, 10 * m, m // 10, m // 100))
        c = choice(reencode_warps=[4, 8, 16][i], reencode_stages=[2, 3, 4][i], reencode_obufs=1 + i % 2,
                   x_staging=i % 3, x8=i % 2, step1_blocks=[0, 152, 38][i])
        cache.put(k, c)
        entries.append((k.as_tuple(), c.as_dict()))
    return entries


def test_save_load_round_trip(lib, tmp_path):
    a = dm.TuneCache()
    entries = _fill(a)
    path = str(tmp_path / "tune.json")
    a.save(path)
    doc = json.load(open(path))   # plain JSON a user can read and edit
    assert doc["format"] == "dmerge-tune-cache" and doc["version"] == 1
    assert len(doc["entries"]) == 3
    b = dm.TuneCache()
    b.load(path)
    assert len(b) == 3
    for kt, cd in entries:
        k = dm.TuneKey(*kt, 0)
        assert b.get(k).as_dict() == cd


def test_load_merges_and_accepts_other_layouts(lib, tmp_path):
    a = dm.TuneCache()
    entries = _fill(a)
    path = str(tmp_path / "tune.json")
    a.save(path)
    doc = json.load(open(path))
    doc["entries"][0]["warps"] = 12
    doc["entries"][0]["some_later_field"] = 7           # ignored
    doc["comment"] = "written by hand"                  # ignored
    open(path, "w").write(json.dumps(doc, indent=4, sort_keys=True))
    b = dm.TuneCache()
    other = dm.dm_tune_key_of(col(8, 77, 7, 770, 7, 7))
    b.put(other, choice(reencode_warps=2))
    b.put(dm.TuneKey(*entries[0][0], 0), choice(reencode_warps=1))
    b.load(path)
    assert len(b) == 4
    assert b.get(other).reencode_warps == 2
    assert b.get(dm.TuneKey(*entries[0][0], 0)).reencode_warps == 12


@pytest.mark.parametrize("mutate", [
    lambda d: d["entries"][1].pop("lnd"),                          # a key field missing
    lambda d: d["entries"][1].update(stages=1),                    # a choice out of range
    lambda d: d["entries"][1].update(warps=-1),                    # not an unsigned integer
    lambda d: d["entries"][1].update(warps=1.5),
    lambda d: d["entries"][1].update(warps=2**32),
    lambda d: d.update(format="something-else"),
    lambda d: d.update(version=2),
    lambda d: d.pop("entries"),
])
def test_malformed_file_changes_nothing(lib, tmp_path, mutate):
    a = dm.TuneCache()
    _fill(a)
    path = str(tmp_path / "tune.json")
    a.save(path)
    doc = json.load(open(path))
    mutate(doc)
    open(path, "w").write(json.dumps(doc))
    b = dm.TuneCache()
    k = dm.dm_tune_key_of(col(8, 5, 3, 50, 1, 1))
    b.put(k, choice(reencode_warps=4))
    g = b.generation
    with pytest.raises(dm.DmError) as e:
        b.load(path)
    assert e.value.status == dm.DM_EINVAL
    assert len(b) == 1 and b.generation == g and b.get(k).reencode_warps == 4


@pytest.mark.parametrize("text", ["", "{", "[]", '{"format": "dmerge-tune-cache", "entries": []} x',
                                  '{"format": "dmerge-tune-cache", "entries": [{]}'])
def test_truncated_or_trailing_text_is_rejected(lib, tmp_path, text):
    path = str(tmp_path / "t.json")
    open(path, "w").write(text)
    with pytest.raises(dm.DmError) as e:
        dm.TuneCache().load(path)
    assert e.value.status == dm.DM_EINVAL


def test_empty_cache_file_and_missing_file(lib, tmp_path):
    path = str(tmp_path / "empty.json")
    dm.TuneCache().save(path)
    b = dm.TuneCache()
    b.load(path)
    assert len(b) == 0
    with pytest.raises(dm.DmError) as e:
        b.load(str(tmp_path / "absent.json"))
    assert e.value.status == dm.DM_ENOENT
