"""The seeded input generator produces what its documentation promises."""
import numpy as np
import pytest

import synth
from tests import _brute


@pytest.mark.parametrize("w", [4, 8, 16])
def test_dictionary_sorted_distinct(w):
    for m in (1, 2, 17, 5000):
        d = synth.dictionary(123, w, m)
        keys = _brute.key_list(d, w)
        assert len(keys) == m
        assert all(a < b for a, b in zip(keys, keys[1:]))


def test_dictionary_dense_4_byte():
    d = synth.dictionary(5, 4, 1_000_000)
    assert np.all(np.diff(d.astype(np.int64)) > 0)


def test_pack_matches_bitwise_definition():
    rng = np.random.default_rng(0)
    for b in range(0, 33):
        n = 97
        top = 2**b
        codes = rng.integers(0, top, n, dtype=np.uint64).astype(np.uint32) if b else \
            np.zeros(n, np.uint32)
        words = synth.pack(codes, b)
        assert np.array_equal(words, _brute.pack_bits(codes.tolist(), b))
        assert words.size % 4 == 0


def test_codes_in_range_and_deterministic():
    a = synth.codes(9, 1000, 100_000, "zipf", 1.0)
    b = synth.codes(9, 1000, 100_000, "zipf", 1.0)
    assert np.array_equal(a, b)
    assert a.max() < 1000
    u = synth.codes(9, 1000, 100_000)
    assert u.max() < 1000 and len(np.unique(u)) == 1000


def test_zipf_rank_frequencies():
    """Sorted frequencies follow (r+1)^-s within sampling noise."""
    m, n, s = 200, 2_000_000, 1.0
    c = synth.codes(11, m, n, "zipf", s)
    freq = np.sort(np.bincount(c, minlength=m))[::-1]
    p = (np.arange(1, m + 1) ** -s)
    p /= p.sum()
    for r in (0, 1, 4, 20):
        assert abs(freq[r] / n - p[r]) < 5 * np.sqrt(p[r] / n) + 1e-4


@pytest.mark.parametrize("w", [4, 8, 16])
def test_delta_partition(w):
    spec = synth.ColumnSpec(n_main=50_000, m=2000, w=w, n_delta=3000, f_new=0.3, seed=4)
    col = synth.make_column(spec)
    um = set(_brute.key_list(col.main_dict, w))
    dd = _brute.key_list(col.delta_dict, w)
    assert len(dd) == len(set(dd))                      # distinct
    assert col.delta_codes.max() < len(dd)
    # first-occurrence order: codes appear for the first time in increasing order
    seen = []
    for c in col.delta_codes.tolist():
        if c not in seen:
            seen.append(c)
    assert seen == list(range(len(dd)))
    new = [v for v in dd if v not in um]
    assert 0 < len(new) <= spec.pool_size()
    fresh_rows = sum(1 for c in col.delta_codes.tolist() if dd[c] not in um)
    assert abs(fresh_rows / spec.n_delta - 0.3) < 0.05


def test_delta_one_new_value_per_fresh_row():
    spec = synth.ColumnSpec(n_main=100_000, m=10_000, w=8, n_delta=1000, f_new=0.5, pool=0, seed=8)
    col = synth.make_column(spec)
    um = set(_brute.key_list(col.main_dict, 8))
    dd = _brute.key_list(col.delta_dict, 8)
    fresh = [c for c in col.delta_codes.tolist() if dd[c] not in um]
    assert len(fresh) == len(set(fresh))                # every fresh row its own value
