"""Pins of the CPU oracle to facts outside itself (no GPU needed).

* the values the paper prints for its worked example (Figures 5/6 prose),
  on a fixture constructed to satisfy them (tests/golden);
* brute force on tiny inputs (tests/_brute.py: bitwise packing, the set of
  Eq. 3, index lookup), exhaustively over small overlap patterns;
* the invariants the paper states or implies (U' sorted and unique, Eq. 2,
  Eq. 3, Eq. 4 minimal width, monotone translation tables, equal values
  share a code, row order kept with the delta appended);
* the unmodified Section 5.2 route (decode then binary search) giving the
  same codes as the Section 5.3 translation-table route;
* special cases: delta contained in the main dictionary with an unchanged
  width leaves the main stream byte-identical.
"""
import itertools
import json
import os
import random

import numpy as np
import pytest

import oracle
import synth
from tests import _brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def ascii_key(s: str) -> int:
    return int.from_bytes(s.encode().ljust(8, b"\0"), "big")


# ---------------------------------------------------------------- worked example

def test_fig5_fig6_constraints():
    fx = json.load(open(os.path.join(GOLDEN, "fig5_fig6_example.json")))
    pr = fx["printed"]
    um = [ascii_key(s) for s in fx["main_dictionary"]]
    assert um == sorted(um)
    main_dict = np.array(um, np.uint64)
    main_codes = [um.index(ascii_key(s)) for s in fx["main_tuples"]]
    dvals = [ascii_key(s) for s in fx["delta_tuples"]]
    ddict = list(dict.fromkeys(dvals))            # first-occurrence order
    dcodes = [ddict.index(v) for v in dvals]
    assert [i for i, s in enumerate(fx["delta_tuples"]) if s == "charlie"] == \
        pr["charlie_delta_positions"]
    b = oracle.new_width(len(um))
    assert b == pr["main_bits"] == 3
    assert len(ddict) == pr["delta_dict_size"]
    assert oracle.new_width(len(ddict)) == pr["delta_bits"] == 2
    assert main_codes[0] == pr["first_main_code_old"] == pr["hotel_old_code"]

    packed = synth.pack(np.array(main_codes, np.uint32), b)
    r = oracle.merge_column(8, main_dict, packed, b, len(main_codes), np.array(ddict, np.uint64),
                            np.array(dcodes, np.uint32))
    assert r.u == pr["merged_size"] == 9
    assert r.new_bits == pr["merged_bits"] == 4
    assert int(r.x_main[4]) == pr["x_main_at_4"] == 6
    new_codes = _brute.unpack_bits(r.new_packed, len(main_codes) + len(dcodes), r.new_bits)
    assert new_codes[0] == pr["first_main_code_new"] == pr["hotel_new_code"]
    hotel = ascii_key("hotel")
    assert int(r.new_dict[pr["hotel_new_code"]]) == hotel
    # every row keeps its value, delta appended after the main rows
    vals = [int(r.new_dict[c]) for c in new_codes]
    assert vals == [ascii_key(s) for s in fx["main_tuples"] + fx["delta_tuples"]]


# ---------------------------------------------------------------- brute force

def run_case(w, um_vals, main_codes, dd_vals, dcodes, b=None):
    um = _brute.key_array(um_vals, w)
    dd = _brute.key_array(dd_vals, w)
    if b is None:
        b = _brute.width(len(um_vals))
    packed = _brute.pack_bits(main_codes, b)
    r = oracle.merge_column(w, um, packed, b, len(main_codes), dd, np.array(dcodes, np.uint32))
    new, xm, xd, codes, bn, words = _brute.merge(w, um, main_codes, dd, dcodes)
    assert _brute.key_list(r.new_dict, w) == new
    assert r.u == len(new)
    assert r.new_bits == bn
    assert r.x_main.tolist() == xm
    assert r.x_delta.tolist() == xd
    assert np.array_equal(r.new_packed, words), (r.new_packed, words)
    return r


def random_keys(rng, n, universe, w):
    top = {4: 2**32, 8: 2**64, 16: 2**128}[w]
    base = rng.randrange(top - universe) if universe < top else 0
    return [base + v for v in rng.sample(range(universe), n)]


@pytest.mark.parametrize("w", [4, 8, 16])
def test_brute_force_random_small(w):
    rng = random.Random(1109 + w)
    for _ in range(300):
        universe = rng.randint(1, 24)
        m = rng.randint(0, min(universe, 10))
        d = rng.randint(0, min(universe, 10))
        pool = random_keys(rng, universe, universe, w)
        um = sorted(rng.sample(pool, m))
        dd = rng.sample(pool, d)                       # insertion order
        n_main = rng.randint(0, 70) if m else 0
        n_delta = rng.randint(0, 40) if d else 0
        mc = [rng.randrange(m) for _ in range(n_main)]
        dc = [rng.randrange(d) for _ in range(n_delta)]
        b = _brute.width(m) + rng.choice([0, 0, 1, 3])
        run_case(w, um, mc, dd, dc, min(b, 32))


def test_brute_force_exhaustive_overlaps():
    """Every main subset x every ordered delta subset of a 4-value universe."""
    universe = [10, 20, 30, 40]
    for w in (4, 16):
        for k in range(5):
            for um in itertools.combinations(universe, k):
                for j in range(5):
                    for dd in itertools.permutations(universe, j):
                        mc = [i % k for i in range(7)] if k else []
                        dc = [i % j for i in range(5)][::-1] if j else []
                        run_case(w, list(um), mc, list(dd), dc)


def test_duplicates_inside_delta_dict():
    """Duplicate delta dictionary entries all take the value's single code."""
    r = run_case(8, [5, 9], [0, 1, 1], [7, 9, 7, 7, 3], [0, 1, 2, 3, 4, 2])
    assert r.x_delta.tolist() == [2, 3, 2, 2, 0]


def test_extreme_keys_and_equal_hi_words():
    top64 = 2**64 - 1
    run_case(8, [0, top64], [1, 0, 1], [top64, 0, 5], [0, 1, 2])
    run_case(4, [0, 2**32 - 1], [1, 0], [2**32 - 1, 7], [1, 0])
    hi = 0xDEADBEEF << 64
    run_case(16, [hi | 1, hi | 5, hi | top64], [2, 0, 1], [hi | 3, hi | 0, (1 << 64) | 9, hi | 5],
             [0, 1, 2, 3, 0])
    run_case(16, [0, 2**128 - 1], [0, 1], [2**127, 2**64 - 1], [0, 1])


@pytest.mark.parametrize("b_new", range(0, 33))
def test_reencode_every_width_pair(b_new):
    """Step 2(b) packing at every (b, b') pair against bitwise brute force."""
    rng = random.Random(b_new)
    for b in range(0, 33):
        m = min(2**b, 7) if b else 1
        n_main, n_delta, d = 67, 13, 3
        mc = [rng.randrange(m) for _ in range(n_main)]
        dc = [rng.randrange(d) for _ in range(n_delta)]
        top = 2**b_new
        xm = [rng.randrange(top) for _ in range(m)]
        xd = [rng.randrange(top) for _ in range(d)]
        packed = _brute.pack_bits(mc, b)
        out = oracle.reencode(packed, b, n_main, np.array(dc, np.uint32), np.array(xm, np.uint32),
                              np.array(xd, np.uint32), b_new)
        want = _brute.pack_bits([xm[c] for c in mc] + [xd[c] for c in dc], b_new)
        assert np.array_equal(out, want), (b, b_new)


# ---------------------------------------------------------------- invariants

def check_invariants(col, r):
    w = col.w
    new = _brute.key_list(r.new_dict, w)
    um = _brute.key_list(col.main_dict, w)
    dd = _brute.key_list(col.delta_dict, w)
    # U' strictly increasing; |U'| = |D u U_M| (Eq. 3)
    assert all(a < b for a, b in zip(new, new[1:]))
    assert len(new) == len(set(um) | set(dd))
    # Eq. 4: minimal width
    assert r.new_bits == _brute.width(len(new))
    assert r.u <= 1 or 2 ** (r.new_bits - 1) < r.u <= 2 ** r.new_bits
    # X_M strictly increasing in the main code; values land where they belong
    xm = r.x_main.astype(np.int64)
    assert np.all(np.diff(xm) > 0)
    assert all(new[x] == v for x, v in zip(r.x_main.tolist(), um))
    assert all(new[x] == v for x, v in zip(r.x_delta.tolist(), dd))
    # X_D follows value order of the delta dictionary
    order = sorted(range(len(dd)), key=lambda k: (dd[k], k))
    xs = [int(r.x_delta[k]) for k in order]
    assert all(a <= b for a, b in zip(xs, xs[1:]))


def decode_identity(col, r):
    """decode(new) == decode(main) ++ decode(delta) (Eq. 2 row count, order kept)."""
    n = col.n_main + col.n_delta
    new_codes = np.array(_brute.unpack_bits(r.new_packed, n, r.new_bits), np.int64)
    main_codes = np.array(_brute.unpack_bits(col.main_packed, col.n_main, col.main_bits), np.int64)
    assert np.array_equal(main_codes, col.main_codes.astype(np.int64))
    if col.w == 16:
        got = r.new_dict[new_codes]
        want = np.concatenate([col.main_dict[main_codes], col.delta_dict[col.delta_codes]])
    else:
        got = r.new_dict[new_codes]
        want = np.concatenate([col.main_dict[main_codes], col.delta_dict[col.delta_codes]])
    assert np.array_equal(got, want)


@pytest.mark.parametrize("w", [4, 8, 16])
@pytest.mark.parametrize("dist", ["uniform", "zipf"])
def test_invariants_and_decode_identity_synth(w, dist):
    spec = synth.ColumnSpec(n_main=3000, m=300, w=w, n_delta=400, f_new=0.4, dist=dist,
                            zipf_s=0.9, seed=77 + w)
    col = synth.make_column(spec)
    r = oracle.merge_synth_column(col)
    check_invariants(col, r)
    decode_identity(col, r)


@pytest.mark.parametrize("w", [4, 8, 16])
def test_naive_route_equals_translation_tables(w):
    """Section 5.2 (binary search, Eq. 5) and Section 5.3 (X tables, Eq. 11) agree."""
    spec = synth.ColumnSpec(n_main=200_000, m=20_000, w=w, n_delta=5000, f_new=0.3,
                            dist="zipf", zipf_s=1.0, seed=5 + w, pool=0)
    col = synth.make_column(spec)
    r = oracle.merge_synth_column(col)
    naive = oracle.naive_reencode(w, col.main_dict, col.main_packed, col.main_bits, col.n_main,
                                  col.delta_dict, col.delta_codes, r.new_dict, r.new_bits)
    assert np.array_equal(naive, r.new_packed)


def test_delta_subset_of_main_keeps_main_stream():
    """D within U_M and b' = b: X_M is the identity and the main bits are unchanged."""
    spec = synth.ColumnSpec(n_main=10_000, m=1000, w=8, n_delta=500, f_new=0.0, seed=3)
    col = synth.make_column(spec)
    r = oracle.merge_synth_column(col)
    assert r.u == 1000 and r.new_bits == col.main_bits
    assert np.array_equal(r.x_main, np.arange(1000, dtype=np.uint32))
    nbits = col.n_main * col.main_bits
    full = nbits // 32
    assert np.array_equal(r.new_packed[:full], col.main_packed[:full])


def test_width_closed_form():
    # Section 4.1: 6 values -> 3 bits, 9 values -> 4 bits; 100,000 -> 17; 1,000,000 -> 20
    for u, b in [(6, 3), (9, 4), (100_000, 17), (1_000_000, 20), (0, 0), (1, 0), (2, 1),
                 (3, 2), (4, 2), (5, 3), (2**32, 32), (2**32 - 1, 32), (2**31 + 1, 32)]:
        assert oracle.new_width(u) == b, u
    for k in range(1, 33):
        assert oracle.new_width(2**k) == k
        assert oracle.new_width(2**k + 1) == k + 1


def test_sort_delta_is_stable_and_sorted():
    dd = np.array([9, 3, 9, 1, 3, 3], np.uint64)
    ud, perm = oracle.sort_delta(8, dd)
    assert ud.tolist() == [1, 3, 3, 3, 9, 9]
    assert perm.tolist() == [3, 1, 4, 5, 0, 2]


def test_empty_and_degenerate():
    run_case(8, [], [], [], [])                      # nothing at all
    run_case(8, [], [], [4, 2], [1, 1, 0])           # empty main
    run_case(8, [4], [0, 0, 0], [], [])              # empty delta, u = 1 -> 0 bits
    run_case(8, [4], [0] * 40, [4], [0] * 9)         # u = 1 with both parts
    r = run_case(4, [1, 2], [1, 0] * 20, [3, 4, 5], [2, 1, 0])  # 2 -> 5 values, 1 -> 3 bits
    assert r.new_bits == 3


def test_validation_errors():
    um = np.array([1, 5, 9], np.uint64)
    good = synth.pack(np.array([0, 1, 2, 1], np.uint32), 2)
    dd = np.array([7], np.uint64)
    dc = np.array([0, 0], np.uint32)
    with pytest.raises(oracle.OracleError) as e:
        oracle.merge_column(8, np.array([1, 9, 5], np.uint64), good, 2, 4, dd, dc)
    assert e.value.code == oracle.UNSORTED
    with pytest.raises(oracle.OracleError) as e:
        oracle.merge_column(8, np.array([1, 5, 5], np.uint64), good, 2, 4, dd, dc)
    assert e.value.code == oracle.UNSORTED
    bad = synth.pack(np.array([0, 3, 2, 1], np.uint32), 2)
    with pytest.raises(oracle.OracleError) as e:
        oracle.merge_column(8, um, bad, 2, 4, dd, dc)
    assert e.value.code == oracle.BAD_CODE
    with pytest.raises(oracle.OracleError) as e:
        oracle.merge_column(8, um, good, 2, 4, dd, np.array([0, 1], np.uint32))
    assert e.value.code == oracle.BAD_CODE
    with pytest.raises(oracle.OracleError) as e:
        oracle.merge_column(8, um, synth.pack(np.array([0, 1, 0, 1], np.uint32), 1), 1, 4, dd, dc)
    assert e.value.code == oracle.BAD_ARG


# ---------------------------------------------------------------- delta ingest (Section 4)

def test_ingest_fig5_delta():
    """Figure 5's delta: five tuples, 'charlie' at positions 1 and 3, four distinct values
    (the Figure 6 prose), coded in order of first arrival."""
    fx = json.load(open(os.path.join(GOLDEN, "fig5_fig6_example.json")))
    vals = np.array([ascii_key(s) for s in fx["delta_tuples"]], np.uint64)
    dd, codes = oracle.ingest_delta(8, vals)
    assert dd.shape[0] == fx["printed"]["delta_dict_size"] == 4
    p = fx["printed"]["charlie_delta_positions"]
    assert codes[p[0]] == codes[p[1]]
    assert list(codes) == [0, 1, 2, 1, 3]
    assert [int(x) for x in dd] == [ascii_key(s) for s in ["zulu", "charlie", "bravo", "echo"]]


def _ingest_brute(values):
    """The definition restated: scan left to right, a value not seen before takes the next code."""
    first, codes = [], []
    for v in values:
        if v not in first:
            first.append(v)
        codes.append(first.index(v))
    return first, codes


@pytest.mark.parametrize("w", [4, 8, 16])
@pytest.mark.parametrize("seed", range(6))
def test_ingest_brute_force(w, seed):
    rng = random.Random(seed * 31 + w)
    n = rng.randint(0, 60)
    pool = [rng.getrandbits(8 * w) for _ in range(rng.randint(1, 12))]
    vals = [rng.choice(pool) for _ in range(n)]
    if w == 16:
        arr = np.array([[v >> 64, v & (2**64 - 1)] for v in vals], np.uint64).reshape(-1, 2)
    else:
        arr = np.array(vals, np.uint32 if w == 4 else np.uint64)
    dd, codes = oracle.ingest_delta(w, arr)
    first, want = _ingest_brute(vals)
    got_dd = [(int(r[0]) << 64) | int(r[1]) for r in dd] if w == 16 else [int(x) for x in dd]
    assert got_dd == first
    assert [int(c) for c in codes] == want


@pytest.mark.parametrize("w", [4, 8, 16])
def test_ingest_invariants(w):
    """On a larger Zipf-shaped column: decoding gives the values back, the dictionary is
    duplicate-free, and the first occurrences of the codes come in order 0, 1, 2, ..."""
    col = synth.make_column(synth.ColumnSpec(n_main=10_000, m=5_000, w=w, n_delta=200_000, f_new=0.4,
                                             dist="zipf", zipf_s=1.0, seed=synth.column_seed(21, w)))
    vals = col.delta_dict[col.delta_codes]
    dd, codes = oracle.ingest_delta(w, vals)
    assert np.array_equal(dd[codes], vals)
    assert np.unique(dd, axis=0).shape[0] == dd.shape[0]
    _, first_pos = np.unique(codes, return_index=True)
    assert np.all(np.diff(first_pos) > 0)
    assert int(codes.max()) + 1 == dd.shape[0]
