"""CUDA path vs the CPU oracle, element by element (exact: all integer work).

Covers each step through its own C-ABI entry point, the whole column merge
on the workload shapes (sizes the oracle finishes in seconds, spanning many
tiles with ragged tails), the edge cases of the method, the error paths
(recorded in the status word, never faulting), determinism, and the
host-buffer and table entry points.
"""
import numpy as np
import pytest

import oracle
import synth
from paper_1109_6885_gb300 import dmerge as dm
from tests import _brute
from tests.gpu_util import assert_parity, column_from_lists, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    from paper_1109_6885_gb300 import build
    build.build()
    c = dm.Context(0, 64 << 20)
    yield c
    c.close()


def kd(w):
    return dm.key_np_dtype(w)


# ------------------------------------------------------------------ Step 1(a)

@pytest.mark.parametrize("w", [4, 8, 16])
@pytest.mark.parametrize("d", [1, 2, 31, 2047, 2048, 2049, 40_000, 300_001])
def test_sort_delta_parity(ctx, w, d):
    import torch
    keys = synth.dictionary(synth.subseed(d, w), w, d)
    rng = np.random.default_rng(d + w)
    order = rng.permutation(d)
    dd = keys[order]
    if d > 10:   # duplicates inside D_dict
        dd[rng.integers(0, d, d // 10)] = dd[rng.integers(0, d, d // 10)]
    ud_ref, perm_ref = oracle.sort_delta(w, dd)
    t_in = dm.to_device(dd)
    ud = dm.key_tensor_empty(d, w)
    perm = torch.empty(d, dtype=torch.int32, device="cuda")
    dm.dm_sort_delta(ctx, w, t_in, d, ud, perm)
    torch.cuda.synchronize()
    assert ctx.sync_status() == dm.DM_OK
    assert np.array_equal(dm.to_host(ud, kd(w)), ud_ref)
    assert np.array_equal(dm.to_host(perm, np.uint32), perm_ref)


@pytest.mark.parametrize("w", [4, 8, 16])
def test_sort_constant_digits(ctx, w):
    """Keys sharing most bytes (skipped passes), all-equal keys, equal hi words."""
    import torch
    rng = np.random.default_rng(7)
    d = 9000
    if w == 16:
        dd = np.zeros((d, 2), np.uint64)
        dd[:, 0] = 0xABCDEF
        dd[:, 1] = rng.integers(0, 300, d).astype(np.uint64)
    else:
        dd = (rng.integers(0, 200, d).astype(kd(w)) << kd(w)(8)) | kd(w)(0x11)
    for arr in (dd, dd[:1].repeat(d, axis=0)):
        ud_ref, perm_ref = oracle.sort_delta(w, arr)
        ud = dm.key_tensor_empty(d, w)
        perm = torch.empty(d, dtype=torch.int32, device="cuda")
        dm.dm_sort_delta(ctx, w, dm.to_device(arr), d, ud, perm)
        torch.cuda.synchronize()
        assert np.array_equal(dm.to_host(ud, kd(w)), ud_ref)
        assert np.array_equal(dm.to_host(perm, np.uint32), perm_ref)


@pytest.mark.parametrize("w", [4, 8, 16])
@pytest.mark.parametrize("lowbits", [1, 6, 12])
def test_sort_skewed_lower_bytes(ctx, w, lowbits):
    """A uniform top byte over few values in the lowest byte(s): the buckets split on
    a low-entropy byte (crowded sub-buckets take the merge sort), with many repeats."""
    import torch
    rng = np.random.default_rng(100 + w + lowbits)
    d = 120_000
    if w == 16:
        dd = np.zeros((d, 2), np.uint64)
        dd[:, 0] = rng.integers(0, 256, d).astype(np.uint64) << np.uint64(56)
        dd[:, 1] = rng.integers(0, 1 << lowbits, d).astype(np.uint64)
    else:
        t = kd(w)
        top = rng.integers(0, 256, d).astype(t) << t(8 * w - 8)
        dd = top | rng.integers(0, 1 << lowbits, d).astype(t)
    ud_ref, perm_ref = oracle.sort_delta(w, dd)
    ud = dm.key_tensor_empty(d, w)
    perm = torch.empty(d, dtype=torch.int32, device="cuda")
    dm.dm_sort_delta(ctx, w, dm.to_device(dd), d, ud, perm)
    torch.cuda.synchronize()
    assert ctx.sync_status() == dm.DM_OK
    assert np.array_equal(dm.to_host(ud, kd(w)), ud_ref)
    assert np.array_equal(dm.to_host(perm, np.uint32), perm_ref)


def _sort_check(ctx, w, dd):
    import torch
    d = dd.shape[0]
    ctx.reserve(max(ctx.arena_bytes, 256 << 20))     # two key buffers and their codes
    ud_ref, perm_ref = oracle.sort_delta(w, dd)
    ud = dm.key_tensor_empty(d, w)
    perm = torch.empty(d, dtype=torch.int32, device="cuda")
    dm.dm_sort_delta(ctx, w, dm.to_device(dd), d, ud, perm)
    torch.cuda.synchronize()
    assert ctx.sync_status() == dm.DM_OK
    assert np.array_equal(dm.to_host(ud, kd(w)), ud_ref)
    assert np.array_equal(dm.to_host(perm, np.uint32), perm_ref)


@pytest.mark.parametrize("w", [4, 8, 16])
@pytest.mark.parametrize("case", ["uniform", "crowded_bin", "one_byte", "two_bytes"])
def test_sort_large_deltas(ctx, w, case):
    """Sorts of 1.6M keys take the split form.  Uniform keys bin on their two
    most significant varying bytes (65,536 bins of about 25 keys) and sort
    groups of bins in place; one bin of 5,000 keys (above what a block sorts
    in shared memory) sends the sort back to the LSD passes; keys varying in
    one byte only, or in two, bin on what varies.  Repeats inside D_dict
    throughout."""
    rng = np.random.default_rng(600 + w + len(case))
    d = 1_600_003
    t = kd(w)
    if case == "uniform":
        dd = synth.dictionary(synth.subseed(d, w), w, d)[rng.permutation(d)]
    elif case == "crowded_bin":
        dd = synth.dictionary(synth.subseed(d + 1, w), w, d)[rng.permutation(d)]
        pick = rng.choice(d, 5000, replace=False)
        if w == 16:
            dd[pick, 0] = (dd[pick, 0] & np.uint64(0x0000FFFFFFFFFFFF)) | np.uint64(0xABCD) << np.uint64(48)
        else:
            hi = t(8 * w - 16)
            mask = t((1 << (8 * w - 16)) - 1)
            dd[pick] = (dd[pick] & mask) | (t(0xABCD) << hi)
    elif case == "one_byte":
        dd = rng.integers(0, 256, d).astype(t) if w < 16 else np.stack(
            [np.zeros(d, np.uint64), rng.integers(0, 256, d).astype(np.uint64)], axis=1)
    else:   # two varying bytes, far apart
        lo = rng.integers(0, 256, d)
        top = rng.integers(0, 256, d)
        if w == 16:
            dd = np.stack([top.astype(np.uint64) << np.uint64(40), lo.astype(np.uint64) << np.uint64(8)], axis=1)
        else:
            dd = (top.astype(t) << t(8 * w - 8)) | (lo.astype(t) << t(8))
    if case in ("uniform", "crowded_bin"):
        dd[rng.integers(0, d, d // 10)] = dd[rng.integers(0, d, d // 10)]
    _sort_check(ctx, w, np.ascontiguousarray(dd))


def test_merge_column_with_a_large_delta(ctx):
    """A whole column whose 1.9M-value delta takes the two-level partition."""
    col = synth.make_column(synth.ColumnSpec(n_main=3_000_000, m=2_500_000, w=8, n_delta=4_000_000, f_new=0.5,
                                             dist="uniform", seed=611))
    assert col.delta_dict.shape[0] > 1_300_000
    assert_parity(ctx, col)


# ------------------------------------------------------------------ Step 1(b) + 2(a)

@pytest.mark.parametrize("w", [4, 8, 16])
@pytest.mark.parametrize("m,d", [(0, 5), (5, 0), (1, 1), (2048, 1), (3000, 5000), (4095, 1), (4096, 1),
                                 (4097, 4096), (100_000, 9_000), (7, 70_000), (250_000, 250_000),
                                 (1_500_000, 200_001)])
def test_merge_dicts_parity(ctx, w, m, d):
    import torch
    um = synth.dictionary(synth.subseed(m, 1), w, m)
    rng = np.random.default_rng(m * 7 + d)
    fresh = synth.dictionary(synth.subseed(d, 2), w, d)
    dd = fresh.copy()
    if m and d:   # about a third of the delta values are main values
        k = d // 3
        dd[:k] = um[rng.integers(0, m, k)]
        dd = dd[rng.permutation(d)]
    ud_ref, perm_ref = oracle.sort_delta(w, dd)
    new_ref, xm_ref, xd_ref = oracle.merge_dicts(w, um, ud_ref, perm_ref)
    new = dm.key_tensor_empty(m + d, w)
    xm = torch.empty(m, dtype=torch.int32, device="cuda")
    xd = torch.empty(d, dtype=torch.int32, device="cuda")
    sc = torch.zeros(2, dtype=torch.int64, device="cuda")
    dm.dm_merge_dicts(ctx, w, dm.to_device(um), m, dm.to_device(ud_ref), dm.to_device(perm_ref), d,
                      new, xm, xd, sc, sc[1:], None)
    torch.cuda.synchronize()
    assert ctx.sync_status() == dm.DM_OK
    u, b = int(sc[0]), int(sc[1]) & 0xFFFFFFFF
    assert u == new_ref.shape[0]
    assert b == oracle.new_width(u)
    assert np.array_equal(dm.to_host(new[:u], kd(w)), new_ref)
    assert np.array_equal(dm.to_host(xm, np.uint32), xm_ref)
    assert np.array_equal(dm.to_host(xd, np.uint32), xd_ref)


# ------------------------------------------------------------------ Step 2(b)

@pytest.mark.parametrize("b", list(range(0, 33)))
def test_reencode_every_width(ctx, b):
    """Every input width, output widths b-1, b, b+1 and a distant one; ragged tails."""
    import torch
    rng = np.random.default_rng(b)
    m = min(2**b, 5000) if b else 1
    n_main, n_delta, d = 70_003, 1_234, 77
    mc = rng.integers(0, m, n_main).astype(np.uint32)
    dc = rng.integers(0, d, n_delta).astype(np.uint32)
    main = synth.pack(mc, b)
    for bo in sorted({max(b - 1, 0), b, min(b + 1, 32), (b + 13) % 33}):
        top = 2**bo
        xm = rng.integers(0, top, m, dtype=np.uint64).astype(np.uint32)
        xd = rng.integers(0, top, d, dtype=np.uint64).astype(np.uint32)
        want = oracle.reencode(main, b, n_main, dc, xm, xd, bo)
        maxb = max(bo, 20)
        out = torch.full((dm.dm_packed_bytes(n_main + n_delta, maxb) // 4,), -1, dtype=torch.int32,
                         device="cuda")
        bits = torch.tensor([bo], dtype=torch.int32, device="cuda")
        for flags in (0, dm.DM_FLAG_GENERIC_REENCODE, dm.DM_FLAG_X_SMEM, dm.DM_FLAG_X_GLOBAL):
            out.fill_(-1)
            dm.dm_reencode(ctx, dm.to_device(main), b, n_main, dm.to_device(dc), n_delta,
                           dm.to_device(xm), m, dm.to_device(xd), d, bits, maxb, out, None, flags)
            torch.cuda.synchronize()
            assert ctx.sync_status() == dm.DM_OK
            got = dm.to_host(out, np.uint32)
            assert np.array_equal(got[:want.size], want), (b, bo, flags)
            assert np.all(got[want.size:] == 0xFFFFFFFF), "wrote past the stream's end"


# ------------------------------------------------------------------ whole column

@pytest.mark.parametrize("w", [4, 8, 16])
@pytest.mark.parametrize("dist", ["uniform", "zipf"])
@pytest.mark.parametrize("n_main,m,n_delta,f_new", [
    (1, 1, 1, 0.5), (31, 5, 33, 0.5), (1023, 40, 1, 1.0), (1025, 1000, 1023, 0.3),
    (33_333, 2_000, 3_333, 0.3), (250_007, 100_000, 20_011, 0.5), (100_000, 60_000, 100_000, 0.9),
])
def test_merge_column_parity(ctx, w, dist, n_main, m, n_delta, f_new):
    spec = synth.ColumnSpec(n_main=n_main, m=m, w=w, n_delta=n_delta, f_new=f_new, dist=dist,
                            zipf_s=0.8, seed=n_main ^ (m << 8) ^ w)
    assert_parity(ctx, synth.make_column(spec))


def test_small_single_column_workload(ctx):
    """1,000,000 rows over 100,000 uint64 values at 17 bits; 10,000 delta rows, half new."""
    spec = synth.ColumnSpec(n_main=1_000_000, m=100_000, w=8, n_delta=10_000, f_new=0.5, pool=0,
                            seed=synth.column_seed(1, 0))
    col = synth.make_column(spec)
    ref = assert_parity(ctx, col)
    assert col.main_bits == 17 and ref.new_bits == 17
    for flags in (dm.DM_FLAG_X_SMEM, dm.DM_FLAG_X_GLOBAL, dm.DM_FLAG_GENERIC_REENCODE):
        assert_parity(ctx, col, flags, ref)


@pytest.mark.parametrize("case", ["delta_empty", "main_empty", "subset_same_width", "all_new",
                                  "u_one", "u_two", "grow_to_pow2", "cross_pow2", "non_minimal_b",
                                  "shrink_width"])
def test_edge_cases(ctx, case):
    rng = np.random.default_rng(len(case))
    if case == "delta_empty":
        col = synth.make_column(synth.ColumnSpec(n_main=5000, m=700, n_delta=0))
    elif case == "main_empty":
        col = synth.make_column(synth.ColumnSpec(n_main=0, m=0, n_delta=5000, f_new=1.0))
    elif case == "subset_same_width":
        col = synth.make_column(synth.ColumnSpec(n_main=50_000, m=1000, n_delta=3000, f_new=0.0))
        ref = assert_parity(ctx, col)
        assert ref.new_bits == col.main_bits
        nb = col.n_main * col.main_bits // 32
        assert np.array_equal(ref.new_packed[:nb], col.main_packed[:nb])
        return
    elif case == "all_new":
        col = synth.make_column(synth.ColumnSpec(n_main=20_000, m=500, n_delta=9000, f_new=1.0,
                                                 pool=0))
    elif case == "u_one":
        col = column_from_lists(8, [42], [0] * 3000, [42], [0] * 77)
    elif case == "u_two":
        col = column_from_lists(8, [42], [0] * 3000, [43], [0] * 77)
    elif case == "grow_to_pow2":      # 1000 + 24 new -> 1024: still 10 bits
        um = sorted(rng.choice(10**6, 1000, replace=False).tolist())
        new = sorted(set(range(10**6, 10**6 + 24)))
        col = column_from_lists(4, um, rng.integers(0, 1000, 9999).tolist(), new,
                                rng.integers(0, 24, 555).tolist())
    elif case == "cross_pow2":        # 1024 + 1 -> 1025: 10 -> 11 bits
        um = list(range(0, 2048, 2))
        col = column_from_lists(4, um, rng.integers(0, 1024, 9999).tolist(), [7],
                                [0] * 555)
    elif case == "non_minimal_b":     # main stored wider than needed
        um = list(range(100, 400))
        col = column_from_lists(8, um, rng.integers(0, 300, 20_000).tolist(), [5, 999],
                                [0, 1] * 100, b=23)
    else:                             # shrink: b' < b
        um = list(range(100, 116))
        col = column_from_lists(8, um, rng.integers(0, 16, 20_000).tolist(), [1],
                                [0] * 100, b=31)
    assert_parity(ctx, col)


def test_extreme_keys_and_equal_hi(ctx):
    top = 2**64 - 1
    rng = np.random.default_rng(3)
    col = column_from_lists(8, [0, 5, top], rng.integers(0, 3, 5000).tolist(), [top, 1, 0, 7],
                            rng.integers(0, 4, 999).tolist())
    assert_parity(ctx, col)
    hi = 0xFEED << 64
    um = [hi | v for v in range(0, 4000, 3)]
    dd = [hi | v for v in range(1, 4000, 5)] + [(1 << 64) | 3, 2**128 - 1]
    col = column_from_lists(16, um, rng.integers(0, len(um), 30_000).tolist(), dd,
                            rng.integers(0, len(dd), 4000).tolist())
    assert_parity(ctx, col)
    # 4-byte keys at collision density: 2^20 main values over a 2^21 range
    um = sorted(rng.choice(2**21, 2**20, replace=False).tolist())
    dd = rng.choice(2**21, 50_000, replace=False).tolist()
    col = column_from_lists(4, um, rng.integers(0, len(um), 300_000).tolist(), dd,
                            rng.integers(0, len(dd), 60_000).tolist())
    assert_parity(ctx, col)


def test_duplicates_in_delta_dict(ctx):
    rng = np.random.default_rng(9)
    um = list(range(0, 30_000, 3))
    dd = rng.integers(0, 40_000, 5000).tolist()           # repeats inside D_dict
    col = column_from_lists(8, um, rng.integers(0, len(um), 40_000).tolist(), dd,
                            rng.integers(0, len(dd), 7000).tolist())
    assert_parity(ctx, col)


def test_determinism(ctx):
    col = synth.make_column(synth.ColumnSpec(n_main=300_000, m=50_000, n_delta=30_000, f_new=0.3,
                                             dist="zipf", seed=11))
    a, _ = run_gpu(ctx, col)
    b, _ = run_gpu(ctx, col)
    for x, y in zip(a, b):
        if isinstance(x, np.ndarray):
            assert np.array_equal(x, y)
        else:
            assert x == y


# ------------------------------------------------------------------ errors (no faults)

def test_unsorted_main_dict_is_reported(ctx):
    col = column_from_lists(8, [5, 3, 9], [0, 1, 2] * 100, [4], [0] * 10)
    _, st = run_gpu(ctx, col)
    assert st == dm.DM_EUNSORTED
    assert ctx.sync_status() == dm.DM_OK          # read-and-clear


def test_out_of_range_codes_are_clamped_and_reported(ctx):
    um = list(range(10, 20))                      # m = 10 at 4 bits: codes 10..15 are invalid
    codes = [3, 15, 7, 12] * 3000
    col = column_from_lists(8, um, codes, [1], [0] * 5, b=4)
    _, st = run_gpu(ctx, col)
    assert st == dm.DM_ECODE
    col = column_from_lists(8, um, [1] * 5000, [1, 2], [0, 1, 5])   # delta code 5 >= d = 2
    _, st = run_gpu(ctx, col)
    assert st == dm.DM_ECODE


def test_argument_errors(ctx):
    col = synth.make_column(synth.ColumnSpec(n_main=1000, m=100, n_delta=10))
    dcol = dm.DeviceColumn.from_numpy(col.w, col.main_dict, col.main_packed, col.main_bits,
                                      col.n_main, col.delta_dict, col.delta_codes)
    res = dm.alloc_result(dcol)
    bad = dcol.cin()
    bad.value_bytes = 6
    with pytest.raises(dm.DmError) as e:
        dm.dm_merge_column(ctx, bad, res.cout())
    assert e.value.status == dm.DM_EINVAL
    bad = dcol.cin()
    bad.main_bits = 3                               # below ceil(log2 100)
    with pytest.raises(dm.DmError) as e:
        dm.dm_merge_column(ctx, bad, res.cout())
    assert e.value.status == dm.DM_EINVAL
    small = dm.Context(0, 1024)
    with pytest.raises(dm.DmError) as e:
        dm.dm_merge_column(small, dcol.cin(), res.cout())
    assert e.value.status == dm.DM_ENOMEM
    small.close()


# ------------------------------------------------------------------ other entry points

# (n_main, m, w, n_delta, f_new, dist): the main vector goes up and the
# result comes back in chunks of whole 1024-row tiles; the cases cover a
# ragged last chunk, an exact multiple, a single short chunk, a delta longer
# than the main vector, the X_M directory lookup, and a zero-width column.
HOST_CASES = [
    (400_003, 30_000, 16, 20_000, 0.4, "zipf"),
    (8 * 1024 * 3, 100, 8, 5_000, 0.9, "uniform"),
    (1_000, 5, 4, 3_000, 0.5, "uniform"),
    (2_000_001, 70_000, 8, 100_000, 0.3, "zipf"),
    (1_500_001, 1, 4, 0, 0.0, "uniform"),
    (3_000_000, 200, 4, 4_096, 0.0, "zipf"),
]


@pytest.mark.parametrize("case", HOST_CASES)
def test_host_buffer_entry_point(ctx, case):
    n_main, m0, w, n_delta, f_new, dist = case
    col = synth.make_column(synth.ColumnSpec(n_main=n_main, m=m0, w=w, n_delta=n_delta,
                                             f_new=f_new, dist=dist, seed=21 + n_main % 97))
    ref = oracle.merge_synth_column(col)
    cin = dm.ColumnIn(col.w, col.main_dict.ctypes.data, col.main_dict.shape[0],
                      col.main_packed.ctypes.data, col.main_bits, col.n_main,
                      col.delta_dict.ctypes.data, col.delta_dict.shape[0],
                      col.delta_codes.ctypes.data, col.n_delta)
    m, d = col.main_dict.shape[0], col.delta_dict.shape[0]
    new_dict = synth.key_array(max(m + d, 1), w)
    nwords = dm.dm_packed_bytes(col.n_main + col.n_delta, dm.dm_bits_for(m + d)) // 4
    packed = np.full(max(nwords, 1), 0xDEADBEEF, np.uint32)
    xm = np.zeros(max(m, 1), np.uint32)
    xd = np.zeros(max(d, 1), np.uint32)
    cout = dm.ColumnOut(new_dict.ctypes.data, packed.ctypes.data, xm.ctypes.data, xd.ctypes.data,
                        None, None)
    ctx.reserve(dm.dm_host_scratch_bytes(cin))
    u, b = dm.dm_merge_column_host(ctx, cin, cout)
    assert ctx.sync_status() == dm.DM_OK
    assert u == ref.u and b == ref.new_bits
    assert np.array_equal(new_dict[:u], ref.new_dict)
    assert np.array_equal(packed[:ref.new_packed.size], ref.new_packed)
    assert np.array_equal(xm[:m], ref.x_main) and np.array_equal(xd[:d], ref.x_delta)


@pytest.mark.parametrize("chunks", [1, 3, 32])
def test_host_buffer_chunk_counts(chunks):
    """The chunk count splits the copies and launches, never the result."""
    col = synth.make_column(synth.ColumnSpec(n_main=1_234_567, m=40_000, w=8, n_delta=30_000,
                                             f_new=0.3, dist="zipf", seed=77))
    ref = oracle.merge_synth_column(col)
    c = dm.Context(0, 1 << 20)
    c.set_tuning(host_chunks=chunks)
    cin = dm.ColumnIn(col.w, col.main_dict.ctypes.data, col.main_dict.shape[0],
                      col.main_packed.ctypes.data, col.main_bits, col.n_main,
                      col.delta_dict.ctypes.data, col.delta_dict.shape[0],
                      col.delta_codes.ctypes.data, col.n_delta)
    m, d = col.main_dict.shape[0], col.delta_dict.shape[0]
    new_dict = synth.key_array(m + d, 8)
    packed = np.zeros(dm.dm_packed_bytes(col.n_main + col.n_delta, dm.dm_bits_for(m + d)) // 4,
                      np.uint32)
    cout = dm.ColumnOut(new_dict.ctypes.data, packed.ctypes.data, None, None, None, None)
    c.reserve(dm.dm_host_scratch_bytes(cin))
    u, b = dm.dm_merge_column_host(c, cin, cout)
    assert c.sync_status() == dm.DM_OK
    c.close()
    assert u == ref.u and b == ref.new_bits
    assert np.array_equal(new_dict[:u], ref.new_dict)
    assert np.array_equal(packed[:ref.new_packed.size], ref.new_packed)


def _table(rng, ncols, n_main, n_delta, max_m, config=4):
    cols, dcols, results = [], [], []
    for j in range(ncols):
        m = int(np.exp(rng.uniform(np.log(2), np.log(max_m))))
        w = int(rng.choice([4, 8, 16]))
        spec = synth.ColumnSpec(n_main=n_main, m=m, w=w, n_delta=n_delta,
                                f_new=float(rng.uniform(0, 0.5)), dist="zipf", zipf_s=0.8,
                                seed=synth.column_seed(config, j))
        col = synth.make_column(spec)
        cols.append(col)
        dc = dm.DeviceColumn.from_numpy(col.w, col.main_dict, col.main_packed, col.main_bits,
                                        col.n_main, col.delta_dict, col.delta_codes)
        dcols.append(dc)
        results.append(dm.alloc_result(dc))
    return cols, dcols, results


def _check_table(cols, results):
    for col, res in zip(cols, results):
        ref = oracle.merge_synth_column(col)
        new_dict, xm, xd, packed, b, u = dm.fetch(res, col.w, col.n_main + col.n_delta)
        assert u == ref.u and b == ref.new_bits
        assert np.array_equal(new_dict, ref.new_dict)
        assert np.array_equal(packed, ref.new_packed)
        assert np.array_equal(xm, ref.x_main) and np.array_equal(xd, ref.x_delta)


@pytest.mark.parametrize("flags", [0, dm.DM_FLAG_SERIAL, dm.DM_FLAG_NO_GRAPH])
def test_merge_table_parity(ctx, flags):
    """Batched (one graph launch, or the same schedule issued directly) and serial table
    merges vs the per-column oracle."""
    import torch
    rng = np.random.default_rng(5)
    cols, dcols, results = _table(rng, 9, 300_007, 3_001, 300_000)
    cins = [c.cin() for c in dcols]
    ctx.reserve(dm.dm_table_scratch_bytes(cins, flags))
    dm.dm_merge_table(ctx, cins, [r.cout() for r in results], flags=flags)
    torch.cuda.synchronize()
    assert ctx.sync_status() == dm.DM_OK
    _check_table(cols, results)


def test_merge_table_graph_replay_sees_new_data(ctx):
    """A replayed table graph reads the buffers' current contents."""
    import torch
    rng = np.random.default_rng(6)
    cols, dcols, results = _table(rng, 5, 200_003, 2_000, 100_000)
    cins = [c.cin() for c in dcols]
    couts = [r.cout() for r in results]
    ctx.reserve(dm.dm_table_scratch_bytes(cins))
    dm.dm_merge_table(ctx, cins, couts)
    torch.cuda.synchronize()
    _check_table(cols, results)
    # same buffers, new codes: rewrite each column's main vector and delta codes in place
    new_cols = []
    for j, (col, dc) in enumerate(zip(cols, dcols)):
        mc = synth.codes(1000 + j, col.main_dict.shape[0], col.n_main)
        packed = synth.pack(mc, col.main_bits)
        dcodes = synth.codes(2000 + j, col.delta_dict.shape[0], col.n_delta)
        dc.main_packed.copy_(dm.to_device(packed))
        dc.delta_codes.copy_(dm.to_device(dcodes))
        new_cols.append(synth.Column(col.spec, col.main_dict, mc, col.main_bits, packed,
                                     col.delta_dict, dcodes))
    dm.dm_merge_table(ctx, cins, couts)
    torch.cuda.synchronize()
    assert ctx.sync_status() == dm.DM_OK
    _check_table(new_cols, results)


# ------------------------------------------------------------------ X_M directory

def _steps_table(m, k, rng, clustered=False):
    """A valid X_M: i + (number of new values inserted at or before main code i)."""
    if clustered:       # several new values at the same insertion points
        pts = np.repeat(rng.integers(0, m + 1, max(k // 4, 1)), 4)[:k]
    else:
        pts = rng.integers(0, m + 1, k)
    pts = np.sort(pts)
    c = np.searchsorted(pts, np.arange(m), side="right")
    return (np.arange(m) + c).astype(np.uint32), m + k


@pytest.mark.parametrize("m,k,clustered", [(20_000, 0, False), (20_000, 150, False),
                                           (20_000, 20_000, False), (300_000, 3_000, True),
                                           (1_000_000, 3_000, False), (1_000_000, 30_000, False),
                                           (1_000_000, 300_000, False), (100_000, 25_000, True),
                                           (16_385, 900, True), (1 << 20, 5_000, False),
                                           ((1 << 20) + 1, 5_000, False), (5_000_000, 40_000, False)])
def test_reencode_directory_mode(ctx, m, k, clustered):
    """X_M looked up through the shared-memory directory (forced) vs the oracle.  The cases
    run from no steps to several per bucket (those buckets read X_M itself), with new
    values that share an insertion point (clustered)."""
    import torch
    rng = np.random.default_rng(m + k)
    xm, u = _steps_table(m, k, rng, clustered)
    b, bo = synth.bits_for(m), synth.bits_for(u)
    n_main, n_delta, d = 1_500_007, 999, 31
    mc = rng.integers(0, m, n_main).astype(np.uint32)
    dc = rng.integers(0, d, n_delta).astype(np.uint32)
    xd = rng.integers(0, u, d).astype(np.uint32)
    main = synth.pack(mc, b)
    want = oracle.reencode(main, b, n_main, dc, xm, xd, bo)
    out = torch.full((dm.dm_packed_bytes(n_main + n_delta, bo) // 4,), -1, dtype=torch.int32,
                     device="cuda")
    bits = torch.tensor([bo], dtype=torch.int32, device="cuda")
    for flags in (dm.DM_FLAG_X_SMEM, dm.DM_FLAG_X_GLOBAL):
        out.fill_(-1)
        dm.dm_reencode(ctx, dm.to_device(main), b, n_main, dm.to_device(dc), n_delta,
                       dm.to_device(xm), m, dm.to_device(xd), d, bits, bo, out, None, flags)
        torch.cuda.synchronize()
        assert ctx.sync_status() == dm.DM_OK
        assert np.array_equal(dm.to_host(out, np.uint32), want), flags


@pytest.mark.parametrize("m,n_delta,f_new,pool", [(50_000, 20_000, 0.3, None),
                                                   (400_000, 100_000, 0.5, 0),
                                                   (1_000_000, 200_000, 0.3, 30_000),
                                                   (2_000_000, 50_000, 0.3, None)])
def test_merge_column_directory_mode(ctx, m, n_delta, f_new, pool):
    spec = synth.ColumnSpec(n_main=3_000_001, m=m, w=8, n_delta=n_delta, f_new=f_new, pool=pool,
                            dist="zipf", zipf_s=1.0, seed=m ^ n_delta)
    col = synth.make_column(spec)
    ref = assert_parity(ctx, col, dm.DM_FLAG_X_SMEM)
    assert_parity(ctx, col, 0, ref)


# ------------------------------------------------------------------ full-size workloads

@pytest.mark.parametrize("w", [8, 16])
def test_full_size_single_column(ctx, w):
    """100,000,000 main rows over 1,000,000 values (1% unique), Zipf(1.0) codes at 20
    bits, 1,000,000 delta rows with 30% new values: every output byte vs the oracle."""
    spec = synth.ColumnSpec(n_main=100_000_000, m=1_000_000, w=w, n_delta=1_000_000, f_new=0.3,
                            dist="zipf", zipf_s=1.0, seed=synth.column_seed(2, 0))
    col = synth.make_column(spec)
    ref = assert_parity(ctx, col)
    assert col.main_bits == 20 and ref.new_bits == 20


def test_full_size_literal_new_fraction(ctx):
    """As above with every fresh delta row a distinct new value (300,000 new: 20 -> 21 bits)."""
    spec = synth.ColumnSpec(n_main=100_000_000, m=1_000_000, w=8, n_delta=1_000_000, f_new=0.3,
                            pool=0, dist="zipf", zipf_s=1.0, seed=synth.column_seed(2, 1))
    col = synth.make_column(spec)
    ref = assert_parity(ctx, col)
    assert ref.new_bits == 21


@pytest.mark.parametrize("warps,stages,obufs", [(4, 2, 1), (8, 4, 2), (12, 3, 2), (16, 2, 1),
                                                (16, 4, 1), (1, 2, 1)])
def test_tuning_changes_nothing(warps, stages, obufs):
    """Launch parameters split the work differently; the bytes stay the same."""
    from paper_1109_6885_gb300 import build
    build.build()
    c = dm.Context(0, 64 << 20)
    c.set_tuning(reencode_warps=warps, reencode_stages=stages, reencode_obufs=obufs)
    spec = synth.ColumnSpec(n_main=2_100_003, m=300_000, w=8, n_delta=30_000, f_new=0.3,
                            dist="zipf", seed=warps * 100 + stages * 10 + obufs)
    col = synth.make_column(spec)
    ref = assert_parity(c, col)
    for flags in (dm.DM_FLAG_X_GLOBAL, dm.DM_FLAG_GENERIC_REENCODE):
        assert_parity(c, col, flags, ref)
    small = synth.make_column(synth.ColumnSpec(n_main=1_500_000, m=3000, w=4, n_delta=999,
                                               seed=warps))
    assert_parity(c, small, dm.DM_FLAG_X_SMEM)
    c.close()


@pytest.mark.parametrize("m,warps", [(5_000_000, 12), (5_000_000, 8), (10_000_000, 10), (10_000_000, 8)])
def test_refined_directory(m, warps):
    """Above 2^22 main codes a block with fewer warps gives its freed shared memory to finer
    directory buckets (halved while the block stays within 196 KB): 5M codes at 23 bits take
    256-code buckets instead of 512, 10M codes at 24 bits 512 instead of 1024.  The delta
    leaves buckets without steps, with one step and with several."""
    from paper_1109_6885_gb300 import build
    build.build()
    c = dm.Context(0, 64 << 20)
    c.set_tuning(reencode_warps=warps)
    spec = synth.ColumnSpec(n_main=3_000_007, m=m, w=8, n_delta=400_000, f_new=0.3, dist="zipf",
                            zipf_s=0.8, seed=synth.column_seed(17, m // 1_000_000 + warps))
    col = synth.make_column(spec)
    ref = assert_parity(c, col)
    assert ref.u > m
    c.close()


@pytest.mark.parametrize("flags", [0, "X_GLOBAL", "X_SMEM"])
def test_merge_repeats_bulk_copy_ring(ctx, flags):
    """A column whose re-encode once read a bulk-copy stage while the copy refilling it
    landed (8M rows at 23 bits over 5.29M values, Zipf(0.8) codes, 80k delta rows): the
    stage is refilled only after every lane's reads of it are done, so each repeat gives
    the same bytes as the oracle."""
    f = 0 if flags == 0 else getattr(dm, "DM_FLAG_" + flags)
    spec = synth.ColumnSpec(n_main=8_000_000, m=5_293_474, w=8, n_delta=80_000, f_new=0.209218938724463,
                            dist="zipf", zipf_s=0.8, seed=synth.column_seed(4, 41))
    col = synth.make_column(spec)
    assert col.main_bits == 23
    ref = assert_parity(ctx, col, f)
    for _ in range(3):
        assert_parity(ctx, col, f, ref)


@pytest.mark.parametrize("n_steps", [60_000, 5_000, 23_137, 23_138])
def test_reencode_byte_table(ctx, n_steps):
    """Above 11 * 2^20 main codes the directory's crowded buckets read a byte table of c[i] - base
    when the steps are dense (two or more a bucket on average), else X_M: 12M codes (11,719
    buckets of 1024) with 60k new values (most buckets crowded, the table), 5k (a few crowded,
    X_M), and counts one below and at the rule's 23,438 steps below the last main code; each
    with one insertion point of 300 new values (more than a byte holds: that bucket reads X_M)."""
    import torch
    rng = np.random.default_rng(8888 + n_steps)
    m = 12_000_000
    pts = np.concatenate([rng.integers(0, m + 1, n_steps), np.full(300, 5_000_001)])
    pts.sort()
    xm = (np.arange(m) + np.searchsorted(pts, np.arange(m), side="right")).astype(np.uint32)
    u = m + pts.size
    b, bo = synth.bits_for(m), synth.bits_for(u)
    n_main, n_delta, d = 3_000_011, 1_000, 50
    mc = rng.integers(0, m, n_main).astype(np.uint32)
    mc[:5000] = rng.integers(4_999_900, 5_000_100, 5000)   # codes around the crowded point
    dc = rng.integers(0, d, n_delta).astype(np.uint32)
    xd = rng.integers(0, u, d).astype(np.uint32)
    main = synth.pack(mc, b)
    want = oracle.reencode(main, b, n_main, dc, xm, xd, bo)
    out = torch.empty((dm.dm_packed_bytes(n_main + n_delta, bo) // 4,), dtype=torch.int32, device="cuda")
    bits = torch.tensor([bo], dtype=torch.int32, device="cuda")
    t = [dm.to_device(x) for x in (main, dc, xm, xd)]
    for flags in (dm.DM_FLAG_X_SMEM, 0):
        out.fill_(-1)
        dm.dm_reencode(ctx, t[0], b, n_main, t[1], n_delta, t[2], m, t[3], d, bits, bo, out, None, flags)
        torch.cuda.synchronize()
        assert ctx.sync_status() == dm.DM_OK
        assert np.array_equal(dm.to_host(out, np.uint32), want), flags


@pytest.mark.parametrize("n_delta,min_new,max_new", [(1_000_000, 100_000, None), (20_000, 1, 20_000)])
def test_merge_column_byte_table(ctx, n_delta, min_new, max_new):
    """Whole merges over 12M main values: with 450k new values X_M's steps are dense and the
    crowded buckets read the byte table; with a few thousand they read X_M."""
    spec = synth.ColumnSpec(n_main=10_000_000, m=12_000_000, w=8, n_delta=n_delta, f_new=0.5,
                            dist="zipf", zipf_s=0.8, seed=synth.column_seed(7, 1 if n_delta >= 1_000_000 else 2))
    col = synth.make_column(spec)
    ref = assert_parity(ctx, col)
    n_new = ref.u - col.main_dict.shape[0]
    assert n_new >= min_new and (max_new is None or n_new <= max_new)


@pytest.mark.parametrize("b_extra", [0, 1, 4])
def test_reencode_directory_width_variants(ctx, b_extra):
    """Directory mode over codes stored wider than needed (covering and not)."""
    import torch
    rng = np.random.default_rng(40 + b_extra)
    m, k = 20_000, 400
    xm, u = _steps_table(m, k, rng)
    b, bo = synth.bits_for(m) + b_extra, synth.bits_for(u)
    n_main = 1_200_001
    mc = rng.integers(0, m, n_main).astype(np.uint32)
    main = synth.pack(mc, b)
    dc = np.zeros(1, np.uint32)
    xd = np.zeros(1, np.uint32)
    want = oracle.reencode(main, b, n_main, dc, xm, xd, bo)
    out = torch.full((dm.dm_packed_bytes(n_main + 1, bo) // 4,), -1, dtype=torch.int32,
                     device="cuda")
    bits = torch.tensor([bo], dtype=torch.int32, device="cuda")
    dm.dm_reencode(ctx, dm.to_device(main), b, n_main, dm.to_device(dc), 1, dm.to_device(xm), m,
                   dm.to_device(xd), 1, bits, bo, out, None, dm.DM_FLAG_X_SMEM)
    torch.cuda.synchronize()
    assert ctx.sync_status() == dm.DM_OK
    assert np.array_equal(dm.to_host(out, np.uint32), want)


def test_directory_mode_flags_codes_past_the_dictionary(ctx):
    """Codes >= |U_M| in a covering directory are flagged, clamped, never faulting."""
    import torch
    rng = np.random.default_rng(77)
    m = 20_000
    xm = np.arange(m, dtype=np.uint32)
    b = synth.bits_for(m)
    mc = rng.integers(0, m, 1_100_000).astype(np.uint32)
    mc[::1000] = rng.integers(m, 2**b, mc[::1000].size)       # invalid codes
    main = synth.pack(mc, b)
    out = torch.zeros(dm.dm_packed_bytes(mc.size, b) // 4, dtype=torch.int32, device="cuda")
    bits = torch.tensor([b], dtype=torch.int32, device="cuda")
    dm.dm_reencode(ctx, dm.to_device(main), b, mc.size, None, 0, dm.to_device(xm), m, None, 0, bits,
                   b, out, None, dm.DM_FLAG_X_SMEM)
    torch.cuda.synchronize()
    assert ctx.sync_status() == dm.DM_ECODE
    got = np.array(_brute.unpack_bits(dm.to_host(out, np.uint32)[:2000], 1000, b))
    want = np.minimum(mc[:1000], m - 1)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("n_hi", [1, 7])
def test_k16_keys_sharing_hi_words_at_scale(ctx, n_hi):
    """16-byte keys whose hi words take only n_hi values (1: all equal), so
    that sorting, merging and deduplication decide on the lo words: 1.4M
    main values, a 300k-row delta of which half repeat main values, 3M main
    rows."""
    rng = np.random.default_rng(160 + n_hi)
    his = np.unique(rng.integers(0, 2**62, 4 * n_hi, dtype=np.uint64))[:n_hi]
    his = his[rng.permutation(his.size)][:n_hi]
    his.sort()
    per = 1_400_000 // n_hi
    groups = []
    for g, h in enumerate(his):
        lo = synth.dictionary(synth.subseed(17, g), 8, per)
        groups.append(np.stack([np.full(per, h, np.uint64), lo], axis=1))
    um = np.concatenate(groups)
    m = um.shape[0]
    n_main, n_delta = 3_000_000, 300_000
    mc = rng.integers(0, m, n_main).astype(np.uint32)
    fresh = np.stack([his[rng.integers(0, n_hi, n_delta)], rng.integers(0, 2**63, n_delta, dtype=np.uint64)],
                     axis=1)
    rows = np.where((rng.random(n_delta) < 0.5)[:, None], um[rng.integers(0, m, n_delta)], fresh)
    # insertion-order dictionary of the delta rows and their codes
    _, first, inv = np.unique(rows, axis=0, return_index=True, return_inverse=True)
    order = np.argsort(first)
    dd = rows[first[order]]
    rank = np.empty_like(order)
    rank[order] = np.arange(order.size)
    dc = rank[inv.reshape(-1)].astype(np.uint32)
    b = synth.bits_for(m)
    spec = synth.ColumnSpec(n_main=n_main, m=m, w=16, n_delta=n_delta)
    col = synth.Column(spec, np.ascontiguousarray(um), mc, b, synth.pack(mc, b), np.ascontiguousarray(dd), dc)
    ref = assert_parity(ctx, col)
    assert ref.u > m


@pytest.mark.parametrize("w,m,d,frac_new,repeats", [
    (4, 4096, 2048, 1.0, False), (8, 4096, 2048, 0.3, False), (16, 4096, 2048, 0.5, True),
    (8, 4097, 2048, 0.3, False), (8, 4096, 2049, 0.3, False), (16, 1, 1, 1.0, False),
    (4, 0, 2048, 1.0, True), (8, 4096, 0, 0.0, False), (8, 1000, 2048, 0.0, True),
    (16, 2, 2048, 0.999, True), (4, 7, 9, 0.3, False), (8, 4096, 1, 1.0, False)])
def test_small_dictionaries_at_and_past_the_one_block_limits(ctx, w, m, d, frac_new, repeats):
    """Dictionaries of at most 4,096 main and 2,048 delta entries take Step 1
    in one block; one entry more takes the tiled kernel.  Both sides of each
    limit, all-new and no-new deltas, repeated delta values, an empty main
    or delta dictionary and 16-byte keys over several hi words."""
    rng = np.random.default_rng(1000 * w + m + d)
    his = [0] if w < 16 else [0, 3, 2**64 - 1]
    span = 2 ** (8 * min(w, 8)) - 1
    vals = set()
    while len(vals) < m + d:
        lo = int(rng.integers(0, span, dtype=np.uint64, endpoint=True))
        vals.add((int(his[int(rng.integers(0, len(his)))]) << 64) | lo if w == 16 else lo)
    vals = list(vals)
    rng.shuffle(vals)
    um = sorted(vals[:m])
    fresh = vals[m:]
    dd = []
    for k in range(d):
        if m == 0 or rng.random() < frac_new:
            dd.append(fresh[int(rng.integers(0, len(fresh)))] if repeats else fresh[k])
        else:
            dd.append(um[int(rng.integers(0, m))])
    if not repeats:
        dd = list(dict.fromkeys(dd))
        while len(dd) < d:                     # refill with unused fresh values
            dd.append(next(v for v in fresh if v not in set(dd)))
    main_codes = rng.integers(0, m, 20_000).tolist() if m else []
    dcodes = rng.integers(0, d, 5000).tolist() if d else []
    col = column_from_lists(w, um, main_codes, dd, dcodes)
    ref = assert_parity(ctx, col)
    assert ref.u == len(set(um) | set(dd))


# ------------------------------------------------------------------ global directory
# Past 2^24 main codes the shared-memory directory cannot cover X_M; Step 2(b)
# then reads an L2-resident directory with one 8-byte entry per bucket of
# 2^s codes (the count of new values below the bucket and the offsets of up
# to four steps), and buckets with more steps read X_M.

GDIR_M = (1 << 24) + 300_001          # b = 25


def _gdir_column(steps, n_random_steps, seed, n_main=1_500_000, above_all=True):
    """GDIR_M main values 4, 8, 12, ... (8-byte keys).  New values 4i + 1,
    4i + 2, 4i + 3 sort right below U_M[i], so k of them put a step of k at
    code i (c = X_M - i grows by k there): `steps` is a list of (code, k),
    plus `n_random_steps` single steps at random codes, one new value above
    every main value, and as many existing main values again in the delta,
    in a shuffled insertion order."""
    rng = np.random.default_rng(seed)
    m = GDIR_M
    um = np.arange(m, dtype=np.uint64) * 4 + 4
    new = [np.uint64(4 * i + j) for i, k in steps for j in range(1, k + 1)]
    rand = np.setdiff1d(rng.integers(0, m, n_random_steps).astype(np.uint64),
                        np.array([i for i, _ in steps], np.uint64))
    new = np.concatenate([np.array(new, np.uint64), rand * 4 + 1])
    if above_all:
        new = np.append(new, np.uint64(4 * m + 9))
    old = um[rng.integers(0, m, new.size)]
    dd = np.concatenate([new, old, new[: new.size // 4]])      # repeats inside D_dict too
    dd = dd[rng.permutation(dd.size)]
    mc = rng.integers(0, m, n_main).astype(np.uint32)
    b = synth.bits_for(m)
    dc = rng.integers(0, dd.size, 20_000).astype(np.uint32)
    spec = synth.ColumnSpec(n_main=n_main, m=m, w=8, n_delta=dc.size)
    return synth.Column(spec, um, mc, b, synth.pack(mc, b), np.ascontiguousarray(dd), dc)


def test_global_directory_steps_at_bucket_edges(ctx):
    """With a small delta the buckets are 64 codes: a step at code 0; one at
    offset 0 and one at offset 63 of their buckets; two; exactly four; five
    (more than an entry holds); three at one code; two double steps; a
    triple and a double (five); the last main code; the first and last
    codes of one bucket."""
    M = GDIR_M
    steps = [(0, 1), (64, 1), (191, 1), (200, 1), (210, 1), (256, 1), (260, 1), (300, 1), (319, 1),
             (320, 1), (321, 1), (322, 1), (330, 1), (383, 1), (400, 3), (448, 2), (460, 2), (512, 3),
             (513, 2), (640, 1), (703, 1), (M - 1, 1)]
    col = _gdir_column(steps, 2_000, seed=31)
    ref = assert_parity(ctx, col)
    new_values = np.unique(col.delta_dict[col.delta_dict % 4 != 0]).size
    assert ref.u == GDIR_M + new_values
    # the plain X_M gather gives the same bytes
    assert_parity(ctx, col, dm.DM_FLAG_X_GLOBAL, ref)


@pytest.mark.parametrize("n_steps", [0, 150_000, 3_000_000])
def test_global_directory_step_densities(ctx, n_steps):
    """No new value below any main value (no bucket with a step), a sparse
    mix, and a dense one (3M steps among 17M codes: the delta's size makes
    the buckets 8 codes, a few of them crowded)."""
    col = _gdir_column([], n_steps, seed=40 + n_steps % 97, above_all=True)
    assert_parity(ctx, col)


def test_global_directory_flags_codes_past_the_dictionary(ctx):
    """Codes >= |U_M| at b = 25 are flagged and clamped, never faulting, on
    the standalone Step 2(b) entry point, which builds the global directory
    itself."""
    import torch
    rng = np.random.default_rng(78)
    m = GDIR_M
    c = np.zeros(m, np.uint32)
    c[rng.integers(0, m, 40_000)] = 1
    xm = (np.arange(m, dtype=np.uint64) + np.cumsum(c)).astype(np.uint32)     # X_M with steps
    b = synth.bits_for(m)
    bo = synth.bits_for(int(xm[-1]) + 1)
    mc = rng.integers(0, m, 1_100_000).astype(np.uint32)
    mc[::1000] = rng.integers(m, 2**b, mc[::1000].size)       # invalid codes
    main = synth.pack(mc, b)
    out = torch.zeros(dm.dm_packed_bytes(mc.size, bo) // 4, dtype=torch.int32, device="cuda")
    bits = torch.tensor([bo], dtype=torch.int32, device="cuda")
    dm.dm_reencode(ctx, dm.to_device(main), b, mc.size, None, 0, dm.to_device(xm), m, None, 0, bits,
                   bo, out, None, 0)
    torch.cuda.synchronize()
    assert ctx.sync_status() == dm.DM_ECODE
    got = np.array(_brute.unpack_bits(dm.to_host(out, np.uint32)[:20_000], 10_000, bo))
    want = xm[np.minimum(mc[:10_000], m - 1)]
    assert np.array_equal(got, want)
