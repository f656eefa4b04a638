"""Delta ingest on the GPU (Section 4): appended values -> the insertion-order
dictionary and codes, element by element against the oracle."""
import numpy as np
import pytest

import oracle
import synth
from paper_1109_6885_gb300 import dmerge as dm

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


def _run(ctx, w, vals):
    import torch
    n = vals.shape[0]
    t = dm.to_device(vals) if n else dm.key_tensor_empty(0, w)
    dd = dm.key_tensor_empty(max(n, 1), w)
    codes = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    dlen = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    dm.dm_ingest_delta(ctx, w, t, n, dd, codes, dlen)
    torch.cuda.synchronize()
    assert ctx.sync_status() == dm.DM_OK
    d = int(dlen.item())
    return dm.to_host(dd[:d], dm.key_np_dtype(w)), dm.to_host(codes[:n], np.uint32), d


def _values(w, n, distinct, seed):
    rng = np.random.default_rng(seed)
    pool = synth.dictionary(synth.subseed(seed, w), w, distinct)
    return pool[rng.integers(0, distinct, n)]


@pytest.mark.parametrize("w", [4, 8, 16])
@pytest.mark.parametrize("n,distinct", [(1, 1), (1000, 37), (1023, 1023), (1025, 5), (300_001, 20_000),
                                        (200_000, 1), (150_000, 150_000)])
def test_ingest_parity(ctx, w, n, distinct):
    vals = _values(w, n, distinct, n + distinct)
    if distinct == n:
        vals = synth.dictionary(synth.subseed(n, w), w, n)[np.random.default_rng(n).permutation(n)]
    want_dd, want_codes = oracle.ingest_delta(w, vals)
    dd, codes, d = _run(ctx, w, vals)
    assert d == want_dd.shape[0]
    assert np.array_equal(dd, want_dd)
    assert np.array_equal(codes, want_codes)


@pytest.mark.parametrize("w", [4, 16])
def test_ingest_reproduces_a_delta_partition(ctx, w):
    """A synthetic delta is stored in order of first arrival: ingesting its expanded
    values gives back its dictionary and codes exactly."""
    col = synth.make_column(synth.ColumnSpec(n_main=100_000, m=20_000, w=w, n_delta=400_000, f_new=0.3,
                                             dist="zipf", zipf_s=1.0, seed=synth.column_seed(17, w)))
    vals = col.delta_dict[col.delta_codes]
    dd, codes, d = _run(ctx, w, vals)
    assert np.array_equal(dd, col.delta_dict)
    assert np.array_equal(codes, col.delta_codes)


def test_ingest_empty(ctx):
    import torch
    dlen = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    dm.dm_ingest_delta(ctx, 8, None, 0, None, None, dlen)
    torch.cuda.synchronize()
    assert int(dlen.item()) == 0


def test_ingest_table_equals_each_column_alone(ctx):
    """A table ingest of 11 columns (more than the eight branches, so
    branches take several columns in turn and reuse their scratch) of every
    width and duplicate density: each column's D_dict, codes and |D_dict|
    equal the oracle's ingest of that column."""
    import torch
    n = 300_007
    shapes = [(4, 7), (8, 20_000), (16, 300_007), (8, 1), (4, 150_000), (16, 37), (8, 299_000), (4, 2),
              (16, 5_000), (8, 64), (4, 300_007)]
    cols, wants, outs = [], [], []
    for k, (w, distinct) in enumerate(shapes):
        vals = _values(w, n, distinct, 900 + k)
        if distinct == n:
            vals = synth.dictionary(synth.subseed(k, w), w, n)[np.random.default_rng(k).permutation(n)]
        wants.append(oracle.ingest_delta(w, vals))
        t = dm.to_device(vals)
        dd = dm.key_tensor_empty(n, w)
        codes = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        dlen = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        cols.append((w, t, dd, codes, dlen))
        outs.append((w, dd, codes, dlen))
    dm.dm_ingest_table(ctx, cols, n)
    torch.cuda.synchronize()
    assert ctx.sync_status() == dm.DM_OK
    for (w, dd, codes, dlen), (want_dd, want_codes) in zip(outs, wants):
        d = int(dlen.item())
        assert d == want_dd.shape[0]
        assert np.array_equal(dm.to_host(dd[:d], dm.key_np_dtype(w)), want_dd)
        assert np.array_equal(dm.to_host(codes, np.uint32), want_codes)


def test_ingest_table_rejects_a_bad_column_before_launching():
    import torch
    from paper_1109_6885_gb300 import build
    build.build()
    c = dm.Context(0, 1 << 20)
    good = dm.key_tensor_empty(16, 8)
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    dlen = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(dm.DmError) as e:
        dm.dm_ingest_table(c, [(8, good, good, out, dlen), (3, good, good, out, dlen)], 16)
    assert e.value.status == dm.DM_EINVAL
    c.close()


def test_ingest_table_of_no_rows_sets_every_length_to_zero(ctx):
    import torch
    lens = [torch.full((1,), -1, dtype=torch.int64, device="cuda") for _ in range(3)]
    dm.dm_ingest_table(ctx, [(w, None, None, None, dl) for w, dl in zip((4, 8, 16), lens)], 0)
    torch.cuda.synchronize()
    assert ctx.sync_status() == dm.DM_OK
    assert [int(dl.item()) for dl in lens] == [0, 0, 0]
    dm.dm_ingest_table(ctx, [], 0)      # no columns: nothing to do
