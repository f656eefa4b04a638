"""Step 2(b) by binary search in U' (Section 5.2, Eq. 5) gives the same packed
bytes as the translation-table route and the oracle."""
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


CASES = [
    dict(n_main=300_007, m=5_000, w=4, n_delta=3_001, f_new=0.4, dist="zipf", zipf_s=0.8),
    dict(n_main=1_000_003, m=100_000, w=8, n_delta=10_007, f_new=0.5, dist="uniform"),
    dict(n_main=700_001, m=60_000, w=16, n_delta=40_000, f_new=0.5, dist="uniform"),
    dict(n_main=0, m=0, w=8, n_delta=50_003, f_new=1.0, dist="uniform"),
    dict(n_main=65_537, m=1_048_576, w=8, n_delta=1_000, f_new=0.9, dist="uniform"),   # E'_C = E_C + 1
    dict(n_main=100_001, m=1, w=4, n_delta=1, f_new=0.0, dist="uniform"),              # one value: 0 bits
]


@pytest.mark.parametrize("k", range(len(CASES)))
def test_search_route_matches(ctx, k):
    import torch
    spec = synth.ColumnSpec(seed=synth.column_seed(13, k), **CASES[k])
    col = synth.make_column(spec)
    ref = oracle.merge_synth_column(col)
    dcol = dm.DeviceColumn.from_numpy(col.w, col.main_dict, col.main_packed, col.main_bits, col.n_main,
                                      col.delta_dict, col.delta_codes)
    res = dm.alloc_result(dcol)
    dm.merge_column(ctx, dcol, res)
    torch.cuda.synchronize()
    assert ctx.sync_status() == dm.DM_OK
    if res.new_packed.numel():
        res.new_packed.fill_(-1)
    dm.dm_reencode_search(ctx, dcol.cin(), res.cout())
    torch.cuda.synchronize()
    assert ctx.sync_status() == dm.DM_OK
    new_dict, xm, xd, packed, b, u = dm.fetch(res, col.w, col.n_main + col.n_delta)
    assert (u, b) == (ref.u, ref.new_bits)
    assert np.array_equal(packed, ref.new_packed)


def test_search_route_flags_bad_codes(ctx):
    """Codes past their dictionary are clamped and flagged, never faulting."""
    import torch
    spec = synth.ColumnSpec(n_main=10_000, m=1_000, w=8, n_delta=100, f_new=0.5, dist="uniform",
                            seed=synth.column_seed(13, 99))
    col = synth.make_column(spec)
    dcol = dm.DeviceColumn.from_numpy(col.w, col.main_dict, col.main_packed, col.main_bits, col.n_main,
                                      col.delta_dict, col.delta_codes)
    res = dm.alloc_result(dcol)
    dm.merge_column(ctx, dcol, res)
    torch.cuda.synchronize()
    assert ctx.sync_status() == dm.DM_OK
    dcol.delta_codes[5] = 1 << 30
    dm.dm_reencode_search(ctx, dcol.cin(), res.cout())
    torch.cuda.synchronize()
    assert ctx.sync_status() == dm.DM_ECODE
