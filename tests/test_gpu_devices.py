"""Merges on a second GPU after the first, in one process.

Kernel attributes (the raised shared-memory limits), occupancy figures and
the allocation-free entry point's scratch address are kept per device; a
process that merges on device 0 and then on device 1 must get exact results
on both.  Skipped unless two GPUs are visible.
"""
import numpy as np
import pytest

import oracle
import synth
from paper_1109_6885_gb300 import dmerge as dm
from tests.gpu_util import assert_parity
from tests.test_zz_no_alloc import _inputs

pytestmark = pytest.mark.gpu


def test_merges_on_device_1_after_device_0():
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("one GPU visible")
    from paper_1109_6885_gb300 import build
    build.build()
    cols = [
        # tiled Step 1, X_M directory
        synth.make_column(synth.ColumnSpec(n_main=2_000_000, m=300_000, w=8, n_delta=40_000, f_new=0.3,
                                           dist="zipf", seed=71)),
        # small-dictionary Step 1, narrow re-encode
        synth.make_column(synth.ColumnSpec(n_main=1_200_000, m=3000, w=4, n_delta=999, seed=72)),
        synth.make_column(synth.ColumnSpec(n_main=1_500_000, m=60_000, w=16, n_delta=20_000, f_new=0.5,
                                           seed=73)),
    ]
    w, m, d = 8, 50_000, 10_000
    um, dd = _inputs(w, m, d, 74)
    r_ud, r_perm = oracle.sort_delta(w, dd)
    r_new, r_xm, r_xd = oracle.merge_dicts(w, um, r_ud, r_perm)
    for dev in (0, 1):
        torch.cuda.set_device(dev)
        ctx = dm.Context(dev, 64 << 20)
        for col in cols:
            assert_parity(ctx, col)
        # the allocation-free Step 1(b) on this device
        t_um, t_dd = dm.to_device(um), dm.to_device(dd)
        ud = dm.key_tensor_empty(d, w)
        perm = torch.empty(d, dtype=torch.int32, device="cuda")
        dm.dm_sort_delta(ctx, w, t_dd, d, ud, perm)
        new = dm.key_tensor_empty(m + d, w)
        xm = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        xd = torch.full((d,), -1, dtype=torch.int32, device="cuda")
        sc = torch.zeros(2, dtype=torch.int64, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        dm.dm_merge_dicts_noalloc(w, t_um, m, ud, perm, d, new, xm, xd, sc, sc[1:], status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0 and ctx.sync_status() == dm.DM_OK
        u = int(sc[0].item())
        assert u == r_new.shape[0]
        assert np.array_equal(dm.to_host(new[:u], r_new.dtype).reshape(r_new.shape), r_new)
        assert np.array_equal(xm.cpu().numpy().view(np.uint32), r_xm)
        assert np.array_equal(xd.cpu().numpy().view(np.uint32), r_xd)
        ctx.close()
    torch.cuda.set_device(0)
