"""The allocation-free Step 1(b) entry point agrees with the regular one.

dm_merge_dicts_noalloc serves callers that cannot allocate device memory
when they merge (their engine owns all of HBM through its own pools, or
cudaMalloc's implicit synchronisation is not acceptable on their path); its
scratch is a fixed array in the library's static device memory.  This test
calls it through the C ABI on merges in a row, the first at exactly the
array's limit of DM_NOALLOC_MAX_ENTRIES entries (every merge tile of the
array in use) and then smaller ones of every key width (each must not see
the previous call's leftovers), and compares every output with
dm_merge_dicts on the same inputs and with the oracle's Step 1(b); merges
are exact integer work, so the comparisons are bit-exact.  This file is
collected last.
"""
import numpy as np
import pytest

import oracle
import synth
from paper_1109_6885_gb300 import dmerge as dm

pytestmark = pytest.mark.gpu


def _inputs(w, m, d, seed):
    um = synth.dictionary(synth.subseed(seed, 1), w, m)
    dd = synth.dictionary(synth.subseed(seed, 2), w, d)
    rng = np.random.default_rng(seed)
    k = d // 3
    dd[:k] = um[rng.integers(0, m, k)]                # a third already in U_M
    dd[k:k + 50] = dd[:50]                            # and some repeats inside D_dict
    return um, dd[rng.permutation(d)]


def test_noalloc_merge_matches_regular_entry_point():
    import torch

    from paper_1109_6885_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    ctx = dm.Context(0, 64 << 20)
    limit = dm.DM_NOALLOC_MAX_ENTRIES
    cases = [(8, limit - (1 << 20), 1 << 20, 3), (4, 700_000, 300_000, 1), (16, 40_000, 9_000, 2),
             (8, 5_000, 1_234, 4)]
    for w, m, d, seed in cases:
        um, dd = _inputs(w, m, d, seed)
        t_um, t_dd = dm.to_device(um), dm.to_device(dd)
        ud = dm.key_tensor_empty(d, w)
        perm = torch.empty(d, dtype=torch.int32, device="cuda")
        dm.dm_sort_delta(ctx, w, t_dd, d, ud, perm)

        outs = []
        for noalloc in (False, True):
            new = dm.key_tensor_empty(m + d, w)
            new.fill_(-1)
            xm = torch.full((m,), -1, dtype=torch.int32, device="cuda")
            xd = torch.full((d,), -1, dtype=torch.int32, device="cuda")
            sc = torch.zeros(2, dtype=torch.int64, device="cuda")
            status = torch.zeros(1, dtype=torch.int32, device="cuda")
            if noalloc:
                dm.dm_merge_dicts_noalloc(w, t_um, m, ud, perm, d, new, xm, xd, sc, sc[1:],
                                          status)
            else:
                dm.dm_merge_dicts(ctx, w, t_um, m, ud, perm, d, new, xm, xd, sc, sc[1:])
            torch.cuda.synchronize()
            outs.append((new.cpu(), xm.cpu(), xd.cpu(), sc.cpu(), int(status.item())))
        assert ctx.sync_status() == dm.DM_OK
        (n0, xm0, xd0, sc0, _), (n1, xm1, xd1, sc1, st1) = outs
        assert st1 == 0
        assert torch.equal(sc0, sc1)
        u = int(sc0[0])
        assert 0 < u <= m + d
        assert torch.equal(n0[:u], n1[:u])
        assert torch.equal(xm0, xm1)
        assert torch.equal(xd0, xd1)
        # and both agree with the oracle's Step 1(b) on the oracle's own sort
        r_ud, r_perm = oracle.sort_delta(w, dd)
        r_new, r_xm, r_xd = oracle.merge_dicts(w, um, r_ud, r_perm)
        assert u == r_new.shape[0]
        assert int(sc1[1]) == oracle.new_width(u)
        assert np.array_equal(dm.to_host(n1[:u], r_new.dtype).reshape(r_new.shape), r_new)
        assert np.array_equal(xm1.numpy().view(np.uint32), r_xm)
        assert np.array_equal(xd1.numpy().view(np.uint32), r_xd)
    ctx.close()


def test_noalloc_rejects_oversized_merge():
    """Sizes above the array's limit are refused before anything is queued."""
    import torch

    from paper_1109_6885_gb300 import build
    build.build()
    small = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(dm.DmError) as e:
        dm.dm_merge_dicts_noalloc(8, small, dm.DM_NOALLOC_MAX_ENTRIES, small, small, 1, small,
                                  small, small, small, small[1:])
    assert e.value.status == dm.DM_EINVAL
