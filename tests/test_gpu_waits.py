"""Bounded device-side waits give up with DM_ETIMEOUT instead of hanging.

Every wait of Step 1 (grid barriers, the look-back words of the sort passes
and of the merge tiles) polls a bounded number of times.  These tests make a
wait run out on purpose without faulting anything: dm_set_wait_test has one
merge tile withhold its look-back word (a flag that nothing else sets) and
lowers the poll limit, so the tiles after it give up.  The kernel must then
finish, the status word must say DM_ETIMEOUT, and the next merge on the same
context, with the setting off, must again match the oracle byte for byte.
"""
import time

import numpy as np
import pytest

import oracle
import synth
from paper_1109_6885_gb300 import dmerge as dm
from tests import gpu_util

pytestmark = pytest.mark.gpu

MERGE_TILE = 4096   # merged positions per Step 1(b) tile


def _dicts(w, m, d, seed):
    um = synth.dictionary(synth.subseed(seed, 1), w, m)
    dd = synth.dictionary(synth.subseed(seed, 2), w, d)
    rng = np.random.default_rng(seed)
    k = d // 4
    dd[:k] = um[rng.integers(0, m, k)]   # a quarter already in U_M
    return um, dd[rng.permutation(d)]


def _merge_dicts(ctx, w, um, dd):
    import torch
    m, d = um.shape[0], dd.shape[0]
    ud, perm = oracle.sort_delta(w, dd)
    t_um, t_ud, t_perm = dm.to_device(um), dm.to_device(ud), dm.to_device(perm)
    new = dm.key_tensor_empty(m + d, w)
    xm = torch.zeros(m, dtype=torch.int32, device="cuda")
    xd = torch.zeros(d, dtype=torch.int32, device="cuda")
    sc = torch.zeros(2, dtype=torch.int64, device="cuda")
    dm.dm_merge_dicts(ctx, w, t_um, m, t_ud, t_perm, d, new, xm, xd, sc, sc[1:])
    torch.cuda.synchronize()
    return new, xm, xd, sc, (ud, perm)


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_1109_6885_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    c = dm.Context(0, 256 << 20)
    yield c
    c.set_wait_test(None)
    c.close()


def test_withheld_lookback_word_times_out_then_merges_are_exact(ctx):
    w, m, d = 8, 250_000, 60_000          # 76 merge tiles: one wave of co-resident blocks
    um, dd = _dicts(w, m, d, seed=11)
    ctx.set_wait_test(3, spin_limit=1 << 10)
    t0 = time.perf_counter()
    _merge_dicts(ctx, w, um, dd)
    elapsed = time.perf_counter() - t0
    assert ctx.sync_status() == dm.DM_ETIMEOUT
    assert elapsed < 30.0, elapsed
    # the status word was read and cleared; a normal merge on the same context is exact
    ctx.set_wait_test(None)
    new, xm, xd, sc, (ud, perm) = _merge_dicts(ctx, w, um, dd)
    assert ctx.sync_status() == dm.DM_OK
    r_new, r_xm, r_xd = oracle.merge_dicts(w, um, ud, perm)
    u = int(sc[0].item())
    assert u == r_new.shape[0] and int(sc[1].item()) == oracle.new_width(u)
    assert np.array_equal(dm.to_host(new[:u], np.uint64), r_new)
    assert np.array_equal(dm.to_host(xm, np.uint32), r_xm)
    assert np.array_equal(dm.to_host(xd, np.uint32), r_xd)


def test_withholding_the_last_tile_delays_nobody(ctx):
    """Only waits time out: the last merge tile has no successor, so
    withholding its word changes nothing."""
    w, m, d = 4, 30_000, 9_000
    um, dd = _dicts(w, m, d, seed=12)
    last = (m + d + MERGE_TILE - 1) // MERGE_TILE - 1
    ctx.set_wait_test(last, spin_limit=1 << 10)
    new, xm, xd, sc, (ud, perm) = _merge_dicts(ctx, w, um, dd)
    ctx.set_wait_test(None)
    assert ctx.sync_status() == dm.DM_OK
    r_new, r_xm, r_xd = oracle.merge_dicts(w, um, ud, perm)
    u = int(sc[0].item())
    assert u == r_new.shape[0]
    assert np.array_equal(dm.to_host(new[:u], np.uint32), r_new)
    assert np.array_equal(dm.to_host(xm, np.uint32), r_xm)
    assert np.array_equal(dm.to_host(xd, np.uint32), r_xd)


def test_whole_column_merge_reports_the_timeout_then_recovers(ctx):
    """The same through dm_merge_column: Step 2(b) runs on the wrong tables
    without faulting, the status says DM_ETIMEOUT, and the next merge of the
    column matches the oracle."""
    spec = synth.ColumnSpec(n_main=400_000, m=40_000, w=16, n_delta=30_000, f_new=0.4,
                            dist="zipf", zipf_s=1.0, seed=0x7E57)
    col = synth.make_column(spec)
    ctx.set_wait_test(2, spin_limit=1 << 10)
    _, st = gpu_util.run_gpu(ctx, col)
    assert st == dm.DM_ETIMEOUT
    ctx.set_wait_test(None)
    gpu_util.assert_parity(ctx, col)
