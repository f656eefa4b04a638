"""Helpers shared by the GPU tests: run the CUDA path on a synth column and
compare it with the CPU oracle byte for byte."""
from __future__ import annotations

import numpy as np

import oracle
import synth
from paper_1109_6885_gb300 import dmerge as dm


def run_gpu(ctx, col, flags=0, with_x=True):
    import torch
    dcol = dm.DeviceColumn.from_numpy(col.w, col.main_dict, col.main_packed, col.main_bits,
                                      col.n_main, col.delta_dict, col.delta_codes)
    res = dm.alloc_result(dcol, with_x=with_x)
    dm.merge_column(ctx, dcol, res, flags=flags)
    torch.cuda.synchronize()
    st = ctx.sync_status()
    return dm.fetch(res, col.w, col.n_main + col.n_delta), st


def assert_parity(ctx, col, flags=0, ref=None):
    """Whole-column parity: U', X_M, X_D, |U'|, E'_C and the packed bytes."""
    if ref is None:
        ref = oracle.merge_synth_column(col)
    (new_dict, xm, xd, packed, b, u), st = run_gpu(ctx, col, flags)
    assert st == dm.DM_OK, dm.load().dm_status_str(st)
    assert u == ref.u, (u, ref.u)
    assert b == ref.new_bits, (b, ref.new_bits)
    assert np.array_equal(new_dict, ref.new_dict)
    assert np.array_equal(xm, ref.x_main)
    assert np.array_equal(xd, ref.x_delta)
    assert packed.size == ref.new_packed.size
    if not np.array_equal(packed, ref.new_packed):
        bad = np.nonzero(packed != ref.new_packed)[0]
        raise AssertionError(f"packed words differ at {bad[:10]} of {packed.size}")
    return ref


def column_from_lists(w, um, main_codes, dd, dcodes, b=None):
    """A synth.Column built from explicit keys and codes."""
    from tests import _brute
    umk = _brute.key_array(um, w)
    ddk = _brute.key_array(dd, w) if dd else synth.key_array(0, w)
    bb = synth.bits_for(len(um)) if b is None else b
    mc = np.array(main_codes, np.uint32)
    spec = synth.ColumnSpec(n_main=len(main_codes), m=len(um), w=w, n_delta=len(dcodes))
    return synth.Column(spec, umk, mc, bb, synth.pack(mc, bb), ddk, np.array(dcodes, np.uint32))
